// C-ABI layer: handle lifetime, host-side set-up, the per-step launch
// sequence and state transfer.  See include/bd.h for the contract of each
// entry point.
//
// A handle advances R >= 1 independent replicas (a single system is R = 1).
// Replicas are concatenated: each owns a contiguous range of internal disk
// slots, its own ghost points (after all disks), its own triangles, j tiles,
// force i blocks and Verlet cells; per-replica parameters live in a device
// table (BdRep).  Every kernel works on the union, so one launch of each
// kernel advances every replica.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <limits>
#include <vector>

#include "bd_handle.h"
#include "bd_internal.h"
#include "predicates.cuh"

namespace bdhost {
int build_delaunay(const double *X, const double *Y, const bdpred::Grid &grid,
                   const std::vector<int> &order, const std::vector<int> &g, std::vector<int> &V,
                   std::vector<int> &N);
void make_ghosts(double L, double a, std::vector<double> &gx, std::vector<double> &gy);
double ghost_extent(double L, double a);
int rsa_place(int n, double lo, double hi, double dmin, uint64_t seed, std::vector<double> &xy);
int lattice_place(int n, double lo, double hi, double dmin, uint64_t seed, std::vector<double> &xy);
int any_overlap(int n, const double *xy, double lo, double hi, double dmin, const double *rad = nullptr);
int any_overlap_periodic(int n, const double *xy, double L, double dmin, const double *rad = nullptr);
int build_torus_delaunay(const double *X, const double *Y, const std::vector<int> &ids, double L,
                         const bdpred::Grid &grid, std::vector<int> &V, std::vector<int> &S,
                         std::vector<int> &N);
uint64_t hilbert_index(uint32_t x, uint32_t y);
}  // namespace bdhost

namespace bdcapi {

int cuda_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? BD_ERR_NOMEM : BD_ERR_CUDA; }

void rep_set_alpha(BdRep &B, const double *alpha, int n_species) {
  for (int i = 0; i < BD_MAX_SPECIES; ++i)
    for (int j = 0; j < BD_MAX_SPECIES; ++j) {
      double v = 0.0;
      if (i < n_species && j < n_species) v = n_species == 1 ? alpha[0] : alpha[i * n_species + j];
      B.alpha_d[BD_MAX_SPECIES * i + j] = v;
      B.alpha[BD_MAX_SPECIES * i + j] = (float)v;
    }
}

}  // namespace bdcapi

using namespace bdcapi;

namespace {

template <class T>
cudaError_t dalloc(bd_handle *h, T **ptr, size_t count) {
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(1, count) * sizeof(T));
  if (e != cudaSuccess) return e;
  h->dev_allocs.push_back(p);
  *ptr = (T *)p;
  return cudaSuccess;
}

size_t pad_to(size_t v, size_t m) { return (v + m - 1) / m * m; }

int grid_shift_for(double E) {
  // every coordinate is below E in magnitude; need E * 2^s < 2^51
  int e = (int)ceil(log2(E + 1.0));
  return 51 - e;
}

int grid_shift(double L, double a) { return grid_shift_for(bdhost::ghost_extent(L, a)); }

double box_side(const bd_params &p) {
  const double L = p.box_L > 0 ? p.box_L : sqrt((double)p.n * M_PI * p.a * p.a / p.area_fraction);
  // periodic box: a side exactly representable in FP32, so that the sweeps'
  // minimum-image subtractions of L are exact
  return p.boundary == BD_BOUNDARY_PERIODIC ? (double)(float)L : L;
}

// largest coordinate magnitude the predicates see: ghost points (walls) or
// corners lifted by one box side (periodic)
double coord_extent(const bd_params &p) {
  const double L = box_side(p);
  return p.boundary == BD_BOUNDARY_PERIODIC ? 4.0 * ceil(L) + 8.0 : bdhost::ghost_extent(L, p.a);
}

int validate(const bd_params *p) {
  if (!p) return BD_ERR_ARG;
  if (p->n < 1 || p->n > (1 << 28)) return BD_ERR_ARG;
  if (p->n_species < 1 || p->n_species > BD_MAX_SPECIES) return BD_ERR_ARG;
  if (!(p->a > 0) || !isfinite(p->a)) return BD_ERR_ARG;
  if (!(p->box_L > 0) && !(p->area_fraction > 0 && p->area_fraction < 0.9)) return BD_ERR_ARG;
  if (p->law < BD_LAW_NONE || p->law > BD_LAW_SHORT) return BD_ERR_ARG;
  if (p->precision < 0 || p->precision > 1) return BD_ERR_ARG;
  if (!(p->dt > 0) || !isfinite(p->dt)) return BD_ERR_ARG;
  if (!(p->D >= 0) || !(p->Dr >= 0) || !isfinite(p->v0)) return BD_ERR_ARG;
  for (int k = 0; k < p->n_species * p->n_species; ++k)
    if (!isfinite(p->alpha[k])) return BD_ERR_ARG;
  if (p->max_corr_iters < 1 || p->max_flip_rounds < 1) return BD_ERR_ARG;
  if (p->law == BD_LAW_SHORT) {
    if (!(p->r_cut > 2.0 * p->a) || !(p->skin > 0) || !(p->eps >= 0) || !(p->kappa >= 0)) return BD_ERR_ARG;
    if (p->precision != 0) return BD_ERR_UNSUPPORTED;
  }
  if (p->overlap_mode < BD_OVERLAP_DELAUNAY || p->overlap_mode > BD_OVERLAP_VERLET) return BD_ERR_ARG;
  if (p->overlap_mode == BD_OVERLAP_VERLET && p->law != BD_LAW_SHORT) return BD_ERR_UNSUPPORTED;
  if (p->max_dt_halvings < 0 || p->max_dt_halvings > 20) return BD_ERR_ARG;
  if (p->boundary < BD_BOUNDARY_WALLS || p->boundary > BD_BOUNDARY_PERIODIC) return BD_ERR_ARG;
  if (p->placement < BD_PLACE_RSA || p->placement > BD_PLACE_LATTICE) return BD_ERR_ARG;
  if (p->boundary == BD_BOUNDARY_PERIODIC) {
    if (p->n < 16) return BD_ERR_UNSUPPORTED;
    const double L = box_side(*p);
    if (!(L >= 16.0 * p->a) || !(L < 1e7)) return BD_ERR_UNSUPPORTED;
    if (p->law == BD_LAW_SHORT && L < 3.0 * (p->r_cut + p->skin)) return BD_ERR_UNSUPPORTED;
  }
  return BD_OK;
}

double snap_host(double v, double q, double inv_q) { return nearbyint(v * inv_q) * q; }

// a periodic coordinate in [0, L) on the grid (L is a multiple of q)
double periodic_coord(double v, double L, double q, double inv_q) {
  double y = snap_host(v - L * floor(v / L), q, inv_q);
  if (y >= L) y -= L;
  if (y < 0.0) y += L;
  return y;
}

// Build the long-range work items: every i block of a long-range replica
// against chunks of at most `tiles` j tiles of the same replica.
void make_items(bd_handle *h, int tiles, std::vector<int4> &items, int &max_chunk) {
  items.clear();
  max_chunk = 1;
  for (size_t r = 0; r < h->reps.size(); ++r) {
    RepHost &R = h->reps[r];
    BdRep &B = h->h_rep[r];
    if (R.p.law != BD_LAW_LONG) {
      B.nchunk = 1;
      continue;
    }
    const int nt_r = R.tile_end - R.tile_begin;
    int nch = std::max(1, (nt_r + tiles - 1) / tiles);
    if (!h->fpart_cap.empty()) nch = std::min(nch, h->fpart_cap[r]);
    // the FP64 sweep walks its chunk's slots, not the items: all its slots
    if (h->c.precision == 1 && !h->fpart_cap.empty()) nch = h->fpart_cap[r];
    B.nchunk = nch;
    max_chunk = std::max(max_chunk, nch);
    for (int ib = 0; ib < R.n_iblocks; ++ib)
      for (int ch = 0; ch < nch; ++ch) {
        int t0 = R.tile_begin + (int)(((long long)nt_r * ch) / nch);
        int t1 = R.tile_begin + (int)(((long long)nt_r * (ch + 1)) / nch);
        if (t1 > t0) items.push_back(make_int4(R.iblock_base + ib, t0, t1, ch));
      }
  }
}

// Work items of the symmetric sweep: block P of a long-range replica against
// its own two tiles (i side only) and every later tile of the replica, in
// chunks of at most `tiles` tiles, plus the reduction lists (per block its
// items, per tile its j-partial tiles, both in item order).
struct SymPlan {
  std::vector<int4> items;
  std::vector<int> iptr, iidx, jptr, jidx;
  int n_jtiles = 0;
};

// Work items of the symmetric sweep: each row of block P (its tiles from 2P
// on) in chunks of `tiles`.  The i side of an item is written as one partial
// (512 disks x 8 B), so long chunks cut the partial traffic; the last part of
// the work is cut into 2-tile items, placed at the end of the launch order, so
// the final waves of resident blocks stay full.
void make_sym(const bd_handle *h, int tiles, int variant, SymPlan &S) {
  const int nblocks = h->np / BD_SB, ntiles = h->np / BD_TJ;
  std::vector<std::vector<int>> bl(nblocks), tl(ntiles);
  S.items.clear();
  S.n_jtiles = 0;
  struct Chunk {
    int P, c0, c1;
  };
  std::vector<Chunk> ch;
  for (const RepHost &R : h->reps) {
    if (R.p.law != BD_LAW_LONG) continue;
    const int tb = R.tile_begin, te = R.tile_end;
    for (int P = tb / 2; P < te / 2; ++P)
      for (int c0 = 2 * P; c0 < te; c0 += tiles) ch.push_back({P, c0, std::min(te, c0 + tiles)});
  }
  if (tiles > 2) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long slots = (long)sms * std::max(1, bd_force_sym_blocks_per_sm(variant, h->c.any_periodic));
    long tail = 4 * slots;   // tile units: two waves of 2-tile items
    std::vector<Chunk> small;
    while (!ch.empty() && tail > 0) {
      const Chunk c = ch.back();
      ch.pop_back();
      for (int s = c.c0; s < c.c1; s += 2) small.push_back({c.P, s, std::min(c.c1, s + 2)});
      tail -= c.c1 - c.c0;
    }
    std::stable_sort(small.begin(), small.end(),
                     [](const Chunk &a, const Chunk &b) { return a.c1 - a.c0 > b.c1 - b.c0; });
    ch.insert(ch.end(), small.begin(), small.end());
  }
  for (const Chunk &c : ch) {
    const int jt0 = std::max(c.c0, 2 * c.P + 2);
    const int it = (int)S.items.size();
    S.items.push_back(make_int4(c.P, c.c0, c.c1, S.n_jtiles));
    bl[c.P].push_back(it);
    for (int t = jt0; t < c.c1; ++t) tl[t].push_back(S.n_jtiles + (t - jt0));
    S.n_jtiles += std::max(0, c.c1 - jt0);
  }
  auto flatten = [](const std::vector<std::vector<int>> &v, std::vector<int> &ptr, std::vector<int> &idx) {
    ptr.assign(v.size() + 1, 0);
    idx.clear();
    for (size_t k = 0; k < v.size(); ++k) {
      idx.insert(idx.end(), v[k].begin(), v[k].end());
      ptr[k + 1] = (int)idx.size();
    }
  };
  flatten(bl, S.iptr, S.iidx);
  flatten(tl, S.jptr, S.jidx);
}

// replace a device array owned by the handle
template <class T>
cudaError_t realloc_dev(bd_handle *h, T **ptr, size_t count) {
  if (*ptr) {
    void *old = (void *)*ptr;
    cudaFree(old);
    h->dev_allocs.erase(std::find(h->dev_allocs.begin(), h->dev_allocs.end(), old));
    *ptr = nullptr;
  }
  return dalloc(h, ptr, std::max<size_t>(1, count));
}

template <class T>
cudaError_t upload_vec(bd_handle *h, T **ptr, const std::vector<T> &v) {
  cudaError_t e = realloc_dev(h, ptr, v.size());
  if (e == cudaSuccess && !v.empty()) e = cudaMemcpy(*ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

cudaError_t upload_sym(bd_handle *h, const SymPlan &S) {
  BdDev &d = h->d;
  cudaError_t e = upload_vec(h, &d.sitems, S.items);
  if (e == cudaSuccess) e = upload_vec(h, &d.red_iptr, S.iptr);
  if (e == cudaSuccess) e = upload_vec(h, &d.red_iidx, S.iidx);
  if (e == cudaSuccess) e = upload_vec(h, &d.red_jptr, S.jptr);
  if (e == cudaSuccess) e = upload_vec(h, &d.red_jidx, S.jidx);
  if (e == cudaSuccess) e = realloc_dev(h, &d.ipart, S.items.size() * BD_SB);
  if (e == cudaSuccess) e = realloc_dev(h, &d.jpart, (size_t)S.n_jtiles * BD_TJ);
  if (e != cudaSuccess) return e;
  h->c.n_sitems = (int)S.items.size();
  h->c.max_nchunk = 1;
  for (size_t r = 0; r < h->reps.size(); ++r) h->h_rep[r].nchunk = 1;
  return cudaMemcpy((void *)h->d.rep, h->h_rep.data(), h->h_rep.size() * sizeof(BdRep), cudaMemcpyHostToDevice);
}

// j tiles per work item for a single system: fill whole waves of resident
// force blocks (the occupancy calculator gives blocks per SM)
int single_system_tiles(const bd_handle *h) {
  const char *env = getenv("BD_NCHUNK");
  const RepHost &R = h->reps[0];
  const int ntiles = std::max(1, R.tile_end - R.tile_begin);
  if (env && atoi(env) > 0) return std::max(1, (ntiles + atoi(env) - 1) / atoi(env));
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (h->c.precision == 1) {
    int blocks = (h->np + 127) / 128;
    int want = std::max(1, (4 * sms) / std::max(1, blocks));
    want = std::max(1, std::min(want, ntiles));
    return std::max(1, (ntiles + want - 1) / want);
  }
  int per_sm = bd_force_blocks_per_sm(h->c.force_variant);
  if (per_sm < 1) per_sm = 1;
  const long slots = (long)sms * per_sm;
  const long ib = std::max(1, R.n_iblocks);
  int best = 1;
  double best_eff = -1.0;
  for (int ch = 1; ch <= std::min(ntiles, 64); ++ch) {
    long ctas = ib * ch;
    long waves = (ctas + slots - 1) / slots;
    double fill = (double)ctas / (double)(waves * slots);
    int tiles_max = (ntiles + ch - 1) / ch;
    double bal = ((double)ntiles / ch) / tiles_max;
    double eff = fill * bal * (waves >= 2 ? 1.0 : 0.9);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = ch;
    }
  }
  return std::max(1, (ntiles + best - 1) / best);
}

cudaError_t upload_items(bd_handle *h, const std::vector<int4> &items, int max_chunk) {
  BdConst &c = h->c;
  c.n_items = (int)items.size();
  c.max_nchunk = max_chunk;
  cudaError_t e = cudaSuccess;
  if (h->d.items) {
    void *old = (void *)h->d.items;
    cudaFree(old);
    h->dev_allocs.erase(std::find(h->dev_allocs.begin(), h->dev_allocs.end(), old));
    h->d.items = nullptr;
  }
  e = dalloc(h, &h->d.items, std::max<size_t>(1, items.size()));
  if (e != cudaSuccess) return e;
  if (!items.empty())
    e = cudaMemcpy(h->d.items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  return cudaMemcpy((void *)h->d.rep, h->h_rep.data(), h->h_rep.size() * sizeof(BdRep),
                    cudaMemcpyHostToDevice);
}

// set up the work list of a sweep variant with `tiles` j tiles per item
cudaError_t use_variant(bd_handle *h, int variant, int tiles) {
  h->c.force_variant = variant;
  h->tune_tiles = tiles;
  if (variant >= 2) {
    SymPlan S;
    make_sym(h, tiles, variant, S);
    return upload_sym(h, S);
  }
  std::vector<int4> items;
  int mc = 1;
  make_items(h, tiles, items, mc);
  return upload_items(h, items, mc);
}

// Autotuner of the all-pairs sweep: time the force launch for each candidate
// (kernel variant, j tiles per work item) and keep the fastest.  Candidates:
// the one-sided sweeps (scalar, packed) and the symmetric sweep over several
// chunk sizes; a single system also tries the wave-filling chunk size.
cudaError_t autotune(bd_handle *h) {
  std::vector<int2> cand;
  if (h->c.any_periodic) {
    // periodic boxes: the scalar one-sided sweep and the symmetric sweep, both
    // with minimum images
    for (int t : {2, 4, 8, 16, 32, 64}) cand.push_back(make_int2(0, t));
    if (h->reps.size() == 1) cand.push_back(make_int2(0, single_system_tiles(h)));
  } else if (h->reps.size() == 1) {
    cand.push_back(make_int2(1, single_system_tiles(h)));
  } else {
    for (int t : {2, 4, 8, 16, 32, 64}) cand.push_back(make_int2(0, t));
    for (int t : {2, 4, 8, 16, 32, 64}) cand.push_back(make_int2(1, t));
  }
  for (int v : {2, 3})
    for (int t : {2, 4, 8, 16, 32}) cand.push_back(make_int2(v, t));
  float best_ms = 1e30f;
  int2 best = cand[0];
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  cudaError_t e = cudaSuccess;
  for (const int2 &cv : cand) {
    e = use_variant(h, cv.x, cv.y);
    if (e != cudaSuccess) break;
    float tot = 0.f;
    for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
      cudaEventRecord(a, h->stream);
      e = bd_launch_force_long_variant(h->d, h->c, cv.x, h->stream);
      cudaEventRecord(b, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0) tot += ms;
    }
    if (e == cudaSuccess && tot < best_ms) {
      best_ms = tot;
      best = cv;
    }
  }
  if (e == cudaSuccess) e = use_variant(h, best.x, best.y);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return e;
}

struct Spec {
  bd_params p;
  const double *xy;
  const uint8_t *sp;
  const float *th;
  const double *rad = nullptr;   // polydisperse disks: one radius each (bd_init_radii)
};

int build_handle(const std::vector<Spec> &specs, void *stream, bd_handle **out);

}  // namespace

extern "C" void bd_free(bd_handle *h);

namespace {

int build_handle(const std::vector<Spec> &specs, void *stream, bd_handle **out) {
  *out = nullptr;
  const int R = (int)specs.size();
  if (R < 1) return BD_ERR_ARG;
  for (const Spec &s : specs) {
    int rc = validate(&s.p);
    if (rc) return rc;
    if (s.p.a != specs[0].p.a || s.p.precision != specs[0].p.precision ||
        s.p.max_corr_iters != specs[0].p.max_corr_iters ||
        s.p.max_flip_rounds != specs[0].p.max_flip_rounds || s.p.overlap_mode != specs[0].p.overlap_mode)
      return BD_ERR_ARG;   // one disk radius, precision, loop caps and overlap mode per handle
    if (R > 1 && s.p.max_dt_halvings > 0) return BD_ERR_UNSUPPORTED;   // halving: one system per handle
    if (s.rad) {
      // polydisperse disks: every radius in (0, a]; over the Delaunay edges
      // the overlap certificate needs a_max <= sqrt(2) a_min
      if (R > 1 || !s.xy) return BD_ERR_ARG;
      double lo = 1e300, hi = 0.0;
      for (int i = 0; i < s.p.n; ++i) {
        const double r = s.rad[i];
        if (!(r > 0.0) || !(r <= s.p.a)) return BD_ERR_ARG;
        lo = std::min(lo, r);
        hi = std::max(hi, r);
      }
      if (s.p.overlap_mode == BD_OVERLAP_DELAUNAY && hi > 1.4142135623730951 * lo) return BD_ERR_UNSUPPORTED;
    }
  }
  bd_handle *h = new (std::nothrow) bd_handle();
  if (!h) return BD_ERR_NOMEM;
  memset(&h->d, 0, sizeof(h->d));
  memset(&h->c, 0, sizeof(h->c));
  h->stream = (cudaStream_t)stream;
  const double a = specs[0].p.a;

  // ---- position grid shared by all replicas ----
  double E = 0.0;
  for (const Spec &s : specs) E = std::max(E, coord_extent(s.p));
  const int s_shift = grid_shift_for(E);
  const double q = ldexp(1.0, -s_shift), inv_q = ldexp(1.0, s_shift);

  h->reps.resize(R);
  std::vector<std::vector<double>> xyr(R);
  std::vector<std::vector<uint8_t>> spr(R);
  std::vector<std::vector<float>> thr(R);
  int ext = 0;
  for (int r = 0; r < R; ++r) {
    const bd_params &p = specs[r].p;
    RepHost &RH = h->reps[r];
    RH.p = p;
    RH.n = p.n;
    RH.ext_base = ext;
    ext += p.n;
    RH.L = box_side(p);
    RH.periodic = p.boundary == BD_BOUNDARY_PERIODIC;
    RH.wall_lo = RH.periodic ? 0.0 : ceil(p.a * inv_q) * q;
    RH.wall_hi = RH.periodic ? RH.L : floor((RH.L - p.a) * inv_q) * q;
    if (!(RH.wall_hi > RH.wall_lo)) { delete h; return BD_ERR_ARG; }
    const double *rad = specs[r].rad;
    // a disk's own walls (polydisperse: a_i from each wall), on the grid
    auto wlo = [&](int i) { return rad && !RH.periodic ? ceil(rad[i] * inv_q) * q : RH.wall_lo; };
    auto whi = [&](int i) { return rad && !RH.periodic ? floor((RH.L - rad[i]) * inv_q) * q : RH.wall_hi; };
    std::vector<double> &xy = xyr[r];
    xy.resize(2 * (size_t)p.n);
    if (specs[r].xy) {
      memcpy(xy.data(), specs[r].xy, sizeof(double) * 2 * (size_t)p.n);
    } else if ((p.placement == BD_PLACE_LATTICE ? bdhost::lattice_place(p.n, p.a, RH.L - p.a, 2.0 * p.a, p.seed, xy)
                                                 : bdhost::rsa_place(p.n, p.a, RH.L - p.a, 2.0 * p.a, p.seed, xy)) != 0) {
      delete h;
      return BD_ERR_ARG;
    }
    if (RH.periodic) {
      // any real coordinate: brought into [0, L) on the grid
      for (size_t k = 0; k < xy.size(); ++k) {
        if (!isfinite(xy[k])) { delete h; return BD_ERR_INIT_OVERLAP; }
        xy[k] = periodic_coord(xy[k], RH.L, q, inv_q);
      }
      if (bdhost::any_overlap_periodic(p.n, xy.data(), RH.L, 2.0 * p.a * (1.0 - 1e-12), rad)) {
        delete h;
        return BD_ERR_INIT_OVERLAP;
      }
    } else {
      for (size_t k = 0; k < xy.size(); ++k) {
        const double ak = rad ? rad[k / 2] : p.a;
        if (!isfinite(xy[k]) || xy[k] < ak - 1e-9 * RH.L || xy[k] > RH.L - ak + 1e-9 * RH.L) {
          delete h;
          return BD_ERR_INIT_OVERLAP;
        }
      }
      if (bdhost::any_overlap(p.n, xy.data(), 0.0, RH.L, 2.0 * p.a * (1.0 - 1e-12), rad)) {
        delete h;
        return BD_ERR_INIT_OVERLAP;
      }
      for (size_t k = 0; k < xy.size(); ++k)
        xy[k] = std::min(whi((int)(k / 2)), std::max(wlo((int)(k / 2)), snap_host(xy[k], q, inv_q)));
    }
    spr[r].assign(p.n, 0);
    if (specs[r].sp)
      for (int i = 0; i < p.n; ++i) {
        if (specs[r].sp[i] >= p.n_species) { delete h; return BD_ERR_ARG; }
        spr[r][i] = specs[r].sp[i];
      }
    thr[r].assign(p.n, 0.f);
    if (specs[r].th) memcpy(thr[r].data(), specs[r].th, sizeof(float) * p.n);
  }
  h->n = ext;

  // ---- internal order: per replica species-major, Hilbert-minor, tile-padded ----
  std::vector<std::vector<int>> byhr(R);   // per replica: disk slots in Hilbert order
  int slot = 0, iblock = 0;
  std::vector<int> iperm;
  std::vector<float2> iorg;
  std::vector<uint8_t> tile_sp;
  std::vector<int> slot_ext, slot_local, slot_rep;
  for (int r = 0; r < R; ++r) {
    RepHost &RH = h->reps[r];
    const int n = RH.n;
    const std::vector<double> &xy = xyr[r];
    const std::vector<uint8_t> &sp = spr[r];
    std::vector<uint64_t> hk(n);
    for (int i = 0; i < n; ++i) {
      uint32_t ux = (uint32_t)std::min(65535.0, std::max(0.0, xy[2 * i] / RH.L * 65536.0));
      uint32_t uy = (uint32_t)std::min(65535.0, std::max(0.0, xy[2 * i + 1] / RH.L * 65536.0));
      hk[i] = bdhost::hilbert_index(ux, uy);
    }
    std::vector<int> by_sp(n);
    std::iota(by_sp.begin(), by_sp.end(), 0);
    std::sort(by_sp.begin(), by_sp.end(), [&](int x, int y) {
      if (sp[x] != sp[y]) return sp[x] < sp[y];
      if (hk[x] != hk[y]) return hk[x] < hk[y];
      return x < y;
    });
    // one segment per species, each a whole number of 512-disk blocks
    int cnt_sp[BD_MAX_SPECIES] = {0, 0, 0, 0}, seg[BD_MAX_SPECIES], seg_begin[BD_MAX_SPECIES + 1];
    for (int i = 0; i < n; ++i) cnt_sp[sp[i]]++;
    seg_begin[0] = slot;
    for (int k = 0; k < BD_MAX_SPECIES; ++k) {
      seg[k] = (int)pad_to(cnt_sp[k], BD_SB);
      seg_begin[k + 1] = seg_begin[k] + seg[k];
    }
    RH.slot_begin = slot;
    RH.slot_end = seg_begin[BD_MAX_SPECIES];
    RH.tile_begin = slot / BD_TJ;
    RH.tile_end = RH.slot_end / BD_TJ;
    slot_ext.resize(RH.slot_end, -1);
    slot_local.resize(RH.slot_end, -1);
    slot_rep.resize(RH.slot_end, -1);
    std::vector<int> local_slot(n);
    {
      int next[BD_MAX_SPECIES];
      for (int k = 0; k < BD_MAX_SPECIES; ++k) next[k] = seg_begin[k];
      for (int k = 0; k < n; ++k) {
        int e = by_sp[k];
        int sl = next[sp[e]]++;
        slot_ext[sl] = RH.ext_base + e;
        slot_local[sl] = e;
        slot_rep[sl] = r;
        local_slot[e] = sl;
      }
    }
    for (int t = RH.tile_begin; t < RH.tile_end; ++t)
    {
      int k = 0;
      while (k + 1 < BD_MAX_SPECIES && t * BD_TJ >= seg_begin[k + 1]) ++k;
      tile_sp.push_back((uint8_t)k);
    }
    slot = RH.slot_end;
    // force i blocks: Hilbert order over the replica's disks
    std::vector<int> by_h(n);
    std::iota(by_h.begin(), by_h.end(), 0);
    std::sort(by_h.begin(), by_h.end(), [&](int x, int y) { return hk[x] != hk[y] ? hk[x] < hk[y] : x < y; });
    const int nib = (int)(pad_to(n, BD_IB) / BD_IB);
    RH.iblock_base = iblock;
    RH.n_iblocks = nib;
    for (int b = 0; b < nib; ++b) {
      double sx = 0, sy = 0;
      int m = 0;
      for (int k = b * BD_IB; k < (b + 1) * BD_IB; ++k) {
        if (k < n) {
          int e = by_h[k];
          iperm.push_back(local_slot[e]);
          sx += xy[2 * e];
          sy += xy[2 * e + 1];
          ++m;
        } else {
          iperm.push_back(-1);
        }
      }
      if (RH.periodic && m) {
        // periodic box: a block may straddle an edge; its origin is the mean
        // of its disks' minimum images about its first disk (the patch
        // centre), which the sweeps re-centre on with minimum images
        const int e0 = by_h[b * BD_IB];
        double mx = 0.0, my = 0.0;
        for (int k = b * BD_IB; k < std::min(n, (b + 1) * BD_IB); ++k) {
          const int e = by_h[k];
          double dx = xy[2 * e] - xy[2 * e0], dy = xy[2 * e + 1] - xy[2 * e0 + 1];
          mx += dx - RH.L * nearbyint(dx / RH.L);
          my += dy - RH.L * nearbyint(dy / RH.L);
        }
        iorg.push_back(make_float2((float)nearbyint(xy[2 * e0] + mx / m), (float)nearbyint(xy[2 * e0 + 1] + my / m)));
      } else {
        iorg.push_back(m ? make_float2((float)nearbyint(sx / m), (float)nearbyint(sy / m)) : make_float2(0.f, 0.f));
      }
    }
    iblock += nib;
    byhr[r].resize(n);
    for (int k = 0; k < n; ++k) byhr[r][k] = local_slot[by_h[k]];
  }
  const int np = slot;
  h->np = np;
  h->np_i = (int)iperm.size();
  h->ext_of_int = slot_ext;
  h->int_of_ext.assign(h->n, -1);
  for (int i = 0; i < np; ++i)
    if (slot_ext[i] >= 0) h->int_of_ext[slot_ext[i]] = i;

  // ---- ghost points (after all disks) and the per-replica triangulations ----
  int ng_total = 0;
  std::vector<std::vector<double>> gxr(R), gyr(R);
  for (int r = 0; r < R; ++r) {
    if (!h->reps[r].periodic) bdhost::make_ghosts(h->reps[r].L, a, gxr[r], gyr[r]);   // a torus needs none
    h->reps[r].ghost_base = np + ng_total;
    h->reps[r].ng = (int)gxr[r].size();
    ng_total += h->reps[r].ng;
  }
  h->ng = ng_total;
  h->host_pos.assign(2 * ((size_t)np + ng_total), 0.0);
  for (int i = 0; i < np; ++i) {
    const int r = slot_rep[i];
    if (r >= 0) {
      int e = slot_local[i];
      h->host_pos[2 * i] = xyr[r][2 * e];
      h->host_pos[2 * i + 1] = xyr[r][2 * e + 1];
    }
  }
  for (int r = 0; r < R; ++r)
    for (int k = 0; k < h->reps[r].ng; ++k) {
      h->host_pos[2 * ((size_t)h->reps[r].ghost_base + k)] = gxr[r][k];
      h->host_pos[2 * ((size_t)h->reps[r].ghost_base + k) + 1] = gyr[r][k];
    }
  std::vector<double> X(np + ng_total), Y(np + ng_total);
  for (int i = 0; i < np + ng_total; ++i) {
    X[i] = h->host_pos[2 * i];
    Y[i] = h->host_pos[2 * i + 1];
  }
  bdpred::Grid grid;
  grid.q = q;
  grid.inv_q = inv_q;
  grid.s = s_shift;
  std::vector<int4> tv_all, tn_all;
  int tri_base = 0;
  for (int r = 0; r < R; ++r) {
    RepHost &RH = h->reps[r];
    std::vector<int> gids(RH.ng);
    for (int k = 0; k < RH.ng; ++k) gids[k] = RH.ghost_base + k;
    std::vector<int> V, N, S;
    if (RH.periodic) {
      if (bdhost::build_torus_delaunay(X.data(), Y.data(), byhr[r], RH.L, grid, V, S, N) != 0) {
        delete h;
        return BD_ERR_TRIANGULATION;
      }
    } else if (bdhost::build_delaunay(X.data(), Y.data(), grid, byhr[r], gids, V, N) != 0) {
      delete h;
      return BD_ERR_TRIANGULATION;
    }
    const int nt_r = (int)(V.size() / 3);
    if (nt_r != (RH.periodic ? 2 * RH.n : 2 * (RH.n + RH.ng) - 6)) {
      delete h;
      return BD_ERR_TRIANGULATION;
    }
    RH.tri_base = tri_base;
    RH.nt = nt_r;
    for (int t = 0; t < nt_r; ++t) {
      int w = 0;
      if (RH.periodic)
        for (int k = 0; k < 3; ++k)
          w |= ((S[6 * t + 2 * k] & 3) << (8 + 4 * k)) | ((S[6 * t + 2 * k + 1] & 3) << (10 + 4 * k));
      tv_all.push_back(make_int4(V[3 * t], V[3 * t + 1], V[3 * t + 2], w));
      auto sh = [&](int o) { return o < 0 ? -1 : o + 3 * tri_base; };
      tn_all.push_back(make_int4(sh(N[3 * t]), sh(N[3 * t + 1]), sh(N[3 * t + 2]), 0));
    }
    tri_base += nt_r;
  }
  const int nt = tri_base;
  h->nt = nt;

  // ---- constants and the replica table ----
  BdConst &c = h->c;
  const bd_params &p0 = specs[0].p;
  c.n = h->n;
  c.np = np;
  c.np_i = h->np_i;
  c.nt = nt;
  c.ntiles = np / BD_TJ;
  c.n_iblocks = iblock;
  c.R = R;
  c.precision = p0.precision;
  c.a = a;
  c.sigma = 2.0 * a;
  c.q = q;
  c.inv_q = inv_q;
  c.qshift = s_shift;
  {
    // fixed-point displacement sums: up to 128 contributions of at most sigma
    // (in grid units below 2^51 * 2 sigma / E) fit in 62 bits with F fraction
    // bits below the grid (F >= 4)
    const double lim = 128.0 * 2.0 * a * inv_q;
    int F = 62 - (int)ceil(log2(std::max(lim, 2.0)));
    F = std::max(4, std::min(F, 40));
    c.disp_scale = ldexp(1.0, s_shift + F);
    c.disp_unscale = ldexp(1.0, -(s_shift + F));
  }
  c.sitem0 = 0;
  {
    // (sigma/q)^2 (1 + 1e-9), rounded up, as a 128-bit integer
    long double sq = (long double)(2.0 * a) * (long double)inv_q;
    long double v = sq * sq * (1.0L + 1e-9L);
    long double two64 = 18446744073709551616.0L;
    unsigned long long hi = (unsigned long long)(v / two64);
    long double rem = v - (long double)hi * two64;
    unsigned long long lo = (unsigned long long)rem;
    if ((long double)lo < rem) ++lo;
    c.sig2q_hi = hi;
    c.sig2q_lo = lo;
  }
  c.max_corr_iters = p0.max_corr_iters;
  c.overlap_verlet = p0.overlap_mode == BD_OVERLAP_VERLET ? 1 : 0;
  {
    const char *tl = getenv("BD_TRI_LISTS");
    c.tri_lists = tl ? std::min(2, std::max(0, atoi(tl))) : 0;
    const char *tf = getenv("BD_TRI_FUSE");
    c.tri_fuse = tf ? (atoi(tf) != 0 ? 1 : 0) : 1;
  }
  {
    // the lists hold every pair within r_cut + skin of the build positions, so
    // every pair closer than sigma while no disk has moved (r_cut + skin - sigma)/2
    double reach = 1e300;
    for (const Spec &sp : specs) reach = std::min(reach, 0.5 * (sp.p.r_cut + sp.p.skin - 2.0 * sp.p.a));
    c.vl_reach2 = c.overlap_verlet ? reach * reach * (1.0 - 1e-9) : 0.0;
  }
  c.max_flip_rounds = p0.max_flip_rounds;
  c.force_variant = 1;
  h->h_rep.resize(R);
  int cell_base = 0;
  for (int r = 0; r < R; ++r) {
    const RepHost &RH = h->reps[r];
    const bd_params &p = RH.p;
    BdRep &B = h->h_rep[r];
    memset(&B, 0, sizeof(B));
    B.L = RH.L;
    B.wall_lo = RH.wall_lo;
    B.wall_hi = RH.wall_hi;
    B.periodic = RH.periodic ? 1 : 0;
    B.Lf = (float)RH.L;
    B.hLf = RH.periodic ? 0.5f * (float)RH.L : std::numeric_limits<float>::infinity();
    B.invLf = RH.periodic ? (float)(1.0 / RH.L) : 0.f;
    B.LQ = (long long)nearbyint(RH.L * inv_q);
    if (RH.periodic) c.any_periodic = 1;
    B.dt = p.dt;
    B.amp = p.literal_noise ? sqrt(p.D * p.dt) : sqrt(2.0 * p.D * p.dt);
    B.amp_r = sqrt(2.0 * p.Dr * p.dt);
    B.v0 = p.v0;
    B.eps = p.eps;
    B.kappa = p.kappa;
    B.r_cut = p.r_cut;
    B.skin = p.skin;
    B.rl2 = (p.r_cut + p.skin) * (p.r_cut + p.skin);
    rep_set_alpha(B, p.alpha, p.n_species);
    B.seed = p.seed;
    B.replica = (unsigned)p.replica;
    B.law = p.law;
    B.slot_begin = RH.slot_begin;
    B.slot_end = RH.slot_end;
    B.n = RH.n;
    B.nchunk = 1;
    if (p.law == BD_LAW_SHORT) {
      B.ncell = std::max(1, std::min(1 << 14, (int)floor(RH.L / (p.r_cut + p.skin))));
      // periodic cells wrap around: at least three per side keep the 3 x 3
      // neighbourhoods free of repeated cells (validate() checks L)
      B.cell_size = RH.L / B.ncell;
      B.cell_base = cell_base;
      cell_base += B.ncell * B.ncell;
      c.any_short = 1;
    }
    if (p.law == BD_LAW_LONG) c.any_long = 1;
    c.n_species = std::max(c.n_species, p.n_species);
  }
  c.ncell_total = cell_base;
  h->step = p0.step0;
  h->graph_off = getenv("BD_NO_GRAPH") != nullptr;

  // ---- device buffers ----
  BdDev &d = h->d;
  cudaError_t e = cudaSuccess;
  const size_t nv = (size_t)np + ng_total;
#define BD_TRY(x)                          \
  do {                                     \
    e = (x);                               \
    if (e != cudaSuccess) goto cuda_error; \
  } while (0)
  {
    BD_TRY(dalloc(h, &d.pos, nv));
    BD_TRY(dalloc(h, &d.prev, nv));
    BD_TRY(dalloc(h, &d.pos0, nv));
    BD_TRY(dalloc(h, &d.work, (size_t)np));
    BD_TRY(dalloc(h, &d.theta, (size_t)np));
    BD_TRY(dalloc(h, &d.theta0, (size_t)np));
    BD_TRY(dalloc(h, &d.species, (size_t)np));
    BD_TRY(dalloc(h, &d.ext_id, (size_t)np));
    BD_TRY(dalloc(h, &d.rep_of, (size_t)np));
    BD_TRY(dalloc(h, &d.ext_glob, (size_t)np));
    BD_TRY(dalloc(h, &d.xfer_xy, (size_t)std::max(1, h->n)));
    BD_TRY(dalloc(h, &d.xfer_th, (size_t)std::max(1, h->n)));
    BD_TRY(dalloc(h, &d.xfer_sp, (size_t)std::max(1, h->n)));
    BD_TRY(dalloc(h, &d.moved, nv));
    BD_TRY(dalloc(h, &d.dmove, (size_t)np));
    // per-replica counters only for batches: a single system's are the
    // call's own counters, and its kernels then skip the per-replica atomics
    d.rep_stats = nullptr;
    d.rep_mark = nullptr;
    if (R > 1) {
      BD_TRY(dalloc(h, &d.rep_stats, 3 * (size_t)R));
      BD_TRY(dalloc(h, &d.rep_mark, (size_t)R));
      BD_TRY(cudaMemsetAsync(d.rep_stats, 0, 3 * (size_t)R * sizeof(long long), h->stream));
      BD_TRY(cudaMemsetAsync(d.rep_mark, 0, (size_t)R * sizeof(unsigned long long), h->stream));
    }
    if (c.any_periodic) {
      BD_TRY(dalloc(h, &d.wrap, (size_t)np));
      BD_TRY(cudaMemsetAsync(d.wrap, 0, (size_t)np, h->stream));
    }
    BD_TRY(dalloc(h, &d.disp, (size_t)np));
    d.rad = nullptr;
    d.radf = nullptr;
    d.wall = nullptr;
    if (specs[0].rad) {
      // polydisperse disks (one replica): radius and grid walls per slot
      const RepHost &RH = h->reps[0];
      const double *rad = specs[0].rad;
      std::vector<double> rs((size_t)np, a);
      std::vector<double2> ws((size_t)np, make_double2(RH.wall_lo, RH.wall_hi));
      for (int sl = 0; sl < np; ++sl) {
        if (slot_rep[sl] < 0) continue;
        const double ri = rad[slot_local[sl]];
        rs[sl] = ri;
        if (!RH.periodic) ws[sl] = make_double2(ceil(ri * inv_q) * q, floor((RH.L - ri) * inv_q) * q);
      }
      std::vector<float2> rf((size_t)np);
      for (int sl = 0; sl < np; ++sl) {
        const float hi = (float)rs[sl];
        rf[sl] = make_float2(hi, (float)(rs[sl] - (double)hi));
      }
      BD_TRY(dalloc(h, &d.rad, (size_t)np));
      BD_TRY(dalloc(h, &d.radf, (size_t)np));
      BD_TRY(dalloc(h, &d.wall, (size_t)np));
      BD_TRY(cudaMemcpy(d.radf, rf.data(), rf.size() * sizeof(float2), cudaMemcpyHostToDevice));
      BD_TRY(cudaMemcpy(d.rad, rs.data(), rs.size() * sizeof(double), cudaMemcpyHostToDevice));
      BD_TRY(cudaMemcpy(d.wall, ws.data(), ws.size() * sizeof(double2), cudaMemcpyHostToDevice));
    }
    {
      BdRep *rp = nullptr;
      BD_TRY(dalloc(h, &rp, (size_t)R));
      d.rep = rp;
    }
    BD_TRY(dalloc(h, &d.tv, (size_t)nt));
    BD_TRY(dalloc(h, &d.tn, (size_t)nt));
    BD_TRY(dalloc(h, &d.jtv, (size_t)nt));
    BD_TRY(dalloc(h, &d.jtn, (size_t)nt));
    BD_TRY(dalloc(h, &d.jmark, (size_t)nt));
    BD_TRY(cudaMemsetAsync(d.jmark, 0, (size_t)nt * sizeof(unsigned), h->stream));
    BD_TRY(dalloc(h, &d.claim, 2 * (size_t)nt));
    BD_TRY(dalloc(h, &d.tinv, (size_t)nt));
    BD_TRY(dalloc(h, &d.clist, 3 * (size_t)nt));
    BD_TRY(dalloc(h, &d.clmark, (size_t)nt));
    BD_TRY(cudaMemsetAsync(d.clmark, 0, (size_t)nt * sizeof(unsigned), h->stream));
    BD_TRY(cudaMemsetAsync(d.tinv, 0, (size_t)nt, h->stream));
    BD_TRY(dalloc(h, &d.vt, nv));
    BD_TRY(dalloc(h, &d.act, 3 * (size_t)nt));
    BD_TRY(dalloc(h, &d.act_mark, 3 * (size_t)nt));
    BD_TRY(cudaMemsetAsync(d.act_mark, 0, 3 * (size_t)nt * sizeof(unsigned), h->stream));
    BD_TRY(dalloc(h, &d.iperm, (size_t)std::max(1, h->np_i)));
    BD_TRY(dalloc(h, &d.iorigin, (size_t)std::max(1, iblock)));
    BD_TRY(dalloc(h, &d.tile_species, std::max<size_t>(1, tile_sp.size())));
    BD_TRY(dalloc(h, &d.ctl, 1));
    BD_TRY(dalloc(h, &h->d_fsum, (size_t)np));
    BD_TRY(cudaMallocHost((void **)&h->h_ctl, sizeof(BdCtl)));
    // partial-force slots: enough for the finest chunking tried (at most 64).
    // The FP64 sweep (one disk per thread) cuts j ranges finer than tiles:
    // into enough chunks for about four blocks per SM
    {
      int slots = 1, sms = 148, dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      const int f64_want = (4 * sms + (np + 127) / 128 - 1) / std::max(1, (np + 127) / 128);
      h->fpart_cap.assign(R, 1);
      for (int r = 0; r < R; ++r) {
        const int nt_r = h->reps[r].tile_end - h->reps[r].tile_begin;
        const int want = c.precision == 1 ? std::max(nt_r, f64_want) : nt_r;
        const int cap = h->reps[r].p.law == BD_LAW_LONG ? std::min(64, std::max(1, want)) : 1;
        h->fpart_cap[r] = cap;
        slots = std::max(slots, cap);
      }
      h->fpart_slots = slots;
      BD_TRY(dalloc(h, &d.fpart, (size_t)slots * np));
    }
    if (c.any_short) {
      const size_t nc2 = (size_t)std::max(1, c.ncell_total);
      BD_TRY(dalloc(h, &d.vl_idx, (size_t)BD_VL_MAX * np));
      BD_TRY(dalloc(h, &d.vl_cnt, (size_t)np));
      BD_TRY(dalloc(h, &d.vl_ref, (size_t)np));
      BD_TRY(dalloc(h, &d.cell_count, nc2));
      BD_TRY(dalloc(h, &d.cell_start, nc2));
      BD_TRY(dalloc(h, &d.cell_cursor, nc2));
      BD_TRY(dalloc(h, &d.cell_idx, (size_t)np));
      BD_TRY(dalloc(h, &d.cell_of, (size_t)np));
      BD_TRY(dalloc(h, &d.scan_sums, (nc2 + 511) / 512 + 1));
    }
    if (c.overlap_verlet) {
      BD_TRY(dalloc(h, &d.vc_hit, (size_t)np));
      BD_TRY(cudaMemsetAsync(d.vc_hit, 0, (size_t)np, h->stream));
    }
    h->max_halvings = specs[0].p.max_dt_halvings;
    if (h->max_halvings > 0) {
      // the state at the start of a step that is being redone in pieces
      BD_TRY(dalloc(h, &h->hs_pos, (size_t)np));
      BD_TRY(dalloc(h, &h->hs_work, (size_t)np));
      BD_TRY(dalloc(h, &h->hs_theta, (size_t)np));
      BD_TRY(dalloc(h, &h->hs_tv, (size_t)nt));
      BD_TRY(dalloc(h, &h->hs_tn, (size_t)nt));
      BD_TRY(dalloc(h, &h->hs_vt, nv));
    }

    cudaStream_t st = h->stream;
    std::vector<float> th_i(np, 0.f);
    std::vector<uint8_t> sp_i(np, 255);
    for (int i = 0; i < np; ++i) {
      const int r = slot_rep[i];
      if (r >= 0) {
        th_i[i] = thr[r][slot_local[i]];
        sp_i[i] = spr[r][slot_local[i]];
      }
    }
    {
      // symmetric-sweep blocks: (replica, species) and an integer origin
      const int nb = np / BD_SB;
      std::vector<int2> sb(std::max(1, nb), make_int2(0, 0));
      std::vector<float2> so(std::max(1, nb), make_float2(0.f, 0.f));
      for (int P = 0; P < nb; ++P) {
        double sx = 0.0, sy = 0.0;
        int m = 0;
        for (int i = P * BD_SB; i < (P + 1) * BD_SB; ++i) {
          if (slot_rep[i] < 0) continue;
          if (m == 0) sb[P] = make_int2(slot_rep[i], sp_i[i]);
          sx += h->host_pos[2 * (size_t)i];
          sy += h->host_pos[2 * (size_t)i + 1];
          ++m;
        }
        if (m && h->reps[sb[P].x].periodic) {
          // periodic box: the mean of the block's minimum images about its
          // first disk (the symmetric sweep re-centres on it with minimum images)
          const double L = h->reps[sb[P].x].L;
          double x0 = 0.0, y0 = 0.0, mx = 0.0, my = 0.0;
          bool have = false;
          for (int i = P * BD_SB; i < (P + 1) * BD_SB; ++i) {
            if (slot_rep[i] < 0) continue;
            const double x = h->host_pos[2 * (size_t)i], y = h->host_pos[2 * (size_t)i + 1];
            if (!have) {
              x0 = x;
              y0 = y;
              have = true;
            }
            mx += (x - x0) - L * nearbyint((x - x0) / L);
            my += (y - y0) - L * nearbyint((y - y0) / L);
          }
          so[P] = make_float2((float)nearbyint(x0 + mx / m), (float)nearbyint(y0 + my / m));
        } else if (m) {
          so[P] = make_float2((float)nearbyint(sx / m), (float)nearbyint(sy / m));
        }
      }
      BD_TRY(dalloc(h, &d.sblock, sb.size()));
      BD_TRY(dalloc(h, &d.sorigin, so.size()));
      BD_TRY(cudaMemcpy(d.sblock, sb.data(), sb.size() * sizeof(int2), cudaMemcpyHostToDevice));
      BD_TRY(cudaMemcpy(d.sorigin, so.data(), so.size() * sizeof(float2), cudaMemcpyHostToDevice));
    }
    BD_TRY(cudaMemcpyAsync(d.pos, h->host_pos.data(), nv * sizeof(double2), cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.prev, d.pos, nv * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.pos0, d.pos, nv * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.theta, th_i.data(), np * sizeof(float), cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.theta0, d.theta, np * sizeof(float), cudaMemcpyDeviceToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.species, sp_i.data(), np, cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.ext_id, slot_local.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.rep_of, slot_rep.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.ext_glob, h->ext_of_int.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemsetAsync(d.moved, 0, nv, st));
    BD_TRY(cudaMemsetAsync(d.disp, 0, np * sizeof(double2), st));
    BD_TRY(cudaMemcpyAsync(d.tv, tv_all.data(), nt * sizeof(int4), cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.tn, tn_all.data(), nt * sizeof(int4), cudaMemcpyHostToDevice, st));
    {
      // one corner per vertex (the star walks of the triangulation kernel start there)
      std::vector<int> vt(nv, -1);
      for (int t = 0; t < nt; ++t) {
        vt[tv_all[t].x] = 3 * t;
        vt[tv_all[t].y] = 3 * t + 1;
        vt[tv_all[t].z] = 3 * t + 2;
      }
      BD_TRY(cudaMemcpy(d.vt, vt.data(), nv * sizeof(int), cudaMemcpyHostToDevice));
    }
    BD_TRY(cudaMemsetAsync(d.claim, 0, 2 * nt * sizeof(unsigned long long), st));
    if (!iperm.empty())
      BD_TRY(cudaMemcpyAsync(d.iperm, iperm.data(), iperm.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    if (!iorg.empty())
      BD_TRY(cudaMemcpyAsync(d.iorigin, iorg.data(), iorg.size() * sizeof(float2), cudaMemcpyHostToDevice, st));
    if (!tile_sp.empty())
      BD_TRY(cudaMemcpyAsync(d.tile_species, tile_sp.data(), tile_sp.size(), cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemsetAsync(d.fpart, 0, (size_t)h->fpart_slots * np * sizeof(double2), st));
    BD_TRY(cudaMemsetAsync(d.ctl, 0, sizeof(BdCtl), st));
    {
      const long long s0 = h->step;
      BD_TRY(cudaMemcpyAsync(&d.ctl->step_dev, &s0, sizeof(s0), cudaMemcpyHostToDevice, st));
      BD_TRY(cudaStreamSynchronize(st));
    }
    if (c.any_short) {
      // reference positions far away: the first force evaluation builds the lists
      std::vector<double2> far(np, make_double2(1e30, 1e30));
      BD_TRY(cudaMemcpyAsync(d.vl_ref, far.data(), np * sizeof(double2), cudaMemcpyHostToDevice, st));
      BD_TRY(cudaMemsetAsync(d.vl_cnt, 0, np * sizeof(int), st));
      BD_TRY(cudaStreamSynchronize(st));
    }
    BD_TRY(cudaStreamSynchronize(st));
    // force work items: the FP64 sweep fills whole waves; the FP32 sweep is
    // chosen by timing (or fixed by BD_FORCE_VARIANT / BD_FORCE_TILES)
    {
      BD_TRY(bd_launch_work_copy(d, c, st));
      BD_TRY(cudaStreamSynchronize(st));
      const char *fv = getenv("BD_FORCE_VARIANT"), *ft = getenv("BD_FORCE_TILES");
      long long nmax = 0;
      for (const RepHost &RH : h->reps)
        if (RH.p.law == BD_LAW_LONG) nmax = std::max<long long>(nmax, RH.n);
      if (c.precision == 1 || !c.any_long) {
        BD_TRY(use_variant(h, c.precision == 1 ? 1 : c.force_variant, R == 1 ? single_system_tiles(h) : 16));
      } else if (fv) {
        int v = std::min(3, std::max(0, atoi(fv)));
        if (c.any_periodic && v == 1) v = 0;   // the packed one-sided sweep has no periodic form
        const int t = ft && atoi(ft) > 0 ? atoi(ft) : (v >= 2 ? 8 : (R == 1 ? single_system_tiles(h) : 16));
        BD_TRY(use_variant(h, v, t));
      } else if (nmax * nmax > 180000000000LL) {
        // a launch takes more than ~50 ms: no timing at init
        BD_TRY(use_variant(h, 2, 16));
      } else {
        BD_TRY(autotune(h));
      }
    }
    if (bd_dt_grid_for(std::max(nt, np), &h->dt_grid, &h->dt_block) != 0 ||
        (c.overlap_verlet && bd_vcorr_grid_for(np, &h->vc_grid, &h->vc_block) != 0)) {
      bd_free(h);
      return BD_ERR_CUDA;
    }
  }
#undef BD_TRY
  *out = h;
  return BD_OK;
cuda_error:
  bd_free(h);
  return cuda_fail(e);
}

}  // namespace

namespace bdcapi {

int read_ctl(bd_handle *h) {
  cudaError_t e = cudaMemcpyAsync(h->h_ctl, h->d.ctl, sizeof(BdCtl), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  return BD_OK;
}

cudaError_t reset_stats(bd_handle *h) {
  // zero everything after the barrier words, the status and the epoch
  char *base = (char *)h->d.ctl;
  size_t off = offsetof(BdCtl, cnt);
  cudaError_t e = cudaMemsetAsync(base + off, 0, offsetof(BdCtl, log_npass) - off, h->stream);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(&h->d.ctl->status, 0, sizeof(int), h->stream);
}

void add_stage_times(bd_handle *h) {
  for (int k = 0; k < 5; ++k) {
    h->stage_ns[k] += (double)h->h_ctl->st_stage_ns[k];
    h->stage_cnt[k] += h->h_ctl->st_stage_cnt[k];
  }
}

int finish_status(bd_handle *h, int status) {
  // clear the sticky status so the handle keeps working from the last good
  // state; after a timed-out barrier the kernel left without undoing its
  // step: undo it (step-start copies, undo journal), and reset the barrier words
  cudaStream_t st = h->stream;
  if (status == BD_ERR_DEVICE_TIMEOUT) {
    bd_launch_restore_step(h->d, h->c, st);
    cudaMemsetAsync(h->d.ctl, 0, offsetof(BdCtl, epoch), st);
  }
  cudaMemsetAsync(&h->d.ctl->cnt[0][0], 0, sizeof(h->d.ctl->cnt), st);
  cudaMemsetAsync(&h->d.ctl->status, 0, sizeof(int), st);
  cudaStreamSynchronize(st);
  return status;
}

// the counters of the call whose control block read_ctl fetched last, as
// bd_step reports them (h->last_stats, returned by bd_last_stats)
void fill_stats(bd_handle *h, int status, int64_t halvings) {
  const BdCtl &k = *h->h_ctl;
  bd_step_stats &o = h->last_stats;
  memset(&o, 0, sizeof(o));
  o.steps_done = k.st_steps;
  o.corr_iters = k.st_corr_iters;
  o.overlap_pairs = k.st_overlap_pairs;
  o.flip_rounds = k.st_flip_rounds;
  o.flips = k.st_flips;
  o.repair_flips = k.st_repair_flips;
  o.inverted = k.st_inverted;
  o.max_corr_iters = k.st_max_corr_iters;
  o.verlet_rebuilds = (int32_t)k.st_verlet_rebuilds;
  o.fail_phase = status ? k.st_fail_phase : 0;
  o.fail_item = k.st_fail_item;
  o.fail_count = k.st_fail_count;
  o.barriers = k.st_barriers;
  o.rejected = status != 0;
  o.substeps = k.st_substeps;
  o.tri_visits = k.st_tri_visits;
  o.exact_tests = k.st_exact;
  o.halvings = halvings;
  double mo;
  unsigned long long bits = k.st_max_overlap_bits;
  memcpy(&mo, &bits, sizeof(mo));
  o.max_overlap = mo;
}

}  // namespace bdcapi

namespace {

// copy the disks' positions / directions / species (internal order)
int fetch_disks(bd_handle *h, std::vector<double2> *pos, std::vector<float> *th,
                std::vector<uint8_t> *sp) {
  cudaStream_t st = h->stream;
  const int np = h->np;
  cudaError_t e = cudaSuccess;
  if (pos) {
    pos->resize(np);
    e = cudaMemcpyAsync(pos->data(), h->d.pos, np * sizeof(double2), cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess && th) {
    th->resize(np);
    e = cudaMemcpyAsync(th->data(), h->d.theta, np * sizeof(float), cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess && sp) {
    sp->resize(np);
    e = cudaMemcpyAsync(sp->data(), h->d.species, np, cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? BD_OK : cuda_fail(e);
}

// the per-step correction stage: triangulation maintenance + Algorithm 2 over
// its edges, or Algorithm 2 over the Verlet lists
cudaError_t launch_correction(bd_handle *h, cudaStream_t s) {
  if (h->c.overlap_verlet) return bd_launch_overlap_verlet(h->d, h->c, s, h->vc_grid, h->vc_block);
  return bd_launch_dt(h->d, h->c, 0, s, h->dt_grid, h->dt_block);
}

// Capture one step (force, integration, triangulation) as a graph on the
// handle's private stream.  The integration reads the step index from the
// device counter, so every replay is the next step.
cudaError_t capture_step_graph(bd_handle *h) {
  cudaError_t e = cudaSuccess;
  if (!h->cap_stream) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k)
    if (!h->graph_ev[k]) e = cudaEventCreate(&h->graph_ev[k]);
  if (e != cudaSuccess) return e;
  if (h->step_graph) {
    cudaGraphExecDestroy(h->step_graph);
    h->step_graph = nullptr;
  }
  cudaStream_t cs = h->cap_stream;
  const bool tm = h->timing && h->c.any_long;
  int launches = 0;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t el = cudaSuccess;
  if (h->c.any_long) {
    if (tm) el = cudaEventRecordWithFlags(h->graph_ev[0], cs, cudaEventRecordExternal);
    if (el == cudaSuccess) el = bd_launch_force_long(h->d, h->c, cs);
    if (el == cudaSuccess && tm) el = cudaEventRecordWithFlags(h->graph_ev[1], cs, cudaEventRecordExternal);
    launches += h->c.precision == 0 ? bd_force_launches(h->c.force_variant) : 1;
  }
  if (el == cudaSuccess && h->c.any_short) {
    el = bd_launch_force_short(h->d, h->c, cs);
    launches += bd_short_launches();
  }
  if (el == cudaSuccess) el = bd_launch_integrate(h->d, h->c, -1, -1, cs);
  if (el == cudaSuccess) el = launch_correction(h, cs);
  launches += 2;
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(cs, &g);
  if (el != cudaSuccess || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();   // clear a launch error of the failed capture
    return el != cudaSuccess ? el : e;
  }
  e = cudaGraphInstantiate(&h->step_graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->step_graph = nullptr;
    cudaGetLastError();
    return e;
  }
  h->graph_d = h->d;
  h->graph_c = h->c;
  h->graph_timed = tm;
  h->graph_launches = launches;
  return cudaSuccess;
}

// the captured graph is usable for the current tables and timing mode
bool step_graph_ready(bd_handle *h) {
  if (h->graph_off) return false;
  const bool tm = h->timing && h->c.any_long;
  if (h->step_graph && tm == h->graph_timed && memcmp(&h->graph_d, &h->d, sizeof(BdDev)) == 0 &&
      memcmp(&h->graph_c, &h->c, sizeof(BdConst)) == 0)
    return true;
  if (capture_step_graph(h) != cudaSuccess) {
    h->graph_off = true;   // fall back to plain launches from now on
    return false;
  }
  return true;
}

// Queue nsteps whole steps (one graph replay each, or plain launches when
// every force launch is timed), wait for them, read the control block and fold
// the force timings in.  A failed step makes the later ones no-ops.
int queue_steps(bd_handle *h, int32_t nsteps, int64_t *launches_out) {
  cudaStream_t st = h->stream;
  cudaError_t e = cudaSuccess;
  int64_t launches = 0;
  int timed = 0;
  const bool long_range = h->c.any_long;
  if (h->timing && long_range) {
    while ((int)h->ev_pool.size() < 2 * nsteps) {
      cudaEvent_t ev;
      if (cudaEventCreate(&ev) != cudaSuccess) return BD_ERR_CUDA;
      h->ev_pool.push_back(ev);
    }
  }
  // one graph replay per step, unless timing wants a launch per step in a
  // multi-step call (the graph holds one pair of timing events)
  const bool use_graph = nsteps > 0 && !(h->timing && long_range && nsteps > 1) && step_graph_ready(h);
  if (use_graph) {
    for (int s = 0; s < nsteps; ++s) {
      e = cudaGraphLaunch(h->step_graph, st);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    launches = (int64_t)nsteps * h->graph_launches;
  }
  for (int s = 0; s < (use_graph ? 0 : nsteps); ++s) {
    if (long_range) {
      bool tm = h->timing;
      if (tm) cudaEventRecord(h->ev_pool[2 * s], st);
      e = bd_launch_force_long(h->d, h->c, st);
      if (e != cudaSuccess) return cuda_fail(e);
      if (tm) {
        cudaEventRecord(h->ev_pool[2 * s + 1], st);
        ++timed;
      }
      launches += h->c.precision == 0 ? bd_force_launches(h->c.force_variant) : 1;
    }
    if (h->c.any_short) {
      e = bd_launch_force_short(h->d, h->c, st);
      if (e != cudaSuccess) return cuda_fail(e);
      launches += bd_short_launches();
    }
    e = bd_launch_integrate(h->d, h->c, h->step + s, -1, st);
    if (e != cudaSuccess) return cuda_fail(e);
    e = launch_correction(h, st);
    if (e != cudaSuccess) return cuda_fail(e);
    launches += 2;
  }
  *launches_out += launches;
  int rc = read_ctl(h);
  if (rc) return rc;
  if (use_graph && h->graph_timed) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->graph_ev[0], h->graph_ev[1]) == cudaSuccess) {
      h->force_ms += ms;
      h->force_launches += 1;
    }
  }
  for (int s = 0; s < timed; ++s) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_pool[2 * s], h->ev_pool[2 * s + 1]) == cudaSuccess) {
      h->force_ms += ms;
      h->force_launches += 1;
    }
  }
  return BD_OK;
}

// ---- Sec. 4.3: a rejected move is repeated with a lower dt ----

// copy the step-start state to (save) or from (restore) the halving snapshot
cudaError_t halving_snapshot(bd_handle *h, bool save) {
  cudaStream_t st = h->stream;
  const size_t np = (size_t)h->np, nt = (size_t)h->nt;
  const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
  cudaError_t e = cudaMemcpyAsync(save ? h->hs_pos : h->d.pos, save ? h->d.pos : h->hs_pos,
                                  np * sizeof(double2), k, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(save ? h->hs_work : h->d.work, save ? h->d.work : h->hs_work, np * sizeof(float4), k, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(save ? h->hs_theta : h->d.theta, save ? h->d.theta : h->hs_theta, np * sizeof(float), k,
                        st);
  if (e == cudaSuccess && !h->c.overlap_verlet) {
    e = cudaMemcpyAsync(save ? h->hs_tv : h->d.tv, save ? h->d.tv : h->hs_tv, nt * sizeof(int4), k, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(save ? h->hs_tn : h->d.tn, save ? h->d.tn : h->hs_tn, nt * sizeof(int4), k, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(save ? h->hs_vt : h->d.vt, save ? h->d.vt : h->hs_vt,
                          ((size_t)h->np + h->ng) * sizeof(int), k, st);
  }
  if (e == cudaSuccess && !save) {
    e = cudaMemcpyAsync(h->d.prev, h->d.pos, np * sizeof(double2), k, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d.moved, 0, np, st);
  }
  return e;
}

// one piece of the step h->step with plain launches: forces at the piece's
// start, the move of length dt / 2^depth(node), the correction stage (which
// undoes the piece itself when it fails)
cudaError_t launch_piece(bd_handle *h, int node, int64_t *launches) {
  cudaStream_t st = h->stream;
  cudaError_t e = cudaSuccess;
  if (h->c.any_long) {
    e = bd_launch_force_long(h->d, h->c, st);
    *launches += h->c.precision == 0 ? bd_force_launches(h->c.force_variant) : 1;
  }
  if (e == cudaSuccess && h->c.any_short) {
    e = bd_launch_force_short(h->d, h->c, st);
    *launches += bd_short_launches();
  }
  if (e == cudaSuccess) e = bd_launch_integrate(h->d, h->c, h->step, -1, st, node);
  if (e == cudaSuccess)
    e = h->c.overlap_verlet ? bd_launch_overlap_verlet(h->d, h->c, st, h->vc_grid, h->vc_block, 0)
                            : bd_launch_dt(h->d, h->c, 2, st, h->dt_grid, h->dt_block);
  *launches += 2;
  return e;
}

// a rejection that a shorter move can avoid: a pair passed through each
// other, an inverted triangle without repair, or a disk beyond its list's reach
bool halvable(const BdCtl &k) {
  return k.status == BD_ERR_STEP_REJECTED &&
         (k.st_fail_phase == 1 || k.st_fail_phase == 2 || k.st_fail_phase == 3 || k.st_fail_phase == 6);
}

// piece `node` was rejected and undone: run its two halves in order, halving
// again a half that is rejected, down to depth max_halvings.  Returns BD_OK
// or the status of the piece that could not be completed (undone by its
// kernel; the caller restores the step's start).
int run_halves(bd_handle *h, int node, int depth, int64_t *launches, int64_t *halvings) {
  *halvings += 1;
  for (int child = 2 * node; child <= 2 * node + 1; ++child) {
    cudaError_t e = launch_piece(h, child, launches);
    if (e != cudaSuccess) return cuda_fail(e);
    int rc = read_ctl(h);
    if (rc) return rc;
    const int status = h->h_ctl->status;
    if (status == BD_OK) continue;
    const bool again = halvable(*h->h_ctl) && depth + 1 < h->max_halvings;
    finish_status(h, status);
    if (!again) return status;
    rc = run_halves(h, child, depth + 1, launches, halvings);
    if (rc) return rc;
  }
  return BD_OK;
}

}  // namespace

extern "C" {

const char *bd_strerror(int code) {
  switch (code) {
    case BD_OK: return "ok";
    case BD_ERR_ARG: return "invalid argument";
    case BD_ERR_CUDA: return "CUDA runtime error";
    case BD_ERR_INIT_OVERLAP: return "initial disks overlap or lie outside [a, L-a]";
    case BD_ERR_STEP_REJECTED: return "step rejected (pair reversal or unrepairable inverted triangle); step undone";
    case BD_ERR_OVERLAP_NOT_CONVERGED: return "overlap correction did not converge; step undone";
    case BD_ERR_FLIP_NOT_CONVERGED: return "edge flips did not converge; step undone";
    case BD_ERR_DEVICE_TIMEOUT: return "a bounded device-side wait timed out";
    case BD_ERR_NOMEM: return "out of memory";
    case BD_ERR_TRIANGULATION: return "initial triangulation failed";
    case BD_ERR_UNSUPPORTED: return "unsupported parameter combination";
    default: return "unknown status";
  }
}

int bd_struct_sizes(int32_t *params_bytes, int32_t *stats_bytes) {
  if (params_bytes) *params_bytes = (int32_t)sizeof(bd_params);
  if (stats_bytes) *stats_bytes = (int32_t)sizeof(bd_step_stats);
  return BD_OK;
}

int bd_default_params(bd_params *p) {
  if (!p) return BD_ERR_ARG;
  memset(p, 0, sizeof(*p));
  p->n_species = 1;
  p->a = 1.0;
  p->area_fraction = 0.3;
  p->law = BD_LAW_NONE;
  p->precision = 0;
  p->eps = 1.0;
  p->kappa = 1.0;
  p->r_cut = 5.0;
  p->skin = 0.6;
  p->D = 1.0;
  p->dt = 1e-4;
  p->max_corr_iters = 1000;
  p->max_flip_rounds = 4096;
  return BD_OK;
}

void bd_free(bd_handle *h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  else cudaDeviceSynchronize();
  bdcapi::rollout_release(h);
  if (h->step_graph) cudaGraphExecDestroy(h->step_graph);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  for (int k = 0; k < 2; ++k)
    if (h->graph_ev[k]) cudaEventDestroy(h->graph_ev[k]);
  for (void *p : h->dev_allocs) cudaFree(p);
  if (h->h_ctl) cudaFreeHost(h->h_ctl);
  for (cudaEvent_t ev : h->ev_pool) cudaEventDestroy(ev);
  delete h;
}

int bd_init(const bd_params *p, const double *xy, const uint8_t *species, const float *theta,
            void *stream, bd_handle **out) {
  if (!out || !p) return BD_ERR_ARG;
  std::vector<Spec> specs(1);
  specs[0] = {*p, xy, species, theta};
  return build_handle(specs, stream, out);
}

int bd_init_radii(const bd_params *p, const double *xy, const uint8_t *species, const float *theta,
                  const double *radii, void *stream, bd_handle **out) {
  if (!out || !p || !xy || !radii) return BD_ERR_ARG;
  std::vector<Spec> specs(1);
  specs[0] = {*p, xy, species, theta, radii};
  return build_handle(specs, stream, out);
}

int bd_batch_init(int32_t R, const bd_params *p, const double *xy, const uint8_t *species,
                  const float *theta, void *stream, bd_handle **out) {
  if (!out || !p || R < 1) return BD_ERR_ARG;
  std::vector<Spec> specs(R);
  size_t off = 0;
  for (int r = 0; r < R; ++r) {
    specs[r] = {p[r], xy ? xy + 2 * off : nullptr, species ? species + off : nullptr,
                theta ? theta + off : nullptr};
    off += (size_t)std::max(0, p[r].n);
  }
  return build_handle(specs, stream, out);
}

int bd_step(bd_handle *h, int32_t nsteps, bd_step_stats *stats) {
  if (!h || nsteps < 0) return BD_ERR_ARG;
  if (h->shard_world > 1) return BD_ERR_UNSUPPORTED;   // a force shard steps by bd_step_begin / bd_step_end
  if (stats) memset(stats, 0, sizeof(*stats));
  cudaError_t e = reset_stats(h);
  if (e != cudaSuccess) return cuda_fail(e);
  const int64_t step_base = h->step;
  int64_t launches = 0, halvings = 0;
  int status = BD_OK;
  int32_t todo = nsteps;
  for (;;) {
    int rc = queue_steps(h, todo, &launches);
    if (rc) return rc;
    const BdCtl &k = *h->h_ctl;
    h->step = step_base + k.st_steps;
    if (k.status == BD_OK) break;
    if (!(h->max_halvings > 0 && halvable(k))) {
      status = k.status;
      break;
    }
    // Sec. 4.3: the rejected step was undone by its kernel; keep its start and
    // repeat it as two halves (each halved again when rejected)
    const int64_t done = k.st_steps;
    finish_status(h, BD_ERR_STEP_REJECTED);
    e = halving_snapshot(h, true);
    if (e != cudaSuccess) return cuda_fail(e);
    rc = run_halves(h, 1, 0, &launches, &halvings);
    if (rc == BD_ERR_CUDA || rc == BD_ERR_NOMEM) return rc;
    if (rc != BD_OK) {
      e = halving_snapshot(h, false);
      if (e != cudaSuccess) return cuda_fail(e);
      status = rc;
      rc = read_ctl(h);
      if (rc) return rc;
      break;
    }
    e = bd_launch_advance_step(h->d, h->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    todo = nsteps - (int32_t)(done + 1);
  }
  h->last_launches = launches;
  const BdCtl &k = *h->h_ctl;
  add_stage_times(h);
  h->step = step_base + k.st_steps;
  if (k.status) status = k.status;
  fill_stats(h, status, halvings);
  if (stats) *stats = h->last_stats;
  if (k.status) return finish_status(h, k.status);
  return status;
}

int bd_get_state(bd_handle *h, double *xy, float *theta, uint8_t *species, int32_t *tri,
                 int32_t *n_tri, int64_t *step) {
  if (!h) return BD_ERR_ARG;
  const int np = h->np, n = h->n;
  if (xy || theta || species) {
    // permuted to the caller's order on the device, then one copy per array
    cudaStream_t st = h->stream;
    cudaError_t e = bd_launch_state_out(h->d, h->c, st);
    if (e == cudaSuccess && xy) e = cudaMemcpyAsync(xy, h->d.xfer_xy, (size_t)n * sizeof(double2), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && theta) e = cudaMemcpyAsync(theta, h->d.xfer_th, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && species) e = cudaMemcpyAsync(species, h->d.xfer_sp, (size_t)n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (tri && !h->c.overlap_verlet) {
    std::vector<int4> tv(h->nt);
    cudaError_t e = cudaMemcpyAsync(tv.data(), h->d.tv, h->nt * sizeof(int4), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    auto ext = [&](int v) { return v < np ? h->ext_of_int[v] : n + (v - np); };
    for (int k = 0; k < h->nt; ++k) {
      tri[3 * k] = ext(tv[k].x);
      tri[3 * k + 1] = ext(tv[k].y);
      tri[3 * k + 2] = ext(tv[k].z);
    }
  }
  if (n_tri) *n_tri = h->c.overlap_verlet ? 0 : h->nt;
  if (step) *step = h->step;
  return BD_OK;
}

int bd_batch_step(bd_handle *h, int32_t nsteps, bd_step_stats *per_replica) {
  if (!h || nsteps < 0) return BD_ERR_ARG;
  const int R = (int)h->reps.size();
  bd_step_stats tot;
  if (!h->d.rep_stats) {
    // one replica: its counters are the call's
    const int rc = bd_step(h, nsteps, &tot);
    if (per_replica) per_replica[0] = tot;
    return rc;
  }
  cudaError_t e = cudaMemsetAsync(h->d.rep_stats, 0, 3 * (size_t)R * sizeof(long long), h->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  const int rc = bd_step(h, nsteps, &tot);
  if (per_replica) {
    std::vector<long long> v(3 * (size_t)R);
    e = cudaMemcpyAsync(v.data(), h->d.rep_stats, v.size() * sizeof(long long), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int r = 0; r < R; ++r) {
      per_replica[r] = tot;
      per_replica[r].corr_iters = v[3 * (size_t)r];
      per_replica[r].flips = v[3 * (size_t)r + 1];
      per_replica[r].inverted = v[3 * (size_t)r + 2];
    }
  }
  return rc;
}

int bd_get_tri_shifts(bd_handle *h, int32_t r, int8_t *shifts) {
  if (!h || !shifts || r >= (int)h->reps.size()) return BD_ERR_ARG;
  if (h->c.overlap_verlet) return BD_OK;
  const int base = r < 0 ? 0 : h->reps[r].tri_base, nt = r < 0 ? h->nt : h->reps[r].nt;
  std::vector<int4> tv(nt);
  cudaError_t e = cudaMemcpyAsync(tv.data(), h->d.tv + base, nt * sizeof(int4), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  auto f = [](int w, int bit) { return (int8_t)((((w >> bit) & 3) ^ 2) - 2); };
  for (int t = 0; t < nt; ++t)
    for (int k = 0; k < 3; ++k) {
      shifts[6 * t + 2 * k] = f(tv[t].w, 8 + 4 * k);
      shifts[6 * t + 2 * k + 1] = f(tv[t].w, 10 + 4 * k);
    }
  return BD_OK;
}

int bd_get_replica(bd_handle *h, int32_t r, double *xy, float *theta, int32_t *tri, int32_t *n_tri,
                   int32_t *n, double *L) {
  if (!h || r < 0 || r >= (int)h->reps.size()) return BD_ERR_ARG;
  const RepHost &RH = h->reps[r];
  if (n) *n = RH.n;
  if (L) *L = RH.L;
  if (n_tri) *n_tri = h->c.overlap_verlet ? 0 : RH.nt;
  if (h->c.overlap_verlet) tri = nullptr;
  if (!xy && !theta && !tri) return BD_OK;
  std::vector<double2> pos;
  std::vector<float> t;
  int rc = fetch_disks(h, xy ? &pos : nullptr, theta ? &t : nullptr, nullptr);
  if (rc) return rc;
  for (int i = 0; i < RH.n; ++i) {
    const int k = h->int_of_ext[RH.ext_base + i];
    if (xy) {
      xy[2 * i] = pos[k].x;
      xy[2 * i + 1] = pos[k].y;
    }
    if (theta) theta[i] = t[k];
  }
  if (tri) {
    std::vector<int4> tv(RH.nt);
    cudaError_t e = cudaMemcpyAsync(tv.data(), h->d.tv + RH.tri_base, RH.nt * sizeof(int4),
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    auto loc = [&](int v) { return v < h->np ? h->ext_of_int[v] - RH.ext_base : RH.n + (v - RH.ghost_base); };
    for (int k = 0; k < RH.nt; ++k) {
      tri[3 * k] = loc(tv[k].x);
      tri[3 * k + 1] = loc(tv[k].y);
      tri[3 * k + 2] = loc(tv[k].z);
    }
  }
  return BD_OK;
}

int bd_set_state(bd_handle *h, const double *xy, const float *theta) {
  if (!h || !xy) return BD_ERR_ARG;
  const BdConst &c = h->c;
  // The caller's arrays are copied as they are; the range checks, the
  // rounding to the grid and the permutation to slot order run on the device
  // (k_state_check, k_state_in).  Pairs closer than sigma are found by the
  // repaired Delaunay triangulation's overlap scan (its edges hold the closest
  // pair), or with Verlet lists by a scan of the lists, rebuilt first if a
  // disk moved more than skin/2 from where they were built (they then hold
  // every pair within r_cut >= sigma).  Any failure leaves the previous state
  // in place.
  cudaStream_t st = h->stream;
  const BdDev &d = h->d;
  // k_state_check also snapshots pos, prev and theta and clears the moved
  // flags; k_state_in also writes the FP32 copy of what it stores
  cudaError_t e = reset_stats(h);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d.xfer_xy, xy, (size_t)h->n * sizeof(double2), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && theta) e = cudaMemcpyAsync(d.xfer_th, theta, (size_t)h->n * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = bd_launch_state_in(d, c, theta ? 1 : 0, st);
  // periodic box: a new coordinate across an edge from the old one re-entered
  if (e == cudaSuccess && c.any_periodic) e = bd_launch_periodic_wraps(d, c, st);
  if (e == cudaSuccess && !c.overlap_verlet) e = bd_launch_dt(d, c, 1, st, h->dt_grid, h->dt_block);
  if (e == cudaSuccess && c.overlap_verlet) {
    e = bd_launch_force_short(d, c, st);
    if (e == cudaSuccess) e = bd_launch_overlap_verlet(d, c, st, h->vc_grid, h->vc_block, -1);
  }
  if (e != cudaSuccess) return cuda_fail(e);
  int rc = read_ctl(h);   // synchronises the stream
  if (rc) return rc;
  fill_stats(h, h->h_ctl->status, 0);
  if (h->h_ctl->status) return finish_status(h, h->h_ctl->status);
  return BD_OK;
}

int bd_noise_sample(uint64_t seed, int32_t replica, int32_t n, const uint32_t *counters, uint32_t *words,
                    float *normals32, double *normals64) {
  if (n < 0 || (n > 0 && !counters)) return BD_ERR_ARG;
  if (n == 0) return BD_OK;
  void *buf = nullptr;
  const size_t nw = (size_t)n * 16, n32 = (size_t)n * 12, n64 = (size_t)n * 24;
  const size_t off64 = (2 * nw + n32 + 7) / 8 * 8;   // the FP64 normals 8-byte aligned
  cudaError_t e = cudaMalloc(&buf, off64 + n64);
  if (e != cudaSuccess) return cuda_fail(e);
  char *b = (char *)buf;
  void *d_ctr = b, *d_words = b + nw;
  float *d_z32 = (float *)(b + 2 * nw);
  double *d_z64 = (double *)(b + off64);
  e = cudaMemcpy(d_ctr, counters, nw, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = bd_launch_noise_sample(seed, (unsigned)replica, n, d_ctr, d_words, d_z32, d_z64, nullptr);
  if (e == cudaSuccess && words) e = cudaMemcpy(words, d_words, nw, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && normals32) e = cudaMemcpy(normals32, d_z32, n32, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && normals64) e = cudaMemcpy(normals64, d_z64, n64, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(buf);
  return e == cudaSuccess ? BD_OK : cuda_fail(e);
}

int bd_set_force_shard(bd_handle *h, int32_t rank, int32_t world) {
  if (!h || world < 1 || rank < 0 || rank >= world) return BD_ERR_ARG;
  if (h->reps.size() != 1 || !h->c.any_long || h->c.precision != 0 || h->max_halvings > 0)
    return BD_ERR_UNSUPPORTED;
  cudaError_t e = cudaSuccess;
  if (h->c.force_variant < 2) e = use_variant(h, 3, 8);   // shards cut the symmetric sweep's plan
  if (e != cudaSuccess) return cuda_fail(e);
  // the plan as uploaded (make_sym is deterministic); an item's cost is its
  // number of j tiles (pairs of a 512-disk block with a 256-disk tile)
  SymPlan S;
  make_sym(h, h->tune_tiles, h->c.force_variant, S);
  const int ni = (int)S.items.size();
  std::vector<double> cum(ni + 1, 0.0);
  for (int k = 0; k < ni; ++k) cum[k + 1] = cum[k] + (S.items[k].z - S.items[k].y);
  // rank r: the items whose cumulative cost starts in [r T / W, (r + 1) T / W)
  auto first = [&](int r) {
    const double target = cum[ni] * r / world;
    return (int)(std::lower_bound(cum.begin(), cum.end() - 1, target) - cum.begin());
  };
  const int b0 = rank == 0 ? 0 : first(rank), b1 = rank + 1 == world ? ni : first(rank + 1);
  // partials of items that are not this rank's stay zero in the reduction
  e = cudaMemsetAsync(h->d.ipart, 0, (size_t)ni * BD_SB * sizeof(float2), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d.jpart, 0, (size_t)S.n_jtiles * BD_TJ * sizeof(float2), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  h->c.sitem0 = b0;
  h->c.n_sitems = b1 - b0;
  h->shard_rank = rank;
  h->shard_world = world;
  return BD_OK;
}

int bd_force_slots(bd_handle *h, int32_t *slots) {
  if (!h || !slots) return BD_ERR_ARG;
  *slots = h->np;
  return BD_OK;
}

int bd_step_begin(bd_handle *h, double *forces) {
  if (!h || !forces || h->reps.size() != 1 || !h->c.any_long || h->c.precision != 0) return BD_ERR_ARG;
  cudaStream_t st = h->stream;
  cudaError_t e = reset_stats(h);
  if (e == cudaSuccess) e = bd_launch_force_long(h->d, h->c, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(forces, h->d.fpart, (size_t)h->np * sizeof(double2), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e == cudaSuccess ? BD_OK : cuda_fail(e);
}

int bd_step_end(bd_handle *h, const double *forces, bd_step_stats *stats) {
  if (!h || !forces || h->reps.size() != 1 || !h->c.any_long || h->c.precision != 0) return BD_ERR_ARG;
  if (stats) memset(stats, 0, sizeof(*stats));
  cudaStream_t st = h->stream;
  const int64_t step_base = h->step;
  cudaError_t e = cudaMemcpyAsync(h->d.fpart, forces, (size_t)h->np * sizeof(double2), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = bd_launch_integrate(h->d, h->c, h->step, -1, st);
  if (e == cudaSuccess) e = launch_correction(h, st);
  if (e != cudaSuccess) return cuda_fail(e);
  h->last_launches = 2;
  int rc = read_ctl(h);
  if (rc) return rc;
  const BdCtl &k = *h->h_ctl;
  add_stage_times(h);
  h->step = step_base + k.st_steps;
  fill_stats(h, k.status, 0);
  if (stats) *stats = h->last_stats;
  if (k.status) return finish_status(h, k.status);
  return BD_OK;
}

int bd_last_stats(bd_handle *h, bd_step_stats *stats) {
  if (!h || !stats) return BD_ERR_ARG;
  *stats = h->last_stats;
  return BD_OK;
}

int bd_set_loop_caps(bd_handle *h, int32_t max_corr_iters, int32_t max_flip_rounds) {
  if (!h || max_corr_iters < 1 || max_flip_rounds < 1) return BD_ERR_ARG;
  // the caps are kernel arguments: the next step recaptures its graph
  h->c.max_corr_iters = max_corr_iters;
  h->c.max_flip_rounds = max_flip_rounds;
  for (auto &r : h->reps) {
    r.p.max_corr_iters = max_corr_iters;
    r.p.max_flip_rounds = max_flip_rounds;
  }
  return BD_OK;
}

int bd_set_wait_limit(bd_handle *h, double seconds, int32_t hold_barrier) {
  if (!h || !(seconds >= 1e-3 && seconds <= 60.0) || hold_barrier < 0) return BD_ERR_ARG;
  // pinned host words: the copies are queued on the handle's stream
  h->h_ctl->bar_hold = (unsigned)hold_barrier;
  h->h_ctl->bar_limit_ns = (unsigned long long)(seconds * 1e9);
  cudaError_t e = cudaMemcpyAsync(&h->d.ctl->bar_hold, &h->h_ctl->bar_hold, sizeof(unsigned),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&h->d.ctl->bar_limit_ns, &h->h_ctl->bar_limit_ns, sizeof(unsigned long long),
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  return e == cudaSuccess ? BD_OK : cuda_fail(e);
}

int bd_compute_forces(bd_handle *h, double *F) {
  if (!h || !F) return BD_ERR_ARG;
  cudaStream_t st = h->stream;
  const int n = h->n, np = h->np;
  cudaError_t e = cudaSuccess;
  if (h->c.any_long) e = bd_launch_force_long(h->d, h->c, st);
  if (e == cudaSuccess && h->c.any_short) e = bd_launch_force_short(h->d, h->c, st);
  if (e == cudaSuccess) e = bd_launch_force_sum(h->d, h->c, h->d_fsum, st);
  std::vector<double2> f(np);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f.data(), h->d_fsum, np * sizeof(double2), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  int rc = read_ctl(h);
  if (rc) return rc;
  if (h->h_ctl->status) return finish_status(h, h->h_ctl->status);
  for (int i = 0; i < n; ++i) {
    double2 v = f[h->int_of_ext[i]];
    F[2 * i] = v.x;
    F[2 * i + 1] = v.y;
  }
  return BD_OK;
}

int bd_get_neighbors(bd_handle *h, int32_t max_per, int32_t *counts, int32_t *idx) {
  if (!h || !counts || max_per < 0 || (max_per > 0 && !idx)) return BD_ERR_ARG;
  if (!h->c.any_short) return BD_ERR_UNSUPPORTED;
  const int np = h->np, n = h->n;
  std::vector<int> cnt(np), vi((size_t)BD_VL_MAX * np);
  cudaStream_t st = h->stream;
  cudaError_t e = cudaMemcpyAsync(cnt.data(), h->d.vl_cnt, np * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(vi.data(), h->d.vl_idx, vi.size() * sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  for (int x = 0; x < n; ++x) {
    int i = h->int_of_ext[x];
    int m = cnt[i];
    counts[x] = m;
    std::vector<int> lst(m);
    for (int t = 0; t < m; ++t) lst[t] = h->ext_of_int[vi[(size_t)t * np + i]];
    std::sort(lst.begin(), lst.end());
    for (int t = 0; t < m && t < max_per; ++t) idx[(size_t)x * max_per + t] = lst[t];
  }
  return BD_OK;
}

int bd_get_geometry(bd_handle *h, double *q, double *L) {
  if (!h) return BD_ERR_ARG;
  if (q) *q = h->c.q;
  if (L) *L = h->reps[0].L;
  return BD_OK;
}

int bd_get_tuning(bd_handle *h, int32_t *tiles_per_item, int32_t *variant, int32_t *n_items) {
  if (!h) return BD_ERR_ARG;
  if (tiles_per_item) *tiles_per_item = h->tune_tiles;
  if (variant) *variant = h->c.force_variant;
  if (n_items) *n_items = h->c.force_variant >= 2 ? h->c.n_sitems : h->c.n_items;
  return BD_OK;
}

int bd_force_timing(bd_handle *h, int enable, int reset, double *total_ms, int64_t *launches) {
  if (!h) return BD_ERR_ARG;
  h->timing = enable != 0;
  if (total_ms) *total_ms = h->force_ms;
  if (launches) *launches = h->force_launches;
  if (reset) {
    h->force_ms = 0.0;
    h->force_launches = 0;
  }
  return BD_OK;
}

int64_t bd_last_launch_count(bd_handle *h) { return h ? h->last_launches : -1; }

int bd_stage_times(bd_handle *h, int reset, double *ms, int64_t *phases) {
  if (!h) return BD_ERR_ARG;
  for (int k = 0; k < 5; ++k) {
    if (ms) ms[k] = (k == 0 ? h->stage_ns[0] + h->stage_ns[4] : h->stage_ns[k]) * 1e-6;
    if (phases) phases[k] = k == 0 ? h->stage_cnt[0] + h->stage_cnt[4] : h->stage_cnt[k];
  }
  if (reset)
    for (int k = 0; k < 5; ++k) {
      h->stage_ns[k] = 0.0;
      h->stage_cnt[k] = 0;
    }
  return BD_OK;
}

int bd_place_disks(int32_t n, double L, double a, int32_t placement, uint64_t seed, double *xy) {
  if (n < 1 || !xy || !(a > 0) || !(L > 2.0 * a) || !isfinite(L)) return BD_ERR_ARG;
  if (placement < BD_PLACE_RSA || placement > BD_PLACE_LATTICE) return BD_ERR_ARG;
  std::vector<double> v;
  const int rc = placement == BD_PLACE_LATTICE ? bdhost::lattice_place(n, a, L - a, 2.0 * a, seed, v)
                                               : bdhost::rsa_place(n, a, L - a, 2.0 * a, seed, v);
  if (rc != 0) return BD_ERR_ARG;
  memcpy(xy, v.data(), sizeof(double) * 2 * (size_t)n);
  return BD_OK;
}

int bd_ghost_points(double L, double a, double *xy, int32_t *count) {
  if (!(L > 0) || !(a > 0) || !count) return BD_ERR_ARG;
  std::vector<double> gx, gy;
  bdhost::make_ghosts(L, a, gx, gy);
  if (xy) {
    if (*count < (int32_t)gx.size()) return BD_ERR_ARG;
    for (size_t k = 0; k < gx.size(); ++k) {
      xy[2 * k] = gx[k];
      xy[2 * k + 1] = gy[k];
    }
  }
  *count = (int32_t)gx.size();
  return BD_OK;
}

int bd_triangulate(int32_t n, const double *xy, double L, double a, double *xy_grid, int32_t *tri,
                   int32_t *n_tri) {
  if (n < 1 || !xy || !tri || !(L > 0) || !(a > 0)) return BD_ERR_ARG;
  const int s = grid_shift(L, a);
  const double q = ldexp(1.0, -s), inv_q = ldexp(1.0, s);
  std::vector<double> gx, gy;
  bdhost::make_ghosts(L, a, gx, gy);
  const int ng = (int)gx.size();
  std::vector<double> X(n + ng), Y(n + ng);
  std::vector<uint64_t> hk(n);
  for (int i = 0; i < n; ++i) {
    X[i] = snap_host(xy[2 * i], q, inv_q);
    Y[i] = snap_host(xy[2 * i + 1], q, inv_q);
    if (!(X[i] > 0 && X[i] < L && Y[i] > 0 && Y[i] < L)) return BD_ERR_ARG;
    if (xy_grid) {
      xy_grid[2 * i] = X[i];
      xy_grid[2 * i + 1] = Y[i];
    }
    uint32_t ux = (uint32_t)std::min(65535.0, std::max(0.0, X[i] / L * 65536.0));
    uint32_t uy = (uint32_t)std::min(65535.0, std::max(0.0, Y[i] / L * 65536.0));
    hk[i] = bdhost::hilbert_index(ux, uy);
  }
  for (int k = 0; k < ng; ++k) {
    X[n + k] = gx[k];
    Y[n + k] = gy[k];
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a_, int b_) { return hk[a_] != hk[b_] ? hk[a_] < hk[b_] : a_ < b_; });
  bdpred::Grid grid;
  grid.q = q;
  grid.inv_q = inv_q;
  grid.s = s;
  std::vector<int> gids(ng);
  for (int k = 0; k < ng; ++k) gids[k] = n + k;
  std::vector<int> V, N;
  if (bdhost::build_delaunay(X.data(), Y.data(), grid, order, gids, V, N) != 0) return BD_ERR_TRIANGULATION;
  const int nt = (int)(V.size() / 3);
  if (nt != 2 * (n + ng) - 6) return BD_ERR_TRIANGULATION;
  memcpy(tri, V.data(), sizeof(int) * V.size());
  if (n_tri) *n_tri = nt;
  return BD_OK;
}

int bd_triangulate_periodic(int32_t n, const double *xy, double L, double *xy_grid, int32_t *tri,
                            int8_t *shifts, int32_t *n_tri) {
  if (n < 3 || !xy || !tri || !shifts || !(L > 0) || !(L < 1e7)) return BD_ERR_ARG;
  bd_params p;
  bd_default_params(&p);
  p.boundary = BD_BOUNDARY_PERIODIC;
  p.box_L = L;
  p.n = n;
  const double Lp = box_side(p);
  const int s = grid_shift_for(coord_extent(p));
  const double q = ldexp(1.0, -s), inv_q = ldexp(1.0, s);
  std::vector<double> X(n), Y(n);
  for (int i = 0; i < n; ++i) {
    if (!isfinite(xy[2 * i]) || !isfinite(xy[2 * i + 1])) return BD_ERR_ARG;
    X[i] = periodic_coord(xy[2 * i], Lp, q, inv_q);
    Y[i] = periodic_coord(xy[2 * i + 1], Lp, q, inv_q);
    if (xy_grid) {
      xy_grid[2 * i] = X[i];
      xy_grid[2 * i + 1] = Y[i];
    }
  }
  std::vector<int> ids(n);
  std::iota(ids.begin(), ids.end(), 0);
  bdpred::Grid grid;
  grid.q = q;
  grid.inv_q = inv_q;
  grid.s = s;
  std::vector<int> V, S, N;
  if (bdhost::build_torus_delaunay(X.data(), Y.data(), ids, Lp, grid, V, S, N) != 0) return BD_ERR_TRIANGULATION;
  memcpy(tri, V.data(), sizeof(int) * V.size());
  for (size_t k = 0; k < S.size(); ++k) shifts[k] = (int8_t)S[k];
  if (n_tri) *n_tri = (int32_t)(V.size() / 3);
  return BD_OK;
}

}  // extern "C"
