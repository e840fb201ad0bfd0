// C-ABI layer: handle lifetime, host-side set-up, the per-step launch
// sequence and state transfer.  See include/bd.h for the contract of each
// entry point.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "bd_internal.h"
#include "predicates.cuh"

namespace bdhost {
int build_delaunay(const double *X, const double *Y, const bdpred::Grid &grid,
                   const std::vector<int> &order, const std::vector<int> &g, std::vector<int> &V,
                   std::vector<int> &N);
void make_ghosts(double L, double a, std::vector<double> &gx, std::vector<double> &gy);
double ghost_extent(double L, double a);
int rsa_place(int n, double lo, double hi, double dmin, uint64_t seed, std::vector<double> &xy);
int any_overlap(int n, const double *xy, double lo, double hi, double dmin);
uint64_t hilbert_index(uint32_t x, uint32_t y);
}  // namespace bdhost

struct bd_handle {
  bd_params p;
  cudaStream_t stream = nullptr;
  BdDev d;
  BdConst c;
  int n = 0, np = 0, np_i = 0, nt = 0, ng = 0;
  std::vector<int> ext_of_int;  // np (-1 = empty slot)
  std::vector<int> int_of_ext;  // n
  std::vector<double> host_pos; // (np + ng) * 2 mirror used for uploads (empty slots, ghost points)
  int dt_grid = 0, dt_block = 0;
  int64_t step = 0;
  double2 *d_fsum = nullptr;
  BdCtl *h_ctl = nullptr;       // pinned
  std::vector<void *> dev_allocs;
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;   // pairs (start, end) per timed launch
  double force_ms = 0.0;
  int64_t force_launches = 0;
  int64_t last_launches = 0;
};

namespace {

int cuda_fail(cudaError_t e) { return e == cudaErrorMemoryAllocation ? BD_ERR_NOMEM : BD_ERR_CUDA; }

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

int grid_shift(double L, double a) {
  // every coordinate (disks and ghost points) is below E in magnitude; need E * 2^s < 2^51
  double E = bdhost::ghost_extent(L, a);
  int e = (int)ceil(log2(E + 1.0));
  return 51 - e;
}

int validate(const bd_params *p) {
  if (!p) return BD_ERR_ARG;
  if (p->n < 1 || p->n > (1 << 28)) return BD_ERR_ARG;
  if (p->n_species < 1 || p->n_species > 2) return BD_ERR_ARG;
  if (!(p->a > 0) || !isfinite(p->a)) return BD_ERR_ARG;
  if (!(p->box_L > 0) && !(p->area_fraction > 0 && p->area_fraction < 0.9)) return BD_ERR_ARG;
  if (p->law < BD_LAW_NONE || p->law > BD_LAW_SHORT) return BD_ERR_ARG;
  if (p->precision < 0 || p->precision > 1) return BD_ERR_ARG;
  if (!(p->dt > 0) || !isfinite(p->dt)) return BD_ERR_ARG;
  if (!(p->D >= 0) || !(p->Dr >= 0) || !isfinite(p->v0)) return BD_ERR_ARG;
  for (int k = 0; k < 4; ++k)
    if (!isfinite(p->alpha[k])) return BD_ERR_ARG;
  if (p->max_corr_iters < 1 || p->max_flip_rounds < 1) return BD_ERR_ARG;
  if (p->law == BD_LAW_SHORT) {
    if (!(p->r_cut > 2.0 * p->a) || !(p->skin > 0) || !(p->eps >= 0) || !(p->kappa >= 0)) return BD_ERR_ARG;
    if (p->precision != 0) return BD_ERR_UNSUPPORTED;
  }
  return BD_OK;
}

double snap_host(double v, double q, double inv_q) { return nearbyint(v * inv_q) * q; }

int pick_nchunk(const BdConst &c) {
  const char *env = getenv("BD_NCHUNK");
  if (env && atoi(env) > 0) return std::min(atoi(env), c.ntiles);
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (c.precision == 1) {
    int blocks = (c.np + 127) / 128;
    int want = std::max(1, (4 * sms) / std::max(1, blocks));
    return std::max(1, std::min(want, c.ntiles));
  }
  // resident force blocks per SM from the occupancy calculator; choose the
  // number of j chunks so the (i block, j chunk) grid fills whole waves
  int per_sm = bd_force_blocks_per_sm(c.force_variant);
  if (per_sm < 1) per_sm = 1;
  const long slots = (long)sms * per_sm;
  const long ib = std::max(1, c.n_iblocks);
  int best = 1;
  double best_eff = -1.0;
  for (int ch = 1; ch <= std::min(c.ntiles, 64); ++ch) {
    long ctas = ib * ch;
    long waves = (ctas + slots - 1) / slots;
    // useful fraction of the last wave, times the tile balance across chunks
    double fill = (double)ctas / (double)(waves * slots);
    int tiles_max = (c.ntiles + ch - 1) / ch;
    double bal = ((double)c.ntiles / ch) / tiles_max;
    // prefer at least two waves of blocks per SM slot for latency hiding
    double eff = fill * bal * (waves >= 2 ? 1.0 : 0.9);
    if (eff > best_eff + 1e-9) {
      best_eff = eff;
      best = ch;
    }
  }
  return best;
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
  for (void *p : h->dev_allocs) cudaFree(p);
  if (h->h_ctl) cudaFreeHost(h->h_ctl);
  for (cudaEvent_t ev : h->ev_pool) cudaEventDestroy(ev);
  delete h;
}

int bd_init(const bd_params *p_in, const double *xy_in, const uint8_t *species_in,
            const float *theta_in, void *stream, bd_handle **out) {
  if (!out) return BD_ERR_ARG;
  *out = nullptr;
  int rc = validate(p_in);
  if (rc) return rc;
  bd_handle *h = new (std::nothrow) bd_handle();
  if (!h) return BD_ERR_NOMEM;
  h->p = *p_in;
  h->stream = (cudaStream_t)stream;
  const bd_params &p = h->p;
  const int n = p.n;
  h->n = n;
  const double L = p.box_L > 0 ? p.box_L : sqrt((double)n * M_PI * p.a * p.a / p.area_fraction);
  const int s = grid_shift(L, p.a);
  const double q = ldexp(1.0, -s), inv_q = ldexp(1.0, s);
  const double wall_lo = ceil(p.a * inv_q) * q, wall_hi = floor((L - p.a) * inv_q) * q;
  if (!(wall_hi > wall_lo)) { delete h; return BD_ERR_ARG; }

  // ---- positions, species, directions (external order) ----
  std::vector<double> xy(2 * (size_t)n);
  if (xy_in) {
    memcpy(xy.data(), xy_in, sizeof(double) * 2 * (size_t)n);
  } else if (bdhost::rsa_place(n, p.a, L - p.a, 2.0 * p.a, p.seed, xy) != 0) {
    delete h;
    return BD_ERR_ARG;
  }
  for (size_t k = 0; k < xy.size(); ++k) {
    if (!isfinite(xy[k]) || xy[k] < p.a - 1e-9 * L || xy[k] > L - p.a + 1e-9 * L) {
      delete h;
      return BD_ERR_INIT_OVERLAP;
    }
  }
  if (bdhost::any_overlap(n, xy.data(), 0.0, L, 2.0 * p.a * (1.0 - 1e-12))) {
    delete h;
    return BD_ERR_INIT_OVERLAP;
  }
  for (size_t k = 0; k < xy.size(); ++k)
    xy[k] = std::min(wall_hi, std::max(wall_lo, snap_host(xy[k], q, inv_q)));
  std::vector<uint8_t> sp(n, 0);
  if (species_in) {
    for (int i = 0; i < n; ++i) {
      if (species_in[i] >= p.n_species) { delete h; return BD_ERR_ARG; }
      sp[i] = species_in[i];
    }
  }
  std::vector<float> th(n, 0.f);
  if (theta_in) memcpy(th.data(), theta_in, sizeof(float) * n);

  // ---- internal order: species-major, Hilbert-minor, tile-padded ----
  std::vector<uint64_t> hk(n);
  for (int i = 0; i < n; ++i) {
    uint32_t ux = (uint32_t)std::min(65535.0, std::max(0.0, xy[2 * i] / L * 65536.0));
    uint32_t uy = (uint32_t)std::min(65535.0, std::max(0.0, xy[2 * i + 1] / L * 65536.0));
    hk[i] = bdhost::hilbert_index(ux, uy);
  }
  std::vector<int> by_sp(n);
  std::iota(by_sp.begin(), by_sp.end(), 0);
  std::sort(by_sp.begin(), by_sp.end(), [&](int a, int b) {
    if (sp[a] != sp[b]) return sp[a] < sp[b];
    if (hk[a] != hk[b]) return hk[a] < hk[b];
    return a < b;
  });
  int cnt_sp[2] = {0, 0};
  for (int i = 0; i < n; ++i) cnt_sp[sp[i]]++;
  const size_t seg0 = pad_to(cnt_sp[0], BD_TJ), seg1 = pad_to(cnt_sp[1], BD_TJ);
  const int np = (int)(seg0 + seg1);
  h->np = np;
  h->ext_of_int.assign(np, -1);
  h->int_of_ext.assign(n, -1);
  {
    size_t k0 = 0, k1 = seg0;
    for (int r = 0; r < n; ++r) {
      int e = by_sp[r];
      size_t slot = sp[e] == 0 ? k0++ : k1++;
      h->ext_of_int[slot] = e;
      h->int_of_ext[e] = (int)slot;
    }
  }
  // i blocks of the force sweep: Hilbert order over all disks
  std::vector<int> by_h(n);
  std::iota(by_h.begin(), by_h.end(), 0);
  std::sort(by_h.begin(), by_h.end(), [&](int a, int b) { return hk[a] != hk[b] ? hk[a] < hk[b] : a < b; });
  const int np_i = (int)pad_to(n, BD_IB);
  h->np_i = np_i;
  std::vector<int> iperm(np_i, -1);
  for (int r = 0; r < n; ++r) iperm[r] = h->int_of_ext[by_h[r]];
  const int n_iblocks = np_i / BD_IB;
  std::vector<float2> iorg(n_iblocks);
  for (int b = 0; b < n_iblocks; ++b) {
    double sx = 0, sy = 0;
    int m = 0;
    for (int k = b * BD_IB; k < std::min(n, (b + 1) * BD_IB); ++k) {
      int e = by_h[k];
      sx += xy[2 * e];
      sy += xy[2 * e + 1];
      ++m;
    }
    iorg[b] = m ? make_float2((float)nearbyint(sx / m), (float)nearbyint(sy / m)) : make_float2(0.f, 0.f);
  }
  std::vector<uint8_t> tile_sp(np / BD_TJ);
  for (size_t t = 0; t < tile_sp.size(); ++t) tile_sp[t] = (t * BD_TJ < seg0) ? 0 : 1;

  // internal position mirror: np slots + ghost points
  std::vector<double> ghx, ghy;
  bdhost::make_ghosts(L, p.a, ghx, ghy);
  const int ng = (int)ghx.size();
  h->ng = ng;
  h->host_pos.assign(2 * ((size_t)np + ng), 0.0);
  for (int i = 0; i < np; ++i) {
    int e = h->ext_of_int[i];
    if (e >= 0) {
      h->host_pos[2 * i] = xy[2 * e];
      h->host_pos[2 * i + 1] = xy[2 * e + 1];
    } else {
      h->host_pos[2 * i] = 0.5 * L;  // never referenced by the triangulation
      h->host_pos[2 * i + 1] = 0.5 * L;
    }
  }
  for (int k = 0; k < ng; ++k) {
    h->host_pos[2 * ((size_t)np + k)] = ghx[k];
    h->host_pos[2 * ((size_t)np + k) + 1] = ghy[k];
  }

  // ---- initial Delaunay triangulation on the host (Sec. 4.1) ----
  std::vector<double> X(np + ng), Y(np + ng);
  for (int i = 0; i < np + ng; ++i) {
    X[i] = h->host_pos[2 * i];
    Y[i] = h->host_pos[2 * i + 1];
  }
  std::vector<int> order(n);
  for (int r = 0; r < n; ++r) order[r] = h->int_of_ext[by_h[r]];
  bdpred::Grid grid;
  grid.q = q;
  grid.inv_q = inv_q;
  grid.s = s;
  std::vector<int> gids(ng);
  for (int k = 0; k < ng; ++k) gids[k] = np + k;
  std::vector<int> V, N;
  if (bdhost::build_delaunay(X.data(), Y.data(), grid, order, gids, V, N) != 0) {
    delete h;
    return BD_ERR_TRIANGULATION;
  }
  const int nt = (int)(V.size() / 3);
  if (nt != 2 * (n + ng) - 6) {
    delete h;
    return BD_ERR_TRIANGULATION;
  }
  h->nt = nt;

  // ---- constants ----
  BdConst &c = h->c;
  memset(&c, 0, sizeof(c));
  c.n = n;
  c.np = np;
  c.np_i = np_i;
  c.nt = nt;
  c.ntiles = np / BD_TJ;
  c.n_iblocks = n_iblocks;
  c.law = p.law;
  c.precision = p.precision;
  c.n_species = p.n_species;
  c.a = p.a;
  c.sigma = 2.0 * p.a;
  c.L = L;
  c.wall_lo = wall_lo;
  c.wall_hi = wall_hi;
  c.q = q;
  c.inv_q = inv_q;
  c.qshift = s;
  {
    // (sigma/q)^2 (1 + 1e-9), rounded up, as a 128-bit integer
    long double sq = (long double)(2.0 * p.a) * (long double)inv_q;
    long double v = sq * sq * (1.0L + 1e-9L);
    long double two64 = 18446744073709551616.0L;
    unsigned long long hi = (unsigned long long)(v / two64);
    long double rem = v - (long double)hi * two64;
    unsigned long long lo = (unsigned long long)rem;
    if ((long double)lo < rem) ++lo;
    c.sig2q_hi = hi;
    c.sig2q_lo = lo;
  }
  for (int k = 0; k < 4; ++k) {
    c.alpha[k] = (float)p.alpha[k];
    c.alpha_d[k] = p.alpha[k];
  }
  if (p.n_species == 1) {
    for (int k = 1; k < 4; ++k) {
      c.alpha[k] = c.alpha[0];
      c.alpha_d[k] = c.alpha_d[0];
    }
  }
  c.eps = p.eps;
  c.kappa = p.kappa;
  c.r_cut = p.r_cut;
  c.skin = p.skin;
  c.rl2 = (p.r_cut + p.skin) * (p.r_cut + p.skin);
  c.ncell = std::max(1, std::min(1 << 14, (int)floor(L / (p.r_cut + p.skin))));
  c.cell_size = L / c.ncell;
  c.D = p.D;
  c.Dr = p.Dr;
  c.v0 = p.v0;
  c.dt = p.dt;
  c.amp = p.literal_noise ? sqrt(p.D * p.dt) : sqrt(2.0 * p.D * p.dt);
  c.amp_r = sqrt(2.0 * p.Dr * p.dt);
  c.seed = p.seed;
  c.replica = (uint32_t)p.replica;
  c.max_corr_iters = p.max_corr_iters;
  c.max_flip_rounds = p.max_flip_rounds;
  c.nchunk = 1;
  h->step = p.step0;

  // ---- device buffers ----
  BdDev &d = h->d;
  memset(&d, 0, sizeof(d));
  cudaError_t e = cudaSuccess;
  const size_t nv = (size_t)np + ng;
#define BD_TRY(x)                         \
  do {                                    \
    e = (x);                              \
    if (e != cudaSuccess) goto cuda_error; \
  } while (0)
  {
    {
      const char *fv = getenv("BD_FORCE_VARIANT");
      c.force_variant = fv ? atoi(fv) : 1;
    }
    c.nchunk = p.law == BD_LAW_SHORT ? 1 : pick_nchunk(c);
    BD_TRY(dalloc(h, &d.pos, nv));
    BD_TRY(dalloc(h, &d.prev, nv));
    BD_TRY(dalloc(h, &d.pos0, nv));
    BD_TRY(dalloc(h, &d.work, (size_t)np));
    BD_TRY(dalloc(h, &d.theta, (size_t)np));
    BD_TRY(dalloc(h, &d.theta0, (size_t)np));
    BD_TRY(dalloc(h, &d.species, (size_t)np));
    BD_TRY(dalloc(h, &d.ext_id, (size_t)np));
    BD_TRY(dalloc(h, &d.moved, nv));
    BD_TRY(dalloc(h, &d.disp, (size_t)np));
    BD_TRY(dalloc(h, &d.tv, (size_t)nt));
    BD_TRY(dalloc(h, &d.tn, (size_t)nt));
    BD_TRY(dalloc(h, &d.tv_snap, (size_t)nt));
    BD_TRY(dalloc(h, &d.tn_snap, (size_t)nt));
    BD_TRY(dalloc(h, &d.claim, (size_t)nt));
    BD_TRY(dalloc(h, &d.partner, (size_t)nt));
    BD_TRY(dalloc(h, &d.iperm, (size_t)np_i));
    BD_TRY(dalloc(h, &d.iorigin, (size_t)n_iblocks));
    BD_TRY(dalloc(h, &d.tile_species, tile_sp.size()));
    BD_TRY(dalloc(h, &d.fpart, (size_t)c.nchunk * np));
    BD_TRY(dalloc(h, &d.ctl, 1));
    if (p.law == BD_LAW_SHORT) {
      const size_t nc2 = (size_t)c.ncell * c.ncell;
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
    BD_TRY(dalloc(h, &h->d_fsum, (size_t)np));
    BD_TRY(cudaMallocHost((void **)&h->h_ctl, sizeof(BdCtl)));

    cudaStream_t st = h->stream;
    std::vector<float> th_i(np, 0.f);
    std::vector<uint8_t> sp_i(np, 255);
    for (int i = 0; i < np; ++i) {
      int ex = h->ext_of_int[i];
      if (ex >= 0) {
        th_i[i] = th[ex];
        sp_i[i] = sp[ex];
      }
    }
    std::vector<int4> tv(nt), tn(nt);
    for (int t = 0; t < nt; ++t) {
      tv[t] = make_int4(V[3 * t], V[3 * t + 1], V[3 * t + 2], 0);
      tn[t] = make_int4(N[3 * t], N[3 * t + 1], N[3 * t + 2], 0);
    }
    BD_TRY(cudaMemcpyAsync(d.pos, h->host_pos.data(), nv * sizeof(double2), cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.prev, d.pos, nv * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.pos0, d.pos, nv * sizeof(double2), cudaMemcpyDeviceToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.theta, th_i.data(), np * sizeof(float), cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.theta0, d.theta, np * sizeof(float), cudaMemcpyDeviceToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.species, sp_i.data(), np, cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.ext_id, h->ext_of_int.data(), np * sizeof(int), cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemsetAsync(d.moved, 0, nv, st));
    BD_TRY(cudaMemsetAsync(d.disp, 0, np * sizeof(double2), st));
    BD_TRY(cudaMemcpyAsync(d.tv, tv.data(), nt * sizeof(int4), cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.tn, tn.data(), nt * sizeof(int4), cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemsetAsync(d.claim, 0, nt * sizeof(unsigned long long), st));
    BD_TRY(cudaMemsetAsync(d.partner, 0, nt * sizeof(unsigned long long), st));
    BD_TRY(cudaMemcpyAsync(d.iperm, iperm.data(), np_i * sizeof(int), cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.iorigin, iorg.data(), n_iblocks * sizeof(float2), cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemcpyAsync(d.tile_species, tile_sp.data(), tile_sp.size(), cudaMemcpyHostToDevice, st));
    BD_TRY(cudaMemsetAsync(d.fpart, 0, (size_t)c.nchunk * np * sizeof(double2), st));
    BD_TRY(cudaMemsetAsync(d.ctl, 0, sizeof(BdCtl), st));
    if (p.law == BD_LAW_SHORT) {
      // reference positions far away: the first force evaluation builds the lists
      std::vector<double2> far(np, make_double2(1e30, 1e30));
      BD_TRY(cudaMemcpyAsync(d.vl_ref, far.data(), np * sizeof(double2), cudaMemcpyHostToDevice, st));
      BD_TRY(cudaMemsetAsync(d.vl_cnt, 0, np * sizeof(int), st));
      BD_TRY(cudaStreamSynchronize(st));
    }
    BD_TRY(bd_launch_work_copy(d, c, st));
    BD_TRY(cudaStreamSynchronize(st));
    if (bd_dt_grid_for(std::max(nt, np), &h->dt_grid, &h->dt_block) != 0) {
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

static int read_ctl(bd_handle *h) {
  cudaError_t e = cudaMemcpyAsync(h->h_ctl, h->d.ctl, sizeof(BdCtl), cudaMemcpyDeviceToHost, h->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return cuda_fail(e);
  return BD_OK;
}

static cudaError_t reset_stats(bd_handle *h) {
  // zero everything after the barrier words, the status and the epoch
  char *base = (char *)h->d.ctl;
  size_t off = offsetof(BdCtl, cnt);
  cudaError_t e = cudaMemsetAsync(base + off, 0, sizeof(BdCtl) - off, h->stream);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(&h->d.ctl->status, 0, sizeof(int), h->stream);
}

int bd_step(bd_handle *h, int32_t nsteps, bd_step_stats *stats) {
  if (!h || nsteps < 0) return BD_ERR_ARG;
  if (stats) memset(stats, 0, sizeof(*stats));
  cudaStream_t st = h->stream;
  cudaError_t e = reset_stats(h);
  if (e != cudaSuccess) return cuda_fail(e);
  int64_t launches = 0;
  int timed = 0;
  if (h->timing && h->c.law == BD_LAW_LONG) {
    while ((int)h->ev_pool.size() < 2 * nsteps) {
      cudaEvent_t ev;
      if (cudaEventCreate(&ev) != cudaSuccess) return BD_ERR_CUDA;
      h->ev_pool.push_back(ev);
    }
  }
  for (int s = 0; s < nsteps; ++s) {
    if (h->c.law == BD_LAW_LONG) {
      bool tm = h->timing;
      if (tm) cudaEventRecord(h->ev_pool[2 * s], st);
      e = bd_launch_force_long(h->d, h->c, st);
      if (e != cudaSuccess) return cuda_fail(e);
      if (tm) {
        cudaEventRecord(h->ev_pool[2 * s + 1], st);
        ++timed;
      }
      ++launches;
    }
    if (h->c.law == BD_LAW_SHORT) {
      e = bd_launch_force_short(h->d, h->c, st);
      if (e != cudaSuccess) return cuda_fail(e);
      launches += bd_short_launches();
    }
    e = bd_launch_integrate(h->d, h->c, h->step + s, st);
    if (e != cudaSuccess) return cuda_fail(e);
    e = bd_launch_dt(h->d, h->c, 0, st, h->dt_grid, h->dt_block);
    if (e != cudaSuccess) return cuda_fail(e);
    launches += 2;
  }
  h->last_launches = launches;
  int rc = read_ctl(h);
  if (rc) return rc;
  for (int s = 0; s < timed; ++s) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_pool[2 * s], h->ev_pool[2 * s + 1]) == cudaSuccess) {
      h->force_ms += ms;
      h->force_launches += 1;
    }
  }
  const BdCtl &k = *h->h_ctl;
  h->step += k.st_steps;
  if (stats) {
    stats->steps_done = k.st_steps;
    stats->corr_iters = k.st_corr_iters;
    stats->overlap_pairs = k.st_overlap_pairs;
    stats->flip_rounds = k.st_flip_rounds;
    stats->flips = k.st_flips;
    stats->repair_flips = k.st_repair_flips;
    stats->inverted = k.st_inverted;
    stats->max_corr_iters = k.st_max_corr_iters;
    stats->verlet_rebuilds = (int32_t)k.st_verlet_rebuilds;
    stats->fail_phase = k.st_fail_phase;
    stats->fail_item = k.st_fail_item;
    stats->fail_count = k.st_fail_count;
    stats->barriers = k.st_barriers;
    stats->rejected = k.status != 0;
    double mo;
    unsigned long long bits = k.st_max_overlap_bits;
    memcpy(&mo, &bits, sizeof(mo));
    stats->max_overlap = mo;
  }
  if (k.status) {
    // clear the sticky status so the handle keeps working from the last good
    // state; after a timed-out barrier also reset the barrier words
    if (k.status == BD_ERR_DEVICE_TIMEOUT) cudaMemsetAsync(h->d.ctl, 0, offsetof(BdCtl, epoch), st);
    cudaMemsetAsync(&h->d.ctl->cnt[0][0], 0, sizeof(h->d.ctl->cnt), st);
    cudaMemsetAsync(&h->d.ctl->status, 0, sizeof(int), st);
    cudaStreamSynchronize(st);
    return k.status;
  }
  return BD_OK;
}

int bd_get_state(bd_handle *h, double *xy, float *theta, uint8_t *species, int32_t *tri,
                 int32_t *n_tri, int64_t *step) {
  if (!h) return BD_ERR_ARG;
  cudaStream_t st = h->stream;
  const int np = h->np, n = h->n;
  cudaError_t e;
  if (xy) {
    std::vector<double2> pos(np);
    e = cudaMemcpyAsync(pos.data(), h->d.pos, np * sizeof(double2), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int i = 0; i < n; ++i) {
      double2 v = pos[h->int_of_ext[i]];
      xy[2 * i] = v.x;
      xy[2 * i + 1] = v.y;
    }
  }
  if (theta) {
    std::vector<float> t(np);
    e = cudaMemcpyAsync(t.data(), h->d.theta, np * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int i = 0; i < n; ++i) theta[i] = t[h->int_of_ext[i]];
  }
  if (species) {
    std::vector<uint8_t> s(np);
    e = cudaMemcpyAsync(s.data(), h->d.species, np, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int i = 0; i < n; ++i) species[i] = s[h->int_of_ext[i]];
  }
  if (tri) {
    std::vector<int4> tv(h->nt);
    e = cudaMemcpyAsync(tv.data(), h->d.tv, h->nt * sizeof(int4), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e);
    auto ext = [&](int v) { return v < np ? h->ext_of_int[v] : n + (v - np); };
    for (int t = 0; t < h->nt; ++t) {
      tri[3 * t] = ext(tv[t].x);
      tri[3 * t + 1] = ext(tv[t].y);
      tri[3 * t + 2] = ext(tv[t].z);
    }
  }
  if (n_tri) *n_tri = h->nt;
  if (step) *step = h->step;
  return BD_OK;
}

int bd_set_state(bd_handle *h, const double *xy, const float *theta) {
  if (!h || !xy) return BD_ERR_ARG;
  const int n = h->n, np = h->np;
  const BdConst &c = h->c;
  for (int i = 0; i < 2 * n; ++i)
    if (!isfinite(xy[i]) || xy[i] < c.a - 1e-9 * c.L || xy[i] > c.L - c.a + 1e-9 * c.L)
      return BD_ERR_INIT_OVERLAP;
  if (bdhost::any_overlap(n, xy, 0.0, c.L, c.sigma * (1.0 - 1e-12))) return BD_ERR_INIT_OVERLAP;
  for (int i = 0; i < n; ++i) {
    int k = h->int_of_ext[i];
    h->host_pos[2 * k] = std::min(c.wall_hi, std::max(c.wall_lo, snap_host(xy[2 * i], c.q, c.inv_q)));
    h->host_pos[2 * k + 1] = std::min(c.wall_hi, std::max(c.wall_lo, snap_host(xy[2 * i + 1], c.q, c.inv_q)));
  }
  cudaStream_t st = h->stream;
  const BdDev &d = h->d;
  cudaError_t e;
  e = cudaMemcpyAsync(d.pos0, d.pos, (size_t)np * sizeof(double2), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d.prev, d.pos, (size_t)np * sizeof(double2), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d.theta0, d.theta, (size_t)np * sizeof(float), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d.pos, h->host_pos.data(), (size_t)np * sizeof(double2), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && theta) {
    std::vector<float> th(np, 0.f);
    // keep the old directions of untouched slots: gather on the host
    e = cudaMemcpyAsync(th.data(), d.theta, (size_t)np * sizeof(float), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    for (int i = 0; i < n && e == cudaSuccess; ++i) th[h->int_of_ext[i]] = theta[i];
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.theta, th.data(), (size_t)np * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(d.moved, 1, (size_t)np, st);
  if (e == cudaSuccess) e = bd_launch_work_copy(d, c, st);
  if (e == cudaSuccess) e = reset_stats(h);
  if (e == cudaSuccess) e = bd_launch_dt(d, c, 1, st, h->dt_grid, h->dt_block);
  if (e != cudaSuccess) return cuda_fail(e);
  int rc = read_ctl(h);
  if (rc) return rc;
  if (h->h_ctl->status) {
    int s = h->h_ctl->status;
    cudaMemsetAsync(&h->d.ctl->status, 0, sizeof(int), st);
    cudaStreamSynchronize(st);
    return s;
  }
  return BD_OK;
}

int bd_compute_forces(bd_handle *h, double *F) {
  if (!h || !F) return BD_ERR_ARG;
  cudaStream_t st = h->stream;
  const int n = h->n, np = h->np;
  if (h->c.law == BD_LAW_NONE) {
    memset(F, 0, sizeof(double) * 2 * (size_t)n);
    return BD_OK;
  }
  cudaError_t e = h->c.law == BD_LAW_SHORT ? bd_launch_force_short(h->d, h->c, st)
                                           : bd_launch_force_long(h->d, h->c, st);
  if (e == cudaSuccess) e = bd_launch_force_sum(h->d, h->c, h->d_fsum, st);
  std::vector<double2> f(np);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f.data(), h->d_fsum, np * sizeof(double2), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  int rc = read_ctl(h);
  if (rc) return rc;
  if (h->h_ctl->status) {
    int s = h->h_ctl->status;
    cudaMemsetAsync(&h->d.ctl->status, 0, sizeof(int), st);
    cudaStreamSynchronize(st);
    return s;
  }
  for (int i = 0; i < n; ++i) {
    double2 v = f[h->int_of_ext[i]];
    F[2 * i] = v.x;
    F[2 * i + 1] = v.y;
  }
  return BD_OK;
}

int bd_get_neighbors(bd_handle *h, int32_t max_per, int32_t *counts, int32_t *idx) {
  if (!h || !counts || max_per < 0 || (max_per > 0 && !idx)) return BD_ERR_ARG;
  if (h->c.law != BD_LAW_SHORT) return BD_ERR_UNSUPPORTED;
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
  if (L) *L = h->c.L;
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

}  // extern "C"
