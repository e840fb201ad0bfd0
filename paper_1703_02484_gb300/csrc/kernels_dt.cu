// Triangulation stages of one time step, as one persistent cooperative
// kernel (Algorithm 1 lines 5-7, Sec. 4.3-4.4):
//
//   A  validity (Sec. 4.3): r0_ij . r1_ij < 0 on any triangulation edge with a
//      moved end point rejects the step; every triangle with a moved corner is
//      re-oriented and flagged "inverted" when not strictly counter-clockwise.
//   R  inversion repair: an edge between an inverted triangle and its
//      neighbour is flipped when both triangles of the other diagonal come out
//      counter-clockwise -- the orientation form of Eq. (predicate) (the
//      moved vertex lies inside the neighbour's triangle, Fig. 4).  Rounds
//      repeat until no triangle is inverted; no candidate left => reject.
//   L  Lawson flips (Sec. 4.1, Navarro et al.): an edge whose opposite vertex
//      lies strictly inside the circumcircle of the other triangle is flipped;
//      rounds repeat until none is left.  Only edges touching a triangle that
//      moved or flipped are re-tested.
//   O  overlap correction (Algorithm 2): every real edge with r < sigma adds
//      -+ (sigma - r) r_hat to its end points' FP64 displacement (atomics); each
//      disk then moves by its sum capped at sigma/4 (Sec. 4.4) and reflects at
//      the walls.  Then A-R-L run again on the moved disks, and the loop ends
//      when a pass over the Delaunay edges of the current positions finds no
//      overlap (the closest pair of a point set is a Delaunay edge, so no pair
//      anywhere is closer than sigma).
//
// Parallel flips follow a claim / flip / re-link scheme: a candidate edge
// claims both its triangles with a 64-bit atomicMax of (round, edge id); an
// edge that holds both claims flips in place (the two triangle slots are
// reused), and a third phase re-links the outer neighbours, matching edges by
// their end points when a neighbour flipped in the same round.
//
// Grid-wide barriers spin with a time limit: a barrier that waits longer
// than BD_BARRIER_TIMEOUT_NS sets BD_ERR_DEVICE_TIMEOUT and every block leaves.
// On any failure the step is undone from the snapshot taken in phase A.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bd_internal.h"
#include "predicates.cuh"

#ifndef BD_BARRIER_TIMEOUT_NS
#define BD_BARRIER_TIMEOUT_NS 2000000000ull
#endif

#define BD_DT_THREADS 256

namespace {

struct Bar {
  unsigned gen;
  int ph;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_status(const int *p) {
  return *(volatile const int *)p;
}

// bounded grid barrier; returns false if the grid must stop
__device__ bool grid_sync(BdCtl *ctl, Bar &b) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    if (ld_status(&ctl->status) == BD_ERR_DEVICE_TIMEOUT) {
      ok = 0;
    } else {
      unsigned target = b.gen + 1;
      __threadfence();
      unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
      if (arrived == gridDim.x - 1) {
        atomicExch(&ctl->bar_count, 0u);
        __threadfence();
        atomicExch(&ctl->bar_gen, target);
      } else {
        unsigned long long t0 = gtimer();
        unsigned it = 0;
        while (ld_acquire(&ctl->bar_gen) != target) {
          if ((++it & 63u) == 0 && gtimer() - t0 > BD_BARRIER_TIMEOUT_NS) {
            atomicExch(&ctl->status, BD_ERR_DEVICE_TIMEOUT);
            ok = 0;
            break;
          }
          __nanosleep(40);
        }
      }
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  b.gen++;
  b.ph++;
  return s_ok != 0;
}

__device__ __forceinline__ int *cnt(BdCtl *ctl, int ph, int slot) { return &ctl->cnt[ph & 3][slot]; }

// reset the counters two phases ahead (see the rotation argument in BdCtl)
__device__ __forceinline__ void phase_begin(BdCtl *ctl, const Bar &b) {
  if (blockIdx.x == 0 && threadIdx.x < 8) ctl->cnt[(b.ph + 2) & 3][threadIdx.x] = 0;
}

// block-aggregated atomic add
__device__ __forceinline__ void block_add(int *dst, int v) {
  __shared__ int s_acc;
  if (threadIdx.x == 0) s_acc = 0;
  __syncthreads();
  // warp reduce
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_acc, v);
  __syncthreads();
  if (threadIdx.x == 0 && s_acc) atomicAdd(dst, s_acc);
}

__device__ __forceinline__ int vk(const int4 &v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }
__device__ __forceinline__ void set_vk(int4 &v, int k, int val) {
  if (k == 0) v.x = val; else if (k == 1) v.y = val; else v.z = val;
}

struct Ctx {
  BdDev d;
  BdConst c;
  bdpred::Grid g;
  int T;
  int np;
};

__device__ __forceinline__ int orient_v(const Ctx &x, int a, int b, int c) {
  double2 pa = x.d.pos[a], pb = x.d.pos[b], pc = x.d.pos[c];
  return bdpred::orient(pa.x, pa.y, pb.x, pb.y, pc.x, pc.y, x.g);
}

__device__ __forceinline__ int incircle_v(const Ctx &x, int a, int b, int c, int p) {
  double2 pa = x.d.pos[a], pb = x.d.pos[b], pc = x.d.pos[c], pp = x.d.pos[p];
  return bdpred::incircle(pa.x, pa.y, pb.x, pb.y, pc.x, pc.y, pp.x, pp.y, x.g);
}

__device__ __forceinline__ double snap(double v, const bdpred::Grid &g) {
  return __dmul_rn(rint(__dmul_rn(v, g.inv_q)), g.q);
}

__device__ __forceinline__ float4 split_pos(double2 p) {
  float xh = __double2float_rn(p.x), yh = __double2float_rn(p.y);
  return make_float4(xh, yh, __double2float_rn(p.x - (double)xh), __double2float_rn(p.y - (double)yh));
}

// flip the edge facing corner c0 (corner table, in place); returns the two
// triangle ids.  Outer-neighbour entries of the two triangles are copied from
// their old slots; the re-link phase makes them consistent.
__device__ void flip_edge(const Ctx &x, int c0, int o0, int &t0, int &t1) {
  t0 = c0 / 3;
  int k0 = c0 % 3;
  t1 = o0 / 3;
  int k1 = o0 % 3;
  int4 V0 = x.d.tv[t0], V1 = x.d.tv[t1], N0 = x.d.tn[t0], N1 = x.d.tn[t1];
  int a = vk(V0, k0), b = vk(V0, (k0 + 1) % 3), c = vk(V0, (k0 + 2) % 3), dd = vk(V1, k1);
  int n_ca = vk(N0, (k0 + 1) % 3), n_ab = vk(N0, (k0 + 2) % 3);
  int n_bd = vk(N1, (k1 + 1) % 3), n_dc = vk(N1, (k1 + 2) % 3);
  set_vk(V0, k0, b);
  set_vk(V0, (k0 + 1) % 3, dd);
  set_vk(V0, (k0 + 2) % 3, a);
  set_vk(V1, k1, c);
  set_vk(V1, (k1 + 1) % 3, a);
  set_vk(V1, (k1 + 2) % 3, dd);
  set_vk(N0, k0, 3 * t1 + k1);
  set_vk(N0, (k0 + 1) % 3, n_ab);
  set_vk(N0, (k0 + 2) % 3, n_bd);
  set_vk(N1, k1, 3 * t0 + k0);
  set_vk(N1, (k1 + 1) % 3, n_dc);
  set_vk(N1, (k1 + 2) % 3, n_ca);
  V0.w = BD_TRI_DIRTY;
  V1.w = BD_TRI_DIRTY;
  x.d.tv[t0] = V0;
  x.d.tv[t1] = V1;
  x.d.tn[t0] = N0;
  x.d.tn[t1] = N1;
}

// re-link the outer neighbours of a triangle flipped in round `epoch`
__device__ void relink(const Ctx &x, int t, unsigned long long epoch) {
  int4 V = x.d.tv[t];
  int4 N = x.d.tn[t];
  int partner = (int)(x.d.partner[t] & 0xFFFFFFFFull);
  bool changed = false;
  for (int k = 0; k < 3; ++k) {
    int o = vk(N, k);
    if (o < 0) continue;
    int tt = o / 3;
    if (tt == partner) continue;  // the new diagonal, already consistent
    int u = vk(V, (k + 1) % 3), w = vk(V, (k + 2) % 3);
    unsigned long long pw = x.d.partner[tt];
    if ((pw >> 32) != epoch) {
      // neighbour unchanged: its corner index is still valid; point it back
      int *slot = ((int *)&x.d.tn[tt]) + (o % 3);
      *slot = 3 * t + k;
    } else {
      // neighbour flipped too: find the triangle and corner now facing edge (w, u)
      int cand[2] = {tt, (int)(pw & 0xFFFFFFFFull)};
      for (int s = 0; s < 2; ++s) {
        int4 W = x.d.tv[cand[s]];
        for (int j = 0; j < 3; ++j) {
          if (vk(W, (j + 1) % 3) == w && vk(W, (j + 2) % 3) == u) {
            set_vk(N, k, 3 * cand[s] + j);
            changed = true;
          }
        }
      }
    }
  }
  if (changed) x.d.tn[t] = N;
}

}  // namespace

// mode 0: full step after the integrator; mode 1: repair + Lawson only
__global__ void __launch_bounds__(BD_DT_THREADS) k_triangulation(BdDev d, BdConst c, int mode) {
  Ctx x;
  x.d = d;
  x.c = c;
  x.g.q = c.q;
  x.g.inv_q = c.inv_q;
  x.T = c.nt;
  x.np = c.np;
  BdCtl *ctl = d.ctl;
  if (ld_status(&ctl->status) != 0) return;
  Bar b;
  b.gen = 0;
  b.ph = 0;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const bool lead = (blockIdx.x == 0 && threadIdx.x == 0);
  unsigned long long epoch = ctl->epoch;   // written only at kernel end by the lead thread
  const double sigma = c.sigma;
  int status = 0;
  int corr_iter = 0;
  long long st_overlap = 0, st_flips = 0, st_rflips = 0, st_inv = 0, st_rounds = 0;
  bool first = true;

  for (;;) {
    // ---------------- A: validity ----------------
    phase_begin(ctl, b);
    {
      int inv = 0, rej = 0;
      for (int t = tid; t < x.T; t += nth) {
        int4 v = d.tv[t];
        int4 nn = d.tn[t];
        if (first) {
          int4 vs = v;
          vs.w = 0;
          d.tv_snap[t] = vs;
          d.tn_snap[t] = nn;
        }
        bool dirty = d.moved[v.x] | d.moved[v.y] | d.moved[v.z];
        if (dirty) {
          int o = orient_v(x, v.x, v.y, v.z);
          int fl = BD_TRI_DIRTY | (o <= 0 ? BD_TRI_INVERTED : 0);
          inv += (o <= 0);
          d.tv[t].w = fl;
        }
        // Sec. 4.3 first criterion on edges with a moved end point
        for (int k = 0; k < 3; ++k) {
          int cc = 3 * t + k;
          int o = vk(nn, k);
          if (o <= cc) continue;
          int u = vk(v, (k + 1) % 3), w = vk(v, (k + 2) % 3);
          if (u >= x.np || w >= x.np) continue;
          if (!(d.moved[u] | d.moved[w])) continue;
          double2 a0 = d.prev[u], b0 = d.prev[w], a1 = d.pos[u], b1 = d.pos[w];
          double r0x = b0.x - a0.x, r0y = b0.y - a0.y, r1x = b1.x - a1.x, r1y = b1.y - a1.y;
          if (r0x * r1x + r0y * r1y < 0.0) {
            rej++;
            atomicExch(&ctl->st_fail_item, cc);
          }
        }
      }
      block_add(cnt(ctl, b.ph, C_INV), inv);
      block_add(cnt(ctl, b.ph, C_REJECT), rej);
    }
    first = false;
    if (!grid_sync(ctl, b)) return;
    int n_inv = *(volatile int *)cnt(ctl, b.ph - 1, C_INV);
    int n_rej = *(volatile int *)cnt(ctl, b.ph - 1, C_REJECT);
    st_inv += n_inv;
    if (n_rej) {
      status = BD_ERR_STEP_REJECTED;
      if (lead) { ctl->st_fail_phase = 1; ctl->st_fail_count = n_rej; }
      break;
    }

    // ---------------- R: inversion repair ----------------
    int rounds = 0;
    while (n_inv > 0) {
      if (rounds++ >= c.max_flip_rounds) {
        status = BD_ERR_STEP_REJECTED;
        if (lead) { ctl->st_fail_phase = 3; ctl->st_fail_count = n_inv; }
        break;
      }
      ++epoch;
      // RM: candidates
      phase_begin(ctl, b);
      {
        int ncand = 0;
        for (int t = tid; t < x.T; t += nth) {
          int4 v = d.tv[t];
          if (!(v.w & BD_TRI_INVERTED)) continue;
          atomicExch(&ctl->st_fail_item, t);
          int4 nn = d.tn[t];
          for (int k = 0; k < 3; ++k) {
            int o = vk(nn, k);
            if (o < 0) continue;
            int p = vk(v, k), u = vk(v, (k + 1) % 3), w = vk(v, (k + 2) % 3);
            int4 v1 = d.tv[o / 3];
            int q = vk(v1, o % 3);
            if (orient_v(x, u, q, p) > 0 && orient_v(x, w, p, q) > 0) {
              int cm = min(3 * t + k, o);
              unsigned long long key = (epoch << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)cm);
              atomicMax(&d.claim[t], key);
              atomicMax(&d.claim[o / 3], key);
              ++ncand;
            }
          }
        }
        block_add(cnt(ctl, b.ph, C_CAND), ncand);
      }
      if (!grid_sync(ctl, b)) return;
      int n_cand = *(volatile int *)cnt(ctl, b.ph - 1, C_CAND);
      if (n_cand == 0) {
        status = BD_ERR_STEP_REJECTED;
        if (lead) { ctl->st_fail_phase = 2; ctl->st_fail_count = n_inv; }
        break;
      }
      // RF: winners flip
      phase_begin(ctl, b);
      {
        int nf = 0;
        for (int t = tid; t < x.T; t += nth) {
          unsigned long long key = d.claim[t];
          if ((key >> 32) != epoch) continue;
          int cm = (int)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull));
          if (cm / 3 != t) continue;
          int o = ((const int *)&d.tn[t])[cm % 3];
          if (d.claim[o / 3] != key) continue;
          int t0, t1;
          flip_edge(x, cm, o, t0, t1);
          d.partner[t0] = (epoch << 32) | (unsigned)t1;
          d.partner[t1] = (epoch << 32) | (unsigned)t0;
          int4 V0 = d.tv[t0], V1 = d.tv[t1];
          if (orient_v(x, V0.x, V0.y, V0.z) <= 0) d.tv[t0].w = BD_TRI_DIRTY | BD_TRI_INVERTED;
          if (orient_v(x, V1.x, V1.y, V1.z) <= 0) d.tv[t1].w = BD_TRI_DIRTY | BD_TRI_INVERTED;
          ++nf;
        }
        block_add(cnt(ctl, b.ph, C_FLIPS), nf);
      }
      if (!grid_sync(ctl, b)) return;
      st_rflips += *(volatile int *)cnt(ctl, b.ph - 1, C_FLIPS);
      // RX: re-link and recount
      phase_begin(ctl, b);
      {
        int inv = 0;
        for (int t = tid; t < x.T; t += nth) {
          if ((d.partner[t] >> 32) == epoch) relink(x, t, epoch);
          inv += (d.tv[t].w & BD_TRI_INVERTED) ? 1 : 0;
        }
        block_add(cnt(ctl, b.ph, C_INV), inv);
      }
      if (!grid_sync(ctl, b)) return;
      n_inv = *(volatile int *)cnt(ctl, b.ph - 1, C_INV);
    }
    if (status) break;

    // ---------------- L: Lawson flips ----------------
    rounds = 0;
    for (;;) {
      if (rounds++ >= c.max_flip_rounds) {
        status = BD_ERR_FLIP_NOT_CONVERGED;
        if (lead) ctl->st_fail_phase = 4;
        break;
      }
      ++epoch;
      phase_begin(ctl, b);
      for (int t = tid; t < x.T; t += nth) {
        int4 v = d.tv[t];
        int4 nn = d.tn[t];
        for (int k = 0; k < 3; ++k) {
          int cc = 3 * t + k;
          int o = vk(nn, k);
          if (o <= cc) continue;
          int4 v1 = d.tv[o / 3];
          if (!((v.w | v1.w) & BD_TRI_DIRTY)) continue;
          int q = vk(v1, o % 3);
          if (incircle_v(x, v.x, v.y, v.z, q) > 0) {
            unsigned long long key = (epoch << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)cc);
            atomicMax(&d.claim[t], key);
            atomicMax(&d.claim[o / 3], key);
          }
        }
      }
      if (!grid_sync(ctl, b)) return;
      phase_begin(ctl, b);
      {
        int nf = 0;
        for (int t = tid; t < x.T; t += nth) {
          unsigned long long key = d.claim[t];
          if ((key >> 32) == epoch) {
            // claimed this round: either this triangle's edge flips, or it
            // stays dirty so a losing illegal edge is tested again next round
            int cm = (int)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull));
            if (cm / 3 == t) {
              int o = ((const int *)&d.tn[t])[cm % 3];
              if (d.claim[o / 3] == key) {
                int t0, t1;
                flip_edge(x, cm, o, t0, t1);
                d.partner[t0] = (epoch << 32) | (unsigned)t1;
                d.partner[t1] = (epoch << 32) | (unsigned)t0;
                ++nf;
              }
            }
          } else if (d.tv[t].w & BD_TRI_DIRTY) {
            // every edge of this triangle was tested and found legal
            d.tv[t].w = 0;
          }
        }
        block_add(cnt(ctl, b.ph, C_FLIPS), nf);
      }
      if (!grid_sync(ctl, b)) return;
      int nf = *(volatile int *)cnt(ctl, b.ph - 1, C_FLIPS);
      if (nf == 0) break;
      st_flips += nf;
      st_rounds += 1;
      phase_begin(ctl, b);
      for (int t = tid; t < x.T; t += nth)
        if ((d.partner[t] >> 32) == epoch) relink(x, t, epoch);
      if (!grid_sync(ctl, b)) return;
    }
    if (status) break;
    if (mode == 1) break;

    // ---------------- O: overlap scan ----------------
    phase_begin(ctl, b);
    {
      int nov = 0;
      double mx = 0.0;
      for (int i = tid; i < x.np; i += nth) d.moved[i] = 0;
      for (int t = tid; t < x.T; t += nth) {
        int4 v = d.tv[t];
        int4 nn = d.tn[t];
        for (int k = 0; k < 3; ++k) {
          int cc = 3 * t + k;
          int o = vk(nn, k);
          if (o <= cc) continue;
          int u = vk(v, (k + 1) % 3), w = vk(v, (k + 2) % 3);
          if (u >= x.np || w >= x.np) continue;
          double2 pu = d.pos[u], pw = d.pos[w];
          double dx = __dsub_rn(pw.x, pu.x), dy = __dsub_rn(pw.y, pu.y);
          double r = sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
          if (r < sigma) {
            double del = sigma - r;
            double nx = dx / r, ny = dy / r;
            atomicAdd(&d.disp[u].x, -del * nx);
            atomicAdd(&d.disp[u].y, -del * ny);
            atomicAdd(&d.disp[w].x, del * nx);
            atomicAdd(&d.disp[w].y, del * ny);
            ++nov;
            mx = fmax(mx, del);
          }
        }
      }
      block_add(cnt(ctl, b.ph, C_OVERLAP), nov);
      if (mx > 0.0) atomicMax(&ctl->st_max_overlap_bits, (unsigned long long)__double_as_longlong(mx));
    }
    if (!grid_sync(ctl, b)) return;
    int n_ov = *(volatile int *)cnt(ctl, b.ph - 1, C_OVERLAP);
    if (n_ov == 0) break;
    st_overlap += n_ov;
    if (corr_iter >= c.max_corr_iters) {
      status = BD_ERR_OVERLAP_NOT_CONVERGED;
      if (lead) ctl->st_fail_phase = 5;
      break;
    }
    ++corr_iter;
    // ---------------- O: apply (capped at sigma/4) ----------------
    phase_begin(ctl, b);
    {
      const double cap = 0.25 * sigma;
      for (int i = tid; i < x.np; i += nth) {
        if (d.ext_id[i] < 0) continue;
        double2 p = d.pos[i];
        d.prev[i] = p;
        double2 dd = d.disp[i];
        if (dd.x == 0.0 && dd.y == 0.0) continue;
        double mag = sqrt(__dadd_rn(__dmul_rn(dd.x, dd.x), __dmul_rn(dd.y, dd.y)));
        double s = mag > cap ? cap / mag : 1.0;
        double nxp = snap(p.x + dd.x * s, x.g), nyp = snap(p.y + dd.y * s, x.g);
        if (nxp < c.wall_lo) nxp = 2.0 * c.wall_lo - nxp;
        if (nxp > c.wall_hi) nxp = 2.0 * c.wall_hi - nxp;
        if (nyp < c.wall_lo) nyp = 2.0 * c.wall_lo - nyp;
        if (nyp > c.wall_hi) nyp = 2.0 * c.wall_hi - nyp;
        double2 np2 = make_double2(nxp, nyp);
        d.pos[i] = np2;
        d.work[i] = split_pos(np2);
        d.disp[i] = make_double2(0.0, 0.0);
        d.moved[i] = 1;
      }
    }
    if (!grid_sync(ctl, b)) return;
  }

  if (status) {
    // undo the step: positions, directions and triangulation from the snapshot
    phase_begin(ctl, b);
    for (int i = tid; i < x.np; i += nth) {
      if (d.ext_id[i] < 0) continue;
      double2 p0 = d.pos0[i];
      d.pos[i] = p0;
      d.prev[i] = p0;
      d.work[i] = split_pos(p0);
      d.theta[i] = d.theta0[i];
      d.disp[i] = make_double2(0.0, 0.0);
      d.moved[i] = 0;
    }
    for (int t = tid; t < x.T; t += nth) {
      d.tv[t] = d.tv_snap[t];
      d.tn[t] = d.tn_snap[t];
    }
    if (lead) atomicCAS(&ctl->status, 0, status);
  } else {
    for (int i = tid; i < x.np; i += nth) d.moved[i] = 0;
  }
  if (lead) {
    ctl->epoch = epoch + 1;
    ctl->st_corr_iters += corr_iter;
    ctl->st_overlap_pairs += st_overlap;
    ctl->st_flips += st_flips;
    ctl->st_repair_flips += st_rflips;
    ctl->st_inverted += st_inv;
    ctl->st_flip_rounds += st_rounds;
    if (corr_iter > ctl->st_max_corr_iters) ctl->st_max_corr_iters = corr_iter;
    if (!status) ctl->st_steps += 1;
  }
}

int bd_dt_grid(int *grid, int *block) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_triangulation, BD_DT_THREADS, 0) !=
      cudaSuccess)
    return -1;
  if (per < 1) return -1;
  *grid = sms * per;
  *block = BD_DT_THREADS;
  return 0;
}

cudaError_t bd_launch_dt(const BdDev &d, const BdConst &c, int mode, cudaStream_t s, int grid,
                         int block) {
  // fresh barrier state for this launch
  cudaError_t e = cudaMemsetAsync(d.ctl, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(&d.ctl->cnt[0][0], 0, sizeof(d.ctl->cnt), s);
  if (e != cudaSuccess) return e;
  BdDev dd = d;
  BdConst cc = c;
  int m = mode;
  void *args[] = {&dd, &cc, &m};
  return cudaLaunchCooperativeKernel((const void *)k_triangulation, dim3(grid), dim3(block), args,
                                     0, s);
}
