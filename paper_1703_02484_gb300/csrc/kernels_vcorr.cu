// Overlap correction over the Verlet lists of the short-range force (the
// paper's short-range path, Sec. 5: no triangulation is maintained).
//
// Algorithm 2 (Sec. 4.4), each pass over every disk i and its list:
//   disp_i = - sum over listed j with r_ij < sigma of (sigma - r_ij) (r_j - r_i)/r_ij,
// then every disk moves by disp_i, scaled to length sigma/4 when longer, and
// reflects at the walls; passes repeat until no listed pair is closer than
// sigma.  Each disk gathers its own sum in list order (the lists are sorted
// and symmetric), so there are no atomics and the result is deterministic.
//
// Which pairs a pass must look at: a pair whose ends both stayed put since the
// previous pass keeps its distance, and was not overlapping then (every disk of
// an overlapping pair is flagged as moved, even when its displacements
// cancel).  So after the first pass (every disk moved by the integrator) only
// entries with a moved end are examined.  An FP32 screen of the squared
// distance (from the FP32 (hi, lo) position pairs, margin 1e-5) discards clearly
// separated pairs; the decision r < sigma itself is FP64, as in the oracle.
//
// The lists hold every pair within r_cut + skin of the positions at their
// build; a pair closer than sigma is in them while no disk has moved more than
// (r_cut + skin - sigma)/2 since.  A disk beyond that reach rejects the step
// (BD_ERR_STEP_REJECTED, fail_phase 6) instead of missing a pair.
//
// One persistent cooperative launch per step with bounded grid barriers, like
// the triangulation kernel; on failure the step is undone from its snapshot.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bd_internal.h"
#include "em.cuh"
#include "gridsync.cuh"

using namespace bdgs;

#define BD_VC_THREADS 256

namespace {

__device__ __forceinline__ float fdiff(float bh, float bl, float ah, float al) {
  return __fadd_rn(__fsub_rn(bh, ah), __fsub_rn(bl, al));
}

// the FP32 screen's coordinate difference; a pair across a periodic box edge
// (hi parts ~L apart, not exact in FP32) reports 0 and is decided exactly
__device__ __forceinline__ float fdiff_p(float bh, float bl, float ah, float al, const BdRep &R) {
  const float h = __fsub_rn(bh, ah);
  if (R.periodic && fabsf(h) > R.hLf) return 0.f;
  return __fadd_rn(h, __fsub_rn(bl, al));
}
__device__ __forceinline__ long long imin_image(long long d, const BdRep &R) {
  if (!R.periodic) return d;
  const long long h = R.LQ / 2;
  return d > h ? d - R.LQ : (d < -h ? d + R.LQ : d);
}

// lead thread only: charge the time since the last mark to a stage
__device__ __forceinline__ void stage_tick(BdCtl *ctl, int stage, unsigned long long &mark) {
  const unsigned long long now = gtimer();
  ctl->st_stage_ns[stage] += now - mark;
  ctl->st_stage_cnt[stage] += 1;
  mark = now;
}

}  // namespace

__global__ void __launch_bounds__(BD_VC_THREADS) k_overlap_verlet(BdDev d, BdConst c, int advance) {
  BdCtl *ctl = d.ctl;
  if (ld_status(&ctl->status) != 0) {
    block_exit(ctl);
    return;
  }
  Bar b;
  b.gen = 0;
  b.ph = 0;
  __shared__ int bc[BC_N];   // phase counters, per barrier
  unsigned long long t_mark = gtimer();
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const bool lead = (blockIdx.x == 0 && threadIdx.x == 0);
  const double sigma = c.sigma;
  const float sig2f = (float)(sigma * sigma * (1.0 + 1e-5));
  int status = 0, corr_iter = 0;
  // launch counter (this kernel's use of the epoch word): stamps of the
  // per-replica pass counts
  const unsigned long long lbase = ctl->epoch;
  long long st_overlap = 0;

  for (;;) {
    // ---------------- scan: every disk gathers its displacement ----------------
    phase_begin(ctl, b);
    {
      int nov = 0, stale = 0;
      double mx = 0.0;
      for (int i = tid; i < c.np; i += nth) {
        if (d.ext_id[i] < 0) continue;
        const bool mi = d.moved[i] != 0;
        const double2 pi = d.pos[i];
        const BdRep &R = d.rep[d.rep_of[i]];
        const bdpred::Grid g{c.q, c.inv_q, c.qshift};
        if (mi) {
          const double2 r0 = d.vl_ref[i];
          const double ex = bdem::grid_to_double(imin_image(bdpred::to_int(pi.x, g) - bdpred::to_int(r0.x, g), R), c.qshift);
          const double ey = bdem::grid_to_double(imin_image(bdpred::to_int(pi.y, g) - bdpred::to_int(r0.y, g), R), c.qshift);
          if (__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)) > c.vl_reach2) {
            ++stale;
            atomicExch(&ctl->st_fail_item, i);
          }
        }
        const float4 wi = d.work[i];
        const int m = d.vl_cnt[i];
        double sx = 0.0, sy = 0.0;
        uint8_t hit = 0;
        for (int t = 0; t < m; ++t) {
          const int j = d.vl_idx[(size_t)t * c.np + i];
          if (!mi && !d.moved[j]) continue;   // neither end moved since the last pass
          const float4 wj = d.work[j];
          const float fx = fdiff_p(wj.x, wj.z, wi.x, wi.z, R), fy = fdiff_p(wj.y, wj.w, wi.y, wi.w, R);
          if (__fadd_rn(__fmul_rn(fx, fx), __fmul_rn(fy, fy)) > sig2f) continue;
          const double2 pj = d.pos[j];
          // the exact difference (grid units), its minimum image in a periodic box
          const double dx = bdem::grid_to_double(imin_image(bdpred::to_int(pj.x, g) - bdpred::to_int(pi.x, g), R), c.qshift);
          const double dy = bdem::grid_to_double(imin_image(bdpred::to_int(pj.y, g) - bdpred::to_int(pi.y, g), R), c.qshift);
          const double r = sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
          const double sg = d.rad ? d.rad[i] + d.rad[j] : sigma;   // polydisperse: a_i + a_j
          if (r < sg) {
            const double del = sg - r;
            sx -= del * (dx / r);
            sy -= del * (dy / r);
            hit = 1;
            if (j > i) ++nov;      // each pair counted once
            mx = fmax(mx, del);
          }
        }
        d.disp[i] = make_double2(sx, sy);
        d.vc_hit[i] = hit;
      }
      block_add(cnt(ctl, b.ph, C_OVERLAP), nov);
      block_add(cnt(ctl, b.ph, C_REJECT), stale);
      if (mx > 0.0) atomicMax(&ctl->st_max_overlap_bits, (unsigned long long)__double_as_longlong(mx));
    }
    if (!grid_sync(ctl, b, bc)) { block_exit(ctl); return; }
    if (lead) stage_tick(ctl, 0, t_mark);
    const int n_rej = bc[BC_CNT + C_REJECT];
    const int n_ov = bc[BC_CNT + C_OVERLAP];
    if (n_rej) {
      status = BD_ERR_STEP_REJECTED;
      if (lead) { ctl->st_fail_phase = 6; ctl->st_fail_count = n_rej; }
      break;
    }
    if (advance < 0) {
      // positions set from outside: any pair closer than sigma rejects them
      if (n_ov) {
        status = BD_ERR_INIT_OVERLAP;
        if (lead) { ctl->st_fail_phase = 7; ctl->st_fail_count = n_ov; }
      }
      break;
    }
    if (n_ov == 0) break;
    if (corr_iter >= c.max_corr_iters) {
      status = BD_ERR_OVERLAP_NOT_CONVERGED;
      if (lead) ctl->st_fail_phase = 5;
      break;
    }
    ++corr_iter;
    st_overlap += n_ov;
    // ---------------- apply (capped at sigma/4), reflect ----------------
    phase_begin(ctl, b);
    {
      const double cap_eq = 0.25 * sigma;
      for (int i = tid; i < c.np; i += nth) {
        if (d.ext_id[i] < 0) continue;
        const double2 dd = d.disp[i];
        d.moved[i] = d.vc_hit[i];
        if (dd.x == 0.0 && dd.y == 0.0) continue;
        if (d.rep_stats) {
          // the first disk of a replica moved by this pass counts the pass
          const int rr = d.rep_of[i];
          // (launch, pass): launches are counted in 32 bits, passes below 2^31
          const unsigned long long stamp = ((lbase + 1ull) << 32) | (unsigned long long)corr_iter;
          if (atomicExch(&d.rep_mark[rr], stamp) != stamp)
            atomicAdd((unsigned long long *)&d.rep_stats[3 * rr], 1ull);
        }
        const double2 p = d.pos[i];
        d.prev[i] = p;
        const double mag = sqrt(__dadd_rn(__dmul_rn(dd.x, dd.x), __dmul_rn(dd.y, dd.y)));
        const double cap = d.rad ? 0.5 * d.rad[i] : cap_eq;   // half the disk's own radius
        const double sc = mag > cap ? cap / mag : 1.0;
        const double2 y = make_double2(bdem::snapd(__dadd_rn(p.x, __dmul_rn(dd.x, sc)), c.q, c.inv_q),
                                       bdem::snapd(__dadd_rn(p.y, __dmul_rn(dd.y, sc)), c.q, c.inv_q));
        int rfl = 0;
        const BdRep &R = d.rep[d.rep_of[i]];
        double2 pn;
        if (R.periodic) {
          const bdpred::Grid g{c.q, c.inv_q, c.qshift};
          long long X = bdpred::to_int(y.x, g), Y = bdpred::to_int(y.y, g);
          bdem::wrap_grid(R.LQ, X, Y);
          pn = make_double2(bdem::grid_to_double(X, c.qshift), bdem::grid_to_double(Y, c.qshift));
        } else {
          pn = bdem::reflect_w(bdem::walls_of(d, R, i), y, &rfl);
        }
        d.pos[i] = pn;
        d.work[i] = bdem::split(pn);
        d.moved[i] = 1;
      }
    }
    if (!grid_sync(ctl, b, bc)) { block_exit(ctl); return; }
    if (lead) stage_tick(ctl, 3, t_mark);
  }

  if (status) {
    // undo the step: positions and directions from the snapshot of the move
    phase_begin(ctl, b);
    for (int i = tid; i < c.np; i += nth) {
      if (d.ext_id[i] < 0) continue;
      const double2 p0 = d.pos0[i];
      d.pos[i] = p0;
      d.prev[i] = p0;
      d.work[i] = bdem::split(p0);
      d.theta[i] = d.theta0[i];
      d.disp[i] = make_double2(0.0, 0.0);
      d.moved[i] = 0;
    }
    if (lead) atomicCAS(&ctl->status, 0, status);
  }
  if (lead) {
    ctl->epoch = lbase + 1;
    ctl->st_corr_iters += corr_iter;
    ctl->st_overlap_pairs += st_overlap;
    ctl->st_barriers += b.gen;
    if (corr_iter > ctl->st_max_corr_iters) ctl->st_max_corr_iters = corr_iter;
    if (!status && advance > 0) {
      ctl->st_steps += 1;
      ctl->step_dev += 1;
    } else if (!status && advance == 0) {
      ctl->st_substeps += 1;
    }
  }
  block_exit(ctl);
}

int bd_vcorr_grid_for(int work_items, int *grid, int *block) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_overlap_verlet, BD_VC_THREADS, 0) != cudaSuccess)
    return -1;
  if (per < 1) return -1;
  int want = (work_items + BD_VC_THREADS - 1) / BD_VC_THREADS;
  if (want < 1) want = 1;
  *grid = want < sms * per ? want : sms * per;
  *block = BD_VC_THREADS;
  return 0;
}

cudaError_t bd_launch_overlap_verlet(const BdDev &d, const BdConst &c, cudaStream_t s, int grid, int block,
                                     int advance) {
  BdDev dd = d;
  BdConst cc = c;
  int adv = advance;
  void *args[] = {&dd, &cc, &adv};
  return cudaLaunchCooperativeKernel((const void *)k_overlap_verlet, dim3(grid), dim3(block), args, 0, s);
}
