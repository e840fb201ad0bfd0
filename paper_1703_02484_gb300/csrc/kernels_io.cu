// State transfers between the caller's order and the internal slot order.
//
// The caller's positions and directions are copied to the device as they are
// (disk e of the concatenated replicas at index e) and permuted there: one
// thread per internal slot gathers its disk, checks it, rounds it to the
// position grid and stores it.  bd_get_state runs the inverse scatter and one
// copy per array to the caller.  The checks and roundings are the same
// operations, in the same order and precision, as the host's at bd_init, so a
// position set here is the one bd_init would have stored.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bd_internal.h"
#include "em.cuh"
#include "predicates.cuh"

namespace {

__device__ __forceinline__ double snap_grid(double v, const BdConst &c) {
  return __dmul_rn(rint(__dmul_rn(v, c.inv_q)), c.q);
}

// a periodic coordinate in [0, L) on the grid (L is a multiple of q)
__device__ __forceinline__ double periodic_grid(double v, double L, const BdConst &c) {
  double y = snap_grid(__dsub_rn(v, __dmul_rn(L, floor(__ddiv_rn(v, L)))), c);
  if (y >= L) y = __dsub_rn(y, L);
  if (y < 0.0) y = __dadd_rn(y, L);
  return y;
}

// a centre must be finite and, with walls, lie in [a, L - a] up to 1e-9 L
// (a_i for polydisperse disks).  Every slot first takes its snapshots (the
// start of the repair, and what a failed repair restores) and clears its
// moved flag.
__global__ void k_state_check(BdDev d, BdConst c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.np) return;
  const double2 o = d.pos[i];
  d.pos0[i] = o;
  d.prev[i] = o;
  d.theta0[i] = d.theta[i];
  d.moved[i] = 0;
  const int e = d.ext_glob[i];
  if (e < 0) return;
  const BdRep &R = d.rep[d.rep_of[i]];
  const double2 p = d.xfer_xy[e];
  bool bad = !isfinite(p.x) || !isfinite(p.y);
  if (!R.periodic) {
    const double tol = __dmul_rn(1e-9, R.L);
    const double ai = d.rad ? d.rad[i] : c.a;
    const double lo = __dsub_rn(ai, tol), hi = __dadd_rn(__dsub_rn(R.L, ai), tol);
    bad = bad || p.x < lo || p.x > hi || p.y < lo || p.y > hi;
  }
  if (bad) atomicCAS(&d.ctl->status, 0, BD_ERR_INIT_OVERLAP);
}

// store the checked positions (and directions) in slot order; nothing is
// written when any disk failed the check
__global__ void k_state_in(BdDev d, BdConst c, int with_theta) {
  if (*(volatile const int *)&d.ctl->status) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.np) return;
  const int e = d.ext_glob[i];
  if (e < 0) return;
  const BdRep &R = d.rep[d.rep_of[i]];
  const double2 p = d.xfer_xy[e];
  double2 y;
  if (R.periodic) {
    y = make_double2(periodic_grid(p.x, R.L, c), periodic_grid(p.y, R.L, c));
  } else {
    const double2 w = bdem::walls_of(d, R, i);
    y = make_double2(fmin(w.y, fmax(w.x, snap_grid(p.x, c))), fmin(w.y, fmax(w.x, snap_grid(p.y, c))));
  }
  {
    // the move from the previous positions, for the triangulation's FP32
    // reversal screen (exact grid difference, one rounding to FP32; in a
    // periodic box its minimum image, and a disk that crossed an edge has its
    // edges tested exactly)
    const double2 o = d.pos[i];
    const bdpred::Grid g{c.q, c.inv_q, c.qshift};
    long long mx = bdpred::to_int(y.x, g) - bdpred::to_int(o.x, g);
    long long my = bdpred::to_int(y.y, g) - bdpred::to_int(o.y, g);
    if (R.periodic) {
      const long long h = R.LQ / 2;
      mx = mx > h ? mx - R.LQ : (mx < -h ? mx + R.LQ : mx);
      my = my > h ? my - R.LQ : (my < -h ? my + R.LQ : my);
    }
    d.dmove[i] = make_float2(bdem::grid_to_float(mx, c.qshift), bdem::grid_to_float(my, c.qshift));
    // only disks that moved mark their triangles for the repair; a state
    // set back unchanged needs none
    const bool changed = (mx | my) != 0;
    d.moved[i] = changed ? 1 : 0;
    const unsigned m = __ballot_sync(__activemask(), changed);
    if (m && (int)(threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(&d.ctl->n_set_moved, __popc(m));
  }
  d.pos[i] = y;
  d.work[i] = bdem::split(y);   // the FP32 (hi, lo) copy the sweeps and filters read
  if (with_theta) d.theta[i] = d.xfer_th[e];
}

__global__ void k_state_out(BdDev d, BdConst c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.np) return;
  const int e = d.ext_glob[i];
  if (e < 0) return;
  d.xfer_xy[e] = d.pos[i];
  d.xfer_th[e] = d.theta[i];
  d.xfer_sp[e] = d.species[i];
}

}  // namespace

cudaError_t bd_launch_state_in(const BdDev &d, const BdConst &c, int with_theta, cudaStream_t s) {
  const int nb = (c.np + 255) / 256;
  k_state_check<<<nb, 256, 0, s>>>(d, c);
  k_state_in<<<nb, 256, 0, s>>>(d, c, with_theta);
  return cudaGetLastError();
}

cudaError_t bd_launch_state_out(const BdDev &d, const BdConst &c, cudaStream_t s) {
  k_state_out<<<(c.np + 255) / 256, 256, 0, s>>>(d, c);
  return cudaGetLastError();
}

// The noise of the time step for given Philox counters (diagnostics and tests
// of the generator): the raw words, and the clamped normals as the FP32 and
// the FP64 step form them.
__global__ void k_noise_sample(unsigned long long seed, unsigned replica, int n, const uint4 *ctr, uint4 *words,
                               float *z32, double *z64) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = ctr[i];
  bdrng::U4 u{c.x, c.y, c.z, c.w};
  const bdrng::U4 r = bdrng::philox(u, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32) ^ replica);
  words[i] = make_uint4(r.x, r.y, r.z, r.w);
  const float3 a = bdem::normals_f32(r);
  const double3 b = bdem::normals_f64(r);
  z32[3 * i] = a.x;
  z32[3 * i + 1] = a.y;
  z32[3 * i + 2] = a.z;
  z64[3 * i] = b.x;
  z64[3 * i + 1] = b.y;
  z64[3 * i + 2] = b.z;
}

cudaError_t bd_launch_noise_sample(unsigned long long seed, unsigned replica, int n, const void *ctr, void *words,
                                   float *z32, double *z64, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  k_noise_sample<<<(n + 255) / 256, 256, 0, s>>>(seed, replica, n, (const uint4 *)ctr, (uint4 *)words, z32, z64);
  return cudaGetLastError();
}
