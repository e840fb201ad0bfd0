// Adjoint of a rollout of the time step (reverse mode), for gradients of a
// loss of the final positions with respect to the pair-force table A (Sec.
// 2.2) and the self-propulsion speed v0 (Sec. 7).  No counterpart in the
// paper.
//
// The differentiated map is the step with its random and discrete choices
// frozen: the Philox noise, the wall reflections of every move, the
// overlapping pairs of every correction pass (Algorithm 2) and which disks
// had their displacement capped at sigma/4.  One step is
//   y   = R0( x + dt (F(x; A) + v0 e(theta)) + amp xi )          (Eq. (integration))
//   z_1 = y,   z_{j+1} = Rj( z_j + cap_j( d_j(z_j) ) )           (Algorithm 2 passes)
//   d_j(z)_u = -sum (sigma - r) r_hat,  d_j(z)_w = +sum (sigma - r) r_hat over the logged
//   pairs (u, w) of pass j, r_hat = (z_w - z_u)/r;  cap(d) = d or (sigma/4) d/|d|.
// Rounding to the position grid is taken as the identity.
//
// Backward through one pass: mu = R^T lambda (a reflected component changes
// sign); mu_d = cap'^T mu (for a capped disk (s/|d|)(I - d_hat d_hat^T) mu);
// lambda <- mu + sum over pairs G (mu_d_u - mu_d_w) at u and its negative at w,
// with G = d/dv [(sigma - |v|) v/|v|] = (sigma/r)(I - n n^T) - I.
// Backward through the move: mu = R0^T lambda; lambda <- mu + dt (dF/dx)^T mu,
//   ((dF/dx)^T mu)_i = sum_j M(r_ij) (A_ij mu_i - A_ji mu_j),  M(r) = I/r^3 - 3 r r^T/r^5,
// and the parameter gradients dL/dA_ab += dt sum_{i in a} mu_i . sum_{j in b} r_ij/r_ij^3,
// dL/dv0 += dt sum_i mu_i . e(theta_i).
// Pair terms are computed in FP32; every accumulation is FP64.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bd_internal.h"
#include "em.cuh"

namespace {

__device__ __forceinline__ double atomic_add_d(double *p, double v) { return atomicAdd(p, v); }

}  // namespace

// ---------------------------------------------------------------- replay

// Euler-Maruyama move with the logged reflections (the forces are in fpart)
__global__ void k_rp_em(BdDev d, BdConst c, long long step, int k_local) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.np) return;
  const int e = d.ext_id[i];
  if (e < 0) return;
  const BdRep &R = d.rep[d.rep_of[i]];
  const double2 F = bdem::force_sum(d, c, R, i);
  const double2 p = d.pos[i];
  const float th = d.theta[i];
  float thn;
  const double2 y = bdem::em_move(c, R, (uint32_t)e, step, p, th, F, R.v0, &thn);
  const double2 pn = bdem::reflect_as(R, y, d.log_refl[(size_t)k_local * c.np + i]);
  d.pos[i] = pn;
  d.work[i] = bdem::split(pn);
  d.theta[i] = thn;
}

// displacements of a logged pass at the current positions (disp must be zero)
__global__ void k_rp_disp(BdDev d, BdConst c, int pair_begin, int pair_end) {
  const int k = pair_begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= pair_end) return;
  const int2 pr = d.log_pairs[k];
  const double2 pu = d.pos[pr.x], pw = d.pos[pr.y];
  const double dx = __dsub_rn(pw.x, pu.x), dy = __dsub_rn(pw.y, pu.y);
  const double r = sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
  const double del = c.sigma - r;
  const double nx = dx / r, ny = dy / r;
  atomic_add_d(&d.disp[pr.x].x, -del * nx);
  atomic_add_d(&d.disp[pr.x].y, -del * ny);
  atomic_add_d(&d.disp[pr.y].x, del * nx);
  atomic_add_d(&d.disp[pr.y].y, del * ny);
}

// apply a logged pass: cap where the log says so, move, reflect as logged
__global__ void k_rp_apply(BdDev d, BdConst c, int pass) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.np || d.ext_id[i] < 0) return;
  const int f = d.log_pflags[(size_t)pass * c.np + i];
  const double2 dd = d.disp[i];
  if (dd.x == 0.0 && dd.y == 0.0 && f == 0) return;
  const double cap = 0.25 * c.sigma;
  const double mag = sqrt(__dadd_rn(__dmul_rn(dd.x, dd.x), __dmul_rn(dd.y, dd.y)));
  const double sc = (f & 16) ? cap / mag : 1.0;
  const double2 p = d.pos[i];
  const double2 y = make_double2(bdem::snapd(__dadd_rn(p.x, __dmul_rn(dd.x, sc)), c.q, c.inv_q),
                                 bdem::snapd(__dadd_rn(p.y, __dmul_rn(dd.y, sc)), c.q, c.inv_q));
  const double2 pn = bdem::reflect_as(d.rep[d.rep_of[i]], y, f & 15);
  d.pos[i] = pn;
  d.work[i] = bdem::split(pn);
  d.disp[i] = make_double2(0.0, 0.0);
}

// ---------------------------------------------------------------- backward

// pass, part 1: mu = R^T lambda; mu_d = cap'^T mu (disp holds d_j(z_j)); lambda = mu
__global__ void k_vjp_pass_mu(BdDev d, BdConst c, int pass, double2 *lam, double2 *mud) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.np || d.ext_id[i] < 0) return;
  const int f = d.log_pflags[(size_t)pass * c.np + i];
  double2 mu = lam[i];
  if (((f & 1) != 0) != ((f & 2) != 0)) mu.x = -mu.x;   // an odd number of mirrors
  if (((f & 4) != 0) != ((f & 8) != 0)) mu.y = -mu.y;
  lam[i] = mu;
  double2 md = mu;
  if (f & 16) {
    const double2 dd = d.disp[i];
    const double m = sqrt(dd.x * dd.x + dd.y * dd.y);
    const double ux = dd.x / m, uy = dd.y / m;
    const double s = 0.25 * c.sigma / m;
    const double dot = ux * mu.x + uy * mu.y;
    md = make_double2(s * (mu.x - dot * ux), s * (mu.y - dot * uy));
  }
  mud[i] = md;
}

// pass, part 2: pair terms lambda_u += G (mu_d_u - mu_d_w), lambda_w -= the same
__global__ void k_vjp_pass_pairs(BdDev d, BdConst c, const double2 *z, int pair_begin, int pair_end,
                                 double2 *lam, const double2 *mud) {
  const int k = pair_begin + blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= pair_end) return;
  const int2 pr = d.log_pairs[k];
  const double2 pu = z[pr.x], pw = z[pr.y];
  const double vx = pw.x - pu.x, vy = pw.y - pu.y;
  const double r = sqrt(vx * vx + vy * vy);
  const double nx = vx / r, ny = vy / r;
  const double a = c.sigma / r;
  // G = a (I - n n^T) - I
  const double gxx = a * (1.0 - nx * nx) - 1.0, gyy = a * (1.0 - ny * ny) - 1.0, gxy = -a * nx * ny;
  const double wx = mud[pr.x].x - mud[pr.y].x, wy = mud[pr.x].y - mud[pr.y].y;
  const double tx = gxx * wx + gxy * wy, ty = gxy * wx + gyy * wy;
  atomic_add_d(&lam[pr.x].x, tx);
  atomic_add_d(&lam[pr.x].y, ty);
  atomic_add_d(&lam[pr.y].x, -tx);
  atomic_add_d(&lam[pr.y].y, -ty);
}

// move, part 1: mu = R0^T lambda (in place)
__global__ void k_vjp_em_refl(BdDev d, BdConst c, int k_local, double2 *lam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.np || d.ext_id[i] < 0) return;
  const int f = d.log_refl[(size_t)k_local * c.np + i];
  double2 mu = lam[i];
  if (((f & 1) != 0) != ((f & 2) != 0)) mu.x = -mu.x;
  if (((f & 4) != 0) != ((f & 8) != 0)) mu.y = -mu.y;
  lam[i] = mu;
}

// move, part 2: all-pairs force adjoint over one chunk of j (blockIdx.y).
// x, th: positions and directions at the step start; mu = R0^T lambda.
// jpart[chunk][i] = sum over the chunk's j of M(r_ij)(A_ij mu_i - A_ji mu_j);
// gpart[block][0..3] = sum over the block's i of mu_i . S_{i,b} sorted by
// (s_i, b), gpart[block][4] = sum mu_i . e(theta_i) (chunk 0 only).  Partial
// sums are reduced in a fixed order by k_vjp_force_sum and k_vjp_grad_sum.
// A single-system handle only: every slot is one system's disk.
__global__ void __launch_bounds__(BD_ADJ_T) k_vjp_force(BdDev d, BdConst c, const double2 *x,
                                                        const float *th, const double2 *mu,
                                                        int jchunk, double2 *jpart, double *gpart) {
  __shared__ float4 sx[BD_ADJ_T];
  __shared__ float2 smu[BD_ADJ_T];
  __shared__ int ssp[BD_ADJ_T];
  __shared__ double sg[5];
  if (threadIdx.x < 5) sg[threadIdx.x] = 0.0;
  const int i = blockIdx.x * BD_ADJ_T + threadIdx.x;
  const bool live = i < c.np && d.ext_id[i] >= 0;
  const BdRep &R = d.rep[0];
  const float4 xi = live ? bdem::split(x[i]) : make_float4(1e18f, 1e18f, 0.f, 0.f);
  const double2 mui_d = live ? mu[i] : make_double2(0.0, 0.0);
  const float2 mui = make_float2((float)mui_d.x, (float)mui_d.y);
  const int si = live ? (d.species[i] ? 1 : 0) : 0;
  const float ai0 = R.alpha[BD_MAX_SPECIES * si], ai1 = R.alpha[BD_MAX_SPECIES * si + 1];
  double jx = 0.0, jy = 0.0, s0x = 0.0, s0y = 0.0, s1x = 0.0, s1y = 0.0;
  const int jb = blockIdx.y * jchunk, je = min(c.np, jb + jchunk);
  for (int j0 = jb; j0 < je; j0 += BD_ADJ_T) {
    const int j = j0 + threadIdx.x;
    const bool okj = j < je && d.ext_id[j] >= 0;
    sx[threadIdx.x] = okj ? bdem::split(x[j]) : make_float4(1e18f, 1e18f, 0.f, 0.f);
    const double2 mj = okj ? mu[j] : make_double2(0.0, 0.0);
    smu[threadIdx.x] = make_float2((float)mj.x, (float)mj.y);
    ssp[threadIdx.x] = okj ? (d.species[j] ? 1 : 0) : 0;
    __syncthreads();
    float ajx = 0.f, ajy = 0.f, t0x = 0.f, t0y = 0.f, t1x = 0.f, t1y = 0.f;
    const int m = min(BD_ADJ_T, je - j0);
    for (int k = 0; k < m; ++k) {
      const float4 xj = sx[k];
      const float rx = __fadd_rn(__fsub_rn(xi.x, xj.x), __fsub_rn(xi.z, xj.z));
      const float ry = __fadd_rn(__fsub_rn(xi.y, xj.y), __fsub_rn(xi.w, xj.w));
      const float r2 = fmaf(rx, rx, fmaf(ry, ry, 1e-20f));
      const float ir = rsqrtf(r2);
      const float ir2 = ir * ir;               // finite: 1e20 for j = i, where r = 0
      // 1/r^3, and 0 for j = i (distinct disks never share a position)
      const float q3 = (rx == 0.f && ry == 0.f) ? 0.f : ir2 * ir;
      const int sj = ssp[k];
      const float aij = sj ? ai1 : ai0;
      const float aji = R.alpha[BD_MAX_SPECIES * sj + si];
      // w = A_ij mu_i - A_ji mu_j;  M w = (w - 3 r (r . w)/r^2) / r^3
      const float wx = aij * mui.x - aji * smu[k].x, wy = aij * mui.y - aji * smu[k].y;
      const float rw = (rx * wx + ry * wy) * ir2;
      ajx += (wx - 3.f * rx * rw) * q3;
      ajy += (wy - 3.f * ry * rw) * q3;
      const float gx = rx * q3, gy = ry * q3;  // r_ij / r^3
      if (sj) {
        t1x += gx;
        t1y += gy;
      } else {
        t0x += gx;
        t0y += gy;
      }
    }
    jx += ajx;
    jy += ajy;
    s0x += t0x;
    s0y += t0y;
    s1x += t1x;
    s1y += t1y;
    __syncthreads();
  }
  if (live) {
    jpart[(size_t)blockIdx.y * c.np + i] = make_double2(jx, jy);
    atomicAdd(&sg[2 * si + 0], mui_d.x * s0x + mui_d.y * s0y);
    atomicAdd(&sg[2 * si + 1], mui_d.x * s1x + mui_d.y * s1y);
    if (blockIdx.y == 0) {
      float st, ct;
      sincosf(th[i], &st, &ct);
      atomicAdd(&sg[4], mui_d.x * (double)ct + mui_d.y * (double)st);
    }
  } else if (i < c.np) {
    jpart[(size_t)blockIdx.y * c.np + i] = make_double2(0.0, 0.0);
  }
  __syncthreads();
  if (threadIdx.x < 5)
    gpart[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 5 + threadIdx.x] = sg[threadIdx.x];
}

// lambda_i = mu_i + dt sum over chunks of jpart
__global__ void k_vjp_force_sum(BdDev d, BdConst c, int nchunk, const double2 *jpart, double2 *lam) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.np || d.ext_id[i] < 0) return;
  double jx = 0.0, jy = 0.0;
  for (int k = 0; k < nchunk; ++k) {
    const double2 v = jpart[(size_t)k * c.np + i];
    jx += v.x;
    jy += v.y;
  }
  const double dt = d.rep[0].dt;
  const double2 mu = lam[i];
  lam[i] = make_double2(mu.x + dt * jx, mu.y + dt * jy);
}

// grad[k] += dt sum over blocks of gpart[.][k] (one block of 32 x 5 threads)
__global__ void k_vjp_grad_sum(BdDev d, int nblocks, const double *gpart, double *grad) {
  __shared__ double s[5][32];
  const int k = threadIdx.y, l = threadIdx.x;
  double v = 0.0;
  for (int b = l; b < nblocks; b += 32) v += gpart[(size_t)b * 5 + k];
  s[k][l] = v;
  __syncthreads();
  if (l == 0) {
    double t = 0.0;
    for (int m = 0; m < 32; ++m) t += s[k][m];
    grad[k] += d.rep[0].dt * t;
  }
}

// ---------------------------------------------------------------- loss

// per-species sums of |x_T - x_0|^2 and counts (acc[0..1] sums, acc[2..3] counts)
// per-species sums of |x_T - x_0|^2 and counts, in a fixed order (one block:
// thread t takes disks t, t + 1024, ...; then a fixed tree), so that the loss
// is the same number on every run
__global__ void __launch_bounds__(1024) k_msd_sums(BdDev d, BdConst c, const double2 *x0, double *acc) {
  __shared__ double sh[4][1024];
  const int t = threadIdx.x;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = t; i < c.np; i += 1024) {
    if (d.ext_id[i] < 0) continue;
    const double2 p = d.pos[i], q = x0[i];
    const double dx = p.x - q.x, dy = p.y - q.y;
    const int s = d.species[i] ? 1 : 0;
    v[s] += dx * dx + dy * dy;
    v[2 + s] += 1.0;
  }
  for (int k = 0; k < 4; ++k) sh[k][t] = v[k];
  __syncthreads();
  for (int w = 512; w > 0; w >>= 1) {
    if (t < w)
      for (int k = 0; k < 4; ++k) sh[k][t] += sh[k][t + w];
    __syncthreads();
  }
  if (t < 4) acc[t] = sh[t][0];
}

// loss = sum_s (MSD_s - target)^2 and its gradient lambda_i = dscale dL/dx_i
__global__ void k_msd_loss_grad(BdDev d, BdConst c, const double2 *x0, const double *acc,
                                double target, double dscale, double2 *lam, double *loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double msd[2], cnt[2];
  for (int s = 0; s < 2; ++s) {
    cnt[s] = acc[2 + s];
    msd[s] = cnt[s] > 0 ? acc[s] / cnt[s] : 0.0;
  }
  if (i == 0 && loss) {
    double L = 0.0;
    for (int s = 0; s < 2; ++s)
      if (cnt[s] > 0) L += (msd[s] - target) * (msd[s] - target);
    *loss = L;
  }
  if (!lam || i >= c.np) return;
  if (d.ext_id[i] < 0) {
    lam[i] = make_double2(0.0, 0.0);
    return;
  }
  const int s = d.species[i] ? 1 : 0;
  const double2 p = d.pos[i], q = x0[i];
  const double f = dscale * 2.0 * (msd[s] - target) * 2.0 / cnt[s];
  lam[i] = make_double2(f * (p.x - q.x), f * (p.y - q.y));
}

// ---------------------------------------------------------------- pair-distance histogram loss
// h_b(x) = (1/n) sum over pairs i < j of K(r_ij - c_b), K(u) = exp(-u^2 / (2 s^2)),
// c_b = 2a + (b + 1/2) a/4 (b = 0..31), s = a/4; L = sum_b (h_b(x_T) - h_b(x_0))^2.
// Pairs farther than 12.5a are skipped: their kernel weight at the last
// centre (9.875a) is exp(-55) ~ 1e-24.  One warp per disk i; its lanes take
// the disks j in a fixed stride, and the warp's sums are combined by a
// shuffle tree, so every sum is in a fixed order (deterministic).

#define BD_HIST_BINS 32

__device__ __forceinline__ double hist_centre(double a, int b) {
  return __dadd_rn(__dmul_rn(2.0, a), __dmul_rn((double)b + 0.5, __dmul_rn(0.25, a)));
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// per-disk partial histograms: hpart[i][b] = sum over j > i of K(r_ij - c_b)
__global__ void k_hist_pairs(BdDev d, BdConst c, const double2 *x, double *hpart) {
  const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= c.np) return;
  double acc[BD_HIST_BINS];
#pragma unroll
  for (int b = 0; b < BD_HIST_BINS; ++b) acc[b] = 0.0;
  if (d.ext_id[i] >= 0) {
    const double a = c.a, s = 0.25 * a, inv2s2 = 1.0 / (2.0 * s * s), rc = 12.5 * a;
    const double2 p = x[i];
    for (int j = i + 1 + lane; j < c.np; j += 32) {
      if (d.ext_id[j] < 0) continue;
      const double2 q = x[j];
      const double dx = __dsub_rn(q.x, p.x), dy = __dsub_rn(q.y, p.y);
      const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
      if (r2 > rc * rc) continue;
      const double r = sqrt(r2);
#pragma unroll
      for (int b = 0; b < BD_HIST_BINS; ++b) {
        const double u = __dsub_rn(r, hist_centre(a, b));
        acc[b] += exp(-__dmul_rn(__dmul_rn(u, u), inv2s2));
      }
    }
  }
  double mine = 0.0;
#pragma unroll
  for (int b = 0; b < BD_HIST_BINS; ++b) {
    const double t = warp_sum_d(acc[b]);
    if (lane == b) mine = t;
  }
  hpart[(size_t)i * BD_HIST_BINS + lane] = mine;
}

// h = sum over disks of hpart / n in a fixed order (8 row groups per bin,
// combined in order); with h0: w_b = 2 (h_b - h0_b) / n and the loss
__global__ void __launch_bounds__(256) k_hist_reduce(BdConst c, const double *hpart, double inv_n,
                                                     const double *h0, double *h, double *w, double *loss) {
  __shared__ double part[8][BD_HIST_BINS];
  __shared__ double sq[BD_HIST_BINS];
  const int b = threadIdx.x & 31, g = threadIdx.x >> 5;
  double t = 0.0;
  for (int i = g; i < c.np; i += 8) t += hpart[(size_t)i * BD_HIST_BINS + b];
  part[g][b] = t;
  __syncthreads();
  if (g != 0) return;
  double hb = 0.0;
  for (int k = 0; k < 8; ++k) hb += part[k][b];
  hb *= inv_n;
  h[b] = hb;
  if (!h0) return;
  const double df = hb - h0[b];
  w[b] = 2.0 * df * inv_n;
  sq[b] = df * df;
  __syncwarp();
  if (b == 0 && loss) {
    double L = 0.0;
    for (int k = 0; k < BD_HIST_BINS; ++k) L += sq[k];
    *loss = L;
  }
}

// lam_i = dscale dL/dx_i = dscale sum_{j != i} g(r_ij) (x_i - x_j) / r_ij,
// g(r) = sum_b w_b dK/du(r - c_b), dK/du = -(u / s^2) K(u)
__global__ void k_hist_grad(BdDev d, BdConst c, const double2 *x, const double *w, double dscale,
                            double2 *lam) {
  const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= c.np) return;
  double gx = 0.0, gy = 0.0;
  if (d.ext_id[i] >= 0) {
    const double a = c.a, s = 0.25 * a, inv_s2 = 1.0 / (s * s), inv2s2 = 0.5 * inv_s2, rc = 12.5 * a;
    double wb[BD_HIST_BINS];
#pragma unroll
    for (int b = 0; b < BD_HIST_BINS; ++b) wb[b] = w[b];
    const double2 p = x[i];
    for (int j = lane; j < c.np; j += 32) {
      if (j == i || d.ext_id[j] < 0) continue;
      const double2 q = x[j];
      const double dx = __dsub_rn(p.x, q.x), dy = __dsub_rn(p.y, q.y);
      const double r2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
      if (r2 > rc * rc) continue;
      const double r = sqrt(r2);
      double g = 0.0;
#pragma unroll
      for (int b = 0; b < BD_HIST_BINS; ++b) {
        const double u = __dsub_rn(r, hist_centre(a, b));
        g += wb[b] * (-u * inv_s2) * exp(-__dmul_rn(__dmul_rn(u, u), inv2s2));
      }
      gx += g / r * dx;
      gy += g / r * dy;
    }
  }
  gx = warp_sum_d(gx);
  gy = warp_sum_d(gy);
  if (lane == 0) lam[i] = make_double2(dscale * gx, dscale * gy);
}

// ---------------------------------------------------------------- launchers

cudaError_t bd_adj_hist(const BdDev &d, const BdConst &c, int n, const double2 *x, double *hpart, double *h,
                        const double *h0, double *w, double *loss, double2 *lam, double dscale, cudaStream_t s) {
  if (n <= 0) return cudaErrorInvalidValue;
  const int blocks = (int)(((size_t)c.np * 32 + 255) / 256);
  k_hist_pairs<<<blocks, 256, 0, s>>>(d, c, x, hpart);
  k_hist_reduce<<<1, 256, 0, s>>>(c, hpart, 1.0 / (double)n, h0, h, w, loss);
  if (h0 && lam) k_hist_grad<<<blocks, 256, 0, s>>>(d, c, x, w, dscale, lam);
  return cudaGetLastError();
}

cudaError_t bd_adj_rp_em(const BdDev &d, const BdConst &c, long long step, int k_local, cudaStream_t s) {
  k_rp_em<<<(c.np + 255) / 256, 256, 0, s>>>(d, c, step, k_local);
  return cudaGetLastError();
}

cudaError_t bd_adj_rp_pass(const BdDev &d, const BdConst &c, int pass, int pb, int pe, cudaStream_t s) {
  if (pe > pb) k_rp_disp<<<(pe - pb + 255) / 256, 256, 0, s>>>(d, c, pb, pe);
  k_rp_apply<<<(c.np + 255) / 256, 256, 0, s>>>(d, c, pass);
  return cudaGetLastError();
}

cudaError_t bd_adj_vjp_pass(const BdDev &d, const BdConst &c, int pass, int pb, int pe, const double2 *z,
                            double2 *lam, double2 *mud, cudaStream_t s) {
  // disp <- d_j(z): positions z are in d.pos for the displacement kernel
  cudaError_t e = cudaMemsetAsync(d.disp, 0, (size_t)c.np * sizeof(double2), s);
  if (e != cudaSuccess) return e;
  BdDev dz = d;
  dz.pos = const_cast<double2 *>(z);
  if (pe > pb) k_rp_disp<<<(pe - pb + 255) / 256, 256, 0, s>>>(dz, c, pb, pe);
  k_vjp_pass_mu<<<(c.np + 255) / 256, 256, 0, s>>>(d, c, pass, lam, mud);
  if (pe > pb) k_vjp_pass_pairs<<<(pe - pb + 255) / 256, 256, 0, s>>>(d, c, z, pb, pe, lam, mud);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(d.disp, 0, (size_t)c.np * sizeof(double2), s);
}

int bd_adj_force_chunks(const BdConst &c, int *jchunk) {
  const int nbi = (c.np + BD_ADJ_T - 1) / BD_ADJ_T;
  const int ntile = nbi;
  int nch = (2 * 152 + nbi - 1) / nbi;
  nch = nch < 1 ? 1 : (nch > ntile ? ntile : nch);
  const int tiles_per = (ntile + nch - 1) / nch;
  *jchunk = tiles_per * BD_ADJ_T;
  return (c.np + *jchunk - 1) / *jchunk;
}

cudaError_t bd_adj_vjp_em(const BdDev &d, const BdConst &c, int k_local, const double2 *x, const float *th,
                          double2 *lam, double2 *jpart, double *gpart, double *grad, cudaStream_t s) {
  k_vjp_em_refl<<<(c.np + 255) / 256, 256, 0, s>>>(d, c, k_local, lam);
  int jchunk = 0;
  const int nch = bd_adj_force_chunks(c, &jchunk);
  const int nbi = (c.np + BD_ADJ_T - 1) / BD_ADJ_T;
  k_vjp_force<<<dim3(nbi, nch), BD_ADJ_T, 0, s>>>(d, c, x, th, lam, jchunk, jpart, gpart);
  k_vjp_force_sum<<<(c.np + 255) / 256, 256, 0, s>>>(d, c, nch, jpart, lam);
  k_vjp_grad_sum<<<1, dim3(32, 5), 0, s>>>(d, nbi * nch, gpart, grad);
  return cudaGetLastError();
}

cudaError_t bd_adj_msd(const BdDev &d, const BdConst &c, const double2 *x0, double *acc, double target,
                       double dscale, double2 *lam, double *loss, cudaStream_t s) {
  k_msd_sums<<<1, 1024, 0, s>>>(d, c, x0, acc);
  k_msd_loss_grad<<<(c.np + 255) / 256, 256, 0, s>>>(d, c, x0, acc, target, dscale, lam, loss);
  return cudaGetLastError();
}
