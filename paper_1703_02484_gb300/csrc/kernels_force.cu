// Long-range all-pairs force sweep and the Euler-Maruyama integrator.
//
// Force (Sec. 2.2): F_i = sum_{j != i} A[s_i][s_j] (r_i - r_j) / |r_i - r_j|^3.
// The paper tiles the O(N^2) sweep through shared memory (Nyland et al.,
// Sec. 4.1) or warp shuffles (Algorithm 3, Sec. 4.5), one thread per disk.
// Here each block owns BD_IB disks i (BD_IPT per thread, in registers) and a
// chunk of j tiles; tiles of BD_TJ disks are staged in shared memory, double
// buffered, and every shared-memory load feeds BD_IPT pair interactions.
//
// Precision (FP32 path):
//  - Disks are stored in internal order: species-major, each species segment
//    padded to a whole number of j tiles with inert far-away slots, so every
//    tile is single-species and A[s_i][s_tile] multiplies the tile's summed
//    r/r^3 once per tile (8 FP32 instructions + 1 MUFU per pair).
//  - i blocks follow a Hilbert order over all disks, so a block covers a
//    compact patch; coordinates are re-centred on the block's origin from
//    the (hi, lo) FP32 pair of each FP64 coordinate, which keeps near pairs
//    at FP32 resolution of the patch size rather than of the box size.
//  - Per-tile FP32 sums are added into (hi, lo) compensated accumulators
//    (TwoSum); chunk partials are summed in FP64 by the integrator.
//  - The self pair contributes exactly zero: r^2 gets a 1e-20 a^2 offset, so
//    its 1/r^3 is finite while its dx is zero.
//
// Integrator (Eq. (integration), Sec. 2.4, Sec. 7): Philox4x32-10 words ->
// Box-Muller -> clamp to [-3, 3]; dr = dt (F + v0 e(theta)) + amp xi in FP32
// (FP64 when precision = 1), added to the FP64 master position, rounded to
// the position grid, reflected at the walls; theta += amp_r n.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bd_internal.h"
#include "em.cuh"
#include "f32x2.cuh"
#include "philox.cuh"

using namespace bdf;

__global__ void __launch_bounds__(BD_FT) k_force_long_f32(BdDev d, BdConst c) {
  if (ctl_failed(d.ctl)) return;
  __shared__ float4 sj[2][BD_TJ / 2];   // (x_j, y_j, x_j+1, y_j+1) re-centred
  const int4 item = d.items[blockIdx.x];  // (i block, first tile, end tile, partial slot)
  const int ib = item.x, slot = item.w, tid = threadIdx.x;
  const float2 org = d.iorigin[ib];
  float xi[BD_IPT], yi[BD_IPT], ax[BD_IPT], ay[BD_IPT];
  float fxh[BD_IPT], fxl[BD_IPT], fyh[BD_IPT], fyl[BD_IPT];
  const float *arow[BD_IPT];   // row A[s_i][.] of the table (the block is one replica's)
  int ii[BD_IPT];
#pragma unroll
  for (int q = 0; q < BD_IPT; ++q) {
    int i = d.iperm[ib * BD_IB + q * BD_FT + tid];
    ii[q] = i;
    arow[q] = d.rep[0].alpha;
    if (i >= 0) {
      float4 w = d.work[i];
      xi[q] = __fadd_rn(__fsub_rn(w.x, org.x), w.z);
      yi[q] = __fadd_rn(__fsub_rn(w.y, org.y), w.w);
      arow[q] = d.rep[d.rep_of[i]].alpha + BD_MAX_SPECIES * d.species[i];
    } else {
      xi[q] = 1.0e18f;
      yi[q] = 1.0e18f;
    }
    ax[q] = ay[q] = 0.f;
    fxh[q] = fxl[q] = fyh[q] = fyl[q] = 0.f;
  }
  const int t_begin = item.y, t_end = item.z;
  const float eps0 = 1e-20f * (float)(c.a * c.a);

  // stage: each thread re-centres 2 disks of the tile (BD_TJ = 2 * BD_FT)
  float2 st0, st1;
  auto fetch = [&](int tile) {
    int j0 = tile * BD_TJ + 2 * tid;
    float4 w0 = d.work[j0], w1 = d.work[j0 + 1];
    st0 = make_float2(__fadd_rn(__fsub_rn(w0.x, org.x), w0.z), __fadd_rn(__fsub_rn(w0.y, org.y), w0.w));
    st1 = make_float2(__fadd_rn(__fsub_rn(w1.x, org.x), w1.z), __fadd_rn(__fsub_rn(w1.y, org.y), w1.w));
  };
  int buf = 0;
  if (t_begin < t_end) {
    fetch(t_begin);
    sj[0][tid] = make_float4(st0.x, st0.y, st1.x, st1.y);
  }
  __syncthreads();
  for (int t = t_begin; t < t_end; ++t) {
    if (t + 1 < t_end) fetch(t + 1);
#pragma unroll 4
    for (int jj = 0; jj < BD_TJ / 2; ++jj) {
      float4 p = sj[buf][jj];
#pragma unroll
      for (int q = 0; q < BD_IPT; ++q) {
        float dx = __fsub_rn(p.x, xi[q]);
        float dy = __fsub_rn(p.y, yi[q]);
        float r2 = __fmaf_rn(dx, dx, eps0);
        r2 = __fmaf_rn(dy, dy, r2);
        float s = rsqrt_apx(r2);
        float s3 = __fmul_rn(__fmul_rn(s, s), s);
        ax[q] = __fmaf_rn(dx, s3, ax[q]);
        ay[q] = __fmaf_rn(dy, s3, ay[q]);
      }
#pragma unroll
      for (int q = 0; q < BD_IPT; ++q) {
        float dx = __fsub_rn(p.z, xi[q]);
        float dy = __fsub_rn(p.w, yi[q]);
        float r2 = __fmaf_rn(dx, dx, eps0);
        r2 = __fmaf_rn(dy, dy, r2);
        float s = rsqrt_apx(r2);
        float s3 = __fmul_rn(__fmul_rn(s, s), s);
        ax[q] = __fmaf_rn(dx, s3, ax[q]);
        ay[q] = __fmaf_rn(dy, s3, ay[q]);
      }
    }
    // (r_j - r_i) was summed: the force on i is -A[s_i][s_tile] times it
    const int sp = d.tile_species[t];
#pragma unroll
    for (int q = 0; q < BD_IPT; ++q) {
      const float al = arow[q][sp];
      two_sum(fxh[q], fxl[q], -al * ax[q]);
      two_sum(fyh[q], fyl[q], -al * ay[q]);
      ax[q] = ay[q] = 0.f;
    }
    if (t + 1 < t_end) sj[buf ^ 1][tid] = make_float4(st0.x, st0.y, st1.x, st1.y);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int q = 0; q < BD_IPT; ++q) {
    int i = ii[q];
    if (i >= 0)
      d.fpart[(size_t)slot * c.np + i] =
          make_double2((double)fxh[q] + (double)fxl[q], (double)fyh[q] + (double)fyl[q]);
  }
}

// Periodic box (Sec. 2.1): the one-sided sweep with minimum images.  Each
// coordinate is re-centred on the block's origin as its minimum image, formed
// exactly in grid units from the FP64 master and kept as an FP32 (hi, lo)
// pair, so a pair vector is (hi_j - hi_i) + (lo_j - lo_i): the hi difference
// is exact for near pairs (and takes its minimum image, one exact addition or
// subtraction of L, when beyond L/2), the sum is rounded once.  This keeps
// near pairs at FP32 resolution of their separation wherever they sit in the
// block.  Inert padding slots are staged far away and never wrapped.
// Replicas with walls in the same batch run here too (no wrap, hL = +inf).
// Per (block, tile) the bounding boxes of the two decide the form used for
// all its pairs: no pair beyond L/2 in a component and no pair closer than
// 6 (box gap) -> the hi parts alone (8 FP32 lane operations + 1 MUFU per
// pair, as the walls sweep); close boxes -> the exact (hi, lo) vector (12);
// boxes straddling L/2 -> (hi, lo) with the per-pair minimum image.
__device__ __forceinline__ float4 stage_q(const BdDev &d, const BdConst &c, int j, long long ox, long long oy,
                                          long long LQ) {
  if (d.ext_id[j] < 0) return make_float4(1.0e18f, 1.0e18f, 0.f, 0.f);
  const bdpred::Grid g{c.q, c.inv_q, c.qshift};
  const double2 p = d.pos[j];
  long long X = bdpred::to_int(p.x, g) - ox, Y = bdpred::to_int(p.y, g) - oy;
  if (LQ > 0) {
    const long long h = LQ / 2;
    X = X > h ? X - LQ : (X < -h ? X + LQ : X);
    Y = Y > h ? Y - LQ : (Y < -h ? Y + LQ : Y);
  }
  const float2 sx = bdem::grid_split(X, c.qshift), sy = bdem::grid_split(Y, c.qshift);
  return make_float4(sx.x, sy.x, sx.y, sy.y);
}

__device__ __forceinline__ float min_image(float dx, float Lf, float hLf) {
  dx = dx > hLf ? __fsub_rn(dx, Lf) : dx;
  return dx < -hLf ? __fadd_rn(dx, Lf) : dx;
}

// bounding box (x_min, x_max, y_min, y_max) of staged coordinates, inert
// slots (1e18) left out; block-wide through per-warp partials in shared memory
__device__ __forceinline__ void box_add(float4 &bx, float x, float y) {
  if (x > 1.0e17f) return;
  bx.x = fminf(bx.x, x);
  bx.y = fmaxf(bx.y, x);
  bx.z = fminf(bx.z, y);
  bx.w = fmaxf(bx.w, y);
}
__device__ __forceinline__ float4 warp_box(float4 bx) {
  for (int o = 16; o > 0; o >>= 1) {
    bx.x = fminf(bx.x, __shfl_xor_sync(0xffffffffu, bx.x, o));
    bx.y = fmaxf(bx.y, __shfl_xor_sync(0xffffffffu, bx.y, o));
    bx.z = fminf(bx.z, __shfl_xor_sync(0xffffffffu, bx.z, o));
    bx.w = fmaxf(bx.w, __shfl_xor_sync(0xffffffffu, bx.w, o));
  }
  return bx;
}
__device__ __forceinline__ float4 empty_box() { return make_float4(3e38f, -3e38f, 3e38f, -3e38f); }
__device__ __forceinline__ float4 merge_box(float4 a, float4 b) {
  return make_float4(fminf(a.x, b.x), fmaxf(a.y, b.y), fminf(a.z, b.z), fmaxf(a.w, b.w));
}

__global__ void __launch_bounds__(BD_FT) k_force_long_per(BdDev d, BdConst c) {
  if (ctl_failed(d.ctl)) return;
  __shared__ float4 sj[2][BD_TJ];   // per j: (x_hi, y_hi, x_lo, y_lo) re-centred
  __shared__ float4 sbox[2][BD_FT / 32];   // per-warp boxes of the staged tile
  __shared__ float4 sibox[BD_FT / 32];     // per-warp boxes of the block's disks i
  const int4 item = d.items[blockIdx.x];  // (i block, first tile, end tile, partial slot)
  const int ib = item.x, slot = item.w, tid = threadIdx.x;
  const float2 org = d.iorigin[ib];
  float Lf = 0.f, hLf = __int_as_float(0x7f800000);
  long long LQ = 0;
  {
    const int i0 = d.iperm[ib * BD_IB];
    const BdRep &R0 = d.rep[i0 >= 0 ? d.rep_of[i0] : 0];
    if (R0.periodic) {
      Lf = R0.Lf;
      hLf = R0.hLf;
      LQ = R0.LQ;
    }
  }
  const long long ox = (long long)org.x * (1ll << c.qshift);   // integer origins: exact in grid units
  const long long oy = (long long)org.y * (1ll << c.qshift);
  float xh[BD_IPT], yh[BD_IPT], xl[BD_IPT], yl[BD_IPT], ax[BD_IPT], ay[BD_IPT];
  float fxh[BD_IPT], fxl[BD_IPT], fyh[BD_IPT], fyl[BD_IPT];
  const float *arow[BD_IPT];   // row A[s_i][.] of the table
  int ii[BD_IPT];
#pragma unroll
  for (int q = 0; q < BD_IPT; ++q) {
    int i = d.iperm[ib * BD_IB + q * BD_FT + tid];
    ii[q] = i;
    arow[q] = d.rep[0].alpha;
    if (i >= 0) {
      const float4 u = stage_q(d, c, i, ox, oy, LQ);
      xh[q] = u.x;
      yh[q] = u.y;
      xl[q] = u.z;
      yl[q] = u.w;
      arow[q] = d.rep[d.rep_of[i]].alpha + BD_MAX_SPECIES * d.species[i];
    } else {
      xh[q] = yh[q] = 1.0e18f;
      xl[q] = yl[q] = 0.f;
    }
    ax[q] = ay[q] = 0.f;
    fxh[q] = fxl[q] = fyh[q] = fyl[q] = 0.f;
  }
  const int t_begin = item.y, t_end = item.z;
  const float eps0 = 1e-20f * (float)(c.a * c.a);
  const int warp = tid >> 5, lane = tid & 31;
  {
    float4 bx = empty_box();
#pragma unroll
    for (int q = 0; q < BD_IPT; ++q) box_add(bx, xh[q], yh[q]);
    bx = warp_box(bx);
    if (lane == 0) sibox[warp] = bx;
  }
  float4 st0, st1;
  auto fetch = [&](int tile) {
    const int j0 = tile * BD_TJ + tid;
    st0 = stage_q(d, c, j0, ox, oy, LQ);
    st1 = stage_q(d, c, j0 + BD_FT, ox, oy, LQ);
  };
  auto store = [&](int b) {
    sj[b][tid] = st0;
    sj[b][tid + BD_FT] = st1;
    float4 bx = empty_box();
    box_add(bx, st0.x, st0.y);
    box_add(bx, st1.x, st1.y);
    bx = warp_box(bx);
    if (lane == 0) sbox[b][warp] = bx;
  };
  int buf = 0;
  if (t_begin < t_end) {
    fetch(t_begin);
    store(0);
  }
  __syncthreads();
  float4 ibx = empty_box();
#pragma unroll
  for (int w = 0; w < BD_FT / 32; ++w) ibx = merge_box(ibx, sibox[w]);
  for (int t = t_begin; t < t_end; ++t) {
    if (t + 1 < t_end) fetch(t + 1);
    float4 jb = empty_box();
#pragma unroll
    for (int w = 0; w < BD_FT / 32; ++w) jb = merge_box(jb, sbox[buf][w]);
    // pair components range over [jmin - imax, jmax - imin]
    const bool wrap = jb.y - ibx.x > hLf || jb.x - ibx.y < -hLf || jb.w - ibx.z > hLf || jb.z - ibx.w < -hLf;
    const float gx = fmaxf(0.f, fmaxf(jb.x - ibx.y, ibx.x - jb.y));
    const float gy = fmaxf(0.f, fmaxf(jb.z - ibx.w, ibx.z - jb.w));
    const bool near = gx * gx + gy * gy < 36.f;
    if (wrap) {
#pragma unroll 4
      for (int jj = 0; jj < BD_TJ; ++jj) {
        const float4 p = sj[buf][jj];
#pragma unroll
        for (int q = 0; q < BD_IPT; ++q) {
          const float dx = __fadd_rn(min_image(__fsub_rn(p.x, xh[q]), Lf, hLf), __fsub_rn(p.z, xl[q]));
          const float dy = __fadd_rn(min_image(__fsub_rn(p.y, yh[q]), Lf, hLf), __fsub_rn(p.w, yl[q]));
          float r2 = __fmaf_rn(dx, dx, eps0);
          r2 = __fmaf_rn(dy, dy, r2);
          const float sv = rsqrt_apx(r2);
          const float s3 = __fmul_rn(__fmul_rn(sv, sv), sv);
          ax[q] = __fmaf_rn(dx, s3, ax[q]);
          ay[q] = __fmaf_rn(dy, s3, ay[q]);
        }
      }
    } else if (near) {
#pragma unroll 4
      for (int jj = 0; jj < BD_TJ; ++jj) {
        const float4 p = sj[buf][jj];
#pragma unroll
        for (int q = 0; q < BD_IPT; ++q) {
          const float dx = __fadd_rn(__fsub_rn(p.x, xh[q]), __fsub_rn(p.z, xl[q]));
          const float dy = __fadd_rn(__fsub_rn(p.y, yh[q]), __fsub_rn(p.w, yl[q]));
          float r2 = __fmaf_rn(dx, dx, eps0);
          r2 = __fmaf_rn(dy, dy, r2);
          const float sv = rsqrt_apx(r2);
          const float s3 = __fmul_rn(__fmul_rn(sv, sv), sv);
          ax[q] = __fmaf_rn(dx, s3, ax[q]);
          ay[q] = __fmaf_rn(dy, s3, ay[q]);
        }
      }
    } else {
#pragma unroll 4
      for (int jj = 0; jj < BD_TJ; ++jj) {
        const float4 p = sj[buf][jj];
#pragma unroll
        for (int q = 0; q < BD_IPT; ++q) {
          const float dx = __fsub_rn(p.x, xh[q]);
          const float dy = __fsub_rn(p.y, yh[q]);
          float r2 = __fmaf_rn(dx, dx, eps0);
          r2 = __fmaf_rn(dy, dy, r2);
          const float sv = rsqrt_apx(r2);
          const float s3 = __fmul_rn(__fmul_rn(sv, sv), sv);
          ax[q] = __fmaf_rn(dx, s3, ax[q]);
          ay[q] = __fmaf_rn(dy, s3, ay[q]);
        }
      }
    }
    // (r_j - r_i) was summed: the force on i is -A[s_i][s_tile] times it
    const int sp = d.tile_species[t];
#pragma unroll
    for (int q = 0; q < BD_IPT; ++q) {
      const float al = arow[q][sp];
      two_sum(fxh[q], fxl[q], -al * ax[q]);
      two_sum(fyh[q], fyl[q], -al * ay[q]);
      ax[q] = ay[q] = 0.f;
    }
    if (t + 1 < t_end) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int q = 0; q < BD_IPT; ++q) {
    const int i = ii[q];
    if (i >= 0)
      d.fpart[(size_t)slot * c.np + i] =
          make_double2((double)fxh[q] + (double)fxl[q], (double)fyh[q] + (double)fyl[q]);
  }
}

// Packed variant: Blackwell's f32x2 instructions (add/sub/mul/fma on a pair
// of FP32 values in one 64-bit register pair) process two i disks per
// instruction, halving the issue slots of the FP32 work.  j disks are staged
// as (x, x, y, y) so one 128-bit shared load yields both packed operands.
template <int IPT>
__global__ void __launch_bounds__(BD_FT) k_force_long_f32x2(BdDev d, BdConst c) {
  if (ctl_failed(d.ctl)) return;
  constexpr int NP = IPT / 2;
  constexpr int IB = BD_FT * IPT;
  __shared__ ulonglong2 sj[2][BD_TJ];   // per j: ((x, x), (y, y)) re-centred
  const int4 item = d.items[blockIdx.x];  // (i block, first tile, end tile, partial slot)
  const int ib = item.x, slot = item.w, tid = threadIdx.x;
  const float2 org = d.iorigin[ib];
  u64 xi2[NP], yi2[NP], ax2[NP], ay2[NP];
  float fxh[IPT], fxl[IPT], fyh[IPT], fyl[IPT];
  const float *arow[IPT];   // row A[s_i][.] of the table
  int ii[IPT];
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    float xs[2], ys[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = 2 * k + h;
      int i = d.iperm[ib * IB + q * BD_FT + tid];
      ii[q] = i;
      arow[q] = d.rep[0].alpha;
      if (i >= 0) {
        float4 w = d.work[i];
        xs[h] = __fadd_rn(__fsub_rn(w.x, org.x), w.z);
        ys[h] = __fadd_rn(__fsub_rn(w.y, org.y), w.w);
        arow[q] = d.rep[d.rep_of[i]].alpha + BD_MAX_SPECIES * d.species[i];
      } else {
        xs[h] = 1.0e18f;
        ys[h] = 1.0e18f;
      }
      fxh[q] = fxl[q] = fyh[q] = fyl[q] = 0.f;
    }
    xi2[k] = pk2(xs[0], xs[1]);
    yi2[k] = pk2(ys[0], ys[1]);
    ax2[k] = ay2[k] = 0ull;
  }
  const int t_begin = item.y, t_end = item.z;
  const float e0 = 1e-20f * (float)(c.a * c.a);
  const u64 eps2 = pk2(e0, e0);
  float2 st0, st1;
  auto fetch = [&](int tile) {
    int j0 = tile * BD_TJ + tid;
    float4 w0 = d.work[j0], w1 = d.work[j0 + BD_FT];
    st0 = make_float2(__fadd_rn(__fsub_rn(w0.x, org.x), w0.z), __fadd_rn(__fsub_rn(w0.y, org.y), w0.w));
    st1 = make_float2(__fadd_rn(__fsub_rn(w1.x, org.x), w1.z), __fadd_rn(__fsub_rn(w1.y, org.y), w1.w));
  };
  auto store = [&](int b) {
    sj[b][tid] = make_ulonglong2(pk2(st0.x, st0.x), pk2(st0.y, st0.y));
    sj[b][tid + BD_FT] = make_ulonglong2(pk2(st1.x, st1.x), pk2(st1.y, st1.y));
  };
  int buf = 0;
  if (t_begin < t_end) {
    fetch(t_begin);
    store(0);
  }
  __syncthreads();
  for (int t = t_begin; t < t_end; ++t) {
    if (t + 1 < t_end) fetch(t + 1);
#pragma unroll 4
    for (int jj = 0; jj < BD_TJ; ++jj) {
      const ulonglong2 p = sj[buf][jj];
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        u64 dx = sub2(p.x, xi2[k]);
        u64 dy = sub2(p.y, yi2[k]);
        u64 r2 = fma2(dx, dx, eps2);
        r2 = fma2(dy, dy, r2);
        float ra, rb;
        up2(r2, ra, rb);
        u64 sv = pk2(rsqrt_apx(ra), rsqrt_apx(rb));
        u64 s3 = mul2(mul2(sv, sv), sv);
        ax2[k] = fma2(dx, s3, ax2[k]);
        ay2[k] = fma2(dy, s3, ay2[k]);
      }
    }
    const int sp = d.tile_species[t];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      float ax0, ax1, ay0, ay1;
      up2(ax2[k], ax0, ax1);
      up2(ay2[k], ay0, ay1);
      const int q0 = 2 * k, q1 = 2 * k + 1;
      const float al0 = arow[q0][sp], al1 = arow[q1][sp];
      two_sum(fxh[q0], fxl[q0], -al0 * ax0);
      two_sum(fyh[q0], fyl[q0], -al0 * ay0);
      two_sum(fxh[q1], fxl[q1], -al1 * ax1);
      two_sum(fyh[q1], fyl[q1], -al1 * ay1);
      ax2[k] = ay2[k] = 0ull;
    }
    if (t + 1 < t_end) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int q = 0; q < IPT; ++q) {
    int i = ii[q];
    if (i >= 0)
      d.fpart[(size_t)slot * c.np + i] =
          make_double2((double)fxh[q] + (double)fxl[q], (double)fyh[q] + (double)fyl[q]);
  }
}

// FP64 variant (precision = 1): one disk per thread, FP64 master positions;
// grid (disk blocks, j chunks), chunk k of a replica covers a k-th of its slots
__global__ void __launch_bounds__(128) k_force_long_f64(BdDev d, BdConst c) {
  if (ctl_failed(d.ctl)) return;
  __shared__ double2 sp[128];
  __shared__ int ss[128];
  const int i = blockIdx.x * 128 + threadIdx.x;
  const int jc = blockIdx.y;
  // a block's disks may span two replicas: each thread keeps its own range
  const int r = i < c.np ? d.rep_of[i] : -1;
  const bool live = r >= 0;
  const BdRep &R = d.rep[live ? r : 0];
  double2 pi = live ? d.pos[i] : make_double2(0.0, 0.0);
  int si = live ? d.species[i] : 0;
  double fx = 0.0, fy = 0.0;
  const int span = R.slot_end - R.slot_begin;
  const int per = (span + R.nchunk - 1) / R.nchunk;
  const int my_begin = R.slot_begin + jc * per, my_end = min(R.slot_end, my_begin + per);
  // the block walks the union of its threads' ranges; a thread skips foreign j
  __shared__ int s_lo, s_hi;
  if (threadIdx.x == 0) {
    s_lo = 0x7FFFFFFF;
    s_hi = -1;
  }
  __syncthreads();
  if (live && jc < R.nchunk && my_begin < my_end) {
    atomicMin(&s_lo, my_begin);
    atomicMax(&s_hi, my_end);
  }
  __syncthreads();
  for (int j0 = s_lo; j0 < s_hi; j0 += 128) {
    int j = j0 + threadIdx.x;
    bool ok = j < s_hi && d.ext_id[j] >= 0;
    sp[threadIdx.x] = ok ? d.pos[j] : make_double2(0.0, 0.0);
    ss[threadIdx.x] = ok ? (int)d.species[j] : -1;
    __syncthreads();
    int m = min(128, s_hi - j0);
    if (live && jc < R.nchunk) {
      for (int k = 0; k < m; ++k) {
        const int jj = j0 + k;
        int sk = ss[k];
        if (sk < 0 || jj == i || jj < my_begin || jj >= my_end) continue;
        double rx = pi.x - sp[k].x, ry = pi.y - sp[k].y;
        if (R.periodic) {
          // minimum image (Sec. 2.1)
          rx -= R.L * rint(rx / R.L);
          ry -= R.L * rint(ry / R.L);
        }
        double r2 = rx * rx + ry * ry;
        // |r|^-3 from the library's reciprocal square root (within an ulp):
        // three multiplies instead of a square root and a division
        const double rs = rsqrt(r2);
        double cf = R.alpha_d[BD_MAX_SPECIES * si + sk] * (rs * rs * rs);
        fx += cf * rx;
        fy += cf * ry;
      }
    }
    __syncthreads();
  }
  if (live && jc < R.nchunk) d.fpart[(size_t)jc * c.np + i] = make_double2(fx, fy);
}

__global__ void k_force_sum(BdDev d, BdConst c, double2 *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.np) return;
  const int r = d.rep_of[i];
  if (r < 0) {
    out[i] = make_double2(0.0, 0.0);
    return;
  }
  const BdRep &R = d.rep[r];
  const int ns = R.law == BD_LAW_LONG ? R.nchunk : (R.law == BD_LAW_SHORT ? 1 : 0);
  double fx = 0.0, fy = 0.0;
  for (int k = 0; k < ns; ++k) {
    double2 f = d.fpart[(size_t)k * c.np + i];
    fx += f.x;
    fy += f.y;
  }
  out[i] = make_double2(fx, fy);
}

// step < 0: the index of the step is the device counter (graph replays)
__global__ void k_integrate(BdDev d, BdConst c, long long step, int log_step, int node) {
  if (ctl_failed(d.ctl)) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.np) return;
  if (step < 0) step = *(volatile const long long *)&d.ctl->step_dev;
  const int e = d.ext_id[i];
  if (e < 0) return;
  const BdRep &R = d.rep[d.rep_of[i]];
  const double2 F = bdem::force_sum(d, c, R, i);
  const double2 p = d.pos[i];
  d.pos0[i] = p;
  d.prev[i] = p;
  const float th = d.theta[i];
  d.theta0[i] = th;
  float thn;
  int flags = 0;
  const bdpred::Grid g{c.q, c.inv_q, c.qshift};
  long long X, Y;
  if (c.precision == 0) {
    // move, reflection and FP32 copy in grid units (no FP64 arithmetic)
    bdem::em_move_grid(c, R, (uint32_t)e, step, p, th, F, R.v0, &thn, (uint32_t)node, &X, &Y);
  } else {
    const double2 y = bdem::em_move(c, R, (uint32_t)e, step, p, th, F, R.v0, &thn, (uint32_t)node);
    X = bdpred::to_int(y.x, g);
    Y = bdpred::to_int(y.y, g);
  }
  const long long X0 = bdpred::to_int(p.x, g), Y0 = bdpred::to_int(p.y, g);
  if (R.periodic) {
    // the move itself (before re-entry), for the triangulation's reversal screen
    d.dmove[i] = make_float2(bdem::grid_to_float(X - X0, c.qshift), bdem::grid_to_float(Y - Y0, c.qshift));
    // re-entry at the opposite side (Sec. 2.1); the triangulation kernel
    // shifts the corners of the disks that re-entered
    const int wr = bdem::wrap_grid(R.LQ, X, Y);
    d.wrap[i] = (uint8_t)wr;
    if (wr && !c.overlap_verlet) atomicAdd(&d.ctl->n_wrapped, 1);
  } else {
    const double2 w = bdem::walls_of(d, R, i);
    flags = bdem::reflect_grid(bdpred::to_int(w.x, g), bdpred::to_int(w.y, g), X, Y);
  }
  d.pos[i] = make_double2(bdem::grid_to_double(X, c.qshift), bdem::grid_to_double(Y, c.qshift));
  if (!R.periodic)
    d.dmove[i] = make_float2(bdem::grid_to_float(X - X0, c.qshift), bdem::grid_to_float(Y - Y0, c.qshift));
  const float2 sx = bdem::grid_split(X, c.qshift), sy = bdem::grid_split(Y, c.qshift);
  d.work[i] = make_float4(sx.x, sy.x, sx.y, sy.y);
  d.theta[i] = thn;
  d.moved[i] = 1;
  if (log_step >= 0 && d.log_refl) d.log_refl[(size_t)log_step * c.np + i] = (uint8_t)flags;
}

// all pieces of a halved step completed: the step counts as one time step
__global__ void k_advance_step(BdCtl *ctl) {
  if (*(volatile int *)&ctl->status) return;
  ctl->step_dev += 1;
  ctl->st_steps += 1;
}

__global__ void k_work_copy(BdDev d, BdConst c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.np) return;
  if (d.ext_id[i] < 0) {
    d.work[i] = make_float4(1.0e18f, 1.0e18f, 0.f, 0.f);
    return;
  }
  d.work[i] = bdem::split(d.pos[i]);
}

int bd_force_blocks_per_sm(int variant) {
  int per = 0;
  cudaError_t e = variant == 1
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_force_long_f32x2<BD_IPT>, BD_FT, 0)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_force_long_f32, BD_FT, 0);
  return e == cudaSuccess ? per : 0;
}

cudaError_t bd_launch_force_long_variant(const BdDev &d, const BdConst &c, int variant, cudaStream_t s) {
  if (c.precision == 0) {
    if (variant >= 2) return bd_launch_force_sym(d, c, variant, s);
    if (c.n_items == 0) return cudaSuccess;
    if (c.any_periodic)
      k_force_long_per<<<c.n_items, BD_FT, 0, s>>>(d, c);   // the one form with minimum images
    else if (variant == 1)
      k_force_long_f32x2<BD_IPT><<<c.n_items, BD_FT, 0, s>>>(d, c);
    else
      k_force_long_f32<<<c.n_items, BD_FT, 0, s>>>(d, c);
  } else {
    k_force_long_f64<<<dim3((c.np + 127) / 128, c.max_nchunk), 128, 0, s>>>(d, c);
  }
  return cudaGetLastError();
}

cudaError_t bd_launch_force_long(const BdDev &d, const BdConst &c, cudaStream_t s) {
  return bd_launch_force_long_variant(d, c, c.force_variant, s);
}

cudaError_t bd_launch_integrate(const BdDev &d, const BdConst &c, int64_t step, int log_step,
                                cudaStream_t s, int node) {
  k_integrate<<<(c.np + 255) / 256, 256, 0, s>>>(d, c, (long long)step, log_step, node);
  return cudaGetLastError();
}

cudaError_t bd_launch_advance_step(const BdDev &d, cudaStream_t s) {
  k_advance_step<<<1, 1, 0, s>>>(d.ctl);
  return cudaGetLastError();
}

// periodic box: a coordinate that moved by more than L/2 crossed an edge
// (stored = geometric - L k, k = round((old - new) / L))
__global__ void k_periodic_wraps(BdDev d, BdConst c) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= c.np) return;
  const int r = d.rep_of[i];
  if (r < 0 || !d.rep[r].periodic) return;
  const long long LQ = d.rep[r].LQ;
  const bdpred::Grid g{c.q, c.inv_q, c.qshift};
  const double2 o = d.pos0[i], p = d.pos[i];
  const long long dx = bdpred::to_int(o.x, g) - bdpred::to_int(p.x, g);
  const long long dy = bdpred::to_int(o.y, g) - bdpred::to_int(p.y, g);
  const int kx = dx > LQ / 2 ? 1 : (dx < -LQ / 2 ? -1 : 0);
  const int ky = dy > LQ / 2 ? 1 : (dy < -LQ / 2 ? -1 : 0);
  const int wr = (kx & 3) | ((ky & 3) << 2);
  d.wrap[i] = (uint8_t)wr;
  if (wr) atomicAdd(&d.ctl->n_wrapped, 1);
}

cudaError_t bd_launch_periodic_wraps(const BdDev &d, const BdConst &c, cudaStream_t s) {
  k_periodic_wraps<<<(c.np + 255) / 256, 256, 0, s>>>(d, c);
  return cudaGetLastError();
}

cudaError_t bd_launch_work_copy(const BdDev &d, const BdConst &c, cudaStream_t s) {
  k_work_copy<<<(c.np + 255) / 256, 256, 0, s>>>(d, c);
  return cudaGetLastError();
}

cudaError_t bd_launch_force_sum(const BdDev &d, const BdConst &c, double2 *out, cudaStream_t s) {
  k_force_sum<<<(c.np + 255) / 256, 256, 0, s>>>(d, c, out);
  return cudaGetLastError();
}
