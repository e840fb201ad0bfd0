// Symmetric all-pairs sweep: the long-range force of Sec. 2.2,
//   F_i = sum_{j != i} A[s_i][s_j] (r_i - r_j) / |r_i - r_j|^3,
// with the geometric factor g_ij = (r_i - r_j)/|r_ij|^3 = -g_ji evaluated
// once per unordered pair and added to both disks (A[s_i][s_j] g_ij to i,
// -A[s_j][s_i] g_ij to j; the table need not be symmetric).
//
// Disks sit in blocks of BD_SB = 512 consecutive slots (two j tiles), each of
// one species.  A work item pairs block P with a range of tiles:
//  - tiles of P itself: the i side only, all ordered pairs inside P;
//  - later tiles (index >= 2P + 2): every pair once, both sides.
// Pairs with an earlier tile are done by that tile's block.
//
// Inside an item each warp holds a share of the disks i of P in registers
// (four or eight per lane, as packed f32x2 pairs).  A tile of 256 disks j is staged
// in shared memory; a warp takes 32 of them, one per lane, and passes them
// round its lanes by shuffles, each j carrying its own accumulator, so after
// 32 steps every j has met all of the warp's i and returned to its lane.  Per
// unordered pair: 2 sub, 2 FMA (r^2), 1 MUFU rsqrt, 2 mul (r^-3), 2 FMA into
// the i accumulators and 2 FMA into the j accumulator -- 10 FP32 lane
// operations for two ordered pair interactions, against 8 per ordered pair in
// the one-sided sweep.
//
// Partial forces are written, not added: the i side of each item to ipart,
// the j side of each (item, tile) to jpart.  k_force_sym_reduce then sums, for
// every disk, its block's i partials and its tile's j partials in a fixed
// order, so the force is deterministic.  Coordinates are re-centred on the
// block's integer origin from the (hi, lo) FP32 pair of each FP64 coordinate,
// as in the one-sided sweep; per-tile FP32 sums are added in (hi, lo) pairs
// within an item on the i side, and partials (FP32) in float-float by the
// reduction.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <type_traits>

#include "bd_internal.h"
#include "em.cuh"
#include "f32x2.cuh"
#include "predicates.cuh"

using namespace bdf;

namespace {

__device__ __forceinline__ float2 recentre(float4 w, float2 org) {
  return make_float2(__fadd_rn(__fsub_rn(w.x, org.x), w.z), __fadd_rn(__fsub_rn(w.y, org.y), w.w));
}

// periodic box: disk j about the block origin (ox, oy) as its minimum image,
// formed exactly in grid units and kept as an FP32 (hi, lo) pair (LQ = 0:
// walls, no wrap); inert slots far away
__device__ __forceinline__ float4 rel_grid(const BdDev &d, const BdConst &c, int j, long long ox, long long oy,
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

// bounding box (x_min, x_max, y_min, y_max), inert slots (1e18) left out
__device__ __forceinline__ void sbox_add(float4 &bx, float x, float y) {
  if (x > 1.0e17f) return;
  bx.x = fminf(bx.x, x);
  bx.y = fmaxf(bx.y, x);
  bx.z = fminf(bx.z, y);
  bx.w = fmaxf(bx.w, y);
}
__device__ __forceinline__ float4 swarp_box(float4 bx) {
  for (int o = 16; o > 0; o >>= 1) {
    bx.x = fminf(bx.x, __shfl_xor_sync(0xffffffffu, bx.x, o));
    bx.y = fmaxf(bx.y, __shfl_xor_sync(0xffffffffu, bx.y, o));
    bx.z = fminf(bx.z, __shfl_xor_sync(0xffffffffu, bx.z, o));
    bx.w = fmaxf(bx.w, __shfl_xor_sync(0xffffffffu, bx.w, o));
  }
  return bx;
}
__device__ __forceinline__ float4 sempty_box() { return make_float4(3e38f, -3e38f, 3e38f, -3e38f); }
__device__ __forceinline__ float4 smerge_box(float4 a, float4 b) {
  return make_float4(fminf(a.x, b.x), fmaxf(a.y, b.y), fminf(a.z, b.z), fmaxf(a.w, b.w));
}

// minimum image of a packed pair of coordinate differences in (-3L/2, 3L/2):
// t = rint(dx / L) by the 1.5 2^23 rounding constant, dx - t L exact (Sterbenz)
__device__ __forceinline__ u64 min_image2(u64 dx, u64 invL2, u64 nL2, u64 M2) {
  const u64 t = sub2(fma2(dx, invL2, M2), M2);
  return fma2(t, nL2, dx);
}
// the same by compares, which leaves the far-away inert slots far away
__device__ __forceinline__ u64 min_image2_cmp(u64 dx, float Lf, float hLf) {
  float a, b;
  up2(dx, a, b);
  a = a > hLf ? __fsub_rn(a, Lf) : (a < -hLf ? __fadd_rn(a, Lf) : a);
  b = b > hLf ? __fsub_rn(b, Lf) : (b < -hLf ? __fadd_rn(b, Lf) : b);
  return pk2(a, b);
}

}  // namespace

// NW warps per block, NP packed i pairs (2 NP disks) per lane, NJ disks j
// carried per lane, COMB: fold the packed halves of a j accumulator before
// passing it (2 shuffles instead of 4), UR: unrolled ring steps.
// NW * 32 * 2 * NP = BD_SB.  Shapes built: (4 warps, 4 disks per lane) and
// (2 warps, 8 disks per lane), one j per lane, halves passed unfolded; the
// second halves the ring's shuffles and register moves per pair.  (Two j per
// lane, folded halves and deeper unrolling measured within 3 % of these.)
//
// PER (periodic boxes, Sec. 2.1): every coordinate is re-centred on the block
// origin as its minimum image, exactly in grid units (near pairs, across an
// edge too, are then plain differences); per (block, tile) the bounding boxes
// tell whether any pair component can exceed L/2, and only such tiles (those
// near the block's antipode) take the per-pair minimum image: 3 packed
// operations per coordinate, or compares when the tile holds inert slots.
// STAGE (walls only): 0 stage the next j tile through registers (re-centred
// on the way to shared memory); 1 copy it raw with cp.async (no registers held
// across the tile's arithmetic) and re-centre each j as it is read.
// ACC: the i side's sum over an item's tiles, 2 in (hi, lo) float-float, 1 in
// FP32 (half the registers).
template <int NW, int NP, int NJ, bool COMB, int UR, bool PER, int STAGE = 0, int ACC = 2>
__device__ __forceinline__ void force_long_sym_body(const BdDev &d, const BdConst &c) {
  static_assert(!(PER && STAGE), "the periodic form stages exact minimum images through registers");
  if (ctl_failed(d.ctl)) return;
  constexpr int T = NW * 32;         // threads
  constexpr int NQ = 2 * NP;         // disks i per thread
  constexpr int NS = BD_TJ / T;      // j disks each thread stages per tile
  static_assert(BD_SB == T * NQ, "a block is BD_SB disks");
  __shared__ float2 sjp[2][STAGE ? 1 : BD_TJ];   // j positions, re-centred (PER: the hi parts)
  __shared__ __align__(16) float4 sraw[2][STAGE ? BD_TJ : 1];   // STAGE 1: j as stored (x_hi, y_hi, x_lo, y_lo)
  __shared__ float2 sjl[2][BD_TJ];   // PER: the lo parts
  __shared__ float2 shw[NW][BD_TJ];  // per-warp j-side sums of the current tile
  const int item_id = c.sitem0 + (int)blockIdx.x;   // this launch's share of the plan (force sharding)
  const int4 item = d.sitems[item_id];
  const int P = item.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int base = P * BD_SB;
  const int tsym = 2 * P + 2;        // first tile met from both sides
  const int2 binfo = d.sblock[P];
  const BdRep &R = d.rep[binfo.x];
  const int a = binfo.y;
  const float2 org = d.sorigin[P];
  long long LQ = 0, ox = 0, oy = 0;
  float Lf = 0.f, hLf = __int_as_float(0x7f800000);
  if (PER) {
    if (R.periodic) {
      LQ = R.LQ;
      Lf = R.Lf;
      hLf = R.hLf;
    }
    ox = (long long)org.x * (1ll << c.qshift);   // integer origins: exact in grid units
    oy = (long long)org.y * (1ll << c.qshift);
  }
  auto rel = [&](int j) -> float4 {
    if (PER) return rel_grid(d, c, j, ox, oy, LQ);
    const float2 v = recentre(d.work[j], org);
    return make_float4(v.x, v.y, 0.f, 0.f);
  };
  __shared__ float4 sbox[2][NW];     // PER: per-warp boxes of the staged tile
  __shared__ int spad[2][NW];        //      and whether it holds inert slots
  __shared__ float4 sibox[NW];       //      per-warp boxes of the block's disks i
  __shared__ int sipad[NW];          //      and whether they include inert slots
  u64 xi2[NP], yi2[NP], ax2[NP], ay2[NP];
  u64 xl2[NP], yl2[NP];              // PER: lo parts of the disks i
  float fxh[NQ], fxl[ACC == 2 ? NQ : 1], fyh[NQ], fyl[ACC == 2 ? NQ : 1];
  float4 ibox = sempty_box();
  bool ipad = false;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const float4 p0 = rel(base + (2 * k) * T + tid);
    const float4 p1 = rel(base + (2 * k + 1) * T + tid);
    xi2[k] = pk2(p0.x, p1.x);
    yi2[k] = pk2(p0.y, p1.y);
    xl2[k] = pk2(p0.z, p1.z);
    yl2[k] = pk2(p0.w, p1.w);
    ax2[k] = ay2[k] = 0ull;
    if (PER) {
      sbox_add(ibox, p0.x, p0.y);
      sbox_add(ibox, p1.x, p1.y);
      ipad = ipad || p0.x > 1.0e17f || p1.x > 1.0e17f;
    }
  }
  if (PER) {
    ibox = swarp_box(ibox);
    ipad = __any_sync(0xffffffffu, ipad);
    if (lane == 0) {
      sibox[warp] = ibox;
      sipad[warp] = ipad ? 1 : 0;
    }
  }
  const u64 invL2 = pk2(Lf > 0.f ? 1.0f / Lf : 0.f, Lf > 0.f ? 1.0f / Lf : 0.f);
  const u64 nL2 = pk2(-Lf, -Lf), M2 = pk2(12582912.0f, 12582912.0f);
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    fxh[q] = fyh[q] = 0.f;
    if (ACC == 2) fxl[q] = fyl[q] = 0.f;
  }
  const float e0 = 1e-20f * (float)(c.a * c.a);   // makes the self pair exactly 0
  const u64 eps2 = pk2(e0, e0);
  const int t_begin = item.y, t_end = item.z;
  const int jt0 = max(t_begin, tsym);
  float4 st[STAGE ? 1 : NS];
  int buf = 0;
  auto fetch = [&](int tile) {
    if constexpr (STAGE == 1) {
      // asynchronous 16-byte copies straight into shared memory
#pragma unroll
      for (int m = 0; m < NS; ++m) {
        const unsigned dst = (unsigned)__cvta_generic_to_shared(&sraw[buf ^ 1][m * T + tid]);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
                     "l"(d.work + (size_t)tile * BD_TJ + m * T + tid)
                     : "memory");
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    } else {
#pragma unroll
      for (int m = 0; m < NS; ++m) st[m] = rel(tile * BD_TJ + m * T + tid);
    }
  };
  auto store = [&](int b) {
    if constexpr (STAGE == 1) {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      return;
    }
#pragma unroll
    for (int m = 0; m < NS; ++m) {
      sjp[b][m * T + tid] = make_float2(st[m].x, st[m].y);
      if (PER) sjl[b][m * T + tid] = make_float2(st[m].z, st[m].w);
    }
    if (PER) {
      float4 bx = sempty_box();
      bool pad = false;
#pragma unroll
      for (int m = 0; m < NS; ++m) {
        sbox_add(bx, st[m].x, st[m].y);
        pad = pad || st[m].x > 1.0e17f;
      }
      bx = swarp_box(bx);
      pad = __any_sync(0xffffffffu, pad);
      if (lane == 0) {
        sbox[b][warp] = bx;
        spad[b][warp] = pad ? 1 : 0;
      }
    }
  };
  buf = STAGE ? 1 : 0;   // STAGE 1: fetch fills sraw[buf ^ 1]
  if (t_begin < t_end) {
    fetch(t_begin);
    store(0);
  }
  buf = 0;
  __syncthreads();
  // the j disk in slot jj of the current staging buffer, re-centred
  auto jpos = [&](int jj) -> float2 {
    if constexpr (STAGE == 1) return recentre(sraw[buf][jj], org);
    else return sjp[buf][jj];
  };
  // pair differences: MODE 0 plain, 1 packed minimum image, 2 minimum image by compares
  // pair differences (r_j - r_i): MODE 0 the hi parts alone; 1 the exact
  // near-pair vector (hi_j - hi_i) + (lo_j - lo_i); 2 the same with the packed
  // minimum image of the hi difference; 3 with the minimum image by compares;
  // 4 near pairs across the antipode (a block spanning the box): the hi
  // difference, about L there, is formed exactly as s + e (TwoDiff), s takes
  // the minimum image (exact: |s| in [L/2, 3L/2]), then e and the lo
  // difference are added
  auto diff = [&](auto MODE, u64 jh2, u64 ih2, u64 jl2, u64 il2) -> u64 {
    constexpr int mode = decltype(MODE)::value;
    u64 dd = sub2(jh2, ih2);
    if constexpr (mode == 4) {
      const u64 v = sub2(dd, jh2);
      const u64 e = sub2(sub2(jh2, sub2(dd, v)), add2(ih2, v));
      return add2(min_image2_cmp(dd, Lf, hLf), add2(e, sub2(jl2, il2)));
    }
    if constexpr (mode == 2) dd = min_image2(dd, invL2, nL2, M2);
    if constexpr (mode == 3) dd = min_image2_cmp(dd, Lf, hLf);
    if constexpr (mode >= 1) dd = add2(dd, sub2(jl2, il2));
    return dd;
  };
  auto own_tile = [&](auto MODE) {
    // the block's own disks: i side only, j broadcast from shared memory
#pragma unroll 4
    for (int jj = 0; jj < BD_TJ; ++jj) {
      const float2 p = jpos(jj);
      const u64 jx2 = pk2(p.x, p.x), jy2 = pk2(p.y, p.y);
      u64 jxl2 = 0ull, jyl2 = 0ull;
      if constexpr (decltype(MODE)::value >= 1) {
        const float2 pl = sjl[buf][jj];
        jxl2 = pk2(pl.x, pl.x);
        jyl2 = pk2(pl.y, pl.y);
      }
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        const u64 dx = diff(MODE, jx2, xi2[k], jxl2, xl2[k]);
        const u64 dy = diff(MODE, jy2, yi2[k], jyl2, yl2[k]);
        u64 r2 = fma2(dx, dx, eps2);
        r2 = fma2(dy, dy, r2);
        float ra, rb;
        up2(r2, ra, rb);
        const u64 sv = pk2(rsqrt_apx(ra), rsqrt_apx(rb));
        const u64 s3 = mul2(mul2(sv, sv), sv);
        ax2[k] = fma2(dx, s3, ax2[k]);
        ay2[k] = fma2(dy, s3, ay2[k]);
      }
    }
  };
  auto ring_tile = [&](auto MODE) {
    // a later tile: every pair once, both sides; each lane carries NJ disks j
    for (int g = 0; g < BD_TJ / (32 * NJ); ++g) {
      constexpr bool LO = decltype(MODE)::value >= 1;
      float jx[NJ], jy[NJ], jxl[NJ], jyl[NJ];
      u64 hx2[NJ], hy2[NJ];
#pragma unroll
      for (int m = 0; m < NJ; ++m) {
        const float2 p = jpos((g * NJ + m) * 32 + lane);
        jx[m] = p.x;
        jy[m] = p.y;
        jxl[m] = jyl[m] = 0.f;
        if constexpr (LO) {
          const float2 pl = sjl[buf][(g * NJ + m) * 32 + lane];
          jxl[m] = pl.x;
          jyl[m] = pl.y;
        }
        hx2[m] = hy2[m] = 0ull;
      }
#pragma unroll UR
      for (int rot = 0; rot < 32; ++rot) {
        const int src = (lane + 1) & 31;
#pragma unroll
        for (int m = 0; m < NJ; ++m) {
          const u64 jx2 = pk2(jx[m], jx[m]), jy2 = pk2(jy[m], jy[m]);
          const u64 jxl2 = LO ? pk2(jxl[m], jxl[m]) : 0ull, jyl2 = LO ? pk2(jyl[m], jyl[m]) : 0ull;
          // the next j position does not depend on this step's arithmetic
          const float njx = __shfl_sync(0xffffffffu, jx[m], src);
          const float njy = __shfl_sync(0xffffffffu, jy[m], src);
          float njxl = 0.f, njyl = 0.f;
          if constexpr (LO) {
            njxl = __shfl_sync(0xffffffffu, jxl[m], src);
            njyl = __shfl_sync(0xffffffffu, jyl[m], src);
          }
#pragma unroll
          for (int k = 0; k < NP; ++k) {
            const u64 dx = diff(MODE, jx2, xi2[k], jxl2, xl2[k]);
            const u64 dy = diff(MODE, jy2, yi2[k], jyl2, yl2[k]);
            u64 r2 = fma2(dx, dx, eps2);
            r2 = fma2(dy, dy, r2);
            float ra, rb;
            up2(r2, ra, rb);
            const u64 sv = pk2(rsqrt_apx(ra), rsqrt_apx(rb));
            const u64 s3 = mul2(mul2(sv, sv), sv);
            ax2[k] = fma2(dx, s3, ax2[k]);
            ay2[k] = fma2(dy, s3, ay2[k]);
            hx2[m] = fma2(dx, s3, hx2[m]);
            hy2[m] = fma2(dy, s3, hy2[m]);
          }
          // pass the j accumulator one lane down the ring, after its disk
          float h0, h1, h2, h3;
          up2(hx2[m], h0, h1);
          up2(hy2[m], h2, h3);
          if (COMB) {
            h0 = __shfl_sync(0xffffffffu, __fadd_rn(h0, h1), src);
            h2 = __shfl_sync(0xffffffffu, __fadd_rn(h2, h3), src);
            hx2[m] = pk2(h0, 0.f);
            hy2[m] = pk2(h2, 0.f);
          } else {
            h0 = __shfl_sync(0xffffffffu, h0, src);
            h1 = __shfl_sync(0xffffffffu, h1, src);
            h2 = __shfl_sync(0xffffffffu, h2, src);
            h3 = __shfl_sync(0xffffffffu, h3, src);
            hx2[m] = pk2(h0, h1);
            hy2[m] = pk2(h2, h3);
          }
          jx[m] = njx;
          jy[m] = njy;
          jxl[m] = njxl;
          jyl[m] = njyl;
        }
      }
      // after 32 passes every j is back in its own lane
#pragma unroll
      for (int m = 0; m < NJ; ++m) {
        float h0, h1, h2, h3;
        up2(hx2[m], h0, h1);
        up2(hy2[m], h2, h3);
        shw[warp][(g * NJ + m) * 32 + lane] = make_float2(__fadd_rn(h0, h1), __fadd_rn(h2, h3));
      }
    }
  };
  float4 ibx = sempty_box();
  int ipd = 0;   // inert slots among the disks i: the packed minimum image would
                 // bring them near, so their tiles take the compares
  if (PER) {
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      ibx = smerge_box(ibx, sibox[w]);
      ipd |= sipad[w];
    }
  }
  for (int t = t_begin; t < t_end; ++t) {
    if (t + 1 < t_end) fetch(t + 1);
    const int b = d.tile_species[t];
    int mode = 0;
    if constexpr (PER) {
      float4 jb = sempty_box();
      int pad = ipd;
#pragma unroll
      for (int w = 0; w < NW; ++w) {
        jb = smerge_box(jb, sbox[buf][w]);
        pad |= spad[buf][w];
      }
      // pair components range over [j_min - i_max, j_max - i_min]
      const bool wrap = LQ > 0 && (jb.y - ibx.x > hLf || jb.x - ibx.y < -hLf || jb.w - ibx.z > hLf ||
                                   jb.z - ibx.w < -hLf);
      // boxes closer than 20: the exact vector keeps their pairs at FP32
      // resolution of their separation (a 512-disk block puts coordinates up
      // to L/2 from its origin, where one rounding costs ulp(L/2) / 2)
      const float gx = fmaxf(0.f, fmaxf(jb.x - ibx.y, ibx.x - jb.y));
      const float gy = fmaxf(0.f, fmaxf(jb.z - ibx.w, ibx.z - jb.w));
      const bool near = gx * gx + gy * gy < 400.f;
      mode = wrap ? (near ? 4 : (pad ? 3 : 2)) : (near ? 1 : 0);
    }
    using M0 = std::integral_constant<int, 0>;
    using M1 = std::integral_constant<int, 1>;
    using M2c = std::integral_constant<int, 2>;
    using M3 = std::integral_constant<int, 3>;
    using M4 = std::integral_constant<int, 4>;
    if (t < tsym) {
      if constexpr (PER) {
        if (mode == 1) own_tile(M1());
        else if (mode == 2) own_tile(M2c());
        else if (mode == 3) own_tile(M3());
        else if (mode == 4) own_tile(M4());
        else own_tile(M0());
      } else {
        own_tile(M0());
      }
    } else {
      if constexpr (PER) {
        if (mode == 1) ring_tile(M1());
        else if (mode == 2) ring_tile(M2c());
        else if (mode == 3) ring_tile(M3());
        else if (mode == 4) ring_tile(M4());
        else ring_tile(M0());
      } else {
        ring_tile(M0());
      }
      __syncthreads();
      // j side of this tile: F_j += A[s_j][s_i] sum_i (r_j - r_i)/r^3
      const float alj = R.alpha[BD_MAX_SPECIES * b + a];
      float2 *out = d.jpart + (size_t)(item.w + (t - jt0)) * BD_TJ;
      for (int jj = tid; jj < BD_TJ; jj += T) {
        float hx = 0.f, hy = 0.f;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
          hx = __fadd_rn(hx, shw[w][jj].x);
          hy = __fadd_rn(hy, shw[w][jj].y);
        }
        out[jj] = make_float2(alj * hx, alj * hy);
      }
    }
    // i side of this tile: F_i -= A[s_i][s_j] sum_j (r_j - r_i)/r^3
    const float ali = R.alpha[BD_MAX_SPECIES * a + b];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      float ax0, ax1, ay0, ay1;
      up2(ax2[k], ax0, ax1);
      up2(ay2[k], ay0, ay1);
      if constexpr (ACC == 2) {
        two_sum(fxh[2 * k], fxl[2 * k], -ali * ax0);
        two_sum(fyh[2 * k], fyl[2 * k], -ali * ay0);
        two_sum(fxh[2 * k + 1], fxl[2 * k + 1], -ali * ax1);
        two_sum(fyh[2 * k + 1], fyl[2 * k + 1], -ali * ay1);
      } else {
        fxh[2 * k] = __fmaf_rn(-ali, ax0, fxh[2 * k]);
        fyh[2 * k] = __fmaf_rn(-ali, ay0, fyh[2 * k]);
        fxh[2 * k + 1] = __fmaf_rn(-ali, ax1, fxh[2 * k + 1]);
        fyh[2 * k + 1] = __fmaf_rn(-ali, ay1, fyh[2 * k + 1]);
      }
      ax2[k] = ay2[k] = 0ull;
    }
    if (t + 1 < t_end) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  float2 *ip = d.ipart + (size_t)item_id * BD_SB;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    if constexpr (ACC == 2) ip[q * T + tid] = make_float2(__fadd_rn(fxh[q], fxl[q]), __fadd_rn(fyh[q], fyl[q]));
    else ip[q * T + tid] = make_float2(fxh[q], fyh[q]);
  }
}

template <int NW, int NP, int NJ, bool COMB, int UR, bool PER>
__global__ void __launch_bounds__(NW * 32) k_force_long_sym(BdDev d, BdConst c) {
  force_long_sym_body<NW, NP, NJ, COMB, UR, PER>(d, c);
}

// the same with a register budget for MINB resident blocks per SM
template <int NW, int NP, int NJ, bool COMB, int UR, bool PER, int MINB, int STAGE, int ACC>
__global__ void __launch_bounds__(NW * 32, MINB) k_force_long_sym_mb(BdDev d, BdConst c) {
  force_long_sym_body<NW, NP, NJ, COMB, UR, PER, STAGE, ACC>(d, c);
}

// F_i = sum of its block's i partials + sum of its tile's j partials, in the
// order the host listed them (item order), into partial-force slot 0.
// A block of 256 threads serves 64 consecutive disks: thread group g (of 4)
// takes every fourth partial (entries g, g + 4, ...) of the 64 disks, so the
// loads stay coalesced and four times as many warps hide their latency; the
// four group sums are added in a fixed order.  Sums are float-float (TwoSum
// into a (hi, lo) FP32 pair, about 48 bits): FP64 adds run at 1/64 of the FP32
// rate on this part and would bound the kernel.
#define BD_RED_D 64   // disks per reduction block
__global__ void __launch_bounds__(4 * BD_RED_D) k_force_sym_reduce(BdDev d, BdConst c) {
  __shared__ float4 part[4][BD_RED_D];
  if (ctl_failed(d.ctl)) return;
  const int g = threadIdx.x / BD_RED_D, dl = threadIdx.x % BD_RED_D;
  const int i = blockIdx.x * BD_RED_D + dl;        // np is a multiple of 512: i < np
  const int P = i / BD_SB, t = i / BD_TJ;           // the same for the whole block
  const float2 *ib = d.ipart + (i - P * BD_SB);
  const float2 *jb = d.jpart + (i - t * BD_TJ);
  float xh[2] = {0.f, 0.f}, xl[2] = {0.f, 0.f}, yh[2] = {0.f, 0.f}, yl[2] = {0.f, 0.f};
  auto run = [&](const int *idx, int k0, int k1, const float2 *b, int stride) {
    int k = k0 + g;
    for (; k + 4 < k1; k += 8) {
      const float2 v0 = b[(size_t)__ldg(idx + k) * stride];
      const float2 v1 = b[(size_t)__ldg(idx + k + 4) * stride];
      two_sum(xh[0], xl[0], v0.x);
      two_sum(yh[0], yl[0], v0.y);
      two_sum(xh[1], xl[1], v1.x);
      two_sum(yh[1], yl[1], v1.y);
    }
    if (k < k1) {
      const float2 v0 = b[(size_t)__ldg(idx + k) * stride];
      two_sum(xh[0], xl[0], v0.x);
      two_sum(yh[0], yl[0], v0.y);
    }
  };
  run(d.red_iidx, d.red_iptr[P], d.red_iptr[P + 1], ib, BD_SB);
  run(d.red_jidx, d.red_jptr[t], d.red_jptr[t + 1], jb, BD_TJ);
  two_sum(xh[0], xl[0], xh[1]);
  two_sum(yh[0], yl[0], yh[1]);
  part[g][dl] = make_float4(xh[0], __fadd_rn(xl[0], xl[1]), yh[0], __fadd_rn(yl[0], yl[1]));
  __syncthreads();
  if (g != 0) return;
  const int r = d.rep_of[i];
  if (r < 0 || d.rep[r].law != BD_LAW_LONG) return;
  double fx = 0.0, fy = 0.0;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const float4 q = part[m][dl];
    fx += (double)q.x + (double)q.y;
    fy += (double)q.z + (double)q.w;
  }
  d.fpart[i] = make_double2(fx, fy);
}

int bd_force_launches(int variant) { return variant >= 2 ? 2 : 1; }

int bd_force_sym_blocks_per_sm(int variant, int periodic) {
  int per = 0;
  cudaError_t e;
  if (periodic)
    e = variant == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                           &per, k_force_long_sym_mb<4, 2, 1, false, 2, true, 8, 0, 2>, 128, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                           &per, k_force_long_sym_mb<2, 4, 1, false, 2, true, 12, 0, 2>, 64, 0);
  else
    e = variant == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                           &per, k_force_long_sym<4, 2, 1, false, 2, false>, 128, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                           &per, k_force_long_sym_mb<2, 4, 1, false, 2, false, 16, 1, 2>, 64, 0);
  return e == cudaSuccess ? per : 0;
}

// variant 2: 4 warps x 4 disks per lane; variant 3: 2 warps x 8 disks per lane
cudaError_t bd_launch_force_sym(const BdDev &d, const BdConst &c, int variant, cudaStream_t s) {
  if (c.n_sitems == 0) return cudaSuccess;
  // periodic boxes (any replica) take the form with minimum images
  if (c.any_periodic) {
    // register budgets measured at N = 1e5 (periodic): <4,2> 2.75 -> 2.67 ms
    // with 8 resident blocks, <2,4> 3.05 -> 2.88 ms with 12
    if (variant == 2)
      k_force_long_sym_mb<4, 2, 1, false, 2, true, 8, 0, 2><<<c.n_sitems, 128, 0, s>>>(d, c);
    else
      k_force_long_sym_mb<2, 4, 1, false, 2, true, 12, 0, 2><<<c.n_sitems, 64, 0, s>>>(d, c);
  } else {
    if (variant == 2)
      k_force_long_sym<4, 2, 1, false, 2, false><<<c.n_sitems, 128, 0, s>>>(d, c);
    else
      // 16 resident blocks (32 warps) per SM in 64 registers, j tiles staged by
      // cp.async: measured 1.776 -> 1.668 ms at N = 1e5 against the
      // register-staged form (120 registers, 16 warps), forces unchanged.
      // Other shapes in the same budget measured slower at N = 1e5: ring
      // unrolled 1 or 4 steps deep (+1.7 %, +1.1 %), two j disks per lane
      // (+1.9 %), folded j accumulators (+3.5 %), one warp of 16 disks per
      // lane (+2.7 %)
      k_force_long_sym_mb<2, 4, 1, false, 2, false, 16, 1, 2><<<c.n_sitems, 64, 0, s>>>(d, c);
  }
  k_force_sym_reduce<<<c.np / BD_RED_D, 4 * BD_RED_D, 0, s>>>(d, c);
  return cudaGetLastError();
}
