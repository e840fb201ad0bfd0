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

using namespace bdf;

namespace {

__device__ __forceinline__ float2 recentre(float4 w, float2 org) {
  return make_float2(__fadd_rn(__fsub_rn(w.x, org.x), w.z), __fadd_rn(__fsub_rn(w.y, org.y), w.w));
}

// periodic box: disk j about the integer block origin o as its minimum
// image, from its stored (x_hi, y_hi, x_lo, y_lo) (tiles are copied to
// shared memory as they are): per coordinate the rounded difference
// s = x_hi - o and its error e (TwoSum), s wrapped by L when beyond L/2
// (exact: L/2 < |s| <= L), then (s, e + x_lo) renormalised (Fast2Sum), so
// that the hi part is the rounded minimum image up to the rounding of the lo
// part; L = 0 (walls): no wrap.  The i side takes the same form, which keeps
// the self pair's difference exactly 0.
__device__ __forceinline__ void rel_raw1(float h, float l, float o, float Lf, float hLf, float &hi, float &lo) {
  const float s = __fsub_rn(h, o);
  const float bb = __fsub_rn(s, h);
  const float e = __fsub_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fadd_rn(o, bb));
  const float w = s > hLf ? __fsub_rn(s, Lf) : (s < -hLf ? __fadd_rn(s, Lf) : s);
  const float t = __fadd_rn(e, l);
  hi = __fadd_rn(w, t);
  lo = __fsub_rn(t, __fsub_rn(hi, w));
}
__device__ __forceinline__ float4 rel_raw(float4 w, float2 org, float Lf, float hLf) {
  if (w.x > 1.0e17f) return make_float4(1.0e18f, 1.0e18f, 0.f, 0.f);   // inert slot
  float4 r;
  rel_raw1(w.x, w.z, org.x, Lf, hLf, r.x, r.z);
  rel_raw1(w.y, w.w, org.y, Lf, hLf, r.y, r.w);
  return r;
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

// lo parts of the disks i, kept in the thread's local memory (read only by
// the rare near tiles, so they hold no registers across the sweep)
__device__ __forceinline__ void st_local4(float4 *p, float4 v) {
  asm volatile("st.local.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(__cvta_generic_to_local(p)), "f"(v.x), "f"(v.y),
               "f"(v.z), "f"(v.w)
               : "memory");
}
__device__ __forceinline__ float4 ld_local4(const float4 *p) {
  float4 v;
  asm volatile("ld.local.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(__cvta_generic_to_local(p)));
  return v;
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
// origin as its minimum image, as an FP32 (hi, lo) pair (rel_raw); each warp
// holds a contiguous quarter (half) of the block's disks i.  Per (warp, group
// of 32 disks j) the warp's box of its disks i and the group's box (taken
// about one of its disks, so a group across the antipode is not mistaken for
// one spanning the box) tell which pair form every pair of the two may take
// (pair_mode): hi parts alone; per-pair minimum image on one axis or both;
// the exact vector for boxes closer than 20.
// STAGE: 0 stage the next j tile through registers (re-centred on the way to
// shared memory); 1 copy it raw with cp.async (no registers held across the
// tile's arithmetic) and re-centre each j as it is read (walls), or, PER,
// re-centre the tile in place once it has landed.  PER takes STAGE 1.
// ACC: the i side's sum over an item's tiles, 2 in (hi, lo) float-float, 1 in
// FP32 (half the registers).
template <int NW, int NP, int NJ, bool COMB, int UR, bool PER, int STAGE = 0, int ACC = 2>
__device__ __forceinline__ void force_long_sym_body(const BdDev &d, const BdConst &c) {
  static_assert(!PER || STAGE == 1, "the periodic form re-centres tiles in shared memory");
  if (ctl_failed(d.ctl)) return;
  constexpr int T = NW * 32;         // threads
  constexpr int NQ = 2 * NP;         // disks i per thread
  constexpr int NS = BD_TJ / T;      // j disks each thread stages per tile
  constexpr int NG = BD_TJ / 32;     // groups of 32 disks j per tile
  static_assert(BD_SB == T * NQ, "a block is BD_SB disks");
  __shared__ float2 sjp[2][STAGE ? 1 : BD_TJ];   // j positions, re-centred
  __shared__ __align__(16) float4 sraw[2][STAGE ? BD_TJ : 1];   // STAGE 1: j as stored (x_hi, y_hi, x_lo, y_lo);
                                                                // PER: re-centred in place (hi, lo)
  __shared__ float2 shw[NW][BD_TJ];  // per-warp j-side sums of the current tile
  __shared__ float4 sgbox[2][PER ? NG : 1];   // PER: per-group boxes of the staged tile
  __shared__ int sgpad[2][PER ? NG : 1];      //      and whether the group holds inert slots
  __shared__ float4 sibox[PER ? NW : 1];      //      per-warp boxes of the block's disks i
  __shared__ int sipad[PER ? NW : 1];         //      and whether they include inert slots
  const int item_id = c.sitem0 + (int)blockIdx.x;   // this launch's share of the plan (force sharding)
  const int4 item = d.sitems[item_id];
  const int P = item.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int base = P * BD_SB;
  const int tsym = 2 * P + 2;        // first tile met from both sides
  const int2 binfo = d.sblock[P];
  const BdRep &R = d.rep[binfo.x];
  const int a = binfo.y;
  const float2 org = d.sorigin[P];
  bool per = false;                  // this block's replica is periodic
  float Lf = 0.f, hLf = __int_as_float(0x7f800000);
  if (PER && R.periodic) {
    per = true;
    Lf = R.Lf;
    hLf = R.hLf;
  }
  auto rel = [&](int j) -> float4 {
    if (PER) return rel_raw(d.work[j], org, Lf, hLf);
    const float2 v = recentre(d.work[j], org);
    return make_float4(v.x, v.y, 0.f, 0.f);
  };
  // slot (in the block) of this thread's disk i number q
  auto islot = [&](int q) -> int { return PER ? warp * (BD_SB / NW) + q * 32 + lane : q * T + tid; };
  u64 xi2[NP], yi2[NP], ax2[NP], ay2[NP];
  float4 ilo[PER ? NP : 1];          // PER: lo parts of the disks i (x0, y0, x1, y1), local memory
  float fxh[NQ], fxl[ACC == 2 ? NQ : 1], fyh[NQ], fyl[ACC == 2 ? NQ : 1];
  float4 ibox = sempty_box();
  bool ipad = false;
#pragma unroll
  for (int k = 0; k < NP; ++k) {
    const float4 p0 = rel(base + islot(2 * k));
    const float4 p1 = rel(base + islot(2 * k + 1));
    xi2[k] = pk2(p0.x, p1.x);
    yi2[k] = pk2(p0.y, p1.y);
    if (PER) st_local4(&ilo[k], make_float4(p0.z, p0.w, p1.z, p1.w));
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
      if constexpr (PER) {
        // each thread re-centres the slots it copied (its own copies are
        // visible to it after the wait), in place; the warp's 32 slots of
        // stage m are group m NW + warp, whose box is taken about its first
        // live disk (minimum images about it), then shifted back
#pragma unroll
        for (int m = 0; m < NS; ++m) {
          const float4 v = rel_raw(sraw[b][m * T + tid], org, Lf, hLf);
          sraw[b][m * T + tid] = v;
          const bool live = v.x < 1.0e17f;
          const unsigned bal = __ballot_sync(0xffffffffu, live);
          float4 bx = sempty_box();
          if (bal) {
            const int src = __ffs(bal) - 1;
            const float rx = __shfl_sync(0xffffffffu, v.x, src), ry = __shfl_sync(0xffffffffu, v.y, src);
            if (live) {
              float dx = __fsub_rn(v.x, rx), dy = __fsub_rn(v.y, ry);
              if (per) {
                dx = dx > hLf ? __fsub_rn(dx, Lf) : (dx < -hLf ? __fadd_rn(dx, Lf) : dx);
                dy = dy > hLf ? __fsub_rn(dy, Lf) : (dy < -hLf ? __fadd_rn(dy, Lf) : dy);
              }
              bx = make_float4(dx, dx, dy, dy);
            }
            bx = swarp_box(bx);
            bx = make_float4(__fadd_rn(rx, bx.x), __fadd_rn(rx, bx.y), __fadd_rn(ry, bx.z), __fadd_rn(ry, bx.w));
          }
          if (lane == 0) {
            sgbox[b][m * NW + warp] = bx;
            sgpad[b][m * NW + warp] = bal != 0xffffffffu ? 1 : 0;
          }
        }
      }
    } else {
#pragma unroll
      for (int m = 0; m < NS; ++m) sjp[b][m * T + tid] = make_float2(st[m].x, st[m].y);
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
    if constexpr (STAGE == 1 && PER) return make_float2(sraw[buf][jj].x, sraw[buf][jj].y);
    else if constexpr (STAGE == 1) return recentre(sraw[buf][jj], org);
    else return sjp[buf][jj];
  };
  // PER: its lo parts
  auto jlo = [&](int jj) -> float2 { return make_float2(sraw[buf][jj].z, sraw[buf][jj].w); };
  // pair differences (r_j - r_i), per axis AX (0: x, 1: y), by the pair form
  // MODE: 0 the hi parts alone; 1 the exact near-pair vector (hi_j - hi_i) +
  // (lo_j - lo_i); 2 the hi difference's packed minimum image on both axes;
  // 3 the same by compares (inert slots, which must stay far away, take part);
  // 5 / 6 the packed minimum image on x / y alone (an inert slot stays far
  // away on the other axis); 4 near pairs across the antipode (boxes of a
  // size near L/2): the hi difference, about L there, is formed exactly as
  // s + e (TwoDiff), s takes the minimum image (exact: |s| in [L/2, 3L/2]),
  // then e and the lo difference are added.  Far pairs (all forms but 1 and
  // 4) drop the lo parts, as form 0 does.
  auto diff = [&](auto MODE, auto AX, u64 jh2, u64 ih2, u64 jl2, u64 il2) -> u64 {
    constexpr int m0 = decltype(MODE)::value, ax = decltype(AX)::value;
    constexpr int mode = m0 == 5 ? (ax == 0 ? 2 : 0) : (m0 == 6 ? (ax == 1 ? 2 : 0) : m0);
    u64 dd = sub2(jh2, ih2);
    if constexpr (mode == 4) {
      const u64 v = sub2(dd, jh2);
      const u64 e = sub2(sub2(jh2, sub2(dd, v)), add2(ih2, v));
      return add2(min_image2_cmp(dd, Lf, hLf), add2(e, sub2(jl2, il2)));
    }
    if constexpr (mode == 2) dd = min_image2(dd, invL2, nL2, M2);
    if constexpr (mode == 3) dd = min_image2_cmp(dd, Lf, hLf);
    if constexpr (mode == 1) dd = add2(dd, sub2(jl2, il2));
    return dd;
  };
  using AXX = std::integral_constant<int, 0>;
  using AXY = std::integral_constant<int, 1>;
  // PER: the pair form of this warp's disks i with the j groups g0 .. g0 +
  // ng - 1 of the current tile.  Pair components range over [j_min - i_max,
  // j_max - i_min]; a plain difference is the minimum image when that range
  // and the j coordinates themselves lie inside (-L/2, L/2) (then each j is
  // stored as the image its box describes), with a margin of 2^-16 L/2 for
  // the rounding of the boxes.  Near: the range comes within 20 of 0 or L.
  auto pair_mode = [&](int g0, int ng) -> int {
    if constexpr (!PER) return 0;
    const float4 ib = sibox[warp];
    if (ib.x > ib.y) return 0;                 // the warp's disks i are all inert
    float4 jb = sempty_box();
    int pad = sipad[warp];
    for (int u = 0; u < ng; ++u) {
      jb = smerge_box(jb, sgbox[buf][g0 + u]);
      pad |= sgpad[buf][g0 + u];
    }
    if (jb.x > jb.y) return 0;                 // inert disks j only: their pairs vanish
    const float lox = __fsub_rn(jb.x, ib.y), hix = __fsub_rn(jb.y, ib.x);
    const float loy = __fsub_rn(jb.z, ib.w), hiy = __fsub_rn(jb.w, ib.z);
    const float hLm = __fmul_rn(hLf, 1.0f - 1.0f / 65536.0f);
    const bool wx = per && (hix > hLm || lox < -hLm || jb.y > hLm || jb.x < -hLm);
    const bool wy = per && (hiy > hLm || loy < -hLm || jb.w > hLm || jb.z < -hLm);
    auto gap = [&](float lo, float hi) -> float {
      float g = fmaxf(0.f, fmaxf(lo, -hi));
      if (per) {
        g = fminf(g, fmaxf(0.f, fmaxf(__fsub_rn(lo, Lf), -__fsub_rn(hi, Lf))));
        g = fminf(g, fmaxf(0.f, fmaxf(__fadd_rn(lo, Lf), -__fadd_rn(hi, Lf))));
      }
      return g;
    };
    const float gx = gap(lox, hix), gy = gap(loy, hiy);
    // boxes closer than 20: the exact vector keeps their pairs at FP32
    // resolution of their separation (coordinates reach L/2 from the block
    // origin, where one rounding costs ulp(L/2) / 2)
    const bool near = gx * gx + gy * gy < 400.f;
    return near ? (wx || wy ? 4 : 1) : (wx && wy ? (pad ? 3 : 2) : (wx ? 5 : (wy ? 6 : 0)));
  };
  using M0 = std::integral_constant<int, 0>;
  using M1 = std::integral_constant<int, 1>;
  using M2c = std::integral_constant<int, 2>;
  using M3 = std::integral_constant<int, 3>;
  using M4 = std::integral_constant<int, 4>;
  using M5 = std::integral_constant<int, 5>;
  using M6 = std::integral_constant<int, 6>;
  auto dispatch = [&](int mode, auto &&fn) {
    if constexpr (PER) {
      if (mode == 1) fn(M1());
      else if (mode == 2) fn(M2c());
      else if (mode == 3) fn(M3());
      else if (mode == 4) fn(M4());
      else if (mode == 5) fn(M5());
      else if (mode == 6) fn(M6());
      else fn(M0());
    } else {
      fn(M0());
    }
  };
  auto own_group = [&](auto MODE, int g) {
    // the block's own disks: i side only, j broadcast from shared memory
    constexpr bool LO = decltype(MODE)::value == 1 || decltype(MODE)::value == 4;
#pragma unroll 4
    for (int jj = g * 32; jj < g * 32 + 32; ++jj) {
      const float2 p = jpos(jj);
      const u64 jx2 = pk2(p.x, p.x), jy2 = pk2(p.y, p.y);
      u64 jxl2 = 0ull, jyl2 = 0ull;
      if constexpr (LO) {
        const float2 pl = jlo(jj);
        jxl2 = pk2(pl.x, pl.x);
        jyl2 = pk2(pl.y, pl.y);
      }
#pragma unroll
      for (int k = 0; k < NP; ++k) {
        u64 ixl2 = 0ull, iyl2 = 0ull;
        if constexpr (LO) {
          const float4 il = ld_local4(&ilo[k]);
          ixl2 = pk2(il.x, il.z);
          iyl2 = pk2(il.y, il.w);
        }
        const u64 dx = diff(MODE, AXX(), jx2, xi2[k], jxl2, ixl2);
        const u64 dy = diff(MODE, AXY(), jy2, yi2[k], jyl2, iyl2);
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
  auto ring_group = [&](auto MODE, int g) {
    // a later tile's group g: every pair once, both sides; each lane carries NJ disks j
    constexpr bool LO = decltype(MODE)::value == 1 || decltype(MODE)::value == 4;
    float jx[NJ], jy[NJ], jxl[NJ], jyl[NJ];
    u64 hx2[NJ], hy2[NJ];
#pragma unroll
    for (int m = 0; m < NJ; ++m) {
      const float2 p = jpos((g * NJ + m) * 32 + lane);
      jx[m] = p.x;
      jy[m] = p.y;
      jxl[m] = jyl[m] = 0.f;
      if constexpr (LO) {
        const float2 pl = jlo((g * NJ + m) * 32 + lane);
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
          u64 ixl2 = 0ull, iyl2 = 0ull;
          if constexpr (LO) {
            const float4 il = ld_local4(&ilo[k]);
            ixl2 = pk2(il.x, il.z);
            iyl2 = pk2(il.y, il.w);
          }
          const u64 dx = diff(MODE, AXX(), jx2, xi2[k], jxl2, ixl2);
          const u64 dy = diff(MODE, AXY(), jy2, yi2[k], jyl2, iyl2);
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
  };
  for (int t = t_begin; t < t_end; ++t) {
    if (t + 1 < t_end) fetch(t + 1);
    const int b = d.tile_species[t];
    if (t < tsym) {
      for (int g = 0; g < NG; ++g)
        dispatch(pair_mode(g, 1), [&](auto M) { own_group(M, g); });
    } else {
      for (int g = 0; g < BD_TJ / (32 * NJ); ++g)
        dispatch(pair_mode(g * NJ, NJ), [&](auto M) { ring_group(M, g); });
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
    if constexpr (ACC == 2) ip[islot(q)] = make_float2(__fadd_rn(fxh[q], fxl[q]), __fadd_rn(fyh[q], fyl[q]));
    else ip[islot(q)] = make_float2(fxh[q], fyh[q]);
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
                           &per, k_force_long_sym_mb<4, 2, 1, false, 2, true, 8, 1, 2>, 128, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                           &per, k_force_long_sym_mb<2, 4, 1, false, 2, true, 12, 1, 2>, 64, 0);
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
    // measured at N = 1e5 (periodic), step times with pair forms chosen per
    // (warp, group of 32 disks j): <2,4> 2.241 ms with 12 resident blocks
    // (2.248 with 16, 2.288 with 10), <4,2> 2.464 ms with 8 (2.519 with 6);
    // 2.86 ms before, with one form per (block, tile) and the tiles staged
    // through registers
    if (variant == 2)
      k_force_long_sym_mb<4, 2, 1, false, 2, true, 8, 1, 2><<<c.n_sitems, 128, 0, s>>>(d, c);
    else
      k_force_long_sym_mb<2, 4, 1, false, 2, true, 12, 1, 2><<<c.n_sitems, 64, 0, s>>>(d, c);
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
