// Euler-Maruyama move of one disk (Eq. (integration), Sec. 2.2; truncated
// noise, Sec. 2.4; self-propulsion, Sec. 7) and the wall reflection, shared
// by the time step and the frozen-contact replay of the adjoint.  In FP32
// mode the move, the reflection and the FP32 copy of the position are formed
// in integer grid units (no FP64 arithmetic).
//   y = x + dt (F + v0 (cos th, sin th)) + amp xi,   th' = th + amp_r n
// Philox4x32-10 words -> Box-Muller -> clamp to [-3, 3]; xi = (z0, z1),
// n = z2.  The increment is formed in FP32 (FP64 when precision = 1), added
// to the FP64 master position and rounded to the position grid.
#pragma once
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "bd_internal.h"
#include "philox.cuh"
#include "predicates.cuh"

namespace bdem {

__device__ __forceinline__ double snapd(double v, double q, double inv_q) {
  return __dmul_rn(rint(__dmul_rn(v, inv_q)), q);
}

__device__ __forceinline__ float4 split(double2 p) {
  float xh = __double2float_rn(p.x), yh = __double2float_rn(p.y);
  return make_float4(xh, yh, __double2float_rn(p.x - (double)xh), __double2float_rn(p.y - (double)yh));
}

// sum of the partial-force slots of disk i (a single slot is read as is)
__device__ __forceinline__ double2 force_sum(const BdDev &d, const BdConst &c, const BdRep &R, int i) {
  const int ns = R.law == BD_LAW_LONG ? R.nchunk : (R.law == BD_LAW_SHORT ? 1 : 0);
  if (ns == 0) return make_double2(0.0, 0.0);
  double2 f = d.fpart[i];
  for (int k = 1; k < ns; ++k) {
    const double2 g = d.fpart[(size_t)k * c.np + i];
    f.x += g.x;
    f.y += g.y;
  }
  return f;
}

// ---- exact position-grid arithmetic without FP64 instructions ----
// Positions are multiples of q = 2^-s held as doubles; X = x / q is an
// integer below 2^51 in magnitude (bdpred::to_int reads it from the bit
// pattern).  The conversions used here run on the conversion pipe, whereas FP64
// arithmetic issues at 1/64 of the FP32 rate on this part.

// X q as a double: exact int64 -> FP64 conversion, then 2^-s on the exponent
__device__ __forceinline__ double grid_to_double(long long X, int s) {
  if (X == 0) return 0.0;
  return __longlong_as_double(__double_as_longlong(__ll2double_rn(X)) - ((long long)s << 52));
}

// X q rounded to FP32 (round to nearest even), for |X q| >= 2^-100
__device__ __forceinline__ float grid_to_float(long long X, int s) {
  if (X == 0) return 0.f;
  return __int_as_float(__float_as_int(__ll2float_rn(X)) - (s << 23));
}

// the (hi, lo) FP32 pair of split(): hi = X q rounded to FP32, lo = the rest
// rounded to FP32
__device__ __forceinline__ float2 grid_split(long long X, int s) {
  const float h = __ll2float_rn(X);          // integer valued
  const long long r = X - __float2ll_rn(h);  // exact
  return make_float2(X == 0 ? 0.f : __int_as_float(__float_as_int(h) - (s << 23)), grid_to_float(r, s));
}

// periodic re-entry in grid units (Sec. 2.1): X, Y brought into [0, LQ).
// Returns the wrap code: bits 0-1 (x) and 2-3 (y) hold k in 2-bit two's
// complement, where the stored coordinate is the geometric one less L k.
__device__ __forceinline__ int wrap_grid(long long LQ, long long &X, long long &Y) {
  int f = 0;
  if (X < 0) { X += LQ; f |= 3; } else if (X >= LQ) { X -= LQ; f |= 1; }
  if (Y < 0) { Y += LQ; f |= 12; } else if (Y >= LQ) { Y -= LQ; f |= 4; }
  return f;
}

// mirror reflection at the walls in grid units (flag bits as reflect())
__device__ __forceinline__ int reflect_grid(long long lo, long long hi, long long &X, long long &Y) {
  int f = 0;
  if (X < lo) { X = 2 * lo - X; f |= 1; }
  if (X > hi) { X = 2 * hi - X; f |= 2; }
  if (Y < lo) { Y = 2 * lo - Y; f |= 4; }
  if (Y > hi) { Y = 2 * hi - Y; f |= 8; }
  return f;
}

// Philox counter word 3 of the noise of piece `node` of a step (Sec. 4.3: a
// rejected move is repeated with a lower dt).  Pieces are numbered as a
// binary heap: 1 is the whole step (noise word TAG_NOISE), 2k and 2k+1 are
// the halves of piece k (word TAG_NOISE + 256 node).
__device__ __forceinline__ uint32_t piece_tag(uint32_t node) {
  return node <= 1u ? bdrng::TAG_NOISE : bdrng::TAG_NOISE + 256u * node;
}

// depth of a piece in the heap numbering: its length is dt / 2^depth
__device__ __forceinline__ int piece_depth(uint32_t node) { return node <= 1u ? 0 : 31 - __clz(node); }

// Philox words -> three clamped standard normals, Sec. 2.4 option (b):
// u = (x + 1/2) 2^-32, Box-Muller on (u0, u1) and (u2, u3), each value
// truncated to [-3, 3]; (z0, z1) drive the translation, z2 the director.
// FP32 form (the FP32 step) and FP64 form (the FP64 step).
__device__ __forceinline__ float3 normals_f32(const bdrng::U4 &r) {
  const float sc = 2.3283064365386963e-10f;  // 2^-32
  float u0 = __fmaf_rn((float)r.x, sc, 0.5f * sc), u1 = __fmaf_rn((float)r.y, sc, 0.5f * sc);
  float u2 = __fmaf_rn((float)r.z, sc, 0.5f * sc), u3 = __fmaf_rn((float)r.w, sc, 0.5f * sc);
  float ra = sqrtf(-2.0f * logf(u0)), rb = sqrtf(-2.0f * logf(u2));
  float s1, c1, s2, c2;
  sincospif(2.0f * u1, &s1, &c1);
  sincospif(2.0f * u3, &s2, &c2);
  return make_float3(fminf(3.0f, fmaxf(-3.0f, ra * c1)), fminf(3.0f, fmaxf(-3.0f, ra * s1)),
                     fminf(3.0f, fmaxf(-3.0f, rb * c2)));
}

__device__ __forceinline__ double3 normals_f64(const bdrng::U4 &r) {
  const double sc = 2.3283064365386962890625e-10;
  double u0 = ((double)r.x + 0.5) * sc, u1 = ((double)r.y + 0.5) * sc;
  double u2 = ((double)r.z + 0.5) * sc, u3 = ((double)r.w + 0.5) * sc;
  double ra = sqrt(-2.0 * log(u0)), rb = sqrt(-2.0 * log(u2));
  double s1, c1, s2, c2;
  sincospi(2.0 * u1, &s1, &c1);
  sincospi(2.0 * u3, &s2, &c2);
  return make_double3(fmin(3.0, fmax(-3.0, ra * c1)), fmin(3.0, fmax(-3.0, ra * s1)),
                      fmin(3.0, fmax(-3.0, rb * c2)));
}

// FP32 move of piece `node` of step `step` in grid units (before
// reflection): X = x/q + rint(dx/q) with the increment dx formed in FP32;
// *thn = new angle
__device__ __forceinline__ void em_move_grid(const BdConst &c, const BdRep &R, uint32_t id,
                                             long long step, double2 p, float th, double2 F,
                                             double v0, float *thn, uint32_t node, long long *X,
                                             long long *Y) {
  bdrng::U4 r = bdrng::draw(id, (int64_t)step, R.seed, R.replica, piece_tag(node));
  const int depth = piece_depth(node);
  // length of this move and its noise amplitudes: dt / 2^depth, amp / 2^(depth/2)
  float dt = (float)R.dt, amp = (float)R.amp, amp_r = (float)R.amp_r;
  if (depth) {
    const double sc = sqrt(ldexp(1.0, -depth));
    dt = (float)ldexp(R.dt, -depth);
    amp = (float)(R.amp * sc);
    amp_r = (float)(R.amp_r * sc);
  }
  const float3 z = normals_f32(r);
  const float z0 = z.x, z1 = z.y, z2 = z.z;
  float st, ct;
  sincosf(th, &st, &ct);
  const float v0f = (float)v0;
  float dxf = dt * ((float)F.x + v0f * ct) + amp * z0;
  float dyf = dt * ((float)F.y + v0f * st) + amp * z1;
  *thn = th + amp_r * z2;
  const bdpred::Grid g{c.q, c.inv_q, c.qshift};
  const float to_grid = __int_as_float((127 + c.qshift) << 23);   // 2^s, exact scaling
  *X = bdpred::to_int(p.x, g) + __float2ll_rn(dxf * to_grid);
  *Y = bdpred::to_int(p.y, g) + __float2ll_rn(dyf * to_grid);
}

// position after the move of piece `node` of step `step` (grid-rounded, before
// reflection); *thn = new angle
__device__ __forceinline__ double2 em_move(const BdConst &c, const BdRep &R, uint32_t id,
                                           long long step, double2 p, float th, double2 F,
                                           double v0, float *thn, uint32_t node = 1u) {
  if (c.precision == 0) {
    long long X, Y;
    em_move_grid(c, R, id, step, p, th, F, v0, thn, node, &X, &Y);
    return make_double2(grid_to_double(X, c.qshift), grid_to_double(Y, c.qshift));
  }
  bdrng::U4 r = bdrng::draw(id, (int64_t)step, R.seed, R.replica, piece_tag(node));
  const int depth = piece_depth(node);
  // length of this move and its noise amplitudes: dt / 2^depth, amp / 2^(depth/2)
  const double dt_p = depth ? ldexp(R.dt, -depth) : R.dt;
  const double amp_scale = depth ? sqrt(ldexp(1.0, -depth)) : 1.0;
  const double amp_p = R.amp * amp_scale, amp_rp = R.amp_r * amp_scale;
  // FP64 mode
  const double3 z = normals_f64(r);
  const double z0 = z.x, z1 = z.y, z2 = z.z;
  double st, ct;
  sincos((double)th, &st, &ct);
  const double nx = p.x + dt_p * (F.x + v0 * ct) + amp_p * z0;
  const double ny = p.y + dt_p * (F.y + v0 * st) + amp_p * z1;
  *thn = (float)((double)th + amp_rp * z2);
  return make_double2(snapd(nx, c.q, c.inv_q), snapd(ny, c.q, c.inv_q));
}

// the walls (lo, hi) that disk i's centre stays between: its own for
// polydisperse disks (a_i from each wall), else the replica's
__device__ __forceinline__ double2 walls_of(const BdDev &d, const BdRep &R, int i) {
  return d.wall ? d.wall[i] : make_double2(R.wall_lo, R.wall_hi);
}

// mirror reflection between walls w = (lo, hi); flags as reflect()
__device__ __forceinline__ double2 reflect_w(double2 w, double2 y, int *flags) {
  int f = 0;
  if (y.x < w.x) { y.x = 2.0 * w.x - y.x; f |= 1; }
  if (y.x > w.y) { y.x = 2.0 * w.y - y.x; f |= 2; }
  if (y.y < w.x) { y.y = 2.0 * w.x - y.y; f |= 4; }
  if (y.y > w.y) { y.y = 2.0 * w.y - y.y; f |= 8; }
  *flags = f;
  return y;
}

// mirror reflection at the walls; flags bits: 1 x<lo, 2 x>hi, 4 y<lo, 8 y>hi
__device__ __forceinline__ double2 reflect(const BdRep &R, double2 y, int *flags) {
  int f = 0;
  if (y.x < R.wall_lo) { y.x = 2.0 * R.wall_lo - y.x; f |= 1; }
  if (y.x > R.wall_hi) { y.x = 2.0 * R.wall_hi - y.x; f |= 2; }
  if (y.y < R.wall_lo) { y.y = 2.0 * R.wall_lo - y.y; f |= 4; }
  if (y.y > R.wall_hi) { y.y = 2.0 * R.wall_hi - y.y; f |= 8; }
  *flags = f;
  return y;
}

// the same reflections as recorded (frozen replay)
__device__ __forceinline__ double2 reflect_as(const BdRep &R, double2 y, int f) {
  if (f & 1) y.x = 2.0 * R.wall_lo - y.x;
  if (f & 2) y.x = 2.0 * R.wall_hi - y.x;
  if (f & 4) y.y = 2.0 * R.wall_lo - y.y;
  if (f & 8) y.y = 2.0 * R.wall_hi - y.y;
  return y;
}

}  // namespace bdem
