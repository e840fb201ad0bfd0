// Euler-Maruyama move of one disk (Eq. (integration), Sec. 2.2; truncated
// noise, Sec. 2.4; self-propulsion, Sec. 7) and the wall reflection, shared
// by the time step and the frozen-contact replay of the adjoint.
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

namespace bdem {

__device__ __forceinline__ double snapd(double v, double q, double inv_q) {
  return __dmul_rn(rint(__dmul_rn(v, inv_q)), q);
}

__device__ __forceinline__ float4 split(double2 p) {
  float xh = __double2float_rn(p.x), yh = __double2float_rn(p.y);
  return make_float4(xh, yh, __double2float_rn(p.x - (double)xh), __double2float_rn(p.y - (double)yh));
}

// sum of the partial-force slots of disk i
__device__ __forceinline__ double2 force_sum(const BdDev &d, const BdConst &c, const BdRep &R, int i) {
  double fx = 0.0, fy = 0.0;
  const int ns = R.law == BD_LAW_LONG ? R.nchunk : (R.law == BD_LAW_SHORT ? 1 : 0);
  for (int k = 0; k < ns; ++k) {
    double2 f = d.fpart[(size_t)k * c.np + i];
    fx += f.x;
    fy += f.y;
  }
  return make_double2(fx, fy);
}

// position after the move (grid-rounded, before reflection); *thn = new angle
__device__ __forceinline__ double2 em_move(const BdConst &c, const BdRep &R, uint32_t id,
                                           long long step, double2 p, float th, double2 F,
                                           double v0, float *thn) {
  bdrng::U4 r = bdrng::draw(id, (int64_t)step, R.seed, R.replica, bdrng::TAG_NOISE);
  double nx, ny;
  if (c.precision == 0) {
    const float sc = 2.3283064365386963e-10f;  // 2^-32
    float u0 = __fmaf_rn((float)r.x, sc, 0.5f * sc), u1 = __fmaf_rn((float)r.y, sc, 0.5f * sc);
    float u2 = __fmaf_rn((float)r.z, sc, 0.5f * sc), u3 = __fmaf_rn((float)r.w, sc, 0.5f * sc);
    float ra = sqrtf(-2.0f * logf(u0)), rb = sqrtf(-2.0f * logf(u2));
    float s1, c1, s2, c2;
    sincospif(2.0f * u1, &s1, &c1);
    sincospif(2.0f * u3, &s2, &c2);
    float z0 = fminf(3.0f, fmaxf(-3.0f, ra * c1));
    float z1 = fminf(3.0f, fmaxf(-3.0f, ra * s1));
    float z2 = fminf(3.0f, fmaxf(-3.0f, rb * c2));
    float st, ct;
    sincosf(th, &st, &ct);
    const float dt = (float)R.dt, v0f = (float)v0, amp = (float)R.amp;
    float dxf = dt * ((float)F.x + v0f * ct) + amp * z0;
    float dyf = dt * ((float)F.y + v0f * st) + amp * z1;
    nx = p.x + (double)dxf;
    ny = p.y + (double)dyf;
    *thn = th + (float)R.amp_r * z2;
  } else {
    const double sc = 2.3283064365386962890625e-10;
    double u0 = ((double)r.x + 0.5) * sc, u1 = ((double)r.y + 0.5) * sc;
    double u2 = ((double)r.z + 0.5) * sc, u3 = ((double)r.w + 0.5) * sc;
    double ra = sqrt(-2.0 * log(u0)), rb = sqrt(-2.0 * log(u2));
    double s1, c1, s2, c2;
    sincospi(2.0 * u1, &s1, &c1);
    sincospi(2.0 * u3, &s2, &c2);
    double z0 = fmin(3.0, fmax(-3.0, ra * c1));
    double z1 = fmin(3.0, fmax(-3.0, ra * s1));
    double z2 = fmin(3.0, fmax(-3.0, rb * c2));
    double st, ct;
    sincos((double)th, &st, &ct);
    nx = p.x + R.dt * (F.x + v0 * ct) + R.amp * z0;
    ny = p.y + R.dt * (F.y + v0 * st) + R.amp * z1;
    *thn = (float)((double)th + R.amp_r * z2);
  }
  return make_double2(snapd(nx, c.q, c.inv_q), snapd(ny, c.q, c.inv_q));
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
