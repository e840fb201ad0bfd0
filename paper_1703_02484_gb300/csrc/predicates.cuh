// Exact orientation and in-circle predicates for the triangulation kernels
// and the host-side initial triangulation.
//
// The triangulation of Sec. 4.1 is maintained by edge flips (Sec. 4.3) whose
// decisions are the signs of two determinants: orient2d (is a triangle
// counter-clockwise?) and incircle (does a point lie inside a triangle's
// circumcircle?).  The paper evaluates them inexactly ("quasi-Delaunay",
// Sec. 4.1); here they are exact.
//
// Exactness comes from the position grid: every stored coordinate is a
// multiple of q = 2^-s with |x / q| < 2^51 (positions are rounded to the grid
// whenever they are written).  Coordinates then convert exactly to int64 and
//   orient2d  = bax*cay - bay*cax            |.| < 2^105  -> signed 128-bit
//   incircle  = sum lift_k * minor_k         |.| < 2^213  -> signed 256-bit
// are evaluated in fixed-width integer arithmetic.  On the host a plain FP64
// evaluation with a conservative error bound decides the clear cases first and
// the integer path runs only when the FP64 value is within the bound of zero.
// On the GPU the integer path always runs: on this part FP64 issues at about
// 1/64 of the FP32/INT32 rate, so the filter costs more than the exact
// evaluation it would skip (BD_PRED_DEVICE_FILTER=1 restores it).  The grid
// integer of a coordinate is read from its bit pattern (mantissa shifted by
// exponent + s), with no floating-point operation.
#pragma once
#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define BD_HD __host__ __device__ __forceinline__
#else
#define BD_HD inline
#endif

namespace bdpred {

// --- FP64 with explicit rounding (no contraction into FMA) -------------------
BD_HD double dmul(double a, double b) {
#if defined(__CUDA_ARCH__)
  return __dmul_rn(a, b);
#else
  return a * b;
#endif
}
BD_HD double dadd(double a, double b) {
#if defined(__CUDA_ARCH__)
  return __dadd_rn(a, b);
#else
  return a + b;
#endif
}
BD_HD double dsub(double a, double b) {
#if defined(__CUDA_ARCH__)
  return __dsub_rn(a, b);
#else
  return a - b;
#endif
}
BD_HD double dabs(double a) { return a < 0 ? -a : a; }

// --- 64x64 -> 128 ---------------------------------------------------------
BD_HD void mul64(uint64_t a, uint64_t b, uint64_t &lo, uint64_t &hi) {
#if defined(__CUDA_ARCH__)
  lo = a * b;
  hi = __umul64hi(a, b);
#else
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  lo = (uint64_t)p;
  hi = (uint64_t)(p >> 64);
#endif
}

// signed 128-bit value in two's complement (lo, hi)
struct i128 {
  uint64_t lo, hi;
};

BD_HD i128 neg128(i128 a) {
  i128 r;
  r.lo = ~a.lo + 1ull;
  r.hi = ~a.hi + (r.lo == 0 ? 1ull : 0ull);
  return r;
}

BD_HD i128 sub128(i128 a, i128 b) {
  i128 r;
  r.lo = a.lo - b.lo;
  r.hi = a.hi - b.hi - (a.lo < b.lo ? 1ull : 0ull);
  return r;
}

BD_HD i128 add128(i128 a, i128 b) {
  i128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1ull : 0ull);
  return r;
}

// product of two int64 values with |a|, |b| < 2^62 (fits in 127 bits)
BD_HD i128 smul64(int64_t a, int64_t b) {
  bool neg = (a < 0) != (b < 0);
  uint64_t ua = a < 0 ? (uint64_t)(-a) : (uint64_t)a;
  uint64_t ub = b < 0 ? (uint64_t)(-b) : (uint64_t)b;
  i128 r;
  mul64(ua, ub, r.lo, r.hi);
  return neg ? neg128(r) : r;
}

BD_HD int sign128(i128 a) {
  if ((int64_t)a.hi < 0) return -1;
  return (a.hi | a.lo) ? 1 : 0;
}

// signed 256-bit two's complement, limbs little-endian
struct i256 {
  uint64_t w[4];
};

// |a| * |b| for non-negative 128-bit magnitudes (each < 2^127) -> 256 bits
BD_HD i256 umul128(i128 a, i128 b) {
  uint64_t p0l, p0h, p1l, p1h, p2l, p2h, p3l, p3h;
  mul64(a.lo, b.lo, p0l, p0h);
  mul64(a.lo, b.hi, p1l, p1h);
  mul64(a.hi, b.lo, p2l, p2h);
  mul64(a.hi, b.hi, p3l, p3h);
  i256 r;
  r.w[0] = p0l;
  // limb 1 = p0h + p1l + p2l
  uint64_t s = p0h + p1l;
  uint64_t c = (s < p0h) ? 1ull : 0ull;
  uint64_t s2 = s + p2l;
  c += (s2 < s) ? 1ull : 0ull;
  r.w[1] = s2;
  // limb 2 = p1h + p2h + p3l + carry
  uint64_t t = p1h + p2h;
  uint64_t c2 = (t < p1h) ? 1ull : 0ull;
  uint64_t t2 = t + p3l;
  c2 += (t2 < t) ? 1ull : 0ull;
  uint64_t t3 = t2 + c;
  c2 += (t3 < t2) ? 1ull : 0ull;
  r.w[2] = t3;
  r.w[3] = p3h + c2;
  return r;
}

BD_HD i256 neg256(i256 a) {
  i256 r;
  uint64_t carry = 1;
  for (int k = 0; k < 4; ++k) {
    uint64_t v = ~a.w[k];
    r.w[k] = v + carry;
    carry = (carry && r.w[k] == 0) ? 1ull : 0ull;
  }
  return r;
}

BD_HD i256 add256(i256 a, i256 b) {
  i256 r;
  uint64_t carry = 0;
  for (int k = 0; k < 4; ++k) {
    uint64_t s = a.w[k] + b.w[k];
    uint64_t c1 = (s < a.w[k]) ? 1ull : 0ull;
    uint64_t s2 = s + carry;
    uint64_t c2 = (s2 < s) ? 1ull : 0ull;
    r.w[k] = s2;
    carry = c1 | c2;
  }
  return r;
}

BD_HD int sign256(i256 a) {
  if ((int64_t)a.w[3] < 0) return -1;
  return (a.w[0] | a.w[1] | a.w[2] | a.w[3]) ? 1 : 0;
}

// signed 128 (|.| < 2^127) times non-negative 128 -> signed 256
BD_HD i256 mul_s128_u128(i128 s, i128 u) {
  bool neg = (int64_t)s.hi < 0;
  i128 m = neg ? neg128(s) : s;
  i256 p = umul128(m, u);
  return neg ? neg256(p) : p;
}

// --- exact predicates on grid integers ----------------------------------------
// inputs: integer coordinates X = x / q, |X| < 2^51

BD_HD int orient_int(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy) {
  i128 l = smul64(bx - ax, cy - ay);
  i128 r = smul64(by - ay, cx - ax);
  return sign128(sub128(l, r));
}

BD_HD int incircle_int(int64_t ax, int64_t ay, int64_t bx, int64_t by, int64_t cx, int64_t cy,
                       int64_t dx, int64_t dy) {
  int64_t adx = ax - dx, ady = ay - dy;
  int64_t bdx = bx - dx, bdy = by - dy;
  int64_t cdx = cx - dx, cdy = cy - dy;
  i128 alift = add128(smul64(adx, adx), smul64(ady, ady));
  i128 blift = add128(smul64(bdx, bdx), smul64(bdy, bdy));
  i128 clift = add128(smul64(cdx, cdx), smul64(cdy, cdy));
  i128 bc = sub128(smul64(bdx, cdy), smul64(bdy, cdx));
  i128 ca = sub128(smul64(cdx, ady), smul64(cdy, adx));
  i128 ab = sub128(smul64(adx, bdy), smul64(ady, bdx));
  i256 t = mul_s128_u128(bc, alift);
  t = add256(t, mul_s128_u128(ca, blift));
  t = add256(t, mul_s128_u128(ab, clift));
  return sign256(t);
}

// --- grid <-> double ------------------------------------------------------------
struct Grid {
  double q;      // grid step 2^-s
  double inv_q;  // 2^s
  int s;
};

// x / q for a grid value x (exact: x = m 2^(e-1075), so x / q = m 2^(e-1075+s))
BD_HD int64_t to_int(double x, const Grid &g) {
  uint64_t b;
#if defined(__CUDA_ARCH__)
  b = (uint64_t)__double_as_longlong(x);
#else
  memcpy(&b, &x, sizeof(b));
#endif
  const int e = (int)((b >> 52) & 0x7FFu);
  if (e == 0) return 0;  // zero (the grid holds no subnormal values)
  const uint64_t m = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = e - 1075 + g.s;
  const uint64_t v = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);
  return (b >> 63) ? -(int64_t)v : (int64_t)v;
}

// --- filtered predicates on grid doubles ------------------------------------------
// FP64 value with a bound on its rounding error relative to the permanent
// (sum of absolute products); Shewchuk's 1997 analysis bounds it by about
// 3.3e-16 for orient2d and 1.1e-15 for incircle; the bounds below carry a
// safety factor of about nine.
#ifndef BD_PRED_FILTER
#define BD_PRED_FILTER 1
#endif
#ifndef BD_PRED_DEVICE_FILTER
#define BD_PRED_DEVICE_FILTER 0
#endif
#if defined(__CUDA_ARCH__)
#define BD_USE_FILTER (BD_PRED_FILTER && BD_PRED_DEVICE_FILTER)
#else
#define BD_USE_FILTER BD_PRED_FILTER
#endif

BD_HD int orient(double ax, double ay, double bx, double by, double cx, double cy, const Grid &g) {
#if BD_USE_FILTER
  double l = dmul(dsub(bx, ax), dsub(cy, ay));
  double r = dmul(dsub(by, ay), dsub(cx, ax));
  double det = dsub(l, r);
  double bound = dmul(3e-15, dadd(dabs(l), dabs(r)));
  if (det > bound) return 1;
  if (-det > bound) return -1;
#endif
  return orient_int(to_int(ax, g), to_int(ay, g), to_int(bx, g), to_int(by, g), to_int(cx, g),
                    to_int(cy, g));
}

BD_HD int incircle(double ax, double ay, double bx, double by, double cx, double cy, double px,
                   double py, const Grid &g) {
#if BD_USE_FILTER
  double adx = dsub(ax, px), ady = dsub(ay, py);
  double bdx = dsub(bx, px), bdy = dsub(by, py);
  double cdx = dsub(cx, px), cdy = dsub(cy, py);
  double bcl = dmul(bdx, cdy), bcr = dmul(bdy, cdx);
  double cal = dmul(cdx, ady), car = dmul(cdy, adx);
  double abl = dmul(adx, bdy), abr = dmul(ady, bdx);
  double al = dadd(dmul(adx, adx), dmul(ady, ady));
  double bl = dadd(dmul(bdx, bdx), dmul(bdy, bdy));
  double cl = dadd(dmul(cdx, cdx), dmul(cdy, cdy));
  double det = dadd(dadd(dmul(al, dsub(bcl, bcr)), dmul(bl, dsub(cal, car))), dmul(cl, dsub(abl, abr)));
  double perm = dadd(dadd(dmul(al, dadd(dabs(bcl), dabs(bcr))), dmul(bl, dadd(dabs(cal), dabs(car)))),
                     dmul(cl, dadd(dabs(abl), dabs(abr))));
  double bound = dmul(1e-14, perm);
  if (det > bound) return 1;
  if (-det > bound) return -1;
#endif
  return incircle_int(to_int(ax, g), to_int(ay, g), to_int(bx, g), to_int(by, g), to_int(cx, g),
                      to_int(cy, g), to_int(px, g), to_int(py, g));
}

// exact sign of the dot product (b0 - a0) . (b1 - a1) of two grid vectors
BD_HD int dot_sign(double a0x, double a0y, double b0x, double b0y, double a1x, double a1y,
                   double b1x, double b1y, const Grid &g) {
  int64_t ux = to_int(b0x, g) - to_int(a0x, g), uy = to_int(b0y, g) - to_int(a0y, g);
  int64_t vx = to_int(b1x, g) - to_int(a1x, g), vy = to_int(b1y, g) - to_int(a1y, g);
  return sign128(add128(smul64(ux, vx), smul64(uy, vy)));
}

}  // namespace bdpred
