// Triangulation stages of one time step, as one persistent cooperative
// kernel (Algorithm 1 lines 5-7, Sec. 4.3-4.4):
//
//   P  validity (Sec. 4.3): r0_ij . r1_ij < 0 on any triangulation edge with a
//      moved end point rejects the step; every triangle with a moved corner is
//      re-oriented and flagged "inverted" when not strictly counter-clockwise;
//      in the same pass the Lawson marks (L) and the overlap scan (O) below.
//   R  inversion repair: an edge between an inverted triangle and its
//      neighbour is flipped when both triangles of the other diagonal come out
//      counter-clockwise -- the orientation form of Eq. (predicate) (the
//      moved vertex lies inside the neighbour's triangle, Fig. 4).  Rounds
//      repeat until no triangle is inverted; no candidate left => reject.
//   F  Lawson flips (Sec. 4.1, Navarro et al.): an edge whose opposite vertex
//      lies strictly inside the circumcircle of the other triangle is flipped;
//      rounds repeat until none is left.  Only edges touching a triangle that
//      moved or flipped are re-tested: by the flip itself, which tests the
//      four outer edges of its quadrilateral and registers the illegal ones
//      for the next round (fused rounds), or by a check pass after the round.
//   A  overlap correction (Algorithm 2): every real edge with r < sigma adds
//      -+ (sigma - r) r_hat to its end points' displacement (fixed-point
//      integer atomics: the sums do not depend on the order); each
//      disk then moves by its sum capped at sigma/4 (Sec. 4.4) and reflects at
//      the walls.  The sums are those of the scan of P, kept through fused
//      Lawson rounds (a flip withdraws the contribution of the diagonal it
//      removes and adds that of the one it draws).  Then P-R-F run again on
//      the moved disks, and the loop ends
//      when a pass over the Delaunay edges of the current positions finds no
//      overlap (the closest pair of a point set is a Delaunay edge, so no pair
//      anywhere is closer than sigma).
//
// Parallel flips: a candidate edge claims the six triangles its flip touches
// (the pair and the four across its outer edges) with a 64-bit atomicMax of
// (round, corner id); an edge that holds all six claims flips in place (the
// two triangle slots are reused) and rewrites its neighbours' back-pointers in
// the same round, since no other flip of the round touches them.
//
// Predicates: orientation and incircle are exact (integer arithmetic on the
// position grid, predicates.cuh), behind an FP32 filter that decides the clear
// cases from the disks' FP32 (hi, lo) position pairs.
//
// Grid-wide barriers spin with a time limit: a barrier that waits longer
// than BD_BARRIER_TIMEOUT_NS sets BD_ERR_DEVICE_TIMEOUT and every block leaves.
// On any failure the step is undone from the launch's undo journal: the first
// change a launch makes to a triangle (a flip, its back-pointers, a periodic
// shift) records the triangle's corners and neighbours as they were.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bd_internal.h"
#include "em.cuh"
#include "gridsync.cuh"
#include "predicates.cuh"

#define BD_DT_THREADS 256

using namespace bdgs;

namespace {

enum { STAGE_P = 0, STAGE_R = 1, STAGE_F = 2, STAGE_A = 3, STAGE_PL = 4 };

// lead thread only: charge the time since the last mark to a stage
__device__ __forceinline__ void stage_tick(BdCtl *ctl, int stage, unsigned long long &mark) {
  const unsigned long long now = gtimer();
  ctl->st_stage_ns[stage] += now - mark;
  ctl->st_stage_cnt[stage] += 1;
  mark = now;
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
  float sig2f;   // sigma^2 (1 + 1e-5): FP32 screen of the overlap scan
  unsigned jstamp;   // this launch's undo-journal mark (odd)
};

// FP32 filters in front of the exact integer predicates.  Every disk's
// position is also held as an FP32 pair (x_hi, x_lo) with x_hi + x_lo equal to
// the FP64 position to ~1e-11 a (the sweeps' copy), so a coordinate
// difference (b_hi - a_hi) + (b_lo - a_lo) carries one FP32 rounding of
// itself (relative 2^-24).  The determinant is then evaluated in FP32 with
// explicit rounding and compared with a bound on its error relative to the
// permanent (the same expression with absolute values): Shewchuk's bounds for
// exact inputs (3e-16 / 1.1e-15 relative in FP64, i.e. about 4 and 11 units
// of the working precision) plus one unit per input factor, times a safety
// factor of about four.  Outside the bound the FP32 sign is the exact sign;
// inside it, or for ghost points (no FP32 copy), the integer path decides.
__device__ __forceinline__ float fdiff(float bh, float bl, float ah, float al) {
  return __fadd_rn(__fsub_rn(bh, ah), __fsub_rn(bl, al));
}

// The exact integer paths are rare (the filters decide almost every case) and
// long; they are kept out of line, one copy each, so that a thread that needs
// one fetches a single shared instruction stream rather than a cold inlined
// copy at every call site (a miss in the instruction cache costs about an L2
// round trip per line, and the slowest thread of a pass sets its length).
__device__ __noinline__ int orient_exact(const double2 *__restrict__ pos, bdpred::Grid g, int a, int b, int c) {
  const double2 pa = pos[a], pb = pos[b], pc = pos[c];
  return bdpred::orient(pa.x, pa.y, pb.x, pb.y, pc.x, pc.y, g);
}

__device__ __noinline__ int incircle_exact(const double2 *__restrict__ pos, bdpred::Grid g, int a, int b, int c,
                                           int p) {
  const double2 pa = pos[a], pb = pos[b], pc = pos[c], pp = pos[p];
  return bdpred::incircle(pa.x, pa.y, pb.x, pb.y, pc.x, pc.y, pp.x, pp.y, g);
}

__device__ __noinline__ int orient_lifted(long long ax, long long ay, long long bx, long long by, long long cx,
                                          long long cy) {
  return bdpred::orient_int(ax, ay, bx, by, cx, cy);
}

__device__ __noinline__ int incircle_lifted(long long ax, long long ay, long long bx, long long by, long long cx,
                                            long long cy, long long px, long long py) {
  return bdpred::incircle_int(ax, ay, bx, by, cx, cy, px, py);
}

// Algorithm 2's per-disk displacement sums as fixed-point integers in the
// disp words: integer adds are associative, so the sum (and every position
// after the pass) does not depend on the order the edges arrive in.  A
// contribution is rounded to disp_unscale (a small fraction of the position
// grid) once; zero is the same bit pattern in both readings of the words.
__device__ __forceinline__ void disp_add(const Ctx &x, int i, double vx, double vy) {
  long long *w = (long long *)&x.d.disp[i];
  atomicAdd((unsigned long long *)&w[0], (unsigned long long)__double2ll_rn(__dmul_rn(vx, x.c.disp_scale)));
  atomicAdd((unsigned long long *)&w[1], (unsigned long long)__double2ll_rn(__dmul_rn(vy, x.c.disp_scale)));
}
__device__ __forceinline__ double2 disp_get(const Ctx &x, int i) {
  const longlong2 w = *(const longlong2 *)&x.d.disp[i];
  return make_double2(__dmul_rn((double)w.x, x.c.disp_unscale), __dmul_rn((double)w.y, x.c.disp_unscale));
}

// Algorithm 2's overlap test of the disk pair (u, w), w's image shifted by
// (rsx, rsy) L: an exact pre-test in grid units, |r_w - r_u|^2 <= (sigma/q)^2
// (1 + 1e-9), then the decision r < a_u + a_w in FP64 as the reference makes
// it (the difference of two grid values is exact in FP64).  On overlap, v is
// the push of w, (a_u + a_w - r) (r_w - r_u) / r; u's is -v.
__device__ __forceinline__ bool edge_overlap(const Ctx &x, int u, int w, int rsx, int rsy, long long LQ, double2 &v,
                                             double &del) {
  const double2 pu = x.d.pos[u], pw = x.d.pos[w];
  const int64_t ix = bdpred::to_int(pw.x, x.g) - bdpred::to_int(pu.x, x.g) + rsx * LQ;
  const int64_t iy = bdpred::to_int(pw.y, x.g) - bdpred::to_int(pu.y, x.g) + rsy * LQ;
  const bdpred::i128 ir2 = bdpred::add128(bdpred::smul64(ix, ix), bdpred::smul64(iy, iy));
  const bool near = ir2.hi < x.c.sig2q_hi || (ir2.hi == x.c.sig2q_hi && ir2.lo <= x.c.sig2q_lo);
  if (!near) return false;
  const double dx = bdem::grid_to_double(ix, x.g.s), dy = bdem::grid_to_double(iy, x.g.s);
  const double r = sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
  const double sg = x.d.rad ? x.d.rad[u] + x.d.rad[w] : x.c.sigma;   // polydisperse: a_u + a_w
  if (!(r < sg)) return false;
  del = sg - r;
  v = make_double2(del * (dx / r), del * (dy / r));
  return true;
}

// a test the FP32 filter could not decide (rare: near-degenerate inputs)
__device__ __forceinline__ void count_exact(const Ctx &x) {
  atomicAdd((unsigned long long *)&x.d.ctl->st_exact, 1ull);
}

// the filters on preloaded FP32 pairs (filt: all corners are disks, whose
// pairs are loaded; ghost points have none)
__device__ __forceinline__ int orient_pre(const Ctx &x, bool filt, const float4 &wa, const float4 &wb,
                                          const float4 &wc, int a, int b, int c) {
  if (filt) {
    const float bax = fdiff(wb.x, wb.z, wa.x, wa.z), bay = fdiff(wb.y, wb.w, wa.y, wa.w);
    const float cax = fdiff(wc.x, wc.z, wa.x, wa.z), cay = fdiff(wc.y, wc.w, wa.y, wa.w);
    const float l = __fmul_rn(bax, cay), r = __fmul_rn(bay, cax);
    const float det = __fsub_rn(l, r);
    const float bound = 1.5e-6f * __fadd_rn(fabsf(l), fabsf(r));
    if (det > bound) return 1;
    if (-det > bound) return -1;
    count_exact(x);
  }
  return orient_exact(x.d.pos, x.g, a, b, c);
}

__device__ __forceinline__ int incircle_pre(const Ctx &x, bool filt, const float4 &wa, const float4 &wb,
                                            const float4 &wc, const float4 &wp, int a, int b, int c, int p) {
  if (filt) {
    const float adx = fdiff(wa.x, wa.z, wp.x, wp.z), ady = fdiff(wa.y, wa.w, wp.y, wp.w);
    const float bdx = fdiff(wb.x, wb.z, wp.x, wp.z), bdy = fdiff(wb.y, wb.w, wp.y, wp.w);
    const float cdx = fdiff(wc.x, wc.z, wp.x, wp.z), cdy = fdiff(wc.y, wc.w, wp.y, wp.w);
    const float bcl = __fmul_rn(bdx, cdy), bcr = __fmul_rn(bdy, cdx);
    const float cal = __fmul_rn(cdx, ady), car = __fmul_rn(cdy, adx);
    const float abl = __fmul_rn(adx, bdy), abr = __fmul_rn(ady, bdx);
    const float al = __fadd_rn(__fmul_rn(adx, adx), __fmul_rn(ady, ady));
    const float bl = __fadd_rn(__fmul_rn(bdx, bdx), __fmul_rn(bdy, bdy));
    const float cl = __fadd_rn(__fmul_rn(cdx, cdx), __fmul_rn(cdy, cdy));
    const float det = __fadd_rn(__fadd_rn(__fmul_rn(al, __fsub_rn(bcl, bcr)), __fmul_rn(bl, __fsub_rn(cal, car))),
                                __fmul_rn(cl, __fsub_rn(abl, abr)));
    const float perm =
        __fadd_rn(__fadd_rn(__fmul_rn(al, __fadd_rn(fabsf(bcl), fabsf(bcr))), __fmul_rn(bl, __fadd_rn(fabsf(cal), fabsf(car)))),
                  __fmul_rn(cl, __fadd_rn(fabsf(abl), fabsf(abr))));
    const float bound = 4e-6f * perm;
    if (det > bound) return 1;
    if (-det > bound) return -1;
    count_exact(x);
  }
  return incircle_exact(x.d.pos, x.g, a, b, c, p);
}

__device__ __forceinline__ float4 work_of(const Ctx &x, int v) {
  return v < x.np ? x.d.work[v] : make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ int orient_v(const Ctx &x, int a, int b, int c) {
  const bool filt = a < x.np && b < x.np && c < x.np;
  return orient_pre(x, filt, work_of(x, a), work_of(x, b), work_of(x, c), a, b, c);
}

__device__ __forceinline__ int incircle_v(const Ctx &x, int a, int b, int c, int p) {
  const bool filt = a < x.np && b < x.np && c < x.np && p < x.np;
  return incircle_pre(x, filt, work_of(x, a), work_of(x, b), work_of(x, c), work_of(x, p), a, b, c, p);
}

// Sec. 4.3 reversal test r0 . r1 < 0 of the edge u -> w, exact on the grid:
// r1 from the present positions, r0 from those before the move (ox, oy: the
// edge's image shift before the move, in units of LQ)
__device__ __noinline__ bool reversed_grid(const double2 *__restrict__ prev, const double2 *__restrict__ pos,
                                           bdpred::Grid g, int u, int w, int ox, int oy, int rsx, int rsy,
                                           long long LQ) {
  const double2 a0 = prev[u], b0 = prev[w], a1 = pos[u], b1 = pos[w];
  const int64_t ux = bdpred::to_int(b0.x, g) - bdpred::to_int(a0.x, g) + ox * LQ;
  const int64_t uy = bdpred::to_int(b0.y, g) - bdpred::to_int(a0.y, g) + oy * LQ;
  const int64_t vx = bdpred::to_int(b1.x, g) - bdpred::to_int(a1.x, g) + rsx * LQ;
  const int64_t vy = bdpred::to_int(b1.y, g) - bdpred::to_int(a1.y, g) + rsy * LQ;
  return bdpred::sign128(bdpred::add128(bdpred::smul64(ux, vx), bdpred::smul64(uy, vy))) < 0;
}

__device__ __forceinline__ bool reversed_exact(const Ctx &x, int u, int w, int ox, int oy, int rsx, int rsy,
                                               long long LQ) {
  return reversed_grid(x.d.prev, x.d.pos, x.g, u, w, ox, oy, rsx, rsy, LQ);
}

// ---- periodic box: image shifts of triangle corners (Sec. 2.1, 4.1) ----
// Corner k of a triangle lies at pos[v_k] + L (sx_k, sy_k); the shifts are
// 2-bit two's-complement fields of tv.w (BD_TRI_SHIFT_BITS), all zero with
// walls, and corner 0 is kept at shift 0.  Straddling triangles are decided
// by the exact integer predicates on lifted grid coordinates.
__device__ __forceinline__ int sh2(int w, int bit) { return (((w >> bit) & 3) ^ 2) - 2; }
__device__ __forceinline__ int shx(int w, int k) { return sh2(w, 8 + 4 * k); }
__device__ __forceinline__ int shy(int w, int k) { return sh2(w, 10 + 4 * k); }
// the kernel is compiled twice: with walls (PER = false) every shift is the
// constant 0 and the shift arithmetic disappears
template <bool PER>
__device__ __forceinline__ int tshx(int w, int k) { return PER ? shx(w, k) : 0; }
template <bool PER>
__device__ __forceinline__ int tshy(int w, int k) { return PER ? shy(w, k) : 0; }
// the check-pass stamp of a triangle (bits 24-31 of tv.w)
__device__ __forceinline__ uint8_t tstamp(int w) { return (uint8_t)((unsigned)w >> BD_TRI_STAMP_SHIFT); }
__device__ __forceinline__ int with_stamp(int w, uint8_t s) {
  return (int)(((unsigned)w & ((1u << BD_TRI_STAMP_SHIFT) - 1u)) | ((unsigned)s << BD_TRI_STAMP_SHIFT));
}
__device__ __forceinline__ int put_shift(int k, int sx, int sy) {
  return ((sx & 3) << (8 + 4 * k)) | ((sy & 3) << (10 + 4 * k));
}
// the wrap of the last move of disk v: stored = geometric - L k
__device__ __forceinline__ int wrapx(uint8_t w) { return ((w & 3) ^ 2) - 2; }
__device__ __forceinline__ int wrapy(uint8_t w) { return (((w >> 2) & 3) ^ 2) - 2; }

struct Lift {
  long long x, y;
};

__device__ __forceinline__ Lift lift(const Ctx &x, int v, int sx, int sy, long long LQ) {
  const double2 p = x.d.pos[v];
  return {bdpred::to_int(p.x, x.g) + sx * LQ, bdpred::to_int(p.y, x.g) + sy * LQ};
}

__device__ __forceinline__ long long rep_LQ(const Ctx &x, int v) { return x.d.rep[x.d.rep_of[v]].LQ; }

// orientation of corners (a, b, c) with shifts (sa, sb, sc)
__device__ __forceinline__ int orient_s(const Ctx &x, int a, int sax, int say, int b, int sbx, int sby, int c,
                                        int scx, int scy) {
  if ((sax | say | sbx | sby | scx | scy) == 0) return orient_v(x, a, b, c);
  const long long LQ = rep_LQ(x, a);
  const Lift A = lift(x, a, sax, say, LQ), B = lift(x, b, sbx, sby, LQ), C = lift(x, c, scx, scy, LQ);
  return orient_lifted(A.x, A.y, B.x, B.y, C.x, C.y);
}

// in-circle test of p (shift sp) against triangle t's corners (shifts in w)
template <bool PER>
__device__ __forceinline__ int incircle_s(const Ctx &x, const int4 &v, int p, int spx, int spy) {
  const int w = v.w;
  if (!PER || ((w & BD_TRI_SHIFT_BITS) | spx | spy) == 0) return incircle_v(x, v.x, v.y, v.z, p);
  const long long LQ = rep_LQ(x, v.x);
  const Lift A = lift(x, v.x, shx(w, 0), shy(w, 0), LQ), B = lift(x, v.y, shx(w, 1), shy(w, 1), LQ);
  const Lift C = lift(x, v.z, shx(w, 2), shy(w, 2), LQ), P = lift(x, p, spx, spy, LQ);
  return incircle_lifted(A.x, A.y, B.x, B.y, C.x, C.y, P.x, P.y);
}

// shift, in the frame of triangle t (corner tab w), of the vertex opposite
// the edge facing corner k, read from the neighbour (tab w1, corner k1):
// t's corner k+1 is the neighbour's corner k1+2
template <bool PER>
__device__ __forceinline__ void opp_shift(int w, int k, int w1, int k1, int &sx, int &sy) {
  if (!PER) {
    sx = sy = 0;
    return;
  }
  const int ku = (k + 1) % 3, ku1 = (k1 + 2) % 3;
  sx = shx(w1, k1) + shx(w, ku) - shx(w1, ku1);
  sy = shy(w1, k1) + shy(w, ku) - shy(w1, ku1);
}

__device__ __forceinline__ double snap(double v, const bdpred::Grid &g) {
  return __dmul_rn(rint(__dmul_rn(v, g.inv_q)), g.q);
}

__device__ __forceinline__ float4 split_pos(double2 p) {
  float xh = __double2float_rn(p.x), yh = __double2float_rn(p.y);
  return make_float4(xh, yh, __double2float_rn(p.x - (double)xh), __double2float_rn(p.y - (double)yh));
}

// Claim the six triangles that flipping the edge facing corner cc touches:
// the pair and the four triangles across its outer edges.  An edge that
// holds all six claims owns them for the round, so its flip can rewrite the
// neighbours' back-pointers directly.
// the claims of the round of epoch e
__device__ __forceinline__ unsigned long long *claims(const Ctx &x, unsigned long long e) {
  return x.d.claim + (size_t)(e & 1ull) * x.T;
}

__device__ __forceinline__ void claim6(const Ctx &x, unsigned long long *cb, int t, int k, const int4 &nn, int o,
                                       unsigned long long key) {
  const int t1 = o / 3, k1 = o % 3;
  const int4 nn1 = x.d.tn[t1];
  atomicMax(&cb[t], key);
  atomicMax(&cb[t1], key);
  int e[4] = {vk(nn, (k + 1) % 3), vk(nn, (k + 2) % 3), vk(nn1, (k1 + 1) % 3), vk(nn1, (k1 + 2) % 3)};
  for (int m = 0; m < 4; ++m)
    if (e[m] >= 0) atomicMax(&cb[e[m] / 3], key);
}

__device__ __forceinline__ bool owns6(const Ctx &x, const unsigned long long *cb, int t0, int k0, const int4 &N0,
                                      int o0, unsigned long long key) {
  const int t1 = o0 / 3, k1 = o0 % 3;
  if (cb[t1] != key) return false;
  const int4 N1 = x.d.tn[t1];
  int e[4] = {vk(N0, (k0 + 1) % 3), vk(N0, (k0 + 2) % 3), vk(N1, (k1 + 1) % 3), vk(N1, (k1 + 2) % 3)};
  for (int m = 0; m < 4; ++m)
    if (e[m] >= 0 && cb[e[m] / 3] != key) return false;
  return true;
}

// Record triangle t, whose corners and neighbours are (V, N), in the undo
// journal before the launch first changes it (in its own slot: no list and no
// shared counter; an undo scans the marks).  A triangle is changed by one
// thread per phase (flips own the triangles they touch; the shift pass visits
// each triangle once), so the test of the mark needs no atomic.  A flip's
// outer neighbours are not journaled: their one change, the back-pointer, is
// rebuilt by the undo from the restored pair (they were adjacent before).
__device__ __forceinline__ void journal(const Ctx &x, int t, const int4 &V, const int4 &N, unsigned mark) {
  if (mark == x.jstamp) return;
  x.d.jmark[t] = x.jstamp;
  x.d.jtv[t] = V;
  x.d.jtn[t] = N;
}
// undo of a journaled triangle t: its corners and neighbours as they were, a
// corner for each of its vertices, and its neighbours' back-pointers
__device__ __forceinline__ void unjournal(const BdDev &d, int t) {
  const int4 vs = d.jtv[t], ns = d.jtn[t];
  d.tv[t] = vs;
  d.tn[t] = ns;
  d.vt[vs.x] = 3 * t;
  d.vt[vs.y] = 3 * t + 1;
  d.vt[vs.z] = 3 * t + 2;
  const int nk[3] = {ns.x, ns.y, ns.z};
  for (int k = 0; k < 3; ++k)
    if (nk[k] >= 0) ((int *)&d.tn[nk[k] / 3])[nk[k] % 3] = 3 * t + k;
}

// Flip the edge facing corner c0 in place (the two triangle slots are reused)
// and point the four outer neighbours, owned by this flip, at the new corners.
// Quad a-b-d-c with t0 = (a, b, c), t1 = (d, c, b) becomes t0 = (b, d, a),
// t1 = (c, a, d): the edge bc is replaced by ad.
template <bool PER>
__device__ void flip_owned(const Ctx &x, int c0, int o0, uint8_t stamp) {
  const int t0 = c0 / 3, k0 = c0 % 3, t1 = o0 / 3, k1 = o0 % 3;
  // the journal marks are loaded with the pair, and the pair's old values
  // journaled after the flip's own stores (they are held in registers)
  const unsigned m0 = x.d.jmark[t0], m1 = x.d.jmark[t1];
  int4 V0 = x.d.tv[t0], V1 = x.d.tv[t1], N0 = x.d.tn[t0], N1 = x.d.tn[t1];
  const int4 oV0 = V0, oV1 = V1, oN0 = N0, oN1 = N1;
  const int a = vk(V0, k0), b = vk(V0, (k0 + 1) % 3), c = vk(V0, (k0 + 2) % 3), dd = vk(V1, k1);
  const int n_ca = vk(N0, (k0 + 1) % 3), n_ab = vk(N0, (k0 + 2) % 3);
  const int n_bd = vk(N1, (k1 + 1) % 3), n_dc = vk(N1, (k1 + 2) % 3);
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
  // image shifts (periodic box): the new corners in t0's frame; d comes from
  // t1's frame, offset by b's shift difference between the two frames
  const int w0 = V0.w, w1 = V1.w;
  int nw0 = 0, nw1 = 0;
  if (PER && ((w0 | w1) & BD_TRI_SHIFT_BITS)) {
    const int Ax = shx(w0, k0), Ay = shy(w0, k0);
    const int Bx = shx(w0, (k0 + 1) % 3), By = shy(w0, (k0 + 1) % 3);
    const int Cx = shx(w0, (k0 + 2) % 3), Cy = shy(w0, (k0 + 2) % 3);
    const int Dx = shx(w1, k1) + Bx - shx(w1, (k1 + 2) % 3), Dy = shy(w1, k1) + By - shy(w1, (k1 + 2) % 3);
    // t0 = (b, d, a) at (k0, k0+1, k0+2); t1 = (c, a, d) at (k1, k1+1, k1+2)
    int sx0[3], sy0[3], sx1[3], sy1[3];
    sx0[k0] = Bx; sy0[k0] = By;
    sx0[(k0 + 1) % 3] = Dx; sy0[(k0 + 1) % 3] = Dy;
    sx0[(k0 + 2) % 3] = Ax; sy0[(k0 + 2) % 3] = Ay;
    sx1[k1] = Cx; sy1[k1] = Cy;
    sx1[(k1 + 1) % 3] = Ax; sy1[(k1 + 1) % 3] = Ay;
    sx1[(k1 + 2) % 3] = Dx; sy1[(k1 + 2) % 3] = Dy;
    for (int k = 0; k < 3; ++k) {
      nw0 |= put_shift(k, sx0[k] - sx0[0], sy0[k] - sy0[0]);
      nw1 |= put_shift(k, sx1[k] - sx1[0], sy1[k] - sy1[0]);
    }
  }
  // both new triangles: their edges are tested by the next check pass
  V0.w = with_stamp(nw0, stamp);
  V1.w = with_stamp(nw1, stamp);
  x.d.tv[t0] = V0;
  x.d.tv[t1] = V1;
  x.d.tn[t0] = N0;
  x.d.tn[t1] = N1;
  x.d.tinv[t0] = 0;
  x.d.tinv[t1] = 0;
  // the four vertices' corners moved: t0 = (b, d, a), t1 = (c, a, d)
  x.d.vt[b] = 3 * t0 + k0;
  x.d.vt[dd] = 3 * t0 + (k0 + 1) % 3;
  x.d.vt[a] = 3 * t0 + (k0 + 2) % 3;
  x.d.vt[c] = 3 * t1 + k1;
  if (n_ab >= 0) ((int *)&x.d.tn[n_ab / 3])[n_ab % 3] = 3 * t0 + (k0 + 1) % 3;
  if (n_bd >= 0) ((int *)&x.d.tn[n_bd / 3])[n_bd % 3] = 3 * t0 + (k0 + 2) % 3;
  if (n_dc >= 0) ((int *)&x.d.tn[n_dc / 3])[n_dc % 3] = 3 * t1 + (k1 + 1) % 3;
  if (n_ca >= 0) ((int *)&x.d.tn[n_ca / 3])[n_ca % 3] = 3 * t1 + (k1 + 2) % 3;
  journal(x, t0, oV0, oN0, m0);
  journal(x, t1, oV1, oN1, m1);
}

__device__ __forceinline__ unsigned long long claim_key(unsigned long long epoch, int corner) {
  return (epoch << 32) | (unsigned long long)(0xFFFFFFFFu - (unsigned)corner);
}
__device__ __forceinline__ int key_corner(unsigned long long key) {
  return (int)(0xFFFFFFFFu - (unsigned)(key & 0xFFFFFFFFull));
}

// Register triangle t as a candidate owner for the round of epoch e, once:
// the marking pass and the previous fused round both register owners for a
// round, and an owner listed twice would be flipped by two threads at once.
__device__ __forceinline__ void push_owner(const Ctx &x, unsigned long long e, int t) {
  if (atomicExch(&x.d.clmark[t], (unsigned)e) == (unsigned)e) return;
  const int l = (int)(e % 3);
  x.d.clist[(size_t)l * x.T + atomicAdd(&x.d.ctl->cl_n[l], 1)] = t;
}

// Stamp triangle t for the check pass of generation byte s.  The word is
// shared with the corners' image shifts, which a flip of t by another thread
// may rewrite meanwhile: compare-and-swap keeps whichever shifts are current.
__device__ __forceinline__ void stamp_tri(const Ctx &x, int t, uint8_t s) {
  int *w = &x.d.tv[t].w;
  int old = *(volatile int *)w, seen;
  do {
    seen = old;
    old = atomicCAS(w, seen, with_stamp(seen, s));
  } while (old != seen);
}

// A fused Lawson round's flip of the edge facing corner c0 (pair and outer
// neighbours owned).  Its loads are issued by level -- the pair and the
// journal marks; the four outer neighbours' corner tables and the quad's
// FP32 pairs; the opposite vertices' FP32 pairs -- before any store.  It
// withdraws the overlap of diagonal bc, adds that of ad, flips, and tests the
// four outer edges, registering the illegal ones (claims in nb, keys of
// epoch ne, owners listed once).  Returns the change in overlapping edges
// and the depth of an added overlap (0 if none).
struct FusedOut {
  int adj;
  double mx;
};
template <bool PER>
__device__ __forceinline__ FusedOut fused_flip(const Ctx &x, int c0, int o0, unsigned long long *nb,
                                             unsigned long long ne) {
  const BdDev &d = x.d;
  const int t0 = c0 / 3, k0 = c0 % 3, t1 = o0 / 3, k1 = o0 % 3;
  const unsigned m0 = d.jmark[t0], m1 = d.jmark[t1];
  const int4 oV0 = d.tv[t0], oV1 = d.tv[t1], oN0 = d.tn[t0], oN1 = d.tn[t1];
  const int a = vk(oV0, k0), b = vk(oV0, (k0 + 1) % 3), c = vk(oV0, (k0 + 2) % 3), dd = vk(oV1, k1);
  const int n_ca = vk(oN0, (k0 + 1) % 3), n_ab = vk(oN0, (k0 + 2) % 3);
  const int n_bd = vk(oN1, (k1 + 1) % 3), n_dc = vk(oN1, (k1 + 2) % 3);
  // outer edges in the order (t0, facing k0+1), (t0, k0+2), (t1, k1+1), (t1, k1+2)
  const int nbr[4] = {n_ab, n_bd, n_dc, n_ca};
  int4 Wn[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) Wn[m] = nbr[m] >= 0 ? d.tv[nbr[m] / 3] : make_int4(0, 0, 0, 0);
  const float4 Pa = work_of(x, a), Pb = work_of(x, b), Pc = work_of(x, c), Pd = work_of(x, dd);
  int q[4];
  float4 Pq[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    q[m] = nbr[m] >= 0 ? vk(Wn[m], nbr[m] % 3) : 0;
    Pq[m] = nbr[m] >= 0 ? work_of(x, q[m]) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  // the new pair: t0 = (b, d, a) at (k0, k0+1, k0+2), t1 = (c, a, d) at (k1, k1+1, k1+2)
  int4 V0 = oV0, V1 = oV1, N0 = oN0, N1 = oN1;
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
  const int w0 = oV0.w, w1 = oV1.w;
  int nw0 = 0, nw1 = 0;
  int Ax = 0, Ay = 0, Bx = 0, By = 0, Cx = 0, Cy = 0, Dx = 0, Dy = 0;
  if (PER && ((w0 | w1) & BD_TRI_SHIFT_BITS)) {
    Ax = shx(w0, k0); Ay = shy(w0, k0);
    Bx = shx(w0, (k0 + 1) % 3); By = shy(w0, (k0 + 1) % 3);
    Cx = shx(w0, (k0 + 2) % 3); Cy = shy(w0, (k0 + 2) % 3);
    Dx = shx(w1, k1) + Bx - shx(w1, (k1 + 2) % 3); Dy = shy(w1, k1) + By - shy(w1, (k1 + 2) % 3);
    int sx0[3], sy0[3], sx1[3], sy1[3];
    sx0[k0] = Bx; sy0[k0] = By;
    sx0[(k0 + 1) % 3] = Dx; sy0[(k0 + 1) % 3] = Dy;
    sx0[(k0 + 2) % 3] = Ax; sy0[(k0 + 2) % 3] = Ay;
    sx1[k1] = Cx; sy1[k1] = Cy;
    sx1[(k1 + 1) % 3] = Ax; sy1[(k1 + 1) % 3] = Ay;
    sx1[(k1 + 2) % 3] = Dx; sy1[(k1 + 2) % 3] = Dy;
    for (int k = 0; k < 3; ++k) {
      nw0 |= put_shift(k, sx0[k] - sx0[0], sy0[k] - sy0[0]);
      nw1 |= put_shift(k, sx1[k] - sx1[0], sy1[k] - sy1[0]);
    }
  }
  V0.w = with_stamp(nw0, tstamp(w0));
  V1.w = with_stamp(nw1, tstamp(w1));
  // overlaps of the old and the new diagonal (a shifted edge takes the exact
  // test directly; a plain one is screened in FP32 first, as in a check pass)
  FusedOut r = {0, 0.0};
  auto diag = [&](int u, int w, const float4 &Pu, const float4 &Pw, int sx, int sy, int sgn) {
    if (u >= x.np || w >= x.np) return;
    if ((sx | sy) == 0) {
      const float fx = fdiff(Pw.x, Pw.z, Pu.x, Pu.z), fy = fdiff(Pw.y, Pw.w, Pu.y, Pu.w);
      if (__fadd_rn(__fmul_rn(fx, fx), __fmul_rn(fy, fy)) > x.sig2f) return;
    }
    const long long LQ = (sx | sy) ? rep_LQ(x, u) : 0;
    double2 v;
    double del;
    if (!edge_overlap(x, u, w, sx, sy, LQ, v, del)) return;
    disp_add(x, u, -sgn * v.x, -sgn * v.y);
    disp_add(x, w, sgn * v.x, sgn * v.y);
    r.adj += sgn;
    if (sgn > 0) r.mx = fmax(r.mx, del);
  };
  diag(b, c, Pb, Pc, Cx - Bx, Cy - By, -1);
  diag(a, dd, Pa, Pd, Dx - Ax, Dy - Ay, 1);
  // the flip
  d.tv[t0] = V0;
  d.tv[t1] = V1;
  d.tn[t0] = N0;
  d.tn[t1] = N1;
  d.tinv[t0] = 0;
  d.tinv[t1] = 0;
  d.vt[b] = 3 * t0 + k0;
  d.vt[dd] = 3 * t0 + (k0 + 1) % 3;
  d.vt[a] = 3 * t0 + (k0 + 2) % 3;
  d.vt[c] = 3 * t1 + k1;
  if (n_ab >= 0) ((int *)&d.tn[n_ab / 3])[n_ab % 3] = 3 * t0 + (k0 + 1) % 3;
  if (n_bd >= 0) ((int *)&d.tn[n_bd / 3])[n_bd % 3] = 3 * t0 + (k0 + 2) % 3;
  if (n_dc >= 0) ((int *)&d.tn[n_dc / 3])[n_dc % 3] = 3 * t1 + (k1 + 1) % 3;
  if (n_ca >= 0) ((int *)&d.tn[n_ca / 3])[n_ca % 3] = 3 * t1 + (k1 + 2) % 3;
  journal(x, t0, oV0, oN0, m0);
  journal(x, t1, oV1, oN1, m1);
  // the four outer edges: the opposite vertex inside the new triangle's
  // circumcircle makes the edge illegal (a candidate of the next round)
  float4 W0[3], W1[3];
  W0[k0] = Pb; W0[(k0 + 1) % 3] = Pd; W0[(k0 + 2) % 3] = Pa;
  W1[k1] = Pc; W1[(k1 + 1) % 3] = Pa; W1[(k1 + 2) % 3] = Pd;
  bool reg0 = false, reg1 = false;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    if (nbr[m] < 0) continue;
    const bool first = m < 2;
    const int tt = first ? t0 : t1, kt = first ? k0 : k1;
    const int k = (kt + 1 + (m & 1)) % 3;
    const int4 &V = first ? V0 : V1;
    const float4 *Wt = first ? W0 : W1;
    int sqx, sqy;
    opp_shift<PER>(V.w, k, Wn[m].w, nbr[m] % 3, sqx, sqy);
    const bool flat = (V.w & BD_TRI_SHIFT_BITS) == 0 && (sqx | sqy) == 0;
    const int ic = flat ? incircle_pre(x, V.x < x.np && V.y < x.np && V.z < x.np && q[m] < x.np, Wt[0], Wt[1],
                                       Wt[2], Pq[m], V.x, V.y, V.z, q[m])
                        : incircle_s<PER>(x, V, q[m], sqx, sqy);
    if (ic > 0) {
      claim6(x, nb, tt, k, first ? N0 : N1, nbr[m], claim_key(ne, 3 * tt + k));
      bool &reg = first ? reg0 : reg1;
      if (!reg) {
        reg = true;
        push_owner(x, ne, tt);
      }
    }
  }
  return r;
}

// Append triangle t to a list once per generation (a list is visited by one
// check pass; its generation tags the members).  The lanes of a warp that
// append together reserve their slots with one atomic on the list length.
__device__ __forceinline__ void push_tri(int *list, unsigned *mark, int *n, unsigned gen, int t) {
  const bool add = atomicExch(&mark[t], gen) != gen;
  const unsigned act = __activemask();
  const unsigned want = __ballot_sync(act, add);
  if (!want) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(want) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(n, __popc(want));
  base = __shfl_sync(act, base, leader);
  if (add) list[base + __popc(want & ((1u << lane) - 1u))] = t;
}

// the replica of a triangle (its first disk corner; -1 if it has none)
__device__ __forceinline__ int tri_rep(const BdDev &d, int np, const int4 &v) {
  const int c = v.x < np ? v.x : (v.y < np ? v.y : (v.z < np ? v.z : -1));
  return c < 0 ? -1 : d.rep_of[c];
}


}  // namespace

// One time step's triangulation work (mode 0), the repair of the
// triangulation after new positions are set (mode 1: no overlap correction; an
// overlapping pair rejects the positions with BD_ERR_INIT_OVERLAP),
// or one piece of a halved step (mode 2: as mode 0, but the step counter does
// not advance).
//
// Phases, each ended by a grid barrier:
//   P  one pass over the triangles: orientation of triangles with a moved
//      corner (inverted => flag), the reversal test on edges with a moved end,
//      Lawson marks on edges touching a dirty triangle, and the overlap scan
//      of every disk-disk edge.  The scan is used only when the pass found no
//      inverted triangle and no illegal edge, i.e. when the triangulation it
//      scanned is the Delaunay triangulation of the current positions.
//   R  inversion repair rounds (candidate marks, owned flips) when P found an
//      inverted triangle; then P again.
//   F  owned Lawson flips of the marked edges; fused: the next round at once
//      with the candidates its flips registered, or, if a candidate lost a
//      claim, P marking without a scan; unfused: P again.
//   A  apply the capped displacements (Algorithm 2) and reflect; then P again.
// Three resident blocks per SM (at most 80 registers): the passes are
// latency-bound chains of dependent loads, and the spills this costs sit in
// the exact-predicate fallbacks (measured: 3 blocks 20 % faster than 2 on
// 2^20 disks; 4 blocks (64 registers) 1.5 % faster on 2^20 disks but 16 %
// slower in the check passes at 1e5; 5 blocks slower on both).
template <bool PER>
__global__ void __launch_bounds__(BD_DT_THREADS, 3) k_triangulation(BdDev d, BdConst c, int mode,
                                                                 int log_step) {
  Ctx x;
  x.d = d;
  x.c = c;
  x.g.q = c.q;
  x.g.inv_q = c.inv_q;
  x.g.s = c.qshift;
  x.T = c.nt;
  x.np = c.np;
  x.sig2f = (float)(c.sigma * c.sigma * (1.0 + 1e-5));
  BdCtl *ctl = d.ctl;
  if (ld_status(&ctl->status) != 0 || (mode == 1 && *(volatile const int *)&ctl->n_set_moved == 0)) {
    // (bd_set_state that moved no disk: the triangulation stands as it was)
    block_exit(ctl);
    return;
  }
  Bar b;
  b.gen = 0;
  b.ph = 0;
  __shared__ int bc[BC_N];                // phase counters and list lengths, per barrier
  unsigned long long t_mark = gtimer();   // stage timing (lead thread)
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  const bool lead = (blockIdx.x == 0 && threadIdx.x == 0);
  unsigned long long epoch = ctl->epoch;   // written only at kernel end by the lead thread
  x.jstamp = ((unsigned)epoch << 1) | 1u;   // distinct per launch: the epoch grows across launches
  const double sigma = c.sigma;
  int status = 0;
  int corr_iter = 0;
  long long st_overlap = 0, st_flips = 0, st_rflips = 0, st_inv = 0, st_rounds = 0;
  bool fresh = true;       // the moved flags describe the latest move
  int lawson_rounds = 0;
  // rollout log (adjoint): committed passes and their overlapping pairs
  const bool logging = log_step >= 0 && d.log_pairs != nullptr;
  int log_head = logging ? ctl->log_npairs : 0;
  int log_npass = logging ? ctl->log_npass : 0;
  int log_pidx = -1;
  // Check-pass domains.  The first pass of a move (and the pass after an
  // inversion repair) visits every triangle; a later pass visits only a list:
  // the triangles a flip touched or left dirty, those with an overlapping
  // edge, and after a correction move the stars of the moved disks.  Every
  // other edge kept its end points and its place in the triangulation since it
  // was last checked, so its earlier verdicts (legal, not overlapping) stand.
  // Lists rotate over three slots: pass kp visits slot kp % 3 (generation
  // g0 + kp) and fills slot (kp + 1) % 3; the lead empties slot (kp + 2) % 3.
  const unsigned g0 = *(volatile unsigned *)&ctl->act_gen;
  int kp = 0;
  bool full = true;
  // Lists pay off when a full pass is bound by the number of triangles per
  // thread; with a few triangles per thread a full pass is as short as one
  // thread's chain of dependent loads, which a list pass (an extra
  // indirection and membership reads) only lengthens (measured: 2^20 disks,
  // 18 triangles per thread, check stage 0.37 -> 0.30 ms per step; 10^5
  // disks, 1.8 per thread, 0.13 -> 0.17 ms).
  const bool use_lists = c.tri_lists == 1 || (c.tri_lists == 0 && x.T > 4 * nth);
  long long tri_visits = 0;
  // the next iteration opens with a check pass (need_p) that scans the
  // overlaps (scan); the overlapping edges of the current triangulation
  // (ov_now); Lawson rounds fused with their re-tests (not while a rollout
  // logs its pairs, which wants every pair of a pass from one scan)
  bool need_p = true, scan = true;
  int ov_now = 0;
  const bool fuse = c.tri_fuse && !logging;

  for (;;) {
    ++epoch;
    if (lead) {
      ctl->cl_n[(epoch + 2) % 3] = 0;   // the candidate list two rounds ahead
      ctl->act_n[(kp + 2) % 3] = 0;     // the triangle list two passes ahead
    }
    const int slot = kp % 3, nslot = (kp + 1) % 3;
    const unsigned gen = g0 + (unsigned)kp, ngen = gen + 1u;
    const uint8_t gen8 = (uint8_t)gen, ngen8 = (uint8_t)ngen;   // check-pass stamps of this pass and the next
    const int *dom = d.act + (size_t)slot * x.T;
    const unsigned *cmark = d.act_mark + (size_t)slot * x.T;
    int *nlist = d.act + (size_t)nslot * x.T;
    unsigned *nmark = d.act_mark + (size_t)nslot * x.T;
    int *ncount = &ctl->act_n[nslot];
    // ---------------- W: shifts of triangles whose corners re-entered (periodic box) ----------------
    if (PER && fresh && *(volatile int *)&ctl->n_wrapped != 0) {
      phase_begin(ctl, b);
      for (int t = tid; t < x.T; t += nth) {
        const int4 v = d.tv[t];
        const uint8_t w0 = d.wrap[v.x], w1 = d.wrap[v.y], w2 = d.wrap[v.z];
        if ((w0 | w1 | w2) == 0) continue;
        journal(x, t, v, d.tn[t], d.jmark[t]);
        // a corner stored L k lower than where it geometrically is: shift += k
        const int kx[3] = {wrapx(w0), wrapx(w1), wrapx(w2)}, ky[3] = {wrapy(w0), wrapy(w1), wrapy(w2)};
        int sx[3], sy[3];
        for (int k = 0; k < 3; ++k) {
          sx[k] = tshx<PER>(v.w, k) + kx[k];
          sy[k] = tshy<PER>(v.w, k) + ky[k];
        }
        int nw = with_stamp(0, tstamp(v.w));
        for (int k = 0; k < 3; ++k) nw |= put_shift(k, sx[k] - sx[0], sy[k] - sy[0]);
        d.tv[t].w = nw;
      }
      if (!grid_sync(ctl, b, bc)) { block_exit(ctl); return; }
      if (lead) ctl->n_wrapped = 0;
    }
    // ---------------- P: check, mark, scan ----------------
    // (skipped between fused Lawson rounds: their flips test the edges they
    // change; a pass that follows such rounds only marks, scan = false, since
    // the rounds keep the overlap sums of the triangulation they leave)
    int n_ov = 0;
    const int dom_n = full ? x.T : bc[BC_ACT + slot];
    if (need_p) {
      if (lead) tri_visits += dom_n;
      phase_begin(ctl, b);
      {
        int inv = 0, rej = 0, cand = 0, nov = 0;
        double mx = 0.0;
        if constexpr (PER)
        for (int it = tid; it < dom_n; it += nth) {
          const int t = full ? it : dom[it];
          const int4 v = d.tv[t];
          const int4 nn = d.tn[t];
          // corners loaded once: FP32 pairs, moved flags and re-entries serve the
          // filters of triangles and edges that carry no image shift
          const int vv[3] = {v.x, v.y, v.z};
          const bool isd[3] = {v.x < x.np, v.y < x.np, v.z < x.np};
          const bool flat = (v.w & BD_TRI_SHIFT_BITS) == 0;
          float4 W[3];
          uint8_t mvd[3], wr[3];
  #pragma unroll
          for (int k = 0; k < 3; ++k) {
            W[k] = work_of(x, vv[k]);
            mvd[k] = fresh ? d.moved[vv[k]] : (uint8_t)0;
            wr[k] = isd[k] ? d.wrap[vv[k]] : (uint8_t)0;
          }
          int fl = tstamp(v.w) == gen8 ? BD_TRI_DIRTY : 0;
          if (mvd[0] | mvd[1] | mvd[2]) {
            const int o = flat ? orient_pre(x, isd[0] && isd[1] && isd[2], W[0], W[1], W[2], v.x, v.y, v.z)
                               : orient_s(x, v.x, tshx<PER>(v.w, 0), tshy<PER>(v.w, 0), v.y, tshx<PER>(v.w, 1),
                                          tshy<PER>(v.w, 1), v.z, tshx<PER>(v.w, 2), tshy<PER>(v.w, 2));
            fl = BD_TRI_DIRTY | (o <= 0 ? BD_TRI_INVERTED : 0);
            if (o <= 0) d.tinv[t] = 1;
          }
          const bool inverted = (fl & BD_TRI_INVERTED) != 0;
          inv += inverted ? 1 : 0;
          bool owner = false;   // t registered a flip candidate
          if (inverted && d.rep_stats) {
            const int rr = tri_rep(d, x.np, v);
            if (rr >= 0) atomicAdd((unsigned long long *)&d.rep_stats[3 * rr + 2], 1ull);
          }
          for (int k = 0; k < 3; ++k) {
            const int cc = 3 * t + k;
            const int o = vk(nn, k);
            // each interior edge once: from its smaller corner, or from this side
            // when the neighbour is not visited by this pass
            if (o < 0 || (o <= cc && (full || cmark[o / 3] == gen))) continue;
            const int ku = (k + 1) % 3, kw = (k + 2) % 3;
            const int u = vv[ku], w = vv[kw];
            const bool disks = isd[ku] && isd[kw];
            const bool mv = (mvd[ku] | mvd[kw]) != 0;
            // image shift of w relative to u in this triangle (periodic box; 0 with walls)
            const int rsx = tshx<PER>(v.w, (k + 2) % 3) - tshx<PER>(v.w, (k + 1) % 3);
            const int rsy = tshy<PER>(v.w, (k + 2) % 3) - tshy<PER>(v.w, (k + 1) % 3);
            long long LQ = 0;
            if (rsx | rsy) LQ = rep_LQ(x, u);
            const bool plain = (rsx | rsy) == 0;   // the edge carries no image shift
            // r1 = r_w - r_u from the FP32 pairs (unshifted edges)
            const float r1x = plain ? fdiff(W[kw].x, W[kw].z, W[ku].x, W[ku].z) : 0.f;
            const float r1y = plain ? fdiff(W[kw].y, W[kw].w, W[ku].y, W[ku].w) : 0.f;
            if (disks && mv) {
              // Sec. 4.3 first criterion: r0 . r1 < 0.  An unshifted edge whose
              // ends did not re-enter is screened in FP32 from r1 and the moves,
              // as with walls; otherwise, and near zero, exact on the grid (the
              // edge's shift before the move is the present one less the
              // re-entries of its end points)
              int dec = 0;   // 1 reversed, -1 not, 0 undecided
              if (plain && (wr[ku] | wr[kw]) == 0) {
                const float2 mu = mvd[ku] ? d.dmove[u] : make_float2(0.f, 0.f);
                const float2 mw = mvd[kw] ? d.dmove[w] : make_float2(0.f, 0.f);
                const float r0x = __fsub_rn(r1x, __fsub_rn(mw.x, mu.x)), r0y = __fsub_rn(r1y, __fsub_rn(mw.y, mu.y));
                const float dot = __fadd_rn(__fmul_rn(r0x, r1x), __fmul_rn(r0y, r1y));
                const float S = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(r0x, r0x), __fmul_rn(r0y, r0y)),
                                                    __fadd_rn(__fmul_rn(r1x, r1x), __fmul_rn(r1y, r1y))),
                                          __fadd_rn(__fadd_rn(__fmul_rn(mu.x, mu.x), __fmul_rn(mu.y, mu.y)),
                                                    __fadd_rn(__fmul_rn(mw.x, mw.x), __fmul_rn(mw.y, mw.y))));
                const float bound = 4e-6f * S;
                dec = dot > bound ? -1 : (-dot > bound ? 1 : 0);
                if (dec == 0) count_exact(x);
              }
              int ox = rsx, oy = rsy;
              if (dec == 0) {
                ox -= wrapx(wr[kw]) - wrapx(wr[ku]);
                oy -= wrapy(wr[kw]) - wrapy(wr[ku]);
                if ((ox | oy) && LQ == 0) LQ = rep_LQ(x, u);
              }
              if (dec == 1 || (dec == 0 && reversed_exact(x, u, w, ox, oy, rsx, rsy, LQ))) {
                ++rej;
                atomicExch(&ctl->st_fail_item, cc);
              }
            }
            if (inverted) continue;   // marks and scan wait for the repair
            const int4 v1 = d.tv[o / 3];
            const int q = vk(v1, o % 3);
            // the edge is tested when a triangle on either side is dirty or one
            // of its four points moved
            const bool d1 = (fl & BD_TRI_DIRTY) || tstamp(v1.w) == gen8 || (mvd[ku] | mvd[kw]) ||
                            (fresh && d.moved[q]);
            if (d1) {
              int sqx, sqy;
              opp_shift<PER>(v.w, k, v1.w, o % 3, sqx, sqy);
              const int ic = (flat && (sqx | sqy) == 0)
                                 ? incircle_pre(x, isd[0] && isd[1] && isd[2] && q < x.np, W[0], W[1], W[2],
                                                work_of(x, q), v.x, v.y, v.z, q)
                                 : incircle_s<PER>(x, v, q, sqx, sqy);
              if (ic > 0) {
                claim6(x, claims(x, epoch), t, k, nn, o, claim_key(epoch, cc));
                ++cand;
                if (!owner) {   // t joins the candidate owners once (candidates are rare)
                  owner = true;
                  push_owner(x, epoch, t);
                }
              }
            }
            if (disks && scan) {
              // FP32 screen: a pair whose FP32 squared distance exceeds
              // sigma^2 (1 + 1e-5) is farther than sigma (FP32 error ~3e-7);
              // edges across a periodic box edge skip it
              if (plain && __fadd_rn(__fmul_rn(r1x, r1x), __fmul_rn(r1y, r1y)) > x.sig2f) continue;
              double2 v;
              double del;
              if (edge_overlap(x, u, w, rsx, rsy, LQ, v, del)) {
                disp_add(x, u, -v.x, -v.y);
                disp_add(x, w, v.x, v.y);
                if (use_lists) push_tri(nlist, nmark, ncount, ngen, t);   // checked again in the next pass
                const int k_ov = atomicAdd(cnt(ctl, b.ph, C_OVERLAP), 1);
                if (logging) {
                  if (log_head + k_ov < c.log_pairs_cap) d.log_pairs[log_head + k_ov] = make_int2(u, w);
                  else atomicExch(&ctl->log_overflow, 1);
                }
                mx = fmax(mx, del);
              }
            }
          }
        }
        else
        for (int it = tid; it < dom_n; it += nth) {
          // walls: the three corners' FP32 pairs and moved flags are loaded once
          // and serve the orientation, the reversal and in-circle filters and the
          // overlap screen of all three edges
          const int t = full ? it : dom[it];
          const int4 v = d.tv[t];
          const int4 nn = d.tn[t];
          const int vv[3] = {v.x, v.y, v.z};
          const bool isd[3] = {v.x < x.np, v.y < x.np, v.z < x.np};
          float4 W[3];
          uint8_t mvd[3];
  #pragma unroll
          for (int k = 0; k < 3; ++k) {
            W[k] = work_of(x, vv[k]);
            mvd[k] = fresh ? d.moved[vv[k]] : (uint8_t)0;
          }
          int fl = tstamp(v.w) == gen8 ? BD_TRI_DIRTY : 0;
          if (mvd[0] | mvd[1] | mvd[2]) {
            const int o = orient_pre(x, isd[0] && isd[1] && isd[2], W[0], W[1], W[2], v.x, v.y, v.z);
            fl = BD_TRI_DIRTY | (o <= 0 ? BD_TRI_INVERTED : 0);
            if (o <= 0) d.tinv[t] = 1;
          }
          const bool inverted = (fl & BD_TRI_INVERTED) != 0;
          inv += inverted ? 1 : 0;
          bool owner = false;   // t registered a flip candidate
          if (inverted && d.rep_stats) {
            const int rr = tri_rep(d, x.np, v);
            if (rr >= 0) atomicAdd((unsigned long long *)&d.rep_stats[3 * rr + 2], 1ull);
          }
  #pragma unroll
          for (int k = 0; k < 3; ++k) {
            const int cc = 3 * t + k;
            const int o = vk(nn, k);
            // each interior edge once: from its smaller corner, or from this side
            // when the neighbour is not visited by this pass
            if (o < 0 || (o <= cc && (full || cmark[o / 3] == gen))) continue;
            const int ku = (k + 1) % 3, kw = (k + 2) % 3;
            const int u = vv[ku], w = vv[kw];
            const bool disks = isd[ku] && isd[kw];
            // r1 = r_w - r_u from the FP32 pairs (one rounding)
            const float r1x = fdiff(W[kw].x, W[kw].z, W[ku].x, W[ku].z);
            const float r1y = fdiff(W[kw].y, W[kw].w, W[ku].y, W[ku].w);
            if (disks && (mvd[ku] | mvd[kw])) {
              // Sec. 4.3 first criterion r0 . r1 < 0; r0 = r1 - (move of w - move
              // of u), screened in FP32, exact on the grid near zero
              bool rev;
              {
                const float2 mu = mvd[ku] ? d.dmove[u] : make_float2(0.f, 0.f);
                const float2 mw = mvd[kw] ? d.dmove[w] : make_float2(0.f, 0.f);
                const float r0x = __fsub_rn(r1x, __fsub_rn(mw.x, mu.x)), r0y = __fsub_rn(r1y, __fsub_rn(mw.y, mu.y));
                // every rounding above is relative (one FP32 rounding of a grid
                // value or of a sum): the computed dot is within ~8 2^-24 S of
                // the exact one, S = |r0|^2 + |r1|^2 + |m_u|^2 + |m_w|^2
                const float dot = __fadd_rn(__fmul_rn(r0x, r1x), __fmul_rn(r0y, r1y));
                const float S = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(r0x, r0x), __fmul_rn(r0y, r0y)),
                                                    __fadd_rn(__fmul_rn(r1x, r1x), __fmul_rn(r1y, r1y))),
                                          __fadd_rn(__fadd_rn(__fmul_rn(mu.x, mu.x), __fmul_rn(mu.y, mu.y)),
                                                    __fadd_rn(__fmul_rn(mw.x, mw.x), __fmul_rn(mw.y, mw.y))));
                const float bound = 4e-6f * S;
                if (dot > bound) {
                  rev = false;
                } else if (-dot > bound) {
                  rev = true;
                } else {
                  count_exact(x);
                  rev = reversed_exact(x, u, w, 0, 0, 0, 0, 0);
                }
              }
              if (rev) {
                ++rej;
                atomicExch(&ctl->st_fail_item, cc);
              }
            }
            if (inverted) continue;   // marks and scan wait for the repair
            const int4 v1 = d.tv[o / 3];
            const int q = vk(v1, o % 3);
            // the edge is tested when a triangle on either side is dirty or one
            // of its four points moved
            const bool d1 = (fl & BD_TRI_DIRTY) || tstamp(v1.w) == gen8 || (mvd[ku] | mvd[kw]) ||
                            (fresh && d.moved[q]);
            if (d1) {
              const bool filt = isd[0] && isd[1] && isd[2] && q < x.np;
              if (incircle_pre(x, filt, W[0], W[1], W[2], work_of(x, q), v.x, v.y, v.z, q) > 0) {
                claim6(x, claims(x, epoch), t, k, nn, o, claim_key(epoch, cc));
                ++cand;
                if (!owner) {   // t joins the candidate owners once (candidates are rare)
                  owner = true;
                  push_owner(x, epoch, t);
                }
              }
            }
            if (disks && scan) {
              // FP32 screen: a pair whose FP32 squared distance exceeds
              // sigma^2 (1 + 1e-5) is farther than sigma (FP32 error ~3e-7)
              if (__fadd_rn(__fmul_rn(r1x, r1x), __fmul_rn(r1y, r1y)) > x.sig2f) continue;
              double2 v;
              double del;
              if (edge_overlap(x, u, w, 0, 0, 0, v, del)) {
                disp_add(x, u, -v.x, -v.y);
                disp_add(x, w, v.x, v.y);
                if (use_lists) push_tri(nlist, nmark, ncount, ngen, t);   // checked again in the next pass
                const int k_ov = atomicAdd(cnt(ctl, b.ph, C_OVERLAP), 1);
                if (logging) {
                  if (log_head + k_ov < c.log_pairs_cap) d.log_pairs[log_head + k_ov] = make_int2(u, w);
                  else atomicExch(&ctl->log_overflow, 1);
                }
                mx = fmax(mx, del);
              }
            }
          }
        }
        block_add(cnt(ctl, b.ph, C_INV), inv);
        block_add(cnt(ctl, b.ph, C_REJECT), rej);
        block_add(cnt(ctl, b.ph, C_CAND), cand);
        (void)nov;
        if (mx > 0.0) atomicMax(&ctl->st_max_overlap_bits, (unsigned long long)__double_as_longlong(mx));
      }
      if (!grid_sync(ctl, b, bc)) { block_exit(ctl); return; }
      if (lead) stage_tick(ctl, full ? STAGE_P : STAGE_PL, t_mark);
      const int n_inv = bc[BC_CNT + C_INV];
      const int n_rej = bc[BC_CNT + C_REJECT];
      n_ov = bc[BC_CNT + C_OVERLAP];
      if (n_rej) {
        status = BD_ERR_STEP_REJECTED;
        if (lead) { ctl->st_fail_phase = 1; ctl->st_fail_count = n_rej; }
        break;
      }

      if (n_inv > 0) {
        // ---------------- R: inversion repair (this pass's marks and scan are void) ----------------
        st_inv += n_inv;
        int rounds = 0;
        bool first_round = true;
        for (;;) {
          ++epoch;
          if (lead) ctl->cl_n[(epoch + 2) % 3] = 0;   // the candidate list two rounds ahead
          phase_begin(ctl, b);
          {
            if (first_round) {
              for (int i = tid; i < x.np; i += nth) d.disp[i] = make_double2(0.0, 0.0);
              // the check pass skipped the marks (and the pass after the repair
              // is not fresh): a triangle with a moved corner stays dirty for it
              for (int t = tid; t < x.T; t += nth) {
                const int4 v = d.tv[t];
                if (d.moved[v.x] | d.moved[v.y] | d.moved[v.z]) d.tv[t].w = with_stamp(v.w, ngen8);
              }
            }
            int inv = 0, ncand = 0;
            for (int t = tid; t < x.T; t += nth) {
              if (!d.tinv[t]) continue;
              const int4 v = d.tv[t];
              ++inv;
              atomicExch(&ctl->st_fail_item, t);
              const int4 nn = d.tn[t];
              for (int k = 0; k < 3; ++k) {
                const int o = vk(nn, k);
                if (o < 0) continue;
                const int p = vk(v, k), u = vk(v, (k + 1) % 3), w = vk(v, (k + 2) % 3);
                const int4 v1 = d.tv[o / 3];
                const int q = vk(v1, o % 3);
                int sqx, sqy;
                opp_shift<PER>(v.w, k, v1.w, o % 3, sqx, sqy);
                const int spx = tshx<PER>(v.w, k), spy = tshy<PER>(v.w, k);
                const int sux = tshx<PER>(v.w, (k + 1) % 3), suy = tshy<PER>(v.w, (k + 1) % 3);
                const int swx = tshx<PER>(v.w, (k + 2) % 3), swy = tshy<PER>(v.w, (k + 2) % 3);
                // orientation form of Eq. (predicate): both triangles of the
                // other diagonal strictly counter-clockwise
                if (orient_s(x, u, sux, suy, q, sqx, sqy, p, spx, spy) > 0 &&
                    orient_s(x, w, swx, swy, p, spx, spy, q, sqx, sqy) > 0) {
                  const int cm = min(3 * t + k, o);
                  const int tt = cm / 3, kk = cm % 3;
                  const int4 ncm = d.tn[tt];
                  claim6(x, claims(x, epoch), tt, kk, ncm, vk(ncm, kk), claim_key(epoch, cm));
                  ++ncand;
                }
              }
            }
            block_add(cnt(ctl, b.ph, C_INV), inv);
            block_add(cnt(ctl, b.ph, C_CAND), ncand);
          }
          if (!grid_sync(ctl, b, bc)) { block_exit(ctl); return; }
          if (lead) stage_tick(ctl, STAGE_R, t_mark);
          first_round = false;
          const int ni = bc[BC_CNT + C_INV];
          const int nc = bc[BC_CNT + C_CAND];
          if (ni == 0) break;
          if (nc == 0 || rounds++ >= c.max_flip_rounds) {
            status = BD_ERR_STEP_REJECTED;
            if (lead) { ctl->st_fail_phase = nc == 0 ? 2 : 3; ctl->st_fail_count = ni; }
            break;
          }
          phase_begin(ctl, b);
          {
            int nf = 0;
            for (int t = tid; t < x.T; t += nth) {
              const unsigned long long key = claims(x, epoch)[t];
              if ((key >> 32) != epoch) continue;
              const int cm = key_corner(key);
              if (cm / 3 != t) continue;
              const int4 N0 = d.tn[t];
              const int o = vk(N0, cm % 3);
              if (!owns6(x, claims(x, epoch), t, cm % 3, N0, o, key)) continue;
              flip_owned<PER>(x, cm, o, ngen8);   // both new triangles are counter-clockwise by the rule
              ++nf;
            }
            block_add(cnt(ctl, b.ph, C_FLIPS), nf);
          }
          if (!grid_sync(ctl, b, bc)) { block_exit(ctl); return; }
          if (lead) stage_tick(ctl, STAGE_R, t_mark);
          st_rflips += bc[BC_CNT + C_FLIPS];
        }
        if (status) break;
        fresh = false;
        full = true;   // the repaired region's marks and scan were skipped: check everything
        need_p = scan = true;
        ++kp;
        continue;
      }
      if (scan) ov_now = n_ov;
    }

    // candidates for this round: the marking pass's and those the previous
    // fused round registered
    if (bc[BC_CL + (int)(epoch % 3)] > 0) {
      // ---------------- F: owned Lawson flips ----------------
      if (lawson_rounds++ >= c.max_flip_rounds) {
        status = BD_ERR_FLIP_NOT_CONVERGED;
        if (lead) ctl->st_fail_phase = 4;
        break;
      }
      phase_begin(ctl, b);
      {
        const bool voided = !fuse && n_ov;   // unfused: the marking pass's scan is void
        if (voided || fresh)
          for (int i = tid; i < x.np; i += nth) {
            if (voided) d.disp[i] = make_double2(0.0, 0.0);
            if (fresh) d.moved[i] = 0;
          }
        int nf = 0, nlose = 0, adj = 0;
        double fmx = 0.0;
        // the triangles that registered a candidate for this round (in the
        // marking pass, or in the previous fused round): each candidate is
        // owned by the triangle that tested it.  An owner whose flip lost a
        // claim is stamped, so its edges are tested again by a check pass.
        // Unfused, a flip stamps its two triangles for the next pass, and
        // every other edge the marking pass tested keeps its verdict unless a
        // flip changes it.  Fused, a flip tests the four outer edges of its
        // quadrilateral itself -- the six triangles it owns do not change
        // during the round -- and registers the illegal ones for the next
        // round (claims of the other parity, the next candidate list); it
        // also withdraws the overlap of the diagonal it removes and adds that
        // of the one it draws (exact fixed-point sums), so the sums stay those
        // of the current triangulation.
        const int cs = (int)(epoch % 3);
        const int ncl = bc[BC_CL + cs];
        const int *cl = d.clist + (size_t)cs * x.T;
        unsigned long long *cb = claims(x, epoch), *nb = claims(x, epoch + 1);
        // consecutive entries go to different blocks (a few hundred flips on
        // one SM would queue on its load/store unit)
        for (int it = blockIdx.x + threadIdx.x * gridDim.x; it < ncl; it += nth) {
          const int t = cl[it];
          const unsigned long long key = cb[t];
          bool flipped = false;
          if ((key >> 32) == epoch) {
            const int cm = key_corner(key);
            if (cm / 3 == t) {
              const int4 N0 = d.tn[t];
              const int k0 = cm % 3;
              const int o = vk(N0, k0);
              if (owns6(x, cb, t, k0, N0, o, key)) {
                if (fuse) {
                  const FusedOut fo = fused_flip<PER>(x, cm, o, nb, epoch + 1);
                  adj += fo.adj;
                  fmx = fmax(fmx, fo.mx);
                } else {
                  flip_owned<PER>(x, cm, o, ngen8);
                }
                if (!fuse && use_lists) {
                  push_tri(nlist, nmark, ncount, ngen, t);
                  push_tri(nlist, nmark, ncount, ngen, o / 3);
                }
                flipped = true;
                ++nf;
                if (d.rep_stats) {
                  // the four points of a flipped edge include a disk (ghost
                  // points never move, so an edge among them stays legal); one
                  // of the two new triangles may hold only ghost points
                  int rr = tri_rep(d, x.np, d.tv[t]);
                  if (rr < 0) rr = tri_rep(d, x.np, d.tv[o / 3]);
                  if (rr >= 0) atomicAdd((unsigned long long *)&d.rep_stats[3 * rr + 1], 1ull);
                }
              }
            }
          }
          if (!flipped) {
            ++nlose;
            stamp_tri(x, t, ngen8);
            if (use_lists) push_tri(nlist, nmark, ncount, ngen, t);
          }
        }
        block_add(cnt(ctl, b.ph, C_FLIPS), nf);
        if (fuse) {
          block_add(cnt(ctl, b.ph, C_LOSE), nlose);
          block_add(cnt(ctl, b.ph, C_OVADJ), adj);
          if (fmx > 0.0) atomicMax(&ctl->st_max_overlap_bits, (unsigned long long)__double_as_longlong(fmx));
        }
      }
      if (!grid_sync(ctl, b, bc)) { block_exit(ctl); return; }
      if (lead) stage_tick(ctl, STAGE_F, t_mark);
      st_flips += bc[BC_CNT + C_FLIPS];
      st_rounds += 1;
      fresh = false;
      full = !use_lists;
      if (!fuse) {
        need_p = scan = true;   // the next pass marks and scans afresh
        ++kp;
        continue;
      }
      ov_now += bc[BC_CNT + C_OVADJ];
      if (bc[BC_CNT + C_LOSE] > 0) {
        need_p = true;          // a pass marks the losers' edges again
        scan = false;
        ++kp;
        continue;
      }
      if (bc[BC_CL + (int)((epoch + 1) % 3)] > 0) {
        need_p = false;         // the next round flips what this one registered
        ++kp;
        continue;
      }
      // no candidate left: the triangulation is Delaunay
    }

    // Delaunay triangulation of the current positions: the overlap sums (the
    // last scan's, kept by the fused rounds) are Algorithm 2's
    if (mode == 1) {
      // new positions set from outside: they must not overlap (the scan of
      // this Delaunay triangulation finds the closest pair)
      if (ov_now) {
        status = BD_ERR_INIT_OVERLAP;
        if (lead) { ctl->st_fail_phase = 7; ctl->st_fail_count = ov_now; }
      }
      break;
    }
    if (ov_now == 0) break;
    if (corr_iter >= c.max_corr_iters) {
      status = BD_ERR_OVERLAP_NOT_CONVERGED;
      if (lead) ctl->st_fail_phase = 5;
      break;
    }
    ++corr_iter;
    st_overlap += ov_now;
    lawson_rounds = 0;
    if (logging) {
      // commit this pass to the rollout log
      log_pidx = log_npass < c.log_pass_cap ? log_npass : -1;
      if (lead) {
        if (log_pidx >= 0) {
          d.log_pass_begin[log_pidx] = log_head;
          d.log_pass_begin[log_pidx + 1] = log_head + n_ov;
        } else {
          atomicExch(&ctl->log_overflow, 1);
        }
      }
      log_head += n_ov;
      ++log_npass;
    }
    // ---------------- A: apply (capped at sigma/4) ----------------
    phase_begin(ctl, b);
    {
      int nwrap = 0;
      for (int i = tid; i < x.np; i += nth) {
        if (d.ext_id[i] < 0) continue;
        const double2 p = d.pos[i];
        d.prev[i] = p;
        const double2 dd = disp_get(x, i);
        if (PER) d.wrap[i] = 0;
        if (dd.x != 0.0 || dd.y != 0.0) {
          // the first disk of a replica moved by this pass counts the pass
          const int rr = d.rep_of[i];
          const unsigned long long stamp = epoch;   // distinct per pass (grows across launches), never 0
          if (d.rep_stats && atomicExch(&d.rep_mark[rr], stamp) != stamp)
            atomicAdd((unsigned long long *)&d.rep_stats[3 * rr], 1ull);
        }
        if (dd.x == 0.0 && dd.y == 0.0) {
          d.moved[i] = 0;
          if (log_pidx >= 0) d.log_pflags[(size_t)log_pidx * x.np + i] = 0;
          continue;
        }
        const double mag = sqrt(__dadd_rn(__dmul_rn(dd.x, dd.x), __dmul_rn(dd.y, dd.y)));
        // Sec. 4.4: sigma/4, half the disk's radius (its own for polydisperse disks)
        const double cap = d.rad ? 0.5 * d.rad[i] : 0.25 * sigma;
        const bool capped = mag > cap;
        const double sc = capped ? cap / mag : 1.0;
        const double2 y = make_double2(snap(__dadd_rn(p.x, __dmul_rn(dd.x, sc)), x.g),
                                       snap(__dadd_rn(p.y, __dmul_rn(dd.y, sc)), x.g));
        int rfl = 0;
        const BdRep &R = d.rep[d.rep_of[i]];
        double2 np2;
        if (PER && R.periodic) {
          // Algorithm 2 "applying the periodic boundary conditions": re-entry
          long long X = bdpred::to_int(y.x, x.g), Y = bdpred::to_int(y.y, x.g);
          d.dmove[i] = make_float2(bdem::grid_to_float(X - bdpred::to_int(p.x, x.g), x.g.s),
                                   bdem::grid_to_float(Y - bdpred::to_int(p.y, x.g), x.g.s));
          const int wr = bdem::wrap_grid(R.LQ, X, Y);
          d.wrap[i] = (uint8_t)wr;
          if (wr) ++nwrap;
          np2 = make_double2(bdem::grid_to_double(X, x.g.s), bdem::grid_to_double(Y, x.g.s));
        } else {
          np2 = bdem::reflect_w(bdem::walls_of(d, R, i), y, &rfl);
        }
        if (log_pidx >= 0) d.log_pflags[(size_t)log_pidx * x.np + i] = (uint8_t)(rfl | (capped ? 16 : 0));
        d.pos[i] = np2;
        d.work[i] = split_pos(np2);
        if (!(PER && R.periodic)) {
          d.dmove[i] = make_float2(bdem::grid_to_float(bdpred::to_int(np2.x, x.g) - bdpred::to_int(p.x, x.g), x.g.s),
                                   bdem::grid_to_float(bdpred::to_int(np2.y, x.g) - bdpred::to_int(p.y, x.g), x.g.s));
        }
        d.disp[i] = make_double2(0.0, 0.0);
        d.moved[i] = 1;
        // the next pass visits the star of the moved disk (walked across the
        // edges (i, p) of its triangles, from the corner vt[i])
        const int c0 = d.vt[i];
        int cw = c0;
        for (int guard = 0; use_lists && guard < 256; ++guard) {
          const int tw = cw / 3;
          push_tri(nlist, nmark, ncount, ngen, tw);
          const int o = ((const int *)&d.tn[tw])[(cw % 3 + 2) % 3];
          if (o < 0) break;
          cw = 3 * (o / 3) + (o % 3 + 2) % 3;
          if (cw == c0) break;
        }
      }
      if (PER) block_add(&ctl->n_wrapped, nwrap);
    }
    if (!grid_sync(ctl, b, bc)) { block_exit(ctl); return; }
    if (lead) stage_tick(ctl, STAGE_A, t_mark);
    fresh = true;
    full = !use_lists;
    need_p = scan = true;
    ++kp;
  }

  if (status) {
    // undo the step: positions and directions from the step start, the
    // triangulation from the undo journal
    phase_begin(ctl, b);
    for (int i = tid; i < x.np; i += nth) {
      if (d.ext_id[i] < 0) continue;
      const double2 p0 = d.pos0[i];
      d.pos[i] = p0;
      d.prev[i] = p0;
      d.work[i] = split_pos(p0);
      d.theta[i] = d.theta0[i];
      d.disp[i] = make_double2(0.0, 0.0);
      d.moved[i] = 0;
    }
    // the journaled triangles as they were; a corner for each of their
    // vertices (flips re-point only the vertices of the triangles they change)
    for (int t = tid; t < x.T; t += nth) {
      d.tinv[t] = 0;
      if (d.jmark[t] == x.jstamp) unjournal(d, t);
    }
    if (lead) atomicCAS(&ctl->status, 0, status);
  } else {
    for (int i = tid; i < x.np; i += nth) d.moved[i] = 0;
  }
  if (lead) {
    if (logging && !status) {
      ctl->log_npairs = log_head;
      ctl->log_npass = log_npass;
      d.log_step_pass[log_step + 1] = log_npass;
    }
    ctl->epoch = epoch + 1;
    ctl->act_gen = g0 + (unsigned)kp + 3u;
    ctl->st_tri_visits += tri_visits;
    ctl->st_corr_iters += corr_iter;
    ctl->st_overlap_pairs += st_overlap;
    ctl->st_flips += st_flips;
    ctl->st_repair_flips += st_rflips;
    ctl->st_inverted += st_inv;
    ctl->st_flip_rounds += st_rounds;
    ctl->st_barriers += b.gen;
    if (corr_iter > ctl->st_max_corr_iters) ctl->st_max_corr_iters = corr_iter;
    if (!status && mode == 2) ctl->st_substeps += 1;
    else if (!status) ctl->st_steps += 1;
    if (!status && mode == 0) ctl->step_dev += 1;
  }
  block_exit(ctl);
}

// Undo a step whose persistent kernel left at a timed-out barrier (the
// kernel's own failure path did not run).  The launch journaled every
// triangle before its first change to it, and all its blocks have finished
// (this kernel runs after it in stream order), so replaying the journal
// restores the triangulation; positions and directions come from pos0 /
// theta0 (the step start, or the positions before bd_set_state).
// bd_launch_restore_step runs it (the header above the launcher declares it).
__global__ void k_restore_step(BdDev d, BdConst c) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nth = gridDim.x * blockDim.x;
  for (int i = tid; i < c.np; i += nth) {
    if (d.ext_id[i] < 0) continue;
    const double2 p0 = d.pos0[i];
    d.pos[i] = p0;
    d.prev[i] = p0;
    d.work[i] = split_pos(p0);
    d.theta[i] = d.theta0[i];
    d.disp[i] = make_double2(0.0, 0.0);
    d.moved[i] = 0;
  }
  if (!c.overlap_verlet) {
    // the journaled triangles as they were, a corner for each of their
    // vertices; their marks cleared (the abandoned launch did not publish its
    // epoch, so the next launch takes the same stamp)
    const unsigned jstamp = ((unsigned)d.ctl->epoch << 1) | 1u;
    for (int t = tid; t < c.nt; t += nth) {
      d.tinv[t] = 0;
      if (d.jmark[t] == jstamp) {
        unjournal(d, t);
        d.jmark[t] = 0u;
      }
      // the abandoned launch did not publish the claim epochs and list
      // generations it used (the next launch starts from the same ones):
      // clear its claims (0 matches no epoch) and list marks (0 matches no
      // generation after the first launch)
      d.claim[t] = 0ull;
      for (int l = 0; l < 3; ++l) d.act_mark[(size_t)l * c.nt + t] = 0u;
    }
  }
}

cudaError_t bd_launch_restore_step(const BdDev &d, const BdConst &c, cudaStream_t s) {
  const int work = c.np > c.nt ? c.np : c.nt;
  int blocks = (work + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 4096) blocks = 4096;
  k_restore_step<<<blocks, 256, 0, s>>>(d, c);
  return cudaGetLastError();
}

int bd_dt_grid_for(int work_items, int *grid, int *block) {
  // all co-resident blocks (the phases are latency-bound chains of dependent
  // loads and integer predicates, so more threads in flight help), but no
  // more than about one work item per thread
  int g = 0, b = 0;
  if (bd_dt_grid(&g, &b) != 0) return -1;
  int want = (work_items + b - 1) / b;
  if (want < 1) want = 1;
  *grid = want < g ? want : g;
  *block = b;
  return 0;
}

int bd_dt_grid(int *grid, int *block) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_triangulation<false>, BD_DT_THREADS, 0) !=
      cudaSuccess)
    return -1;
  if (per < 1) return -1;
  *grid = sms * per;
  *block = BD_DT_THREADS;
  return 0;
}

cudaError_t bd_launch_dt(const BdDev &d, const BdConst &c, int mode, cudaStream_t s, int grid,
                         int block, int log_step) {
  // the barrier words and phase counters were reset by the previous
  // launch's last block (and zeroed at allocation)
  BdDev dd = d;
  BdConst cc = c;
  int m = mode, ls = log_step;
  void *args[] = {&dd, &cc, &m, &ls};
  const void *fn = c.any_periodic ? (const void *)k_triangulation<true> : (const void *)k_triangulation<false>;
  return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(block), args, 0, s);
}
