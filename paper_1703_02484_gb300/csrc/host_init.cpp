// Host-side initialisation: seeded placement, spatial ordering and the
// initial Delaunay triangulation.
//
// Sec. 4.1: "the Delaunay triangulation of the particle positions is built
// only once from scratch on the host" and then maintained on the device.
// The paper uses CGAL's periodic triangulation; this build uses reflecting
// walls and closes the hull with fixed ghost points outside the box (see
// make_ghosts), and builds the triangulation by incremental insertion: each point
// splits the triangle (or edge) that contains it and Lawson flips restore
// the empty-circle property around it.  Predicates are exact (predicates.cuh).
//
// Layout ("corner table"): triangle t has corners 3t+0..3t+2 holding vertex
// ids in counter-clockwise order; opp[3t+k] is the corner of the neighbouring
// triangle facing the edge opposite corner k (-1 on the outer square).
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "philox.cuh"
#include "predicates.cuh"

namespace bdhost {

static inline int nxt(int c) { return c - c % 3 + (c % 3 + 1) % 3; }
static inline int prv(int c) { return c - c % 3 + (c % 3 + 2) % 3; }

struct Tri {
  const double *X, *Y;
  bdpred::Grid g;
  std::vector<int> V, N;

  int orient(int a, int b, int c) const {
    return bdpred::orient(X[a], Y[a], X[b], Y[b], X[c], Y[c], g);
  }
  int orient_pt(int a, int b, double px, double py) const {
    return bdpred::orient(X[a], Y[a], X[b], Y[b], px, py, g);
  }
  // > 0 iff vertex d lies strictly inside the circumcircle of triangle t
  int incircle_tri(int t, int d) const {
    int a = V[3 * t], b = V[3 * t + 1], c = V[3 * t + 2];
    return bdpred::incircle(X[a], Y[a], X[b], Y[b], X[c], Y[c], X[d], Y[d], g);
  }
  int new_tri() {
    V.push_back(-1); V.push_back(-1); V.push_back(-1);
    N.push_back(-1); N.push_back(-1); N.push_back(-1);
    return (int)(V.size() / 3) - 1;
  }
  void link(int c, int o) {
    N[c] = o;
    if (o >= 0) N[o] = c;
  }

  // flip the edge facing corner c0 (its triangle and the neighbour across it
  // become the other diagonal of their quadrilateral)
  void flip(int c0) {
    int o0 = N[c0];
    int t0 = c0 / 3, k0 = c0 % 3, t1 = o0 / 3, k1 = o0 % 3;
    int a = V[c0], b = V[nxt(c0)], c = V[prv(c0)], d = V[o0];
    int n_ca = N[3 * t0 + (k0 + 1) % 3], n_ab = N[3 * t0 + (k0 + 2) % 3];
    int n_bd = N[3 * t1 + (k1 + 1) % 3], n_dc = N[3 * t1 + (k1 + 2) % 3];
    V[3 * t0 + k0] = b; V[3 * t0 + (k0 + 1) % 3] = d; V[3 * t0 + (k0 + 2) % 3] = a;
    V[3 * t1 + k1] = c; V[3 * t1 + (k1 + 1) % 3] = a; V[3 * t1 + (k1 + 2) % 3] = d;
    link(3 * t0 + k0, 3 * t1 + k1);
    link(3 * t0 + (k0 + 1) % 3, n_ab);
    link(3 * t0 + (k0 + 2) % 3, n_bd);
    link(3 * t1 + (k1 + 1) % 3, n_dc);
    link(3 * t1 + (k1 + 2) % 3, n_ca);
  }

  void legalize(std::vector<int> &stack) {
    while (!stack.empty()) {
      int c = stack.back();
      stack.pop_back();
      int o = N[c];
      if (o < 0) continue;
      int t = c / 3;
      if (incircle_tri(t, V[o]) > 0) {
        int t0 = t, k0 = c % 3, t1 = o / 3, k1 = o % 3;
        flip(c);
        // the inserted point sits at corner k0+2 of t0 and k1+1 of t1
        stack.push_back(3 * t0 + (k0 + 2) % 3);
        stack.push_back(3 * t1 + (k1 + 1) % 3);
      }
    }
  }

  // walk from triangle t towards (px, py); returns the containing triangle
  // and in *on_edge the corner facing the edge the point lies on (-1 if
  // strictly inside, -2 if it coincides with a vertex, -3 if outside)
  int locate(int t, double px, double py, int *on_edge) const {
    int rot = 0;
    long guard = 0;
    for (;;) {
      int moved = 0;
      for (int kk = 0; kk < 3; ++kk) {
        int k = (kk + rot) % 3;
        int a = V[3 * t + (k + 1) % 3], b = V[3 * t + (k + 2) % 3];
        if (orient_pt(a, b, px, py) < 0) {
          int o = N[3 * t + k];
          if (o < 0) { *on_edge = -3; return t; }
          t = o / 3;
          moved = 1;
          break;
        }
      }
      rot = (rot + 1) % 3;
      if (!moved) break;
      if (++guard > 100000000L) { *on_edge = -3; return t; }
    }
    int zeros = 0, zk = -1;
    for (int k = 0; k < 3; ++k) {
      int a = V[3 * t + (k + 1) % 3], b = V[3 * t + (k + 2) % 3];
      if (orient_pt(a, b, px, py) == 0) { ++zeros; zk = k; }
    }
    *on_edge = zeros == 0 ? -1 : (zeros == 1 ? 3 * t + zk : -2);
    return t;
  }

  int insert(int p, int start, std::vector<int> &stack) {
    int on = 0;
    int t = locate(start, X[p], Y[p], &on);
    if (on == -3 || on == -2) return on;
    if (on == -1) {
      int a = V[3 * t], b = V[3 * t + 1], c = V[3 * t + 2];
      int na = N[3 * t], nb = N[3 * t + 1], nc = N[3 * t + 2];
      int T0 = t, T1 = new_tri(), T2 = new_tri();
      V[3 * T0] = a; V[3 * T0 + 1] = b; V[3 * T0 + 2] = p;
      V[3 * T1] = b; V[3 * T1 + 1] = c; V[3 * T1 + 2] = p;
      V[3 * T2] = c; V[3 * T2 + 1] = a; V[3 * T2 + 2] = p;
      link(3 * T0 + 0, 3 * T1 + 1);
      link(3 * T0 + 1, 3 * T2 + 0);
      link(3 * T1 + 0, 3 * T2 + 1);
      link(3 * T0 + 2, nc);
      link(3 * T1 + 2, na);
      link(3 * T2 + 2, nb);
      stack.push_back(3 * T0 + 2);
      stack.push_back(3 * T1 + 2);
      stack.push_back(3 * T2 + 2);
      legalize(stack);
      return T0;
    }
    // on the edge facing corner `on`: split both triangles
    int c0 = on, o = N[c0];
    if (o < 0) return -3;
    int t0 = c0 / 3, k = c0 % 3, t1 = o / 3, k1 = o % 3;
    int a = V[c0], b = V[3 * t0 + (k + 1) % 3], c = V[3 * t0 + (k + 2) % 3], d = V[o];
    int n_ca = N[3 * t0 + (k + 1) % 3], n_ab = N[3 * t0 + (k + 2) % 3];
    int n_bd = N[3 * t1 + (k1 + 1) % 3], n_dc = N[3 * t1 + (k1 + 2) % 3];
    int T0 = t0, T1 = new_tri(), T2 = t1, T3 = new_tri();
    V[3 * T0] = a; V[3 * T0 + 1] = b; V[3 * T0 + 2] = p;
    V[3 * T1] = a; V[3 * T1 + 1] = p; V[3 * T1 + 2] = c;
    V[3 * T2] = d; V[3 * T2 + 1] = c; V[3 * T2 + 2] = p;
    V[3 * T3] = d; V[3 * T3 + 1] = p; V[3 * T3 + 2] = b;
    link(3 * T0 + 0, 3 * T3 + 0);
    link(3 * T0 + 1, 3 * T1 + 2);
    link(3 * T1 + 0, 3 * T2 + 0);
    link(3 * T2 + 1, 3 * T3 + 2);
    link(3 * T0 + 2, n_ab);
    link(3 * T1 + 1, n_ca);
    link(3 * T2 + 2, n_dc);
    link(3 * T3 + 1, n_bd);
    stack.push_back(3 * T0 + 2);
    stack.push_back(3 * T1 + 1);
    stack.push_back(3 * T2 + 2);
    stack.push_back(3 * T3 + 1);
    legalize(stack);
    return T0;
  }
};

// Points that close the triangulation around the box (ids after the disks).
// The paper's box is periodic (a torus has no hull); with walls the hull is
// closed here by four far corners plus a ring of fixed points just outside
// the walls.  The ring keeps the triangles at the walls well shaped: with the
// corners alone, disks along a wall form long slivers that a noise step
// inverts.  Layout, with C = ceil(L), W = S = ceil(2a):
//   [0..3] far corners (-F,-F), (G,-F), (G,G), (-F,G), F = C + 3W, G = 2C + 3W
//   rows   y = -W - off(k, 4+side) (bottom, side 0), y = C + W + off(k, 4+side) (top, side 1),
//          x = -W + k S + off(k, side)
//   cols   x = -W - off(k, 4+side) (left, side 2),   x = C + W + off(k, 4+side) (right, side 3),
//          y = -W + S/2 + k S + off(k, side)
// off(k, s) = ((7919 k + 104729 s) mod 257) / 1024 in [0, 1/4] breaks the
// symmetries that would make four ghost points cocircular.  All values are
// dyadic, hence exact on the position grid.
void make_ghosts(double L, double a, std::vector<double> &gx, std::vector<double> &gy) {
  const double C = ceil(L), W = ceil(2.0 * a), S = W;
  const double F = C + 3.0 * W, G = 2.0 * C + 3.0 * W;
  gx.assign({-F, G, G, -F});
  gy.assign({-F, -F, G, G});
  auto off = [](long k, long side) { return (double)((7919L * k + 104729L * side) % 257L) / 1024.0; };
  for (int side = 0; side < 2; ++side) {
    for (long k = 0; -W + k * S <= C + W; ++k) {
      gx.push_back(-W + k * S + off(k, side));
      gy.push_back(side == 0 ? -W - off(k, 4 + side) : C + W + off(k, 4 + side));
    }
  }
  for (int side = 2; side < 4; ++side) {
    for (long k = 0; -W + 0.5 * S + k * S < C + W; ++k) {
      gx.push_back(side == 2 ? -W - off(k, 4 + side) : C + W + off(k, 4 + side));
      gy.push_back(-W + 0.5 * S + k * S + off(k, side));
    }
  }
}

// largest coordinate magnitude among disks and ghost points
double ghost_extent(double L, double a) { return 2.0 * ceil(L) + 3.0 * ceil(2.0 * a); }

// Hilbert-curve index of (x, y) on a 2^16 x 2^16 grid (locality order only)
uint64_t hilbert_index(uint32_t x, uint32_t y) {
  const uint32_t n = 1u << 16;
  uint64_t d = 0;
  for (uint32_t s = n / 2; s > 0; s /= 2) {
    uint32_t rx = (x & s) ? 1u : 0u;
    uint32_t ry = (y & s) ? 1u : 0u;
    d += (uint64_t)s * (uint64_t)s * ((3u * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) {
        x = n - 1 - x;
        y = n - 1 - y;
      }
      uint32_t t = x;
      x = y;
      y = t;
    }
  }
  return d;
}

// Delaunay triangulation of the points listed in `order` (ids into X/Y)
// plus the ghost points `g` (g[0..3] a counter-clockwise square enclosing
// everything, the rest inserted first).  Fills V/N (corner table).  Returns 0
// or a negative code (-2 duplicate point, -3 point outside the corner square).
int build_delaunay(const double *X, const double *Y, const bdpred::Grid &grid,
                   const std::vector<int> &order, const std::vector<int> &g, std::vector<int> &V,
                   std::vector<int> &N) {
  Tri T;
  T.X = X;
  T.Y = Y;
  T.g = grid;
  T.V.reserve(3 * (2 * order.size() + 4));
  T.N.reserve(3 * (2 * order.size() + 4));
  int t0 = T.new_tri(), t1 = T.new_tri();
  T.V[0] = g[0]; T.V[1] = g[1]; T.V[2] = g[2];
  T.V[3] = g[0]; T.V[4] = g[2]; T.V[5] = g[3];
  T.link(3 * t0 + 1, 3 * t1 + 2);
  std::vector<int> stack;
  int last = t0;
  for (size_t i = 4; i < g.size(); ++i) {
    int r = T.insert(g[i], last, stack);
    if (r < 0) return r;
    last = r;
  }
  for (size_t i = 0; i < order.size(); ++i) {
    int r = T.insert(order[i], last, stack);
    if (r < 0) return r;
    last = r;
  }
  V.swap(T.V);
  N.swap(T.N);
  return 0;
}

// seeded random sequential addition of n centres in [lo, hi]^2, pairwise
// distance >= dmin, cell-grid accelerated; Philox stream TAG_PLACE
int rsa_place(int n, double lo, double hi, double dmin, uint64_t seed, std::vector<double> &xy) {
  double W = hi - lo;
  if (W <= 0) return -1;
  int nc = std::max(1, (int)floor(W / dmin));
  double cs = W / nc;
  std::vector<std::vector<int>> cells((size_t)nc * nc);
  xy.assign(2 * (size_t)n, 0.0);
  uint64_t attempt = 0;
  const uint64_t max_attempts = 1000ull * (uint64_t)n + 1000000ull;
  int k = 0;
  while (k < n) {
    if (attempt >= max_attempts) return -2;
    bdrng::U4 r = bdrng::draw((uint32_t)(attempt & 0xFFFFFFFFu), (int64_t)(attempt >> 32), seed, 0,
                              bdrng::TAG_PLACE);
    ++attempt;
    double ux = ((double)r.x + 0.5) * (1.0 / 4294967296.0);
    double uy = ((double)r.y + 0.5) * (1.0 / 4294967296.0);
    double x = lo + W * ux, y = lo + W * uy;
    int cx = std::min(nc - 1, (int)((x - lo) / cs)), cy = std::min(nc - 1, (int)((y - lo) / cs));
    bool ok = true;
    for (int gx = cx - 1; gx <= cx + 1 && ok; ++gx)
      for (int gy = cy - 1; gy <= cy + 1 && ok; ++gy) {
        if (gx < 0 || gy < 0 || gx >= nc || gy >= nc) continue;
        for (int j : cells[(size_t)gx * nc + gy]) {
          double dx = xy[2 * j] - x, dy = xy[2 * j + 1] - y;
          if (dx * dx + dy * dy < dmin * dmin) { ok = false; break; }
        }
      }
    if (!ok) continue;
    xy[2 * k] = x;
    xy[2 * k + 1] = y;
    cells[(size_t)cx * nc + cy].push_back(k);
    ++k;
  }
  return 0;
}

// minimum pair distance check with a cell grid: returns 1 if some pair is
// closer than dmin
int any_overlap(int n, const double *xy, double lo, double hi, double dmin) {
  double W = hi - lo;
  int nc = std::max(1, std::min(4096, (int)floor(W / dmin)));
  double cs = W / nc;
  std::vector<std::vector<int>> cells((size_t)nc * nc);
  for (int i = 0; i < n; ++i) {
    int cx = std::min(nc - 1, std::max(0, (int)((xy[2 * i] - lo) / cs)));
    int cy = std::min(nc - 1, std::max(0, (int)((xy[2 * i + 1] - lo) / cs)));
    for (int gx = cx - 1; gx <= cx + 1; ++gx)
      for (int gy = cy - 1; gy <= cy + 1; ++gy) {
        if (gx < 0 || gy < 0 || gx >= nc || gy >= nc) continue;
        for (int j : cells[(size_t)gx * nc + gy]) {
          double dx = xy[2 * j] - xy[2 * i], dy = xy[2 * j + 1] - xy[2 * i + 1];
          if (dx * dx + dy * dy < dmin * dmin) return 1;
        }
      }
    cells[(size_t)cx * nc + cy].push_back(i);
  }
  return 0;
}

}  // namespace bdhost
