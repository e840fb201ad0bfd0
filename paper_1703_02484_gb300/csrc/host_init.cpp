// Host-side initialisation: seeded placement, spatial ordering and the
// initial Delaunay triangulation.
//
// Sec. 4.1: "the Delaunay triangulation of the particle positions is built
// only once from scratch on the host" and then maintained on the device.
// The paper uses CGAL's periodic triangulation; with reflecting walls (the
// benchmark configurations) the hull is closed with fixed ghost points
// outside the box (see make_ghosts).  The triangulation is built by
// incremental insertion: each point splits the triangle (or edge) that
// contains it and Lawson flips restore the empty-circle property around it.  Predicates are exact (predicates.cuh).
//
// Layout ("corner table"): triangle t has corners 3t+0..3t+2 holding vertex
// ids in counter-clockwise order; opp[3t+k] is the corner of the neighbouring
// triangle facing the edge opposite corner k (-1 on the outer square).
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <unordered_map>
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

// ---- periodic box (Sec. 2.1; the triangulation lives on a flat torus, Sec. 4.1) ----
//
// The torus triangulation is read off the planar Delaunay triangulation of
// the points plus their images within a band of width w around the box
// (shifted by L in x, y or both), closed by four far corners.  A torus
// triangle is kept once, as the lifted triangle whose smallest point id sits
// in the box itself (shift 0).  Corners carry integer image shifts: corner k
// lies at (X, Y)[id] + L shift_k; each triangle is stored with corner 0 at
// shift 0.  The result is accepted only if it is a closed torus triangulation
// (2n triangles, every edge shared by exactly two, matched by vertex pair
// and relative shift), every triangle is counter-clockwise and every edge is
// locally Delaunay (exact predicates on the lifted grid coordinates); a band
// too narrow for that is doubled and the build repeated.

namespace {

struct TorusPt {
  int id, sx, sy;
};

inline uint64_t edge_key(int u, int w, int sx, int sy) {
  return ((uint64_t)(uint32_t)u << 34) | ((uint64_t)(uint32_t)w << 6) | ((uint64_t)(sx + 2) << 3) |
         (uint64_t)(sy + 2);
}

}  // namespace

int build_torus_delaunay(const double *X, const double *Y, const std::vector<int> &ids, double L,
                         const bdpred::Grid &grid, std::vector<int> &V, std::vector<int> &S,
                         std::vector<int> &N) {
  const int n = (int)ids.size();
  if (n < 3) return -4;
  const int64_t LQ = bdpred::to_int(L, grid);
  double w = std::min(L, 8.0 * L / sqrt((double)n) + 1.0);
  for (int attempt = 0; attempt < 6; ++attempt, w = std::min(L, 2.0 * w)) {
    // points: the box's own, then images within the band, then 4 far corners
    std::vector<TorusPt> pts;
    std::vector<double> px, py;
    pts.reserve(n + n / 2);
    for (int k = 0; k < n; ++k) {
      const int i = ids[k];
      for (int sy = -1; sy <= 1; ++sy)
        for (int sx = -1; sx <= 1; ++sx) {
          const double x = X[i] + sx * L, y = Y[i] + sy * L;
          if (x < -w || x >= L + w || y < -w || y >= L + w) continue;
          if (sx == 0 && sy == 0) continue;
          pts.push_back({i, sx, sy});
          px.push_back(x);
          py.push_back(y);
        }
    }
    std::vector<TorusPt> all;
    std::vector<double> ax, ay;
    all.reserve(n + pts.size() + 4);
    for (int k = 0; k < n; ++k) {
      all.push_back({ids[k], 0, 0});
      ax.push_back(X[ids[k]]);
      ay.push_back(Y[ids[k]]);
    }
    for (size_t k = 0; k < pts.size(); ++k) {
      all.push_back(pts[k]);
      ax.push_back(px[k]);
      ay.push_back(py[k]);
    }
    const int m = (int)all.size();
    const double F = 3.0 * L + 3.0 * w;
    const double cx[4] = {-F, L + F, L + F, -F}, cy[4] = {-F, -F, L + F, L + F};
    for (int k = 0; k < 4; ++k) {
      all.push_back({-1, 0, 0});
      ax.push_back(cx[k]);
      ay.push_back(cy[k]);
    }
    std::vector<int> order(m), gids(4);
    for (int k = 0; k < m; ++k) order[k] = k;
    // insertion in a locality order keeps the point-location walks short
    std::vector<uint64_t> hk(m);
    for (int k = 0; k < m; ++k) {
      uint32_t ux = (uint32_t)std::min(65535.0, std::max(0.0, (ax[k] + w) / (L + 2 * w) * 65536.0));
      uint32_t uy = (uint32_t)std::min(65535.0, std::max(0.0, (ay[k] + w) / (L + 2 * w) * 65536.0));
      hk[k] = hilbert_index(ux, uy);
    }
    std::sort(order.begin(), order.end(), [&](int a, int b) { return hk[a] != hk[b] ? hk[a] < hk[b] : a < b; });
    for (int k = 0; k < 4; ++k) gids[k] = m + k;
    std::vector<int> PV, PN;
    if (build_delaunay(ax.data(), ay.data(), grid, order, gids, PV, PN) != 0) return -2;
    // keep one lift per torus triangle
    V.clear();
    S.clear();
    const int ntp = (int)(PV.size() / 3);
    for (int t = 0; t < ntp; ++t) {
      const int a = PV[3 * t], b = PV[3 * t + 1], c = PV[3 * t + 2];
      if (a >= m || b >= m || c >= m) continue;
      const TorusPt *q[3] = {&all[a], &all[b], &all[c]};
      int k0 = 0;
      for (int k = 1; k < 3; ++k)
        if (q[k]->id < q[k0]->id) k0 = k;
      if (q[k0]->sx != 0 || q[k0]->sy != 0) continue;
      // rotate so that corner 0 is the one at shift 0 with the smallest id
      for (int k = 0; k < 3; ++k) {
        const TorusPt *r = q[(k0 + k) % 3];
        V.push_back(r->id);
        S.push_back(r->sx);
        S.push_back(r->sy);
      }
    }
    const int T = (int)(V.size() / 3);
    if (T != 2 * n) continue;
    // neighbours: the edge opposite corner k runs from corner k+1 to k+2 with
    // relative shift s; its twin in the neighbour runs back with shift -s
    std::unordered_map<uint64_t, int> dir;
    dir.reserve(3 * (size_t)T * 2);
    bool ok = true;
    for (int t = 0; t < T && ok; ++t)
      for (int k = 0; k < 3; ++k) {
        const int c1 = 3 * t + (k + 1) % 3, c2 = 3 * t + (k + 2) % 3;
        const uint64_t key = edge_key(V[c1], V[c2], S[2 * c2] - S[2 * c1], S[2 * c2 + 1] - S[2 * c1 + 1]);
        if (!dir.emplace(key, 3 * t + k).second) { ok = false; break; }
      }
    if (!ok) continue;
    N.assign(3 * (size_t)T, -1);
    for (int t = 0; t < T && ok; ++t)
      for (int k = 0; k < 3; ++k) {
        const int c1 = 3 * t + (k + 1) % 3, c2 = 3 * t + (k + 2) % 3;
        auto it = dir.find(edge_key(V[c2], V[c1], S[2 * c1] - S[2 * c2], S[2 * c1 + 1] - S[2 * c2 + 1]));
        if (it == dir.end()) { ok = false; break; }
        N[3 * t + k] = it->second;
      }
    if (!ok) continue;
    // exact checks on lifted grid coordinates
    auto lx = [&](int c) { return bdpred::to_int(X[V[c]], grid) + (int64_t)S[2 * c] * LQ; };
    auto ly = [&](int c) { return bdpred::to_int(Y[V[c]], grid) + (int64_t)S[2 * c + 1] * LQ; };
    for (int t = 0; t < T && ok; ++t) {
      const int c0 = 3 * t;
      if (bdpred::orient_int(lx(c0), ly(c0), lx(c0 + 1), ly(c0 + 1), lx(c0 + 2), ly(c0 + 2)) <= 0) ok = false;
      for (int k = 0; k < 3 && ok; ++k) {
        const int o = N[3 * t + k], t1 = o / 3, k1 = o % 3;
        // the neighbour's frame: its corner k1+2 is this triangle's corner k+1
        const int cu = 3 * t + (k + 1) % 3, cu1 = 3 * t1 + (k1 + 2) % 3;
        const int64_t ox = (int64_t)(S[2 * cu] - S[2 * cu1]) * LQ, oy = (int64_t)(S[2 * cu + 1] - S[2 * cu1 + 1]) * LQ;
        if (bdpred::incircle_int(lx(c0), ly(c0), lx(c0 + 1), ly(c0 + 1), lx(c0 + 2), ly(c0 + 2), lx(o) + ox,
                                 ly(o) + oy) > 0)
          ok = false;
      }
    }
    if (ok) return 0;
    if (w >= L) break;
  }
  return -5;
}

// Cell list as a counting sort (flat arrays): cell of each centre, start of
// each cell's run in `order`.  Cells of side >= dmin, nc per side.
static void cell_sort(int n, const double *xy, double lo, double cs, int nc, std::vector<int> &cell,
                      std::vector<int> &start, std::vector<int> &order) {
  cell.resize(n);
  start.assign((size_t)nc * nc + 1, 0);
  for (int i = 0; i < n; ++i) {
    const int cx = std::min(nc - 1, std::max(0, (int)((xy[2 * i] - lo) / cs)));
    const int cy = std::min(nc - 1, std::max(0, (int)((xy[2 * i + 1] - lo) / cs)));
    cell[i] = cy * nc + cx;
    ++start[cell[i] + 1];
  }
  for (size_t k = 0; k + 1 < start.size(); ++k) start[k + 1] += start[k];
  order.resize(n);
  std::vector<int> fill(start.begin(), start.end() - 1);
  for (int i = 0; i < n; ++i) order[fill[cell[i]]++] = i;
}

// a pair's overlap test: closer than dmin, or for polydisperse disks (rad
// given) closer than (rad_i + rad_j)(1 - 1e-12); dmin is then the largest
// contact distance (the cell size)
static inline bool too_close(double d2, double dmin, const double *rad, int i, int j) {
  if (!rad) return d2 < dmin * dmin;
  const double s = (rad[i] + rad[j]) * (1.0 - 1e-12);
  return d2 < s * s;
}

// periodic minimum-image overlap check (centres in [0, L)): 1 if some pair
// is closer than dmin (polydisperse: than rad_i + rad_j)
int any_overlap_periodic(int n, const double *xy, double L, double dmin, const double *rad) {
  int nc = std::max(1, std::min(4096, (int)floor(L / dmin)));
  if (nc < 3) {
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j) {
        double dx = xy[2 * j] - xy[2 * i], dy = xy[2 * j + 1] - xy[2 * i + 1];
        dx -= L * nearbyint(dx / L);
        dy -= L * nearbyint(dy / L);
        if (too_close(dx * dx + dy * dy, dmin, rad, i, j)) return 1;
      }
    return 0;
  }
  const double cs = L / nc;
  std::vector<int> cell, start, order;
  cell_sort(n, xy, 0.0, cs, nc, cell, start, order);
  for (int i = 0; i < n; ++i) {
    const int cx = cell[i] % nc, cy = cell[i] / nc;
    for (int gy = cy - 1; gy <= cy + 1; ++gy)
      for (int gx = cx - 1; gx <= cx + 1; ++gx) {
        const int c = ((gy + nc) % nc) * nc + (gx + nc) % nc;
        for (int k = start[c]; k < start[c + 1]; ++k) {
          const int j = order[k];
          if (j >= i) continue;
          double dx = xy[2 * j] - xy[2 * i], dy = xy[2 * j + 1] - xy[2 * i + 1];
          dx -= L * nearbyint(dx / L);
          dy -= L * nearbyint(dy / L);
          if (too_close(dx * dx + dy * dy, dmin, rad, i, j)) return 1;
        }
      }
  }
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

// The paper's initial placement (Sec. 4.1): a triangular lattice over
// [lo, hi]^2 with N* >= n sites (the widest spacing s >= dmin that gives
// enough sites; rows s sqrt(3)/2 apart, odd rows offset by s/2), n of them
// chosen by reservoir sampling (Vitter's algorithm R: the first n sites fill
// the reservoir, site k >= n replaces a uniform slot j in [0, k] when j < n),
// each moved by a uniform offset in the disk of radius (s - dmin)/2, so that
// no two come closer than dmin and the set is in general position; an offset
// that would leave [lo, hi] keeps the site.  Philox stream TAG_LATTICE.
// Returns -1 when even spacing dmin gives fewer than n sites.
int lattice_place(int n, double lo, double hi, double dmin, uint64_t seed, std::vector<double> &xy) {
  const double W = hi - lo;
  if (!(W > 0) || n < 1) return -1;
  const double h3 = 0.5 * sqrt(3.0);
  auto count = [&](double sp, int &nx0, int &nx1, int &ny) -> long long {
    nx0 = (int)floor(W / sp) + 1;                                  // even rows
    nx1 = W >= 0.5 * sp ? (int)floor((W - 0.5 * sp) / sp) + 1 : 0;  // odd rows
    ny = (int)floor(W / (sp * h3)) + 1;
    return (long long)((ny + 1) / 2) * nx0 + (long long)(ny / 2) * nx1;
  };
  int nx0 = 0, nx1 = 0, ny = 0;
  if (count(dmin, nx0, nx1, ny) < n) return -1;
  double s_lo = dmin, s_hi = std::max(dmin, W);   // count(s_lo) >= n
  for (int it = 0; it < 100; ++it) {
    const double mid = 0.5 * (s_lo + s_hi);
    if (count(mid, nx0, nx1, ny) >= n) s_lo = mid; else s_hi = mid;
  }
  const double sp = s_lo;
  const long long nsites = count(sp, nx0, nx1, ny);
  auto site = [&](long long k, double &x, double &y) {
    const long long pair = (long long)nx0 + nx1;
    const long long r2 = k / pair, rem = k % pair;
    const int row = (int)(2 * r2 + (rem < nx0 ? 0 : 1));
    const int col = (int)(rem < nx0 ? rem : rem - nx0);
    x = lo + (row & 1 ? 0.5 * sp : 0.0) + col * sp;
    y = lo + row * sp * h3;
  };
  std::vector<long long> res((size_t)n);
  for (int k = 0; k < n; ++k) res[k] = k;
  for (long long k = n; k < nsites; ++k) {
    bdrng::U4 r = bdrng::draw((uint32_t)(k & 0xFFFFFFFF), (int64_t)(k >> 32), seed, 0, bdrng::TAG_LATTICE);
    const double u = ((double)r.x * 4294967296.0 + (double)r.y + 0.5) * (1.0 / 18446744073709551616.0);
    const long long j = std::min(k, (long long)(u * (double)(k + 1)));
    if (j < n) res[(size_t)j] = k;
  }
  std::sort(res.begin(), res.end());
  const double jr = 0.5 * (sp - dmin);
  // an (almost) unjittered triangular lattice has four sites on one circle
  // everywhere: too close to the lattice's packing limit for a start in
  // general position
  if (!(jr >= 1e-6 * dmin)) return -1;
  xy.assign(2 * (size_t)n, 0.0);
  for (int i = 0; i < n; ++i) {
    double x, y;
    site(res[i], x, y);
    bdrng::U4 r = bdrng::draw((uint32_t)(res[i] & 0xFFFFFFFF), (int64_t)(res[i] >> 32), seed, 1u,
                              bdrng::TAG_LATTICE);
    const double u0 = ((double)r.x + 0.5) * (1.0 / 4294967296.0), u1 = ((double)r.y + 0.5) * (1.0 / 4294967296.0);
    const double rad = jr * sqrt(u0), ang = 6.283185307179586 * u1;
    // an offset that would leave the box is mirrored (same length, so every
    // pair stays at least dmin apart and every site is jittered)
    double ox = rad * cos(ang), oy = rad * sin(ang);
    if (x + ox < lo || x + ox > hi) ox = -ox;
    if (y + oy < lo || y + oy > hi) oy = -oy;
    x += ox;
    y += oy;
    xy[2 * i] = x;
    xy[2 * i + 1] = y;
  }
  return 0;
}

// minimum pair distance check with a cell grid: returns 1 if some pair is
// closer than dmin (polydisperse: than rad_i + rad_j)
int any_overlap(int n, const double *xy, double lo, double hi, double dmin, const double *rad) {
  double W = hi - lo;
  int nc = std::max(1, std::min(4096, (int)floor(W / dmin)));
  double cs = W / nc;
  std::vector<int> cell, start, order;
  cell_sort(n, xy, lo, cs, nc, cell, start, order);
  for (int i = 0; i < n; ++i) {
    const int cx = cell[i] % nc, cy = cell[i] / nc;
    for (int gy = std::max(0, cy - 1); gy <= std::min(nc - 1, cy + 1); ++gy)
      for (int gx = std::max(0, cx - 1); gx <= std::min(nc - 1, cx + 1); ++gx) {
        const int c = gy * nc + gx;
        for (int k = start[c]; k < start[c + 1]; ++k) {
          const int j = order[k];
          if (j >= i) continue;
          const double dx = xy[2 * j] - xy[2 * i], dy = xy[2 * j + 1] - xy[2 * i + 1];
          if (too_close(dx * dx + dy * dy, dmin, rad, i, j)) return 1;
        }
      }
  }
  return 0;
}

}  // namespace bdhost
