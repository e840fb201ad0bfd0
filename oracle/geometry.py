"""Triangulation geometry -- oracle (test infrastructure).

* Exact orientation and in-circle signs: small cases in Python rationals
  (`fractions.Fraction`, exact by construction), bulk work in the oracle's C
  expansion arithmetic (oracle/csrc).
* The Delaunay triangulation (Sec. 4.1) of the disk centres together with
  fixed ghost points outside the box.  The paper's box is periodic and its
  triangulation lives on a torus; with reflecting walls the hull is closed
  with four far corners and a ring of points just outside the walls
  (layout in `ghost_points`).  Any pair of disks closer than sigma is a
  Delaunay edge of this point set (its diametral circle lies at y, x >= 0 and
  holds no other point), so the overlap search over triangulation edges still
  finds every overlap.
* A brute-force Delaunay (every empty-circumcircle triangle, O(n^4)) for tiny
  inputs, which pins the builder.
* The inverted-triangle flip predicate of Sec. 4.3, Eq. (predicate).
"""
import ctypes
import math
from fractions import Fraction

import numpy as np

from . import _clib


# ---------------------------------------------------------------- predicates

def orient_frac(a, b, c):
    """sign((b - a) x (c - a)) in exact rationals; > 0 iff a, b, c turn left."""
    ax, ay, bx, by, cx, cy = (Fraction(float(v)) for v in (*a, *b, *c))
    d = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax)
    return (d > 0) - (d < 0)


def incircle_frac(a, b, c, d):
    """> 0 iff d lies strictly inside the circle through a, b, c (a, b, c
    counter-clockwise), exact rationals."""
    ax, ay, bx, by, cx, cy, dx, dy = (Fraction(float(v)) for v in (*a, *b, *c, *d))
    m = [[ax - dx, ay - dy], [bx - dx, by - dy], [cx - dx, cy - dy]]
    lift = [u * u + v * v for u, v in m]
    det = (lift[0] * (m[1][0] * m[2][1] - m[1][1] * m[2][0])
           - lift[1] * (m[0][0] * m[2][1] - m[0][1] * m[2][0])
           + lift[2] * (m[0][0] * m[1][1] - m[0][1] * m[1][0]))
    return (det > 0) - (det < 0)


def orient(a, b, c):
    return _clib.lib().oracle_orient2d(float(a[0]), float(a[1]), float(b[0]), float(b[1]),
                                       float(c[0]), float(c[1]))


def incircle(a, b, c, d):
    return _clib.lib().oracle_incircle(float(a[0]), float(a[1]), float(b[0]), float(b[1]),
                                       float(c[0]), float(c[1]), float(d[0]), float(d[1]))


def orient_exact_c(a, b, c):
    return _clib.lib().oracle_orient2d_exact(*(float(v) for v in (*a, *b, *c)))


def incircle_exact_c(a, b, c, d):
    return _clib.lib().oracle_incircle_exact(*(float(v) for v in (*a, *b, *c, *d)))


# ------------------------------------------------------------- ghost points

def ghost_points(L, a=1.0):
    """Fixed points closing the triangulation, in this order: the far corners
    (-F,-F), (G,-F), (G,G), (-F,G) with F = C + 3W, G = 2C + 3W; then the
    bottom row (side 0) at y = -W - off(k, 4) and the top row (side 1) at
    y = C + W + off(k, 5), x = -W + k S + off(k, side); then the left column
    (side 2) at x = -W - off(k, 6) and the right column (side 3) at
    x = C + W + off(k, 7), y = -W + S/2 + k S + off(k, side); C = ceil(L),
    W = S = ceil(2a), off(k, s) = ((7919 k + 104729 s) mod 257) / 1024."""
    C = float(math.ceil(L))
    W = float(math.ceil(2.0 * a))
    S = W
    F, G = C + 3 * W, 2 * C + 3 * W
    pts = [(-F, -F), (G, -F), (G, G), (-F, G)]

    def off(k, s):
        return ((7919 * k + 104729 * s) % 257) / 1024.0

    for side in (0, 1):
        k = 0
        while -W + k * S <= C + W:
            y = -W - off(k, 4 + side) if side == 0 else C + W + off(k, 4 + side)
            pts.append((-W + k * S + off(k, side), y))
            k += 1
    for side in (2, 3):
        k = 0
        while -W + 0.5 * S + k * S < C + W:
            x = -W - off(k, 4 + side) if side == 2 else C + W + off(k, 4 + side)
            pts.append((x, -W + 0.5 * S + k * S + off(k, side)))
            k += 1
    return np.array(pts, dtype=np.float64)


def with_ghosts(xy, L, a=1.0):
    return np.concatenate([np.asarray(xy, dtype=np.float64), ghost_points(L, a)], axis=0)


def _insertion_order(xy):
    """Serpentine sweep over a coarse grid: any order gives the same
    triangulation; this one keeps the point-location walks short."""
    n = len(xy)
    if n == 0:
        return np.zeros(0, dtype=np.int32)
    k = max(1, int(math.sqrt(n / 4.0)))
    lo = xy.min(axis=0)
    span = np.maximum(xy.max(axis=0) - lo, 1e-300)
    gx = np.minimum((xy[:, 0] - lo[0]) / span[0] * k, k - 1).astype(np.int64)
    gy = np.minimum((xy[:, 1] - lo[1]) / span[1] * k, k - 1).astype(np.int64)
    xkey = np.where(gy % 2 == 0, xy[:, 0], -xy[:, 0])
    return np.lexsort((xkey, gy)).astype(np.int32)


def delaunay(xy, L, a=1.0):
    """Triangles (T, 3) of the Delaunay triangulation of the disks plus the
    ghost points, counter-clockwise; ghost ids follow the disks (n + k for the
    k-th point of ghost_points)."""
    xy = np.asarray(xy, dtype=np.float64)
    n = len(xy)
    g = ghost_points(L, a)
    ring = g[4:]
    R = len(ring)
    # the C builder wants the enclosing square last; it triangulates
    # [disks, ring] inside it
    pts = np.concatenate([xy, ring, g[:4]], axis=0)
    x = np.ascontiguousarray(pts[:, 0])
    y = np.ascontiguousarray(pts[:, 1])
    order = np.ascontiguousarray(np.concatenate([np.arange(n, n + R, dtype=np.int32),
                                                 _insertion_order(xy)]))
    m = n + R
    out = np.zeros(3 * (2 * m + 8), dtype=np.int32)
    p = lambda arr: arr.ctypes.data_as(ctypes.c_void_p)
    nt = _clib.lib().oracle_delaunay(m, p(x), p(y), p(order), p(out))
    if nt < 0:
        raise ValueError("oracle_delaunay failed with code %d" % nt)
    tris = out[: 3 * nt].reshape(nt, 3).copy()
    # builder ids: disks 0..n-1, ring n..n+R-1, corners m..m+3 -> canonical
    remap = np.concatenate([np.arange(n), n + 4 + np.arange(R), n + np.arange(4)]).astype(np.int32)
    return remap[tris]


def delaunay_generic(points, corner_square):
    """Delaunay triangulation of arbitrary points inside a given enclosing
    counter-clockwise square of 4 corners (ids n..n+3)."""
    pts = np.concatenate([np.asarray(points, float), np.asarray(corner_square, float)], axis=0)
    n = len(points)
    x = np.ascontiguousarray(pts[:, 0])
    y = np.ascontiguousarray(pts[:, 1])
    order = np.ascontiguousarray(np.arange(n, dtype=np.int32))
    out = np.zeros(3 * (2 * n + 8), dtype=np.int32)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    nt = _clib.lib().oracle_delaunay(n, p(x), p(y), p(order), p(out))
    if nt < 0:
        raise ValueError("oracle_delaunay failed with code %d" % nt)
    return out[: 3 * nt].reshape(nt, 3).copy()


def edges(tris):
    """Sorted unique undirected edges (E, 2), i < j."""
    t = np.asarray(tris, dtype=np.int64)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]], axis=0)
    e = np.sort(e, axis=1)
    e = np.unique(e, axis=0)
    return e


def canonical_triangles(tris):
    """Triangles as a set of frozensets (orientation-free comparison)."""
    return {frozenset(int(v) for v in t) for t in np.asarray(tris)}


def delaunay_bruteforce(points):
    """Every triangle whose circumcircle contains no other point strictly
    inside (exact rationals).  O(n^4); for tiny inputs in general position."""
    pts = [tuple(map(float, p)) for p in points]
    n = len(pts)
    out = set()
    for i in range(n):
        for j in range(i + 1, n):
            for k in range(j + 1, n):
                o = orient_frac(pts[i], pts[j], pts[k])
                if o == 0:
                    continue
                a, b, c = (i, j, k) if o > 0 else (i, k, j)
                if all(incircle_frac(pts[a], pts[b], pts[c], pts[m]) <= 0
                       for m in range(n) if m not in (i, j, k)):
                    out.add(frozenset((i, j, k)))
    return out


def is_valid_triangulation(points, tris):
    """Every triangle strictly counter-clockwise and the triangles' areas sum
    to the hull area (no overlaps, no holes) -- exact signs, area in FP64."""
    P = np.asarray(points, float)
    for t in tris:
        if orient(P[t[0]], P[t[1]], P[t[2]]) <= 0:
            return False
    area = 0.0
    for t in tris:
        a, b, c = P[t[0]], P[t[1]], P[t[2]]
        area += 0.5 * ((b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0]))
    from scipy.spatial import ConvexHull  # hull area only
    hull = ConvexHull(P)
    return abs(area - hull.volume) <= 1e-9 * hull.volume


def non_delaunay_edges(points, tris):
    """Interior edges whose opposite vertex lies strictly inside the
    neighbour's circumcircle (exact)."""
    P = np.asarray(points, float)
    opp = {}
    for t in tris:
        t = [int(v) for v in t]
        for k in range(3):
            u, v, w = t[(k + 1) % 3], t[(k + 2) % 3], t[k]
            opp[(u, v)] = (w, t)
    bad = []
    for (u, v), (w, t) in opp.items():
        if (v, u) in opp and u < v:
            q = opp[(v, u)][0]
            if incircle(P[t[0]], P[t[1]], P[t[2]], P[q]) > 0:
                bad.append((u, v))
    return bad


def general_position(points, tris):
    """True if no triangulation edge has its four quad vertices cocircular."""
    P = np.asarray(points, float)
    opp = {}
    for t in tris:
        t = [int(v) for v in t]
        for k in range(3):
            opp[(t[(k + 1) % 3], t[(k + 2) % 3])] = (t[k], t)
    for (u, v), (w, t) in opp.items():
        if (v, u) in opp and u < v:
            q = opp[(v, u)][0]
            if incircle(P[t[0]], P[t[1]], P[t[2]], P[q]) == 0:
                return False
    return True


# ------------------------------------------------- Eq. (predicate), Sec. 4.3

def _cross(u, v):
    return u[0] * v[1] - u[1] * v[0]


def flip_predicate(v1, v2, v3, v4):
    """Sec. 4.3, Eq. (predicate): should edge (v1, v2), with opposite
    vertices v3 and v4, be flipped to (v3, v4)?  True iff v4 lies in the
    triangle (v1, v2, v3).  Barycentric form with e0 = v2 - v1, e1 = v3 - v1,
    e2 = v4 - v1, d = e1 x e0, s = e1 x e2, t = e2 x e0 (so v4 = v1 +
    (s/d) e0 + (t/d) e1):
      d <  0:  s <= 0, t <= 0, s + t >= d
      d >= 0:  s >= 0, t >= 0, s + t <= d
    The typeset d2, s2, t2 pair the vectors differently and reject the
    inverted configuration of Fig. 4(b); this is the reading that accepts it.
    Evaluated in exact rationals."""
    v1, v2, v3, v4 = ([Fraction(float(c)) for c in v] for v in (v1, v2, v3, v4))
    e0 = (v2[0] - v1[0], v2[1] - v1[1])
    e1 = (v3[0] - v1[0], v3[1] - v1[1])
    e2 = (v4[0] - v1[0], v4[1] - v1[1])
    d = _cross(e1, e0)
    s = _cross(e1, e2)
    t = _cross(e2, e0)
    if d < 0:
        return s <= 0 and t <= 0 and s + t >= d
    return s >= 0 and t >= 0 and s + t <= d


def flip_predicate_as_typeset(v1, v2, v3, v4):
    """Eq. (predicate) with d2 = e2 x e0, s2 = e1 x e0, t2 = e2 x e1 exactly
    as printed (kept to document that the printed pairing is garbled)."""
    v1, v2, v3, v4 = ([Fraction(float(c)) for c in v] for v in (v1, v2, v3, v4))
    e0 = (v2[0] - v1[0], v2[1] - v1[1])
    e1 = (v3[0] - v1[0], v3[1] - v1[1])
    e2 = (v4[0] - v1[0], v4[1] - v1[1])
    d = _cross(e2, e0)
    s = _cross(e1, e0)
    t = _cross(e2, e1)
    if d < 0:
        return s <= 0 and t <= 0 and s + t >= d
    return s >= 0 and t >= 0 and s + t <= d
