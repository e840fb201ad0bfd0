"""Pins for the oracle's predicates and Delaunay triangulation (Sec. 4.1-4.3)."""
import math

import numpy as np
import pytest

from oracle import geometry
from paper_1703_02484_gb300 import workloads


def _tri_ids(names, tris):
    return {frozenset(names.index(v) for v in t) for t in tris}


def test_fig4_flip_predicate(golden):
    g = golden("fig4_predicate.json")
    for case in g["cases"]:
        assert geometry.flip_predicate(g["v1"], g["v2"], g["v3"], case["v4"]) == case["flip"]
    # the pairing as typeset rejects Fig. 4(b), so it cannot be the intended test
    assert geometry.flip_predicate_as_typeset(g["v1"], g["v2"], g["v3"], [2, 0]) is False


def test_flip_predicate_is_point_in_triangle():
    rng = np.random.default_rng(8)
    for _ in range(2000):
        v = rng.integers(-6, 7, size=(4, 2)).astype(float)
        if geometry.orient_frac(v[0], v[1], v[2]) == 0:
            continue
        o = [geometry.orient_frac(v[0], v[1], v[3]), geometry.orient_frac(v[1], v[2], v[3]),
             geometry.orient_frac(v[2], v[0], v[3])]
        inside = all(x >= 0 for x in o) or all(x <= 0 for x in o)
        assert geometry.flip_predicate(v[0], v[1], v[2], v[3]) == inside


def test_fig5_one_flip(golden):
    g = golden("fig5_one_flip.json")
    names = list(g["points"])
    P = np.array([g["points"][k] for k in names], dtype=float)
    assert geometry.delaunay_bruteforce(P) == _tri_ids(names, g["start_triangles"])
    P[names.index("b")] = g["b_moved"]
    assert geometry.delaunay_bruteforce(P) == _tri_ids(names, g["final_triangles"])
    # the moved point inverts triangle bcd of the start triangulation
    b, c, d = (P[names.index(k)] for k in "bcd")
    assert geometry.orient_frac(b, c, d) < 0
    # and the paper's first flip (ab <-> cd) is the one Eq. (predicate) selects:
    # edge (c, d) with opposite vertices a and b, b inside triangle (c, d, a)
    a = P[names.index("a")]
    assert geometry.flip_predicate(c, d, a, b)
    # the C builder agrees (inside a far corner square)
    sq = [[-100, -100], [100, -100], [100, 100], [-100, 100]]
    tris = geometry.delaunay_generic(P, sq)
    real = {frozenset(t) for t in tris.tolist() if max(t) < len(P)}
    assert real == _tri_ids(names, g["final_triangles"])


def test_fig6_two_flips(golden):
    g = golden("fig6_two_flips.json")
    names = list(g["points"])
    P = np.array([g["points"][k] for k in names], dtype=float)
    assert geometry.delaunay_bruteforce(P) == _tri_ids(names, g["start_triangles"])
    P[names.index("f")] = g["f_moved"]
    dt = _tri_ids(names, g["delaunay_after_move"])
    assert geometry.delaunay_bruteforce(P) == dt
    rep = [[names.index(v) for v in t] for t in g["repaired_triangles"]]
    rep = [t if geometry.orient_frac(*P[t]) > 0 else [t[0], t[2], t[1]] for t in rep]
    assert geometry.is_valid_triangulation(P, rep)
    bad = geometry.non_delaunay_edges(P, rep)
    assert [tuple(sorted(e)) for e in bad] == [(names.index("a"), names.index("f"))]
    # Eq. (predicate) alone does not pick the first flip of Fig. 6 (edge be,
    # opposite vertices f and c): f is not inside (b, e, c) -- the paper notes
    # this case is detected and the step reverted
    b, c, e, f = (P[names.index(k)] for k in "bcef")
    assert not geometry.flip_predicate(b, e, c, f)


def test_exact_predicates_vs_rationals():
    rng = np.random.default_rng(3)
    for _ in range(300):
        p = rng.uniform(-3, 3, size=(4, 2))
        # near-degenerate: put d almost on the circle / c almost on the line
        if rng.uniform() < 0.5:
            t = rng.uniform()
            p[2] = p[0] + t * (p[1] - p[0]) + rng.normal(size=2) * 1e-15
        assert geometry.orient(p[0], p[1], p[2]) == geometry.orient_frac(p[0], p[1], p[2])
        assert geometry.orient_exact_c(p[0], p[1], p[2]) == geometry.orient_frac(p[0], p[1], p[2])
        a, b, c = p[0], p[1], p[2]
        if geometry.orient_frac(a, b, c) < 0:
            b, c = c, b
        if geometry.orient_frac(a, b, c) == 0:
            continue
        # a point on the circumcircle, perturbed by an ulp or so
        ax, ay, bx, by, cx, cy = a[0], a[1], b[0], b[1], c[0], c[1]
        dd = 2 * (ax * (by - cy) + bx * (cy - ay) + cx * (ay - by))
        if abs(dd) < 1e-3:
            continue
        ux = ((ax * ax + ay * ay) * (by - cy) + (bx * bx + by * by) * (cy - ay) + (cx * cx + cy * cy) * (ay - by)) / dd
        uy = ((ax * ax + ay * ay) * (cx - bx) + (bx * bx + by * by) * (ax - cx) + (cx * cx + cy * cy) * (bx - ax)) / dd
        R = math.hypot(ax - ux, ay - uy)
        ang = rng.uniform(0, 2 * math.pi)
        d = np.array([ux + R * math.cos(ang), uy + R * math.sin(ang)])
        d = d + rng.integers(-2, 3, size=2) * np.spacing(d)
        want = geometry.incircle_frac(a, b, c, d)
        assert geometry.incircle(a, b, c, d) == want
        assert geometry.incircle_exact_c(a, b, c, d) == want


def test_delaunay_vs_bruteforce_tiny():
    rng = np.random.default_rng(5)
    sq = [[-60.0, -60.0], [80.0, -60.0], [80.0, 80.0], [-60.0, 80.0]]
    for trial in range(6):
        n = 14
        xy = rng.uniform(1, 19, size=(n, 2))
        tris = geometry.delaunay_generic(xy, sq)
        P = np.concatenate([xy, sq])
        assert geometry.canonical_triangles(tris) == geometry.delaunay_bruteforce(P)
        assert len(tris) == 2 * n + 2


def test_delaunay_with_ghost_ring_vs_bruteforce():
    # a small box: disks plus its ghost points, brute-forced over all points
    rng = np.random.default_rng(6)
    L = 7.0
    xy = rng.uniform(1, L - 1, size=(4, 2))
    tris = geometry.delaunay(xy, L)
    P = geometry.with_ghosts(xy, L)
    assert geometry.canonical_triangles(tris) == geometry.delaunay_bruteforce(P)
    assert len(tris) == 2 * len(P) - 6


def test_delaunay_vs_qhull_and_properties():
    from scipy.spatial import Delaunay
    cfg = workloads.CONFIGS["c5"]
    xy, _, _ = workloads.initial_state(cfg, n=3000)
    L = workloads.box_side(3000, cfg.rho)
    tris = geometry.delaunay(xy, L)
    P = geometry.with_ghosts(xy, L)
    assert np.array_equal(geometry.edges(tris), geometry.edges(Delaunay(P).simplices))
    assert geometry.general_position(P, tris)
    assert geometry.non_delaunay_edges(P, tris) == []
    V = len(P)
    assert len(tris) == 2 * V - 6
    assert len(geometry.edges(tris)) == 3 * V - 7


def test_box_side_formula():
    # Sec. 7: N = 10^4 ABP disks with sigma = 1 at rho = 0.7 in a box L = 105.9
    assert abs(workloads.box_side(10000, 0.7, a=0.5) - 105.9) < 0.05
