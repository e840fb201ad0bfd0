"""Pins for the oracle's polydisperse disks (Sec. 2.3: the method extends to
disks whose radii "do not differ too much").

Readings pinned here: a pair overlaps when closer than a_i + a_j; each disk
of an overlapping pair moves a_i + a_j - r (the bounce of Eq. (overlaps));
a disk's summed displacement is truncated at half its own radius (Sec. 4.4's
"sigma/4 (half the particle radius)"); centres reflect a_i from the walls;
the short-range law's length scale is a_i + a_j.

The Delaunay certificate: with a_max <= sqrt(2) a_min the overlapping pair
with the smallest centre distance is a Delaunay edge (a third disk k inside
the pair's diametral disk would be closer than r / sqrt(2) < sqrt(2) a_max
<= 2 a_min to one of them, an overlapping pair closer than the closest),
so no overlapping Delaunay edge means no overlap anywhere.  Pinned by brute
force on random sets, and by a configuration with a larger ratio where an
overlapping pair is not a Delaunay edge."""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

from oracle import dynamics, forces, geometry, overlap, periodic
from oracle import step as ostep
from paper_1703_02484_gb300 import workloads


def brute_overlaps(xy, radii):
    xy = np.asarray(xy)
    out = []
    for i, j in cKDTree(xy).query_pairs(2.0 * float(np.max(radii))):
        r = math.hypot(*(xy[j] - xy[i]))
        if r < radii[i] + radii[j]:
            out.append((r, min(i, j), max(i, j)))
    return sorted(out)


def test_two_disk_bounce_unequal_radii():
    # a = 1 and 1.3 at r = 2.2 (contact 2.3): each moves 0.1 apart (below its
    # cap), the new separation is 2 (a1 + a2) - r = 2.4
    xy = np.array([[10.0, 10.0], [12.2, 10.0]])
    radii = np.array([1.0, 1.3])
    new, pairs, capped, disp = overlap.correction_pass(xy, np.array([[0, 1]]), 2.6, 1.3, 30.0, radii)
    assert len(pairs) == 1 and not capped.any()
    assert np.allclose(new, [[9.9, 10.0], [12.3, 10.0]], atol=1e-14)
    assert math.isclose(new[1, 0] - new[0, 0], 2.4, rel_tol=1e-14)
    # touching pairs do not overlap
    xy = np.array([[10.0, 10.0], [12.3, 10.0]])
    _, pairs, _, _ = overlap.correction_pass(xy, np.array([[0, 1]]), 2.6, 1.3, 30.0, radii)
    assert len(pairs) == 0


def test_cap_is_half_the_own_radius():
    # a small disk (a = 0.75) pushed by two disks of radius 1 at distance 1.3,
    # 120 degrees apart (contact 1.75): two pushes of 0.45 add to 0.45,
    # truncated to 0.375 = 0.75 / 2; each large disk moves 0.45, below its cap
    # of 0.5, and the large disks (2.25 apart) do not overlap each other
    c = np.array([10.0, 10.0])
    u = np.array([math.cos(2 * math.pi / 3), math.sin(2 * math.pi / 3)])
    xy = np.array([c, c + [1.3, 0.0], c + 1.3 * u])
    radii = np.array([0.75, 1.0, 1.0])
    E = np.array([[0, 1], [0, 2], [1, 2]])
    new, pairs, capped, disp = overlap.correction_pass(xy, E, 2.0, 1.0, 30.0, radii)
    assert len(pairs) == 2 and capped.tolist() == [True, False, False]
    assert math.isclose(float(np.hypot(*disp[0])), 0.45, rel_tol=1e-13)
    assert math.isclose(float(np.hypot(*(new[0] - xy[0]))), 0.375, rel_tol=1e-13)
    assert math.isclose(float(np.hypot(*(new[1] - xy[1]))), 0.45, rel_tol=1e-13)


def test_walls_reflect_at_own_radius():
    xy = np.array([[0.5, 5.0], [5.0, 19.7]])
    out = dynamics.reflect(xy, np.array([0.8, 0.5]), 20.0)
    assert np.allclose(out, [[1.1, 5.0], [5.0, 19.3]], atol=1e-14)


def test_short_range_law_mixes_radii():
    # a_i = 1, a_j = 1.5: length scale 2.5; at contact, eps = kappa = 1:
    # WCA 24/2.5 = 9.6, Yukawa -2.5 (1/6.25 + 1/2.5) = -1.4, together 8.2
    xy = np.array([[5.0, 5.0], [7.5, 5.0]])
    f = forces.short_range_pairs(xy, np.array([1]), np.array([0]), 1.0, 1.0, 2.0, 5.0,
                                 radii=np.array([1.0, 1.5]))
    assert math.isclose(float(f[1, 0]), 8.2, rel_tol=1e-13)


@pytest.mark.parametrize("seed", range(6))
def test_closest_overlapping_pair_is_a_delaunay_edge(seed):
    # radii ratio up to sqrt(2); near-contact start, then noise moves that
    # create deep overlaps
    n = 600
    radii = workloads.poly_radii(n, 1.0, math.sqrt(2.0), seed)
    L = workloads.box_side(n, 0.3)
    xy = workloads.poly_positions(radii, L, seed, near_frac=0.4)
    rng = np.random.default_rng(seed)
    for scale in (0.05, 0.15, 0.3):
        moved = dynamics.reflect(xy + rng.normal(scale=scale, size=xy.shape), radii, L)
        ov = brute_overlaps(moved, radii)
        if not ov:
            continue
        _, i, j = ov[0]
        E = {tuple(sorted(e)) for e in geometry.edges(geometry.delaunay(moved, L, 1.0)).tolist()}
        assert (i, j) in E


def test_certificate_needs_the_radius_bound():
    # large disks i, j (a = 1) overlapping at r = 1.95; small disks k, k'
    # (a = 0.3) inside their diametral disk on either side, touching neither:
    # the Delaunay triangulation takes the diagonal kk', so the overlapping
    # pair is not an edge and a Delaunay-edge correction misses it
    c = np.array([15.0, 15.0])
    h = 0.95
    xy = np.array([c + [-0.975, 0.0], c + [0.975, 0.0], c + [0.0, h], c + [0.0, -h]])
    radii = np.array([1.0, 1.0, 0.3, 0.3])
    ov = brute_overlaps(xy, radii)
    assert len(ov) == 1 and ov[0][1:] == (0, 1) and math.isclose(ov[0][0], 1.95, rel_tol=1e-14)
    E = {tuple(sorted(e)) for e in geometry.edges(geometry.delaunay(xy, 30.0, 1.0)).tolist()}
    assert (0, 1) not in E and (2, 3) in E
    out, _, it, _, rej = overlap.correct(xy, 30.0, 1.0, radii=radii)
    assert it == 0 and rej == 0 and len(brute_overlaps(out, radii)) == 1


@pytest.mark.parametrize("law,pairs_from", [(ostep.LAW_LONG, "delaunay"), (ostep.LAW_SHORT, "delaunay"),
                                            (ostep.LAW_SHORT, "allpairs")])
def test_polydisperse_step_leaves_no_overlap(law, pairs_from):
    n = 1500
    radii = workloads.poly_radii(n, 1.0, 1.35, 7)
    L = workloads.box_side(n, 0.3)
    xy = workloads.poly_positions(radii, L, 7, near_frac=0.3)
    sp = (np.arange(n) % 2).astype(np.uint8)
    th = np.zeros(n)
    p = ostep.Params(L=L, a=1.0, law=law, alpha=(0.05, 0.2, -0.1, 0.05), D=1.0, v0=1.0, dt=1e-3, seed=3,
                     radii=radii)
    r = ostep.step(xy, th, sp, 0, p, pairs_from=pairs_from)
    assert not r["rejected"] and r["corr_iters"] >= 1
    assert brute_overlaps(r["xy"], radii) == []
    assert np.all(r["xy"] >= radii[:, None] - 1e-12) and np.all(r["xy"] <= L - radii[:, None] + 1e-12)
    if pairs_from == "delaunay":
        assert np.array_equal(geometry.edges(r["tris"]), geometry.edges(geometry.delaunay(r["xy"], L, 1.0)))


def test_polydisperse_periodic_step_leaves_no_overlap():
    n = 800
    radii = workloads.poly_radii(n, 1.0, 1.3, 9)
    L = workloads.box_side(n, 0.3)
    xy = workloads.poly_positions(radii, L, 9, near_frac=0.3)
    p = ostep.Params(L=L, a=1.0, law=ostep.LAW_NONE, D=1.0, dt=1e-3, seed=5, periodic=True, radii=radii)
    r = ostep.step(xy, np.zeros(n), np.zeros(n, np.uint8), 0, p)
    assert not r["rejected"] and r["corr_iters"] >= 1
    assert len(periodic.close_pairs(r["xy"], 2.0, L, radii=radii)) == 0
    # the same positions do overlap under the largest radius: the test is not vacuous
    assert len(periodic.close_pairs(r["xy"], 2.0, L)) > 0
