"""Pins for the overlap correction (Eq. (overlaps), Algorithm 2, Sec. 4.4)."""
import math

import numpy as np
from scipy.spatial import cKDTree

from oracle import geometry, overlap, step
from paper_1703_02484_gb300 import workloads


def test_two_disk_bounce():
    xy = np.array([[10.0, 10.0], [11.9, 10.0]])
    E = np.array([[0, 1]])
    new, pairs, capped, disp = overlap.correction_pass(xy, E, 2.0, 1.0, 50.0)
    # each disk moves by the full overlap sigma - r: separation 2 sigma - r
    assert math.isclose(new[1, 0] - new[0, 0], 2 * 2.0 - 1.9, rel_tol=1e-14)
    assert math.isclose(new[0, 0], 10.0 - 0.1, rel_tol=1e-14)
    assert len(pairs) == 1 and not capped.any()


def test_fig7_cap(golden):
    g = golden("fig7_overlap_cap.json")
    names = list(g["points"])
    P = np.array([g["points"][k] for k in names], dtype=float) + 10.0
    E = np.array([[i, j] for i in range(4) for j in range(i + 1, 4)])
    new, pairs, capped, disp = overlap.correction_pass(P, E, g["sigma"], 1.0, 100.0)
    C = names.index("C")
    # uncapped push on C from A and B is longer than sigma/4 ...
    assert np.hypot(*disp[C]) > g["sigma"] / 4
    # ... so C moves exactly sigma/4 along it
    mv = new[C] - P[C]
    assert math.isclose(np.hypot(*mv), g["sigma"] / 4, rel_tol=1e-14)
    assert abs(mv[0] * disp[C][1] - mv[1] * disp[C][0]) < 1e-14
    assert capped[C]
    assert np.array_equal(new[names.index("D")], P[names.index("D")])


def test_jacobi_sum_cancels_symmetric_pushes():
    xy = np.array([[10.0, 10.0], [11.8, 10.0], [13.6, 10.0]])
    E = np.array([[0, 1], [1, 2]])
    new, pairs, capped, disp = overlap.correction_pass(xy, E, 2.0, 1.0, 50.0)
    assert np.allclose(disp[1], 0.0, atol=1e-14) and np.allclose(new[1], xy[1], atol=1e-14)
    assert np.allclose(new[0], [9.8, 10.0]) and np.allclose(new[2], [13.8, 10.0])


def test_full_step_leaves_no_overlap_and_a_delaunay_triangulation():
    cfg = workloads.CONFIGS["c2"]
    n = 2000
    L = workloads.box_side(n, cfg.rho)
    xy = workloads.near_contact_state(n, L, 1.0, seed=3)
    _, sp, th = workloads.initial_state(cfg, n=n)
    p = step.Params(L=L, alpha=cfg.alpha, D=cfg.D, Dr=cfg.Dr, v0=cfg.v0, dt=cfg.dt, seed=1)
    r = step.step(xy, th, sp, 0, p)
    assert not r["rejected"]
    assert r["corr_iters"] >= 1 and r["overlap_pairs"] > 0
    assert len(cKDTree(r["xy"]).query_pairs(2.0 * (1 - 1e-12))) == 0
    # without correction the Euler-Maruyama positions overlap
    assert len(cKDTree(r["xy_em"]).query_pairs(2.0)) > 0
    P = geometry.with_ghosts(r["xy"], L)
    assert geometry.non_delaunay_edges(P, r["tris"]) == []
    assert np.all(r["xy"] >= 1.0) and np.all(r["xy"] <= L - 1.0)


def test_close_pairs_is_brute_force():
    rng = np.random.default_rng(11)
    xy = rng.uniform(0, 12, (300, 2))
    E = overlap.close_pairs(xy, 2.0)
    ref = {(i, j) for i in range(300) for j in range(i + 1, 300)
           if (xy[j, 0] - xy[i, 0]) ** 2 + (xy[j, 1] - xy[i, 1]) ** 2 < 4.0}
    assert {tuple(e) for e in E.tolist()} == ref


def test_allpairs_two_disk_bounce():
    # one overlapping pair: each disk moves by the full depth (final separation 2 sigma - r)
    xy = np.array([[10.0, 10.0], [11.5, 10.0]])
    out, it, tot, rej = overlap.correct_allpairs(xy, 40.0, 1.0)
    assert not rej and it == 1 and tot == 1
    assert np.allclose(out, [[9.5, 10.0], [12.0, 10.0]], atol=1e-15)


def test_allpairs_equals_delaunay_correction_when_overlaps_are_edges():
    # mild overlaps: every overlapping pair is a Delaunay edge (Gabriel), so
    # both neighbour sources give the same passes and the same result
    from paper_1703_02484_gb300 import workloads
    L = workloads.box_side(400, 0.3)
    xy = workloads.near_contact_state(400, L, 1.0, seed=5)
    rng = np.random.default_rng(6)
    xy = np.clip(xy + rng.normal(scale=0.01, size=xy.shape), 1.0, L - 1.0)
    a, it_a, tot_a, rej_a = overlap.correct_allpairs(xy, L, 1.0)
    b, _, it_b, tot_b, rej_b = overlap.correct(xy, L, 1.0)
    assert not rej_a and not rej_b and it_a >= 1
    assert it_a == it_b and tot_a == tot_b
    assert np.max(np.abs(a - b)) <= 1e-12
    assert len(overlap.close_pairs(a, 2.0 * (1 - 1e-12))) == 0
