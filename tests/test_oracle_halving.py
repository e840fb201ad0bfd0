"""Pins for repeating a rejected move with a lower dt (Sec. 4.3).

Sec. 4.3 rejects a move in which two disks passed through each other
(r0_ij . r1_ij < 0 on a triangulation edge) and integrates again with a lower
dt.  The oracle halves the rejected move (oracle.step, Params.max_halvings).
The pins use a pair that only attracts itself, so the criterion can be worked
out by hand: two disks at distance r that pull each other with A/r^2 close by
2 dt_p A / r^2 in a move of length dt_p, so they pass through each other iff
2 dt_p A / r^2 > r (the noise, ~1e-2, is far from the margins used here)."""
import math

import numpy as np

from oracle import dynamics, noise, overlap, philox
from oracle import step as ostep
from paper_1703_02484_gb300 import workloads

VC = noise.clamped_normal_variance()


def attracting_pair_case(n=300, rho=0.3, seed=5, depth_ok=2):
    """n disks by random sequential addition; the two closest disks form
    species 1 and attract each other with A11 = -K, every other coefficient
    is zero.  K is chosen so that moves of length dt / 2^(depth_ok - 1) make
    the pair pass through each other and moves of dt / 2^depth_ok do not:
    dt K = 1.5 * 2^(depth_ok - 2) r^3."""
    L = workloads.box_side(n, rho)
    xy = workloads.initial_positions(n, L, 1.0, rho, seed=seed)
    d = np.linalg.norm(xy[:, None, :] - xy[None, :, :], axis=2)
    np.fill_diagonal(d, np.inf)
    i, j = np.unravel_index(np.argmin(d), d.shape)
    r = float(d[i, j])
    sp = np.zeros(n, dtype=np.uint8)
    sp[[i, j]] = 1
    dt = 1e-4
    K = 1.5 * 2.0 ** (depth_ok - 2) * r ** 3 / dt
    p = ostep.Params(L=L, a=1.0, law=ostep.LAW_LONG, alpha=(0.0, 0.0, 0.0, -K), D=1.0, Dr=0.0,
                     v0=0.0, dt=dt, seed=17)
    return xy, sp, np.zeros(n), (int(i), int(j)), r, p


def test_whole_step_keeps_its_noise_stream():
    # piece 1 (the whole step) draws the stream of an ordinary step
    assert philox.substep_tag(1) == philox.TAG_NOISE == 0
    ids = np.arange(64)
    a = noise.normals(ids, 7, 3)
    b = noise.normals(ids, 7, 3, tag=philox.substep_tag(1))
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    # halves draw other numbers
    c = noise.normals(ids, 7, 3, tag=philox.substep_tag(2))
    assert not np.array_equal(a[0], c[0])


def test_halves_add_up_to_the_variance_of_a_whole_move():
    # Brownian increments over dt/2 + dt/2 have the variance of one over dt:
    # each half's amplitude is sqrt(2 D dt / 2) per component (clamped normals)
    n, D, dt, L = 200000, 1.0, 1e-4, 1e7
    ids = np.arange(n)
    xy = np.full((n, 2), L / 2)
    F = np.zeros((n, 2))
    th = np.zeros(n)
    y1, _ = dynamics.em_move(xy, th, F, ids, 0, 11, D, 0.0, 0.0, dt / 2, tag=philox.substep_tag(2))
    y2, _ = dynamics.em_move(y1, th, F, ids, 0, 11, D, 0.0, 0.0, dt / 2, tag=philox.substep_tag(3))
    d = y2 - xy
    var = d.var(axis=0)
    want = 2 * D * dt * VC
    se = want * math.sqrt(2.0 / n)
    assert np.all(np.abs(var - want) < 5 * se), (var, want)
    # the two halves' normals are uncorrelated with each other and with the whole step's
    a = noise.normals(ids, 0, 11, tag=philox.substep_tag(2))[0]
    b = noise.normals(ids, 0, 11, tag=philox.substep_tag(3))[0]
    c = noise.normals(ids, 0, 11, tag=philox.substep_tag(1))[0]
    assert abs(np.corrcoef(a, b)[0, 1]) < 5 / math.sqrt(n)
    assert abs(np.corrcoef(a, c)[0, 1]) < 5 / math.sqrt(n)


def test_pass_through_rejected_without_halving():
    xy, sp, th, (i, j), r, p = attracting_pair_case()
    res = ostep.step(xy, th, sp, 0, p)
    assert res["rejected"] == overlap.REJ_REVERSAL
    assert np.array_equal(res["xy"], xy)
    assert res["substeps"] == 0 and res["halvings"] == 0


def test_halving_depth_follows_the_reversal_criterion():
    xy, sp, th, (i, j), r, p = attracting_pair_case(depth_ok=2)
    # moves of dt/2 still let the pair pass through each other: one halving is not enough
    p.max_halvings = 1
    res = ostep.step(xy, th, sp, 0, p)
    assert res["rejected"] == overlap.REJ_REVERSAL and np.array_equal(res["xy"], xy)
    # moves of dt/4 do not: two halvings complete the step
    p.max_halvings = 2
    res = ostep.step(xy, th, sp, 0, p)
    assert not res["rejected"]
    assert res["halvings"] >= 2 and res["substeps"] >= 3
    out = res["xy"]
    # the pair kept its order along the axis joining it (no pass-through)
    r0 = xy[j] - xy[i]
    r1 = out[j] - out[i]
    assert float(r0 @ r1) > 0
    # no two disks overlap after the step, and the pair did approach
    assert len(overlap.close_pairs(out, 2.0)) == 0
    assert np.linalg.norm(r1) < r + 1.0
    # deeper limits change nothing once depth 2 suffices
    p.max_halvings = 5
    res5 = ostep.step(xy, th, sp, 0, p)
    assert np.array_equal(res5["xy"], out) and res5["substeps"] == res["substeps"]


def test_deeper_case_needs_deeper_halving():
    # K doubled: moves of dt/4 pass through, dt/8 do not
    xy, sp, th, _, r, p = attracting_pair_case(depth_ok=3)
    p.max_halvings = 2
    assert ostep.step(xy, th, sp, 0, p)["rejected"] == overlap.REJ_REVERSAL
    p.max_halvings = 3
    res = ostep.step(xy, th, sp, 0, p)
    assert not res["rejected"] and res["halvings"] >= 3
    assert len(overlap.close_pairs(res["xy"], 2.0)) == 0
