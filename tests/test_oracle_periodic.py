"""Pins for the periodic box (Sec. 2.1: minimum image, re-entry at the
opposite side; Sec. 4.1: the triangulation lives on a flat torus).

Test configurations are RSA starts translated by a seeded offset modulo L, so
that disks, pairs and triangles straddle the box edges."""
import math

import numpy as np
import pytest
from scipy.spatial import Delaunay, cKDTree

from oracle import forces, geometry, overlap, periodic, verlet
from oracle import step as ostep
from paper_1703_02484_gb300 import workloads


def translated_start(n, rho, seed, near_contact=False):
    L = workloads.box_side(n, rho)
    if near_contact:
        xy = workloads.near_contact_state(n, L, 1.0, seed=seed, rho=rho)
    else:
        xy = workloads.initial_positions(n, L, 1.0, rho, seed=seed)
    off = np.random.default_rng(seed + 1000).uniform(0, L, 2)
    return periodic.wrap(xy + off, L), L


def incircle_frac_tiled(a, b, c, P):
    return [geometry.incircle_frac(a, b, c, p) for p in P]


def test_torus_triangulation_is_delaunay_by_brute_force():
    xy, L = translated_start(36, 0.3, seed=1)
    tri, sh = periodic.delaunay_torus(xy, L)
    assert periodic.is_torus_triangulation(tri, sh)
    tiled = np.concatenate([xy + L * s for s in periodic.SHIFTS], axis=0)
    corners = periodic.lifted(xy, tri, sh, L)
    for a, b, c in corners:
        assert geometry.orient_frac(a, b, c) > 0
        # no point of the 3 x 3 tiling strictly inside the circumcircle
        near = tiled[np.linalg.norm(tiled - (a + b + c) / 3.0, axis=1) < 0.6 * L]
        assert max(incircle_frac_tiled(a, b, c, near)) <= 0


def test_torus_triangulation_matches_qhull_of_the_tiling():
    xy, L = translated_start(400, 0.3, seed=2)
    tri, sh = periodic.delaunay_torus(xy, L)
    tiled = np.concatenate([xy + L * s for s in periodic.SHIFTS], axis=0)
    src = np.tile(np.arange(len(xy)), 9)
    shf = np.repeat(periodic.SHIFTS, len(xy), axis=0)
    q = Delaunay(tiled).simplices
    s_id, s_sh = src[q], shf[q]
    k0 = np.argmin(s_id, axis=1)
    keep = np.all(s_sh[np.arange(len(q)), k0] == 0, axis=1)
    ref = periodic.edge_keys(s_id[keep], s_sh[keep])
    assert np.array_equal(periodic.edge_keys(tri, sh), ref)


def test_torus_triangulation_follows_a_translation():
    # translating every disk by d (mod L) keeps the torus triangulation; an
    # edge's shift changes by the wraps of its ends: s' = s + k_w - k_u
    xy, L = translated_start(300, 0.3, seed=3)
    d = np.array([0.37 * L, 0.81 * L])
    moved = xy + d
    k = np.floor(moved / L).astype(np.int64)
    xy2 = moved - L * k
    K1 = periodic.edge_keys(*periodic.delaunay_torus(xy, L))
    K2 = periodic.edge_keys(*periodic.delaunay_torus(xy2, L))
    want = K1.copy()
    want[:, 2:4] = K1[:, 2:4] + k[K1[:, 1]] - k[K1[:, 0]]
    want = np.unique(want, axis=0)
    assert np.array_equal(want, K2)


def test_min_image_two_body_closed_form():
    L = 20.0
    xy = np.array([[0.4, 10.0], [19.1, 10.3]])   # 1.3 apart across x = 0 / L
    A = (0.7, 0.7, 0.7, 0.7)
    F = forces.long_range_numpy(xy, np.zeros(2, np.uint8), A, L=L)
    d = np.array([0.4 - (19.1 - 20.0), 10.0 - 10.3])   # r_0 - r_1 (nearest image)
    r = math.hypot(*d)
    assert np.allclose(F[0], 0.7 * d / r ** 3, rtol=1e-14)
    assert np.allclose(F[1], -F[0], rtol=1e-14)
    # the C loop agrees with the numpy sum
    assert np.allclose(forces.long_range(xy, np.zeros(2, np.uint8), A, L=L), F, rtol=1e-14)


def test_periodic_forces_translation_invariant_and_reciprocal():
    xy, L = translated_start(500, 0.3, seed=4)
    sp = (np.arange(500) % 2).astype(np.uint8)
    A = (0.05, 0.2, -0.1, 0.05)
    F = forces.long_range_numpy(xy, sp, A, L=L)
    xy2 = periodic.wrap(xy + np.array([0.5 * L + 0.123, 0.25 * L]), L)
    F2 = forces.long_range_numpy(xy2, sp, A, L=L)
    scale = np.sqrt(np.mean(np.sum(F ** 2, axis=1)))
    assert np.max(np.abs(F - F2)) <= 1e-11 * scale
    # a symmetric table: Newton's third law over minimum-image pairs
    Fs = forces.long_range(xy, sp, (0.1, 0.1, 0.1, 0.1), L=L)
    assert np.max(np.abs(Fs.sum(axis=0))) <= 1e-11 * np.abs(Fs).sum()
    # the short-range law too
    S1 = forces.short_range(xy, 1.0, 1.0, 2.0, 5.0, L=L)
    S2 = forces.short_range(xy2, 1.0, 1.0, 2.0, 5.0, L=L)
    assert np.max(np.abs(S1 - S2)) <= 1e-11 * np.sqrt(np.mean(np.sum(S1 ** 2, axis=1)))


def test_overlapping_pair_across_the_edge_bounces():
    # Eq. (overlaps): each disk of a pair at r < sigma moves by sigma - r along
    # the pair (final separation 2 sigma - r); the pair straddles x = 0 / L
    L = 30.0
    xy = np.array([[0.3, 15.0], [28.6, 15.0], [10.0, 5.0], [20.0, 25.0], [15.0, 15.0],
                   [5.0, 25.0], [25.0, 5.0], [8.0, 15.0], [22.0, 14.0]])
    r = 1.7
    out, tris, it, tot, rej = overlap.correct_periodic(xy, L, 1.0)
    assert not rej and it == 1 and tot == 1
    assert np.allclose(out[0], [0.3 + (2.0 - r), 15.0], atol=1e-12)
    assert np.allclose(out[1], [28.6 - (2.0 - r), 15.0], atol=1e-12)
    d = periodic.min_image(out[0] - out[1], L)
    assert math.isclose(float(np.hypot(*d)), 2 * 2.0 - r, rel_tol=1e-12)
    # a deeper overlap: the sigma/4 cap (Sec. 4.4) limits each move, and a
    # disk pushed across x = 0 re-enters at the right edge
    xy[0] = [0.2, 15.0]
    xy[1] = [29.0, 15.0]                  # r = 1.2
    out, tris, it, tot, rej = overlap.correct_periodic(xy, L, 1.0)
    assert not rej and it == 1
    assert np.allclose(out[1], [28.5, 15.0], atol=1e-12)
    assert np.allclose(out[0], [0.7, 15.0], atol=1e-12)
    xy[0] = [0.1, 15.0]
    xy[1] = [0.9, 15.0]                   # r = 0.8: disk 0 is pushed below x = 0
    out, tris, it, tot, rej = overlap.correct_periodic(xy, L, 1.0)
    assert not rej and it == 2           # r: 0.8 -> 1.8 (capped moves) -> 2 sigma - 1.8 = 2.2
    assert np.allclose(out[0], [29.4, 15.0], atol=1e-9)
    assert np.allclose(out[1], [1.6, 15.0], atol=1e-9)
    assert len(periodic.close_pairs(out, 2.0, L)) == 0


def test_periodic_step_leaves_no_overlap_and_a_torus_delaunay():
    xy, L = translated_start(600, 0.35, seed=6, near_contact=True)
    sp = (np.arange(600) % 2).astype(np.uint8)
    p = ostep.Params(L=L, law=ostep.LAW_LONG, alpha=(0.05, 0.2, -0.1, 0.05), D=1.0, Dr=0.5, v0=1.0,
                     dt=1e-4, seed=3, periodic=True)
    res = ostep.step(xy, np.zeros(600), sp, 0, p)
    assert not res["rejected"] and res["corr_iters"] >= 1
    out = res["xy"]
    assert np.all((out >= 0) & (out < L))
    assert len(periodic.close_pairs(out, 2.0, L)) == 0
    tree = cKDTree(out, boxsize=L)
    assert len(tree.query_pairs(2.0 * (1 - 1e-12))) == 0
    tri, sh = res["tris"]
    assert periodic.is_torus_triangulation(tri, sh)
    assert np.array_equal(periodic.edge_keys(tri, sh), periodic.edge_keys(*periodic.delaunay_torus(out, L)))


def test_periodic_verlet_lists_match_periodic_kdtree():
    xy, L = translated_start(3000, 0.5, seed=7)
    lists = verlet.build(xy, 5.0, 0.6, L=L)
    tree = cKDTree(xy, boxsize=L)
    for i in range(0, 3000, 7):
        ref = sorted(j for j in tree.query_ball_point(xy[i], 5.6 * (1 - 1e-12)) if j != i)
        assert lists[i].tolist() == ref


@pytest.mark.parametrize("seed", [8, 9])
def test_wrap_keeps_coordinates_in_the_box(seed):
    L = 17.3
    x = np.random.default_rng(seed).uniform(-3 * L, 4 * L, (1000, 2))
    w = periodic.wrap(x, L)
    assert np.all((w >= 0) & (w < L))
    assert np.allclose(periodic.min_image(w - x, L), 0.0, atol=1e-12)
