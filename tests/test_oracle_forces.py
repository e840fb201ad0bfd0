"""Pins for the oracle's pair forces (Sec. 2.2 and the short-range law)."""
import math

import numpy as np
import pytest

from oracle import forces

A2 = (0.05, 0.2, -0.1, 0.05)    # on A from A, on A from B, on B from A, on B from B


def test_two_body_closed_form_and_index_order():
    # disk 0 (species A) at origin, disk 1 (species B) at (3, 4): r = 5
    xy = np.array([[0.0, 0.0], [3.0, 4.0]])
    s = np.array([0, 1], dtype=np.uint8)
    F = forces.long_range_numpy(xy, s, A2)
    # force on 0 from 1: A[A][B] * (r0 - r1)/r^3 = 0.2 * (-3,-4)/125
    assert np.allclose(F[0], 0.2 * np.array([-3.0, -4.0]) / 125.0, rtol=1e-15, atol=0)
    # force on 1 from 0: A[B][A] * (r1 - r0)/r^3 = -0.1 * (3,4)/125 (attractive)
    assert np.allclose(F[1], -0.1 * np.array([3.0, 4.0]) / 125.0, rtol=1e-15, atol=0)
    # magnitude alpha / r^2
    assert math.isclose(np.hypot(*F[0]), 0.2 / 25.0, rel_tol=1e-14)


def test_c_and_numpy_paths_and_newton3_for_reciprocal_law():
    rng = np.random.default_rng(2)
    n = 700
    xy = rng.uniform(0, 60, size=(n, 2))
    s = rng.integers(0, 2, n).astype(np.uint8)
    A = (0.1, 0.03, 0.03, -0.07)   # symmetric table = reciprocal pair law
    F1 = forces.long_range_numpy(xy, s, A)
    F2 = forces.long_range(xy, s, A, threads=2)
    assert np.allclose(F1, F2, rtol=1e-12, atol=1e-15)
    tot = F1.sum(axis=0)
    assert np.all(np.abs(tot) <= 1e-12 * np.abs(F1).sum())


def test_symmetric_ring_cancels():
    k = 12
    ang = 2 * math.pi * np.arange(k) / k
    ring = np.stack([5 * np.cos(ang), 5 * np.sin(ang)], axis=1)
    xy = np.concatenate([[[0.0, 0.0]], ring])
    s = np.zeros(k + 1, dtype=np.uint8)
    F = forces.long_range_numpy(xy, s, (1.0, 0, 0, 0))
    assert np.all(np.abs(F[0]) < 1e-15)
    # every ring disk is pushed radially outward
    radial = (F[1:] * ring).sum(axis=1) / 5.0
    tang = np.abs(F[1:, 0] * ring[:, 1] - F[1:, 1] * ring[:, 0]) / 5.0
    assert np.all(radial > 0) and np.all(tang < 1e-14)


def test_nonreciprocal_pair_self_propels():
    # Sec. 2.2: with alpha != mu action and reaction differ; a lone A-B pair
    # with A[A][B] = -A[B][A] moves as a unit (net force nonzero)
    xy = np.array([[0.0, 0.0], [2.5, 0.0]])
    s = np.array([0, 1], dtype=np.uint8)
    F = forces.long_range_numpy(xy, s, (0.0, 0.3, -0.3, 0.0))
    assert np.allclose(F[0], F[1])
    assert abs(F.sum(axis=0)[0]) > 0.09


@pytest.mark.parametrize("r", [2.0, 2.1, 2.2, 2.4, 3.0, 4.5])
def test_short_range_force_is_minus_potential_gradient(r):
    h = 1e-6
    dU = (forces.short_range_potential(r + h, 1.0, 1.0, 2.0)
          - forces.short_range_potential(r - h, 1.0, 1.0, 2.0)) / (2 * h)
    assert abs(float(forces.short_range_magnitude(r, 1.0, 1.0, 2.0)) + float(dU)) < 1e-6


def test_short_range_cutoff_and_newton3():
    rng = np.random.default_rng(4)
    xy = rng.uniform(0, 30, size=(300, 2))
    F = forces.short_range(xy, 1.0, 1.0, 2.0, 5.0)
    assert np.all(np.abs(F.sum(axis=0)) < 1e-9 * np.abs(F).sum())
    two = np.array([[0.0, 0.0], [5.0 + 1e-9, 0.0]])
    assert np.all(forces.short_range(two, 1.0, 1.0, 2.0, 5.0) == 0.0)
    two = np.array([[0.0, 0.0], [4.9, 0.0]])
    f = forces.short_range(two, 1.0, 1.0, 2.0, 5.0)
    # Yukawa tail attracts: force on 0 points toward +x
    assert f[0, 0] > 0 and f[1, 0] < 0


def test_more_species_two_body_and_relabelling():
    # Sec. 2.2's force mu_i alpha_k f(r_i - r_k) allows any number of species;
    # the oracle takes an n x n table A[s_i][s_k]
    rng = np.random.default_rng(4)
    A3 = rng.normal(size=(3, 3))
    xy = np.array([[1.0, 2.0], [4.0, 6.0]])          # 5 apart
    F = forces.long_range_numpy(xy, np.array([0, 2], np.uint8), A3.reshape(-1))
    d = xy[0] - xy[1]
    assert np.allclose(F[0], A3[0, 2] * d / 125.0, rtol=1e-14)
    assert np.allclose(F[1], -A3[2, 0] * d / 125.0, rtol=1e-14)
    # a third species that copies species 0's rows and columns changes nothing
    A2 = rng.normal(size=(2, 2))
    A3 = np.zeros((3, 3))
    A3[:2, :2] = A2
    A3[2, :2] = A2[0]
    A3[:2, 2] = A2[:, 0]
    A3[2, 2] = A2[0, 0]
    n = 300
    xy = rng.uniform(0, 60, (n, 2))
    s2 = rng.integers(0, 2, n).astype(np.uint8)
    s3 = s2.copy()
    s3[(s2 == 0) & (rng.random(n) < 0.5)] = 2
    F2 = forces.long_range_numpy(xy, s2, A2.reshape(-1))
    F3 = forces.long_range_numpy(xy, s3, A3.reshape(-1))
    assert np.max(np.abs(F2 - F3)) <= 1e-12 * np.max(np.abs(F2))
    # the C loop takes the same table
    F3c = forces.long_range(xy, s3, A3.reshape(-1))
    assert np.max(np.abs(F3c - F3)) <= 1e-12 * np.max(np.abs(F3))


def test_factorised_table_matches_charges():
    # A[s_i][s_k] = mu_{s_i} alpha_{s_k} (Sec. 2.2): F_i = mu_i sum_k alpha_k r_ik / r^3
    rng = np.random.default_rng(5)
    mu, al = rng.normal(size=4), rng.normal(size=4)
    n = 200
    xy = rng.uniform(0, 50, (n, 2))
    s = rng.integers(0, 4, n).astype(np.uint8)
    F = forces.long_range_numpy(xy, s, np.outer(mu, al).reshape(-1))
    d = xy[:, None, :] - xy[None, :, :]
    r = np.linalg.norm(d, axis=2)
    np.fill_diagonal(r, np.inf)
    ref = mu[s][:, None] * np.einsum("k,ikc->ic", al[s], d / r[:, :, None] ** 3)
    assert np.allclose(F, ref, rtol=1e-11, atol=1e-14)


# Literal values of the short-range law (WCA core 4 eps[(s/r)^12 - (s/r)^6] + eps
# below 2^(1/6) s, Yukawa tail -eps (s/r) exp(-kappa (r - s)), s = 2a), worked
# by hand.  Each catches one plausible slip: a wrong WCA coefficient, a missing
# +eps shift, the WCA cut at s instead of 2^(1/6) s, a wrong Yukawa prefactor
# (eps and kappa swapped, a missing 1/r^2 or kappa/r term).

def test_short_range_contact_value():
    # at r = s = 2, eps = kappa = 1: WCA 24/2 (2 - 1) = 12, Yukawa -2 (1/4 + 1/2) = -1.5
    assert float(forces.short_range_magnitude(2.0, 1.0, 1.0, 2.0)) == pytest.approx(10.5, rel=1e-14)
    # U(s) = 4 (1 - 1) + 1 - 1 = 0
    assert abs(float(forces.short_range_potential(2.0, 1.0, 1.0, 2.0))) < 1e-15


def test_short_range_wca_cut_and_shift():
    # kappa = 200 makes the tail below 1e-17 beyond r = 2.2, leaving the WCA part
    k = 200.0
    rw = 2.0 ** (7.0 / 6.0)          # 2^(1/6) s = 2.2449...
    # (10/11)^6 = 0.564473930, (10/11)^12 = 0.318630818:
    # -U'(2.2) = (24/2.2)(2 x 0.318630818 - 0.564473930) = 10.9090909 x 0.072787706 = 0.79404770
    assert float(forces.short_range_magnitude(2.2, 1.0, k, 2.0)) == pytest.approx(0.79404770, rel=2e-8)
    # U(2.2) = 4 (0.318630818 - 0.564473930) + 1 = 0.016627552 (the +eps shift)
    assert float(forces.short_range_potential(2.2, 1.0, k, 2.0)) == pytest.approx(0.016627552, rel=1e-7)
    # the WCA part is exactly zero at and past 2^(1/6) s, and both force and
    # potential are continuous there
    for r in (rw, rw * (1 + 1e-12), 2.3, 3.0):
        assert abs(float(forces.short_range_magnitude(r, 1.0, k, 2.0))) < 1e-15
        assert abs(float(forces.short_range_potential(r, 1.0, k, 2.0))) < 1e-15
    assert 0 < float(forces.short_range_magnitude(rw * (1 - 1e-9), 1.0, k, 2.0)) < 1e-6
    assert abs(float(forces.short_range_potential(rw * (1 - 1e-9), 1.0, k, 2.0))) < 1e-15


def test_short_range_yukawa_values():
    # r = 4, eps = kappa = 1, s = 2: -U' = -2 e^-2 (1/16 + 1/4) = -0.625 e^-2,
    # U = -(2/4) e^-2; e^-2 = 0.1353352832366127
    assert float(forces.short_range_magnitude(4.0, 1.0, 1.0, 2.0)) == pytest.approx(-0.0845845520228829, rel=1e-13)
    assert float(forces.short_range_potential(4.0, 1.0, 1.0, 2.0)) == pytest.approx(-0.06766764161830635, rel=1e-13)
    # r = 3, eps = 2, kappa = 0.5: -U' = -(2 x 2) e^-0.5 (1/9 + 0.5/3) = -4 e^-0.5 (5/18),
    # e^-0.5 = 0.6065306597126334
    assert float(forces.short_range_magnitude(3.0, 2.0, 0.5, 2.0)) == pytest.approx(-0.6739229552362594, rel=1e-13)
    # U = -2 (2/3) e^-0.5
    assert float(forces.short_range_potential(3.0, 2.0, 0.5, 2.0)) == pytest.approx(-0.8087075462835112, rel=1e-13)
