"""Pins for the Euler-Maruyama / ABP update (Eq. (integration), Sec. 7)."""
import math

import numpy as np

from oracle import dynamics, noise

VC = noise.clamped_normal_variance()


def _run(n, steps, D, Dr, v0, dt, seed=9):
    L = 1e7
    xy = np.full((n, 2), L / 2)
    xy0 = xy.copy()
    th = np.zeros(n)
    F = np.zeros((n, 2))
    ids = np.arange(n)
    for k in range(steps):
        xy, th = dynamics.em_step(xy, th, F, ids, k, seed, D, Dr, v0, dt, 1.0, L)
    d = xy - xy0
    return (d ** 2).sum(axis=1)


def test_free_diffusion_msd():
    n, steps, D, dt = 20000, 50, 1.0, 1e-4
    sq = _run(n, steps, D, 0.0, 0.0, dt)
    t = steps * dt
    want = 4 * D * t * VC
    se = sq.std() / math.sqrt(n)
    assert abs(sq.mean() - want) < 4 * se
    # the paper's literal amplitude sqrt(D dt) would give half of it
    assert abs(sq.mean() - 2 * D * t * VC) > 20 * se


def test_abp_msd_closed_form():
    n, steps, D, Dr, v0, dt = 4000, 400, 0.05, 1.0, 1.0, 0.01
    sq = _run(n, steps, D, Dr, v0, dt, seed=21)
    t = steps * dt
    De, Dre = D * VC, Dr * VC
    want = 4 * De * t + 2 * v0 ** 2 / Dre ** 2 * (Dre * t - 1 + math.exp(-Dre * t))
    se = sq.std() / math.sqrt(n)
    assert abs(sq.mean() - want) < 4 * se + 0.01 * want


def test_deterministic_part_and_reflection():
    xy = np.array([[5.0, 5.0], [1.00001, 9.0]])
    th = np.array([0.0, math.pi / 2])
    F = np.array([[10.0, -20.0], [-5.0, 3.0]])
    new, th2 = dynamics.em_step(xy, th, F, np.arange(2), 0, 0, 0.0, 0.0, 2.0, 1e-2, 1.0, 10.0)
    assert np.allclose(new[0], [5.0 + 1e-2 * (10 + 2), 5.0 - 0.2])
    # x = 1.00001 - 0.05 = 0.95001 < a = 1  ->  2a - x = 1.04999;
    # y = 9 + 0.05 > L - a = 9  ->  2(L - a) - y = 8.95
    assert np.allclose(new[1], [2.0 - (1.00001 - 0.05), 18.0 - (9.0 + 1e-2 * (3 + 2))])
    assert np.array_equal(th2, th)
    r = dynamics.reflect(np.array([[9.5, 0.2]]), 1.0, 10.0)
    assert np.allclose(r, [[8.5, 1.8]])
