"""Pins of the oracle's differentiated rollout (oracle/adjoint.py).

The forward-mode tangent gradient is checked against central differences of
the frozen replay (an independent definition of the derivative), in a regime
where every frozen choice occurs (overlap passes, capped disks, reflections
of moves and of passes); the force Jacobian products against differences of
the oracle's own force sum; the free-flight case against its closed form."""
import numpy as np
import pytest

from oracle import adjoint
from oracle import forces as oforces
from oracle import step as ostep
from paper_1703_02484_gb300 import workloads


def _system(n=60, rho=0.45, seed=3, v0=150.0, dt=2e-3, alpha=(0.5, 1.0, -0.4, 0.3)):
    L = workloads.box_side(n, rho)
    xy = workloads.near_contact_state(n, L, 1.0, seed=seed, gap=0.02, frac=0.5)
    sp = (np.arange(n) % 2).astype(np.uint8)
    th = np.random.default_rng(seed + 1).uniform(0, 2 * np.pi, n)
    p = ostep.Params(L=L, a=1.0, alpha=alpha, D=1.0, Dr=0.5, v0=v0, dt=dt, seed=7)
    return xy, sp, th, p


def _counts(rec):
    caps = sum(int(ps["capped"].sum()) for s in rec["steps"] for ps in s["passes"])
    pairs = sum(len(ps["pairs"]) for s in rec["steps"] for ps in s["passes"])
    r0 = sum(int((s["flags"] != 0).sum()) for s in rec["steps"])
    rp = sum(int((ps["flags"] != 0).sum()) for s in rec["steps"] for ps in s["passes"])
    return caps, pairs, r0, rp


@pytest.fixture(scope="module")
def fast_rollout():
    xy, sp, th, p = _system()
    rec = adjoint.record(xy, th, sp, p, 12)
    return rec, sp, p


def test_replay_reproduces_recorded_rollout(fast_rollout):
    rec, sp, p = fast_rollout
    xr = adjoint.replay(rec, sp, p)
    assert np.max(np.abs(xr - rec["xT"])) <= 1e-11


def test_all_frozen_choices_occur(fast_rollout):
    caps, pairs, r0, rp = _counts(fast_rollout[0])
    assert caps > 0 and pairs > 0 and r0 > 0 and rp > 0


def test_tangent_gradient_matches_central_differences(fast_rollout):
    rec, sp, p = fast_rollout
    g, xT = adjoint.tangent_gradient(rec, sp, p, target=0.1)
    assert np.max(np.abs(xT - rec["xT"])) <= 1e-11
    fd = adjoint.fd_gradient(rec, sp, p, target=0.1, h=1e-4)
    scale = np.max(np.abs(fd))
    assert scale > 0
    assert np.max(np.abs(g - fd)) <= 1e-6 * scale, (g, fd)


def test_tangent_gradient_slow_regime():
    # ordinary speeds: passes without caps
    xy, sp, th, p = _system(v0=5.0)
    rec = adjoint.record(xy, th, sp, p, 10)
    g, _ = adjoint.tangent_gradient(rec, sp, p, target=0.1)
    fd = adjoint.fd_gradient(rec, sp, p, target=0.1, h=1e-4)
    assert np.max(np.abs(g - fd)) <= 1e-6 * np.max(np.abs(fd))


def test_force_jvp_matches_differences():
    rng = np.random.default_rng(0)
    n = 40
    xy = rng.uniform(0, 30, (n, 2))
    sp = (np.arange(n) % 2).astype(np.uint8)
    A = (0.7, -0.2, 0.4, 1.1)
    Tm = rng.normal(size=(n, 2, 3))
    J = adjoint.force_jvp(xy, sp, A, Tm)
    eps = 1e-6
    for k in range(3):
        fd = (oforces.long_range_numpy(xy + eps * Tm[:, :, k], sp, A)
              - oforces.long_range_numpy(xy - eps * Tm[:, :, k], sp, A)) / (2 * eps)
        assert np.max(np.abs(J[:, :, k] - fd)) <= 1e-6 * np.max(np.abs(fd))


def test_force_dA_is_the_unit_table_force():
    rng = np.random.default_rng(1)
    n = 33
    xy = rng.uniform(0, 20, (n, 2))
    sp = (rng.uniform(size=n) < 0.4).astype(np.uint8)
    D = adjoint.force_dA(xy, sp)
    for col in range(4):
        E = np.zeros(4)
        E[col] = 1.0
        assert np.allclose(D[:, :, col], oforces.long_range_numpy(xy, sp, E), rtol=1e-12, atol=1e-14)


def test_free_flight_closed_form():
    # no forces, no contacts, no walls: x_T = x_0 + sum_t (dt v0 e_t + amp xi_t),
    # so dx_T/dv0 = dt sum_t e(theta_t) and dx_T/dA[a][b] = dt sum_t S_ab(x_t)
    n = 12
    L = 400.0
    rng = np.random.default_rng(2)
    xy = np.stack([np.linspace(150, 250, n), 200 + 30 * np.sin(np.arange(n))], axis=1)
    sp = (np.arange(n) % 2).astype(np.uint8)
    th = rng.uniform(0, 2 * np.pi, n)
    p = ostep.Params(L=L, a=1.0, alpha=(0.0, 0.0, 0.0, 0.0), D=0.5, Dr=1.0, v0=2.0, dt=1e-3, seed=11)
    rec = adjoint.record(xy, th, sp, p, 15)
    assert _counts(rec) == (0, 0, 0, 0)
    g, xT = adjoint.tangent_gradient(rec, sp, p, target=0.05)
    gl = adjoint.msd_loss_grad(xT, rec["x0"], sp, 0.05)
    e_sum = np.zeros((n, 2))
    S_sum = np.zeros((n, 2, 4))
    x = rec["x0"].copy()
    xs = [x]
    for st in rec["steps"]:
        e_sum += np.stack([np.cos(st["th"]), np.sin(st["th"])], axis=1)
    # positions along the free flight (independent of A when A = 0)
    for t, st in enumerate(rec["steps"]):
        for col in range(4):
            E = np.zeros(4)
            E[col] = 1.0
            S_sum[:, :, col] += oforces.long_range_numpy(xs[-1], sp, E)
        xs.append(adjoint.replay({**rec, "steps": rec["steps"][:t + 1]}, sp, p))
    ref = np.zeros(5)
    ref[4] = p.dt * np.sum(gl * e_sum)
    for col in range(4):
        ref[col] = p.dt * np.sum(gl * S_sum[:, :, col])
    assert np.allclose(g, ref, rtol=1e-10, atol=1e-16)


def test_msd_loss_gradient_matches_differences():
    rng = np.random.default_rng(4)
    n = 20
    x0 = rng.uniform(0, 10, (n, 2))
    xT = x0 + rng.normal(scale=0.3, size=(n, 2))
    sp = (np.arange(n) % 3 == 0).astype(np.uint8)
    g = adjoint.msd_loss_grad(xT, x0, sp, 0.07)
    eps = 1e-6
    for i in (0, 3, 7):
        for c in (0, 1):
            a = xT.copy()
            b = xT.copy()
            a[i, c] += eps
            b[i, c] -= eps
            fd = (adjoint.msd_loss(a, x0, sp, 0.07) - adjoint.msd_loss(b, x0, sp, 0.07)) / (2 * eps)
            assert abs(fd - g[i, c]) <= 1e-7 * max(1e-3, abs(fd))


def test_reflection_flags_reproduce_walls():
    from oracle import dynamics
    rng = np.random.default_rng(5)
    y = rng.uniform(-1.0, 12.0, (200, 2))
    r, f = adjoint.reflect_flags(y, 1.0, 10.0)
    assert np.array_equal(r, dynamics.reflect(y, 1.0, 10.0))
    assert np.array_equal(adjoint.apply_flags(y, f, 1.0, 10.0), r)
    # the derivative of a mirror is -1 in its component
    s = adjoint.flag_signs(f)
    assert np.all(s[(y[:, 0] < 1.0) | (y[:, 0] > 9.0), 0] == -1.0)
    assert np.all(s[(y[:, 0] >= 1.0) & (y[:, 0] <= 9.0), 0] == 1.0)


# ---- pair-distance histogram loss ----

def test_hist_single_pair_peaks_at_its_bin():
    # one pair at the centre of bin 5: K(0) = 1 gives h_5 = 1/n, and the bins
    # either side are equal (the centres are evenly spaced about it)
    a = 1.0
    c = adjoint.hist_centres(a)
    assert c[0] == 2.125 and c[-1] == 9.875 and np.allclose(np.diff(c), 0.25)
    x = np.array([[10.0, 10.0], [10.0 + c[5], 10.0]])
    h = adjoint.pair_histogram(x, a)
    assert int(np.argmax(h)) == 5 and h[5] == 0.5
    assert abs(h[4] - h[6]) <= 1e-15 and abs(h[2] - h[8]) <= 1e-15
    assert h[4] < h[5] and h[3] < h[4]


@pytest.mark.parametrize("side", [6.0, 5.3, 7.11])
def test_hist_bins_sum_to_the_gaussian_integral(side):
    # bins spaced one kernel width s apart: for a distance r well inside
    # [2a, 10a] the sum over bins of exp(-(r - c_b)^2 / 2 s^2) is, by Poisson
    # summation, sqrt(2 pi) (1 + 2 exp(-2 pi^2) cos(2 pi (r - c_0) / s)) (the
    # next term is exp(-8 pi^2) ~ 1e-34; the 32-bin truncation cuts tails
    # beyond 11 s)
    a = 1.0
    s = 0.25 * a
    tri = side * np.array([[0.0, 0.0], [1.0, 0.0], [0.5, np.sqrt(3.0) / 2.0]])
    h = adjoint.pair_histogram(tri + 20.0, a)
    c0 = adjoint.hist_centres(a)[0]
    want = np.sqrt(2.0 * np.pi) * (1.0 + 2.0 * np.exp(-2.0 * np.pi ** 2) * np.cos(2.0 * np.pi * (side - c0) / s))
    assert abs(h.sum() - want) <= 1e-13     # 3 pairs at distance side, n = 3


def test_hist_is_rigid_motion_invariant():
    rng = np.random.default_rng(8)
    x = rng.uniform(0.0, 14.0, (40, 2))
    phi = 0.7
    R = np.array([[np.cos(phi), -np.sin(phi)], [np.sin(phi), np.cos(phi)]])
    y = x @ R.T + np.array([3.0, -5.0])
    assert np.max(np.abs(adjoint.pair_histogram(x, 1.0) - adjoint.pair_histogram(y, 1.0))) <= 1e-13
    assert adjoint.hist_loss(y, x, 1.0) <= 1e-26


def test_hist_loss_gradient_matches_differences():
    rng = np.random.default_rng(9)
    n = 30
    x0 = rng.uniform(0.0, 12.0, (n, 2))
    xT = x0 + rng.normal(scale=0.4, size=(n, 2))
    g = adjoint.hist_loss_grad(xT, x0, 1.0)
    eps = 1e-6
    for i in (0, 11, 29):
        for c in (0, 1):
            a, b = xT.copy(), xT.copy()
            a[i, c] += eps
            b[i, c] -= eps
            fd = (adjoint.hist_loss(a, x0, 1.0) - adjoint.hist_loss(b, x0, 1.0)) / (2 * eps)
            assert abs(fd - g[i, c]) <= 1e-6 * max(1e-6, np.max(np.abs(g)))
    # a rigid translation of x_T changes nothing: the gradient sums to zero
    assert np.max(np.abs(g.sum(axis=0))) <= 1e-12 * np.max(np.abs(g))


def test_tangent_gradient_hist_loss_matches_central_differences(fast_rollout):
    rec, sp, p = fast_rollout
    g, _ = adjoint.tangent_gradient(rec, sp, p, target=0.1, loss="hist")
    fd = adjoint.fd_gradient(rec, sp, p, target=0.1, h=1e-4, loss="hist")
    scale = np.max(np.abs(fd))
    assert scale > 0
    assert np.max(np.abs(g - fd)) <= 1e-6 * scale, (g, fd)
