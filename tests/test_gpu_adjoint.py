"""GPU parity of the differentiated rollout against the FP64 oracle.

The oracle records its own FP64 rollout from the same start and noise,
differentiates its frozen map by forward-mode tangents (pinned to central
differences in test_oracle_adjoint.py), and the GPU's reverse-mode gradient
must agree: relative error <= 1e-3 for the FP32 path (the stated bar for the
differentiated rollout), <= 1e-5 for the FP64 path.  The GPU's own frozen
replay is also differenced centrally (h = 1e-4) against its adjoint."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1703_02484_gb300 as bd  # noqa: E402
from paper_1703_02484_gb300 import workloads  # noqa: E402
from oracle import adjoint  # noqa: E402
from oracle import step as ostep  # noqa: E402

THREADS = max(1, min(16, os.cpu_count() or 1))
TARGET = 0.1


def stream():
    return torch.cuda.current_stream().cuda_stream


def _setup(n, precision, seed, near_contact=True, rho=None):
    cfg = workloads.CONFIGS["c5"]
    rho = cfg.rho if rho is None else rho
    L = workloads.box_side(n, rho)
    if near_contact:
        xy = workloads.near_contact_state(n, L, cfg.a, seed=seed, rho=rho)
    else:
        xy = workloads.initial_positions(n, L, cfg.a, rho, seed)
    _, sp, th = workloads.initial_state(cfg, n=n)
    p = bd.params_from_config(cfg, n=n)
    p.box_L = L
    p.precision = precision
    s = bd.System(p, xy, sp, th, stream=stream())
    st = s.state(want_tri=False)
    P = ostep.Params(L=L, a=cfg.a, law=cfg.law, alpha=cfg.alpha, D=cfg.D, Dr=cfg.Dr, v0=cfg.v0, dt=cfg.dt,
                     seed=cfg.seed)
    return s, st["xy"], st["theta"].astype(np.float64), sp, P


def _log_size(rec):
    return (sum(len(s["passes"]) for s in rec["steps"]),
            sum(len(ps["pairs"]) for s in rec["steps"] for ps in s["passes"]))


def _rel(g, ref):
    return float(np.max(np.abs(g - ref)) / np.max(np.abs(ref)))


def test_fp64_rollout_gradient_matches_oracle():
    s, x0, th0, sp, P = _setup(500, 1, seed=21)
    loss, stats = s.rollout(30, ckpt_every=7, target=TARGET)     # ragged last segment
    assert stats["steps_done"] == 30 and stats["corr_iters"] > 0
    g = s.rollout_vjp()
    rec = adjoint.record(x0, th0, sp, P, 30, threads=THREADS)
    assert s.rollout_log_size() == _log_size(rec)
    ref_loss = adjoint.msd_loss(rec["xT"], rec["x0"], sp, TARGET)
    assert abs(loss - ref_loss) <= 1e-8 * abs(ref_loss)
    gref, _ = adjoint.tangent_gradient(rec, sp, P, TARGET, threads=THREADS)
    assert _rel(g, gref) <= 1e-5, (g, gref)
    # the reverse pass leaves the state alone, and the frozen replay ends where
    # the forward did
    fin = s.state(want_tri=False)["xy"]
    assert abs(s.rollout_replay() - loss) <= 1e-12 * abs(loss)
    assert np.max(np.abs(s.rollout_positions(1) - fin)) <= 1e-11
    assert np.array_equal(s.rollout_positions(0), x0)
    # a second reverse pass gives the same gradient up to the order of the
    # FP64 atomic sums of the pass adjoint
    assert np.allclose(s.rollout_vjp(), g, rtol=1e-10, atol=0)


def test_gpu_replay_differences_match_adjoint():
    s, x0, th0, sp, P = _setup(400, 1, seed=22)
    loss, _ = s.rollout(25, ckpt_every=10, target=TARGET)
    assert abs(s.rollout_replay() - loss) <= 1e-12 * abs(loss)
    g = s.rollout_vjp()
    base = np.array(list(P.alpha) + [P.v0])
    h = 1e-4
    fd = np.zeros(5)
    for k in range(5):
        up, dn = base.copy(), base.copy()
        up[k] += h
        dn[k] -= h
        fd[k] = (s.rollout_replay(up[:4], up[4]) - s.rollout_replay(dn[:4], dn[4])) / (2 * h)
    assert _rel(g, fd) <= 1e-5, (g, fd)


def test_fp32_rollout_gradient_matches_oracle():
    s, x0, th0, sp, P = _setup(1024, 0, seed=23)
    s.rollout(40, ckpt_every=20, target=TARGET)
    g = s.rollout_vjp()
    rec = adjoint.record(x0, th0, sp, P, 40, threads=THREADS)
    assert s.rollout_log_size() == _log_size(rec)
    gref, _ = adjoint.tangent_gradient(rec, sp, P, TARGET, threads=THREADS)
    assert _rel(g, gref) <= 1e-3, (g, gref)


def test_full_size_rollout_gradient_matches_oracle():
    # 4096 disks, area fraction 0.35, two species, v0 = 1, 200 steps, checkpoints
    # every 20; both losses, from the same start and noise
    cfg = workloads.CONFIGS["c5"]
    xy, sp, th = workloads.initial_state(cfg)
    s = bd.System(bd.params_from_config(cfg), xy, sp, th, stream=stream())
    st = s.state(want_tri=False)
    loss, stats = s.rollout(cfg.steps, ckpt_every=20, target=TARGET)
    assert stats["steps_done"] == cfg.steps
    g = s.rollout_vjp()
    s.set_state(st["xy"], st["theta"])
    s.set_step(0)
    loss_h, _ = s.rollout(cfg.steps, ckpt_every=20, loss_kind=bd.LOSS_HIST)
    g_h = s.rollout_vjp()
    L = workloads.box_side(cfg.n, cfg.rho)
    P = ostep.Params(L=L, a=cfg.a, law=cfg.law, alpha=cfg.alpha, D=cfg.D, Dr=cfg.Dr, v0=cfg.v0, dt=cfg.dt,
                     seed=cfg.seed)
    rec = adjoint.record(st["xy"], st["theta"].astype(np.float64), sp, P, cfg.steps, threads=THREADS)
    assert s.rollout_log_size() == _log_size(rec)
    assert abs(loss - adjoint.msd_loss(rec["xT"], rec["x0"], sp, TARGET)) <= 1e-6 * loss
    assert abs(loss_h - adjoint.hist_loss(rec["xT"], rec["x0"], cfg.a)) <= 1e-4 * loss_h
    Tm, xT = adjoint.tangent_map(rec, sp, P, threads=THREADS)
    # every component to 1e-3 of its own size
    gref = np.einsum("ia,iak->k", adjoint.msd_loss_grad(xT, rec["x0"], sp, TARGET), Tm)
    assert np.all(np.abs(g - gref) <= 1e-3 * np.abs(gref)), (g, gref)
    gref_h = np.einsum("ia,iak->k", adjoint.hist_loss_grad(xT, rec["x0"], cfg.a), Tm)
    # each component to 1e-3 of its own size, or to 1e-4 of the largest for a
    # component that nearly cancels
    tol = np.maximum(1e-3 * np.abs(gref_h), 1e-4 * np.max(np.abs(gref_h)))
    assert np.all(np.abs(g_h - gref_h) <= tol), (g_h, gref_h)


def test_fp64_hist_loss_gradient_matches_oracle():
    s, x0, th0, sp, P = _setup(500, 1, seed=27)
    loss, stats = s.rollout(30, ckpt_every=7, loss_kind=bd.LOSS_HIST)
    assert stats["steps_done"] == 30 and stats["corr_iters"] > 0
    g = s.rollout_vjp()
    rec = adjoint.record(x0, th0, sp, P, 30, threads=THREADS)
    assert s.rollout_log_size() == _log_size(rec)
    ref_loss = adjoint.hist_loss(rec["xT"], rec["x0"], P.a)
    assert ref_loss > 0 and abs(loss - ref_loss) <= 1e-8 * ref_loss
    gref, _ = adjoint.tangent_gradient(rec, sp, P, TARGET, threads=THREADS, loss="hist")
    assert _rel(g, gref) <= 1e-5, (g, gref)
    assert abs(s.rollout_replay() - loss) <= 1e-12 * loss
    # the GPU's own frozen replay, differenced centrally
    base = np.array(list(P.alpha) + [P.v0])
    h = 1e-4
    fd = np.zeros(5)
    for k in range(5):
        up, dn = base.copy(), base.copy()
        up[k] += h
        dn[k] -= h
        fd[k] = (s.rollout_replay(up[:4], up[4]) - s.rollout_replay(dn[:4], dn[4])) / (2 * h)
    assert _rel(g, fd) <= 1e-5, (g, fd)


def test_fp32_hist_loss_gradient_matches_oracle():
    s, x0, th0, sp, P = _setup(1024, 0, seed=28)
    s.rollout(40, ckpt_every=20, loss_kind=bd.LOSS_HIST)
    g = s.rollout_vjp()
    rec = adjoint.record(x0, th0, sp, P, 40, threads=THREADS)
    gref, _ = adjoint.tangent_gradient(rec, sp, P, TARGET, threads=THREADS, loss="hist")
    assert _rel(g, gref) <= 1e-3, (g, gref)


def test_rollout_forward_is_the_step():
    s1, x0, th0, sp, P = _setup(700, 0, seed=24)
    s2, _, _, _, _ = _setup(700, 0, seed=24)
    s1.rollout(15, ckpt_every=4)
    s2.step(15)
    a, b = s1.state(), s2.state()
    assert np.array_equal(a["xy"], b["xy"]) and a["step"] == b["step"] == 15
    assert np.array_equal(a["tri"], b["tri"])


def test_autograd_function():
    s, x0, th0, sp, P = _setup(300, 0, seed=25)
    params = torch.tensor(list(P.alpha) + [P.v0], dtype=torch.float64, requires_grad=True)
    loss = bd.rollout_loss(params, s, x0, th0, 0, 20, 5, TARGET)
    loss.backward()
    g = s.rollout_vjp()
    assert np.allclose(params.grad.numpy(), g, rtol=1e-10, atol=0)
    # same parameters and start: same loss
    loss2 = bd.rollout_loss(params.detach(), s, x0, th0, 0, 20, 5, TARGET)
    assert float(loss2) == float(loss.detach())
    # the histogram loss through the same function
    p2 = params.detach().clone().requires_grad_(True)
    lh = bd.rollout_loss(p2, s, x0, th0, 0, 20, 5, TARGET, bd.LOSS_HIST)
    lh.backward()
    assert np.allclose(p2.grad.numpy(), s.rollout_vjp(), rtol=1e-10, atol=0)


def test_rollout_argument_errors():
    s, *_ = _setup(64, 0, seed=26, near_contact=False)
    with pytest.raises(bd.BDError) as e:
        s.rollout_vjp()
    assert e.value.code == -1
    with pytest.raises(bd.BDError) as e:
        s.rollout(0)
    assert e.value.code == -1
    with pytest.raises(bd.BDError) as e:
        s.rollout(3, loss_kind=7)
    assert e.value.code == -10
    loss, st = s.rollout(1, ckpt_every=50)
    assert st["steps_done"] == 1 and np.all(np.isfinite(s.rollout_vjp()))
    cfg = workloads.CONFIGS["c3"]
    xy, sp, th = workloads.initial_state(cfg, n=256)
    short = bd.System(bd.params_from_config(cfg, n=256), xy, sp, th, stream=stream())
    with pytest.raises(bd.BDError) as e:
        short.rollout(2)
    assert e.value.code == -10
