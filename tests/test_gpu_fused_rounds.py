"""GPU tests of the fused Lawson rounds (a flip tests the outer edges of its
quadrilateral and keeps the overlap sums, so no check pass runs between
rounds) against the unfused order (a check pass, marking and scanning, after
every round).  Both reach the Delaunay triangulation of the same positions,
which is unique for points in general position, and Algorithm 2's sums over
its overlapping edges are exact fixed-point sums, so the two runs agree bit
for bit: positions, directions and triangulations, step after step, with
walls, in the periodic box, with list-mode check passes and under the
inversion repair of bd_set_state."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1703_02484_gb300 as bd  # noqa: E402
from paper_1703_02484_gb300 import workloads  # noqa: E402
from oracle import geometry, periodic  # noqa: E402


def stream():
    return torch.cuda.current_stream().cuda_stream


def edges(tri):
    return geometry.edges(tri)


def pair(monkeypatch, make):
    # the switch is read when a handle is made
    monkeypatch.setenv("BD_TRI_FUSE", "1")
    fused = make()
    monkeypatch.setenv("BD_TRI_FUSE", "0")
    plain = make()
    monkeypatch.delenv("BD_TRI_FUSE")
    return fused, plain


def run_and_compare(fused, plain, steps, chunk=1):
    rounds = flips = 0
    for _ in range(steps // chunk):
        sf = fused.step(chunk)
        sp = plain.step(chunk)
        a, b = fused.state(), plain.state()
        assert np.array_equal(a["xy"], b["xy"])
        assert np.array_equal(a["theta"], b["theta"])
        assert np.array_equal(edges(a["tri"]), edges(b["tri"]))
        assert sf["corr_iters"] == sp["corr_iters"] and sf["overlap_pairs"] == sp["overlap_pairs"]
        rounds += sf["flip_rounds"]
        flips += sf["flips"]
    return rounds, flips


@pytest.mark.parametrize("n,seed", [(4000, 1), (2500, 2)])
def test_fused_rounds_match_unfused_walls(monkeypatch, n, seed):
    cfg = workloads.CONFIGS["c2"]
    L = workloads.box_side(n, cfg.rho)
    xy = workloads.near_contact_state(n, L, cfg.a, seed=seed)
    _, sp, th = workloads.initial_state(cfg, n=n)
    p = bd.params_from_config(cfg, n=n)
    fused, plain = pair(monkeypatch, lambda: bd.System(p, xy, sp, th, stream=stream()))
    rounds, flips = run_and_compare(fused, plain, 12)
    assert flips > 0 and rounds > 0


def test_fused_rounds_match_unfused_periodic(monkeypatch):
    cfg = workloads.CONFIGS["c2"]
    n = 3000
    L = workloads.box_side(n, cfg.rho)
    xy = workloads.near_contact_state(n, L, cfg.a, seed=5)
    xy = periodic.wrap(xy + np.random.default_rng(6).uniform(0, L, 2), L)   # disks across the edges
    _, sp, th = workloads.initial_state(cfg, n=n)
    p = bd.make_params(n, L=L, a=cfg.a, law=cfg.law, alpha=cfg.alpha, n_species=cfg.n_species, D=cfg.D,
                       Dr=cfg.Dr, v0=cfg.v0, dt=cfg.dt, seed=cfg.seed, boundary=bd.BOUNDARY_PERIODIC)
    fused, plain = pair(monkeypatch, lambda: bd.System(p, xy, sp, th, stream=stream()))
    rounds, flips = run_and_compare(fused, plain, 12)
    assert flips > 0


def test_fused_rounds_match_unfused_list_passes(monkeypatch):
    # check passes after the first of a move visit lists (forced at this size)
    monkeypatch.setenv("BD_TRI_LISTS", "1")
    cfg = workloads.CONFIGS["c3"]
    n = 20000
    L = workloads.box_side(n, cfg.rho)
    xy = workloads.near_contact_state(n, L, cfg.a, seed=3, rho=cfg.rho)
    _, sp, th = workloads.initial_state(cfg, n=n)
    p = bd.params_from_config(cfg, n=n)
    fused, plain = pair(monkeypatch, lambda: bd.System(p, xy, sp, th, stream=stream()))
    rounds, flips = run_and_compare(fused, plain, 10)
    assert flips > 0


@pytest.mark.parametrize("delta", [0.0, -1e-9])
def test_fused_rounds_match_unfused_after_set_state(monkeypatch, delta):
    # bd_set_state moves that flatten or invert triangles (disks moved onto
    # or just across the line of two neighbours): inversion repair, then
    # Lawson rounds, in both orders
    from test_gpu_repair import _collinear_moves
    cfg = workloads.CONFIGS["c5"]
    n = 2500
    xy0, sp, th = workloads.initial_state(cfg, n=n)
    p = bd.params_from_config(cfg, n=n)
    p.law = bd.LAW_NONE
    fused, plain = pair(monkeypatch, lambda: bd.System(p, xy0, sp, th, stream=stream()))
    q, L = fused.geometry()
    start = fused.state()
    moved, count = _collinear_moves(start["xy"], start["tri"], n, q, delta, np.random.default_rng(11))
    assert count >= 10
    codes = []
    for s in (fused, plain):
        try:
            s.set_state(moved)
            codes.append(0)
        except bd.BDError as e:
            codes.append(e.code)
    assert codes[0] == codes[1]
    assert fused.last_stats()["repair_flips"] == plain.last_stats()["repair_flips"] > 0
    a, b = fused.state(), plain.state()
    assert np.array_equal(a["xy"], b["xy"])
    assert np.array_equal(edges(a["tri"]), edges(b["tri"]))
    if codes[0] == 0:
        assert np.array_equal(edges(a["tri"]), edges(geometry.delaunay(a["xy"], L, cfg.a)))
