"""GPU parity: the CUDA time step against the FP64 oracle, through the C ABI.

Tolerances (the accuracy bar set for this method): per-disk force error <= 1e-5
relative to the force norm (read as the RMS of |F_i| over the system), and
position error <= 1e-5 a after one step; the Delaunay edge set must match
exactly for points in general position."""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1703_02484_gb300 as bd  # noqa: E402
from paper_1703_02484_gb300 import workloads  # noqa: E402
from oracle import forces as oforces  # noqa: E402
from oracle import geometry, overlap  # noqa: E402
from oracle import step as ostep  # noqa: E402
from scipy.spatial import cKDTree  # noqa: E402

POS_TOL = 1e-5
FORCE_TOL = 1e-5


def stream():
    return torch.cuda.current_stream().cuda_stream


def oracle_params(cfg, L, seed=None):
    return ostep.Params(L=L, a=cfg.a, law=cfg.law, alpha=cfg.alpha, eps=cfg.eps, kappa=cfg.kappa,
                        r_cut=cfg.r_cut, D=cfg.D, Dr=cfg.Dr, v0=cfg.v0, dt=cfg.dt,
                        seed=cfg.seed if seed is None else seed)


def force_error(F, ref):
    scale = math.sqrt(float(np.mean(np.sum(ref ** 2, axis=1))))
    return float(np.max(np.linalg.norm(F - ref, axis=1))) / scale


@pytest.mark.parametrize("cfgname,n", [("c2", 3001), ("c2", 777), ("c1", 1024), ("c5", 4096)])
def test_forces_match_oracle(cfgname, n):
    cfg = workloads.CONFIGS[cfgname]
    xy, sp, th = workloads.initial_state(cfg, n=n)
    s = bd.System(bd.params_from_config(cfg, n=n), xy, sp, th, stream=stream())
    F = s.forces()
    grid = s.state(want_tri=False)["xy"]
    ref = oforces.long_range_numpy(grid, sp, cfg.alpha if cfg.n_species == 2 else (cfg.alpha[0],) * 4)
    err = force_error(F, ref)
    assert err <= FORCE_TOL, err
    if cfg.precision == 1:
        assert err <= 1e-12


@pytest.mark.parametrize("variant,tiles", [(0, 3), (1, 5), (2, 1), (2, 2), (2, 7), (3, 1), (3, 4)])
@pytest.mark.parametrize("cfgname,n", [("c2", 3001), ("c2", 1300), ("c1", 1024)])
def test_force_variants_match_oracle(monkeypatch, variant, tiles, cfgname, n):
    # every FP32 sweep, chunk sizes that split rows unevenly, ragged species segments
    monkeypatch.setenv("BD_FORCE_VARIANT", str(variant))
    monkeypatch.setenv("BD_FORCE_TILES", str(tiles))
    cfg = workloads.CONFIGS[cfgname]
    xy, sp, th = workloads.initial_state(cfg, n=n)
    p = bd.params_from_config(cfg, n=n)
    p.precision = 0
    s = bd.System(p, xy, sp, th, stream=stream())
    assert s.tuning()["variant"] == variant and s.tuning()["tiles_per_item"] == tiles
    F = s.forces()
    grid = s.state(want_tri=False)["xy"]
    A = cfg.alpha if cfg.n_species == 2 else (cfg.alpha[0],) * 4
    assert force_error(F, oforces.long_range_numpy(grid, sp, A)) <= FORCE_TOL
    # deterministic: a second evaluation gives the same bits
    assert np.array_equal(s.forces(), F)


@pytest.mark.parametrize("cfgname", ["n1e5", "c2"])
def test_forces_full_size_every_disk(cfgname):
    # the full workload in the configuration the benchmark times (autotuned
    # sweep), every disk against the oracle's FP64 sum (OpenMP C loop)
    cfg = workloads.CONFIGS[cfgname]
    xy, sp, th = workloads.initial_state(cfg)
    s = bd.System(bd.params_from_config(cfg), xy, sp, th, stream=stream())
    F = s.forces()
    grid = s.state(want_tri=False)["xy"]
    ref = oforces.long_range(grid, sp, cfg.alpha, threads=max(1, os.cpu_count() or 1))
    err = force_error(F, ref)
    assert err <= FORCE_TOL, (err, s.tuning())


def _one_step(cfgname, n, seed_state, step_index=0, near_contact=True):
    cfg = workloads.CONFIGS[cfgname]
    L = workloads.box_side(n, cfg.rho)
    if near_contact:
        xy = workloads.near_contact_state(n, L, cfg.a, seed=seed_state)
    else:
        xy = workloads.initial_positions(n, L, cfg.a, cfg.rho, seed_state)
    _, sp, th = workloads.initial_state(cfg, n=n)
    p = bd.params_from_config(cfg, n=n)
    p.step0 = step_index
    s = bd.System(p, xy, sp, th, stream=stream())
    st = s.step(1)
    out = s.state()
    ref = ostep.step(xy, th, sp, step_index, oracle_params(cfg, L))
    return cfg, L, s, st, out, ref


@pytest.mark.parametrize("cfgname,n,seed,k", [("c2", 4000, 1, 0), ("c2", 2500, 2, 12345),
                                               ("c1", 1024, 3, 7), ("c5", 4096, 4, 99)])
def test_one_step_parity(cfgname, n, seed, k):
    cfg, L, s, st, out, ref = _one_step(cfgname, n, seed, k)
    assert not ref["rejected"]
    assert ref["corr_iters"] >= 1          # the start had overlaps to correct
    err = float(np.max(np.abs(out["xy"] - ref["xy"])))
    assert err <= POS_TOL * cfg.a, err
    assert st["corr_iters"] == ref["corr_iters"]
    # theta: FP32 director update
    assert np.max(np.abs(out["theta"] - ref["theta"])) <= 1e-5
    # Delaunay edge set: the GPU's triangulation equals the oracle's Delaunay
    # triangulation of the oracle's own final positions
    assert np.array_equal(geometry.edges(out["tri"]), geometry.edges(ref["tris"]))
    # and no pair overlaps anywhere
    assert len(cKDTree(out["xy"]).query_pairs(2 * cfg.a * (1 - 1e-12))) == 0


def test_multi_step_invariants():
    cfg = workloads.CONFIGS["c5"]
    n = 4096
    xy, sp, th = workloads.initial_state(cfg, n=n)
    L = workloads.box_side(n, cfg.rho)
    s = bd.System(bd.params_from_config(cfg, n=n), xy, sp, th, stream=stream())
    total = 0
    for _ in range(10):
        st = s.step(10)
        assert st["steps_done"] == 10
        total += st["corr_iters"]
        out = s.state()
        assert len(cKDTree(out["xy"]).query_pairs(2 * cfg.a * (1 - 1e-12))) == 0
        assert np.all(out["xy"] >= cfg.a) and np.all(out["xy"] <= L - cfg.a)
        P = geometry.with_ghosts(out["xy"], L)
        # the maintained triangulation is the Delaunay triangulation of the positions
        assert np.array_equal(geometry.edges(out["tri"]), geometry.edges(geometry.delaunay(out["xy"], L)))
    assert out["step"] == 100


def test_trajectory_step_parity_from_state():
    # feed a state reached by the GPU after some steps back to both sides as a
    # new start (through the public entry points) and compare one more step
    cfg = workloads.CONFIGS["c2"]
    n = 3000
    L = workloads.box_side(n, cfg.rho)
    xy = workloads.near_contact_state(n, L, 1.0, seed=9)
    _, sp, th = workloads.initial_state(cfg, n=n)
    p = bd.params_from_config(cfg, n=n)
    s = bd.System(p, xy, sp, th, stream=stream())
    s.step(20)
    mid = s.state()
    ref = ostep.step(mid["xy"], mid["theta"], mid["species"], mid["step"], oracle_params(cfg, L))
    s.step(1)
    out = s.state()
    assert np.max(np.abs(out["xy"] - ref["xy"])) <= POS_TOL
    assert np.array_equal(geometry.edges(out["tri"]), geometry.edges(ref["tris"]))


def test_set_state_repairs_triangulation():
    cfg = workloads.CONFIGS["c5"]
    n = 2000
    xy, sp, th = workloads.initial_state(cfg, n=n)
    L = workloads.box_side(n, cfg.rho)
    s = bd.System(bd.params_from_config(cfg, n=n), xy, sp, th, stream=stream())
    rng = np.random.default_rng(5)
    moved = xy + rng.normal(scale=0.05, size=xy.shape)
    moved = np.clip(moved, 1.0, L - 1.0)
    keep = len(cKDTree(moved).query_pairs(2.0)) == 0
    if not keep:
        # push overlapping pairs back to the original positions
        for i, j in cKDTree(moved).query_pairs(2.0):
            moved[i], moved[j] = xy[i], xy[j]
    assert len(cKDTree(moved).query_pairs(2.0)) == 0
    s.set_state(moved)
    out = s.state()
    assert np.max(np.abs(out["xy"] - moved)) <= 1e-11 * L
    assert np.array_equal(geometry.edges(out["tri"]), geometry.edges(geometry.delaunay(out["xy"], L)))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 257, 513])
def test_tiny_and_ragged_sizes(n):
    cfg = workloads.CONFIGS["c2"]
    L = workloads.box_side(max(n, 16), cfg.rho)
    xy = workloads.initial_positions(n, L, 1.0, cfg.rho, seed=n)
    sp = (np.arange(n) % 2).astype(np.uint8)
    th = np.zeros(n, np.float32)
    p = bd.params_from_config(cfg, n=n)
    p.box_L = L
    s = bd.System(p, xy, sp, th, stream=stream())
    st = s.step(5)
    assert st["steps_done"] == 5
    out = s.state()
    assert len(out["tri"]) == 2 * (n + len(geometry.ghost_points(L))) - 6
    assert np.array_equal(geometry.edges(out["tri"]), geometry.edges(geometry.delaunay(out["xy"], L)))
    if n >= 2:
        assert len(cKDTree(out["xy"]).query_pairs(2.0 * (1 - 1e-12))) == 0


def test_init_rejects_overlap():
    p = bd.make_params(2, L=20.0)
    with pytest.raises(bd.BDError) as e:
        bd.System(p, np.array([[5.0, 5.0], [6.0, 5.0]]))
    assert e.value.code == -3


@pytest.mark.parametrize("cfgname,n", [("c5", 4096), ("c3", 30000)])
def test_graph_replay_equals_plain_launches(monkeypatch, cfgname, n):
    # bd_step replays one captured graph per step; with graphs disabled the
    # same kernels are launched one by one: identical trajectories
    cfg = workloads.CONFIGS[cfgname]
    xy, sp, th = workloads.initial_state(cfg, n=n)
    out = []
    for off in (False, True):
        if off:
            monkeypatch.setenv("BD_NO_GRAPH", "1")
        else:
            monkeypatch.delenv("BD_NO_GRAPH", raising=False)
        s = bd.System(bd.params_from_config(cfg, n=n), xy, sp, th, stream=stream())
        s.step(7)
        s.step(1)
        out.append(s.state())
    assert out[0]["step"] == out[1]["step"] == 8
    assert np.array_equal(out[0]["xy"], out[1]["xy"])
    assert np.array_equal(out[0]["tri"], out[1]["tri"])


@pytest.mark.parametrize("cfgname,n,seed,k", [("c2", 4000, 1, 0), ("c5", 4096, 4, 99)])
def test_one_step_parity_with_check_lists(monkeypatch, cfgname, n, seed, k):
    # the check passes after the first of a move visit only listed triangles
    # (used by default when a full pass has many triangles per thread, i.e. at
    # 2^20 disks); BD_TRI_LISTS=1 forces them at sizes the oracle steps fully
    monkeypatch.setenv("BD_TRI_LISTS", "1")
    cfg, L, s, st, out, ref = _one_step(cfgname, n, seed, k)
    assert not ref["rejected"] and ref["corr_iters"] >= 1
    assert float(np.max(np.abs(out["xy"] - ref["xy"]))) <= POS_TOL * cfg.a
    assert st["corr_iters"] == ref["corr_iters"]
    assert np.array_equal(geometry.edges(out["tri"]), geometry.edges(ref["tris"]))
    assert len(cKDTree(out["xy"]).query_pairs(2 * cfg.a * (1 - 1e-12))) == 0
    # the later passes visited far fewer triangles than full passes would
    passes = s.stage_times()["check"][1]
    assert passes >= 2 and st["tri_visits"] < s.n_tri * (1 + 0.5 * (passes - 1))


def test_multi_step_with_check_lists_matches_full_passes(monkeypatch):
    # 60 steps with lists and with full passes: the same trajectory (up to the
    # order of FP64 atomic additions in Algorithm 2) and the same
    # triangulation, Delaunay every 20 steps
    cfg = workloads.CONFIGS["c5"]
    n = 4096
    xy, sp, th = workloads.initial_state(cfg, n=n)
    L = workloads.box_side(n, cfg.rho)
    monkeypatch.setenv("BD_TRI_LISTS", "1")
    a = bd.System(bd.params_from_config(cfg, n=n), xy, sp, th, stream=stream())
    monkeypatch.setenv("BD_TRI_LISTS", "2")
    b = bd.System(bd.params_from_config(cfg, n=n), xy, sp, th, stream=stream())
    for _ in range(3):
        sa, sb = a.step(20), b.step(20)
        assert sa["steps_done"] == sb["steps_done"] == 20
        assert sa["tri_visits"] < sb["tri_visits"]
        oa, ob = a.state(), b.state()
        assert float(np.max(np.abs(oa["xy"] - ob["xy"]))) <= 1e-9
        assert np.array_equal(geometry.edges(oa["tri"]), geometry.edges(ob["tri"]))
        assert np.array_equal(geometry.edges(oa["tri"]), geometry.edges(geometry.delaunay(oa["xy"], L)))
    a.close()
    b.close()


@pytest.mark.parametrize("boundary", [0, 1])
def test_set_state_rejects_overlapping_positions(boundary):
    # the device finds the overlap on the repaired Delaunay triangulation's
    # edges; the handle keeps its state
    cfg = workloads.CONFIGS["c5"]
    n = 2000
    xy, sp, th = workloads.initial_state(cfg, n=n)
    L = workloads.box_side(n, cfg.rho)
    p = bd.params_from_config(cfg, n=n)
    if boundary:
        L = float(np.float32(L))
        p.box_L = L
        p.boundary = bd.BOUNDARY_PERIODIC
    s = bd.System(p, xy, sp, th, stream=stream())
    before = s.state()
    dist, nb = cKDTree(xy).query(xy, k=2)
    i = int(np.argmin(dist[:, 1]))          # a disk and its nearest neighbour
    j = int(nb[i, 1])
    bad = xy.copy()
    bad[j] = xy[i] + 1.9 * (xy[j] - xy[i]) / np.linalg.norm(xy[j] - xy[i])   # 1.9 < sigma apart
    with pytest.raises(bd.BDError) as e:
        s.set_state(bad)
    assert e.value.code == -3
    after = s.state()
    assert np.array_equal(after["xy"], before["xy"]) and np.array_equal(after["tri"], before["tri"])
    s.step(3)                       # still usable
    s.close()


@pytest.mark.parametrize("eps", [1e-3, 2e-9])
@pytest.mark.parametrize("turn", [-1, 1])
def test_reversal_test_near_perpendicular_moves(eps, turn):
    # Sec. 4.3's criterion r0 . r1 < 0 on one edge, through bd_set_state (its
    # repair pass tests every edge of the move): w turned about u by 90 deg
    # - turn * eps gives r0 . r1 = |r|^2 sin(turn * eps).  At eps = 1e-3 the
    # FP32 screen decides; at 2e-9 the product lies inside its bound and the
    # exact grid test decides.  Either way the outcome follows the exact sign.
    # Small disks (a = 0.01, |r| = 0.03): the turn moves w by 0.04, far less
    # than its distance to any other point, so no triangle inverts.
    L, r = 60.0, 0.03
    xy = np.array([[30.0, 30.0], [30.0 + r, 30.0], [12.0, 45.0], [48.0, 14.0]])
    p = bd.make_params(n=4, L=L, a=0.01, D=0.0, dt=1e-4, seed=3)
    s = bd.System(p, xy, np.zeros(4, np.uint8), np.zeros(4, np.float32), stream=stream())
    q, _ = s.geometry()
    before = s.state()
    u, w = before["xy"][0], before["xy"][1]
    th = np.pi / 2 - turn * eps
    new = before["xy"].copy()
    new[1] = u + r * np.array([np.cos(th), np.sin(th)])
    gi = lambda v: [int(round(c / q)) for c in v]     # noqa: E731  (grid integers)
    U0, W0, W1 = gi(u), gi(w), gi(np.rint(new[1] / q) * q)
    dot = (W0[0] - U0[0]) * (W1[0] - U0[0]) + (W0[1] - U0[1]) * (W1[1] - U0[1])
    assert dot != 0 and (dot > 0) == (turn > 0)
    if dot > 0:
        s.set_state(new)
        assert np.max(np.abs(s.state()["xy"][1] - new[1])) <= q
    else:
        with pytest.raises(bd.BDError) as e:
            s.set_state(new)
        assert e.value.code == -4
        after = s.state()
        assert np.array_equal(after["xy"], before["xy"]) and np.array_equal(after["tri"], before["tri"])
    s.close()


def test_one_step_parity_full_size_n1e5():
    # the benchmark's system (N = 1e5, two species, active) from a near-contact
    # start, in the configuration the benchmark times: one step against the
    # oracle's (positions, passes of Algorithm 2, Delaunay edge set)
    cfg = workloads.CONFIGS["n1e5"]
    n = cfg.n
    L = workloads.box_side(n, cfg.rho)
    xy = workloads.near_contact_state(n, L, cfg.a, seed=21, frac=0.1)
    _, sp, th = workloads.initial_state(cfg)
    s = bd.System(bd.params_from_config(cfg), xy, sp, th, stream=stream())
    st = s.step(1)
    out = s.state()
    ref = ostep.step(xy, th, sp, 0, oracle_params(cfg, L), threads=max(1, os.cpu_count() or 1))
    assert not ref["rejected"] and ref["corr_iters"] >= 1
    err = float(np.max(np.abs(out["xy"] - ref["xy"])))
    assert err <= POS_TOL * cfg.a, err
    assert st["corr_iters"] == ref["corr_iters"]
    assert np.max(np.abs(out["theta"] - ref["theta"])) <= 1e-5
    assert np.array_equal(geometry.edges(out["tri"]), geometry.edges(ref["tris"]))
    assert len(cKDTree(out["xy"]).query_pairs(2 * cfg.a * (1 - 1e-12))) == 0
