"""GPU parity of the short-range path (Verlet lists + WCA/Yukawa force)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1703_02484_gb300 as bd  # noqa: E402
from paper_1703_02484_gb300 import workloads  # noqa: E402
from oracle import forces as oforces  # noqa: E402
from oracle import geometry, verlet  # noqa: E402
from oracle import step as ostep  # noqa: E402
from scipy.spatial import cKDTree  # noqa: E402

CFG = workloads.CONFIGS["c3"]


def stream():
    return torch.cuda.current_stream().cuda_stream


def rel_err(F, ref):
    scale = math.sqrt(float(np.mean(np.sum(ref ** 2, axis=1))))
    return float(np.max(np.linalg.norm(F - ref, axis=1))) / scale


def system(n, xy=None, skin=None, seed=2):
    L = workloads.box_side(n, CFG.rho)
    if xy is None:
        xy = workloads.initial_positions(n, L, 1.0, CFG.rho, seed)
    _, sp, th = workloads.initial_state(CFG, n=n)
    p = bd.params_from_config(CFG, n=n)
    if skin is not None:
        p.skin = skin
    return bd.System(p, xy, sp, th, stream=stream()), L, xy, sp, th


@pytest.mark.parametrize("n", [3000, 20000])
def test_verlet_lists_and_forces_match_oracle(n):
    s, L, xy, sp, th = system(n)
    F = s.forces()                          # first evaluation builds the lists
    grid = s.state(want_tri=False)["xy"]
    lists = s.neighbors()
    ref_lists = verlet.build(grid, CFG.r_cut, CFG.skin)
    for i in range(n):
        assert np.array_equal(lists[i], ref_lists[i]), i
    ref = oforces.short_range(grid, CFG.eps, CFG.kappa, 2.0, CFG.r_cut)
    assert rel_err(F, ref) <= 1e-5


def test_rebuild_trigger_and_lists_after_rebuild():
    n = 4000
    s, L, xy, sp, th = system(n, skin=0.04)
    s.forces()
    rebuilt = 0
    for _ in range(20):
        before = s.state(want_tri=False)["xy"]
        st = s.step(1)
        if st["verlet_rebuilds"]:
            rebuilt += 1
            lists = s.neighbors()
            ref_lists = verlet.build(before, CFG.r_cut, 0.04)
            for i in range(0, n, 3):
                assert np.array_equal(lists[i], ref_lists[i])
    assert rebuilt >= 2


def test_short_one_step_parity():
    n = 6000
    L = workloads.box_side(n, CFG.rho)
    xy = workloads.near_contact_state(n, L, 1.0, seed=5, rho=CFG.rho)
    s, L, _, sp, th = system(n, xy=xy)
    s.step(1)
    out = s.state()
    op = ostep.Params(L=L, a=1.0, law=CFG.law, eps=CFG.eps, kappa=CFG.kappa, r_cut=CFG.r_cut,
                      D=CFG.D, Dr=CFG.Dr, v0=CFG.v0, dt=CFG.dt, seed=CFG.seed)
    ref = ostep.step(xy, th, sp, 0, op)
    assert ref["corr_iters"] >= 1
    assert np.max(np.abs(out["xy"] - ref["xy"])) <= 1e-5
    assert np.array_equal(geometry.edges(out["tri"]), geometry.edges(ref["tris"]))


def test_full_size_c3_forces_sampled_and_steps():
    n = CFG.n
    s, L, xy, sp, th = system(n)
    F = s.forces()
    grid = s.state(want_tri=False)["xy"]
    rng = np.random.default_rng(1)
    idx = rng.choice(n, 2000, replace=False)
    tree = cKDTree(grid)
    pi, pj = [], []
    for i in idx:
        for j in tree.query_ball_point(grid[i], CFG.r_cut * (1 + 1e-9)):
            if j != i:
                pi.append(i)
                pj.append(j)
    ref = oforces.short_range_pairs(grid, np.array(pi), np.array(pj), CFG.eps, CFG.kappa, 2.0,
                                    CFG.r_cut)[idx]
    assert rel_err(F[idx], ref) <= 1e-5
    st = s.step(20)
    assert st["steps_done"] == 20
    out = s.state()
    assert len(cKDTree(out["xy"]).query_pairs(2.0 * (1 - 1e-12))) == 0
    assert np.array_equal(geometry.edges(out["tri"]), geometry.edges(geometry.delaunay(out["xy"], L)))


# ---- Algorithm 2 over the Verlet lists (the paper's short-range path) ----

def verlet_system(n, xy=None, seed=None):
    L = workloads.box_side(n, CFG.rho)
    if xy is None:
        xy, sp, th = workloads.initial_state(CFG, n=n)
    else:
        _, sp, th = workloads.initial_state(CFG, n=n)
    p = bd.params_from_config(CFG, n=n)
    p.overlap_mode = bd.OVERLAP_VERLET
    return bd.System(p, xy, sp, th, stream=stream()), L, xy, sp, th


@pytest.mark.parametrize("n,seed", [(3000, 7), (12000, 8)])
def test_verlet_correction_one_step_parity(n, seed):
    L = workloads.box_side(n, CFG.rho)
    xy = workloads.near_contact_state(n, L, 1.0, seed=seed, rho=CFG.rho)
    s, L, _, sp, th = verlet_system(n, xy=xy)
    st = s.step(1)
    out = s.state()
    assert out["n_tri"] == 0
    op = ostep.Params(L=L, a=1.0, law=CFG.law, eps=CFG.eps, kappa=CFG.kappa, r_cut=CFG.r_cut,
                      D=CFG.D, Dr=CFG.Dr, v0=CFG.v0, dt=CFG.dt, seed=CFG.seed)
    ref = ostep.step(xy, th, sp, 0, op, pairs_from="allpairs")
    assert ref["corr_iters"] >= 1 and not ref["rejected"]
    assert st["corr_iters"] == ref["corr_iters"]
    assert st["overlap_pairs"] == ref["overlap_pairs"]
    assert np.max(np.abs(out["xy"] - ref["xy"])) <= 1e-5
    assert len(cKDTree(out["xy"]).query_pairs(2.0 * (1 - 1e-12))) == 0


def test_verlet_correction_trajectory_state_parity():
    # a state reached on the GPU fed back as a new start: one more step on both sides
    n = 5000
    s, L, xy, sp, th = verlet_system(n)
    s.step(15)
    mid = s.state(want_tri=False)
    op = ostep.Params(L=L, a=1.0, law=CFG.law, eps=CFG.eps, kappa=CFG.kappa, r_cut=CFG.r_cut,
                      D=CFG.D, Dr=CFG.Dr, v0=CFG.v0, dt=CFG.dt, seed=CFG.seed)
    ref = ostep.step(mid["xy"], mid["theta"], mid["species"], mid["step"], op, pairs_from="allpairs")
    s.step(1)
    out = s.state(want_tri=False)
    assert np.max(np.abs(out["xy"] - ref["xy"])) <= 1e-5


def test_verlet_correction_full_size_steps():
    s, L, xy, sp, th = verlet_system(CFG.n)
    st = s.step(30)
    assert st["steps_done"] == 30 and st["rejected"] == 0
    out = s.state(want_tri=False)
    assert len(cKDTree(out["xy"]).query_pairs(2.0 * (1 - 1e-12))) == 0
    assert np.all(out["xy"] >= 1.0) and np.all(out["xy"] <= L - 1.0)


def test_verlet_mode_requires_short_range():
    cfg = workloads.CONFIGS["c2"]
    p = bd.params_from_config(cfg, n=500)
    p.overlap_mode = bd.OVERLAP_VERLET
    xy, sp, th = workloads.initial_state(cfg, n=500)
    with pytest.raises(bd.BDError) as e:
        bd.System(p, xy, sp, th, stream=stream())
    assert e.value.code == -10


@pytest.mark.parametrize("far", [False, True])
def test_verlet_set_state_checks_overlaps_on_the_device(far):
    # bd_set_state on a Verlet-list handle: the lists (rebuilt when a disk moved
    # more than skin/2 from where they were built) are scanned for pairs closer
    # than sigma; a good state is taken, an overlapping one rejected with the
    # previous state kept
    n = 4000
    s, L, xy, sp, th = verlet_system(n)
    s.step(3)
    before = s.state(want_tri=False)
    good = before["xy"].copy()
    if far:
        # one disk moved by more than skin/2 (0.3): the lists must be rebuilt
        dist, _ = cKDTree(good).query(good, k=2)
        for k in np.argsort(-dist[:, 1])[:20]:
            for step in ((0.45, 0.0), (-0.45, 0.0), (0.0, 0.45), (0.0, -0.45)):
                trial = good.copy()
                trial[k] += step
                if np.all(trial[k] >= 1.0) and np.all(trial[k] <= L - 1.0) and \
                        len(cKDTree(trial).query_pairs(2.0)) == 0:
                    good = trial
                    break
            else:
                continue
            break
        assert not np.array_equal(good, before["xy"])
    s.set_state(good)
    q, _ = s.geometry()
    got = s.state(want_tri=False)["xy"]
    assert np.max(np.abs(got - good)) <= q      # rounded to the position grid
    good = got
    dist, nb = cKDTree(good).query(good, k=2)
    i = int(np.argmin(dist[:, 1]))
    j = int(nb[i, 1])
    bad = good.copy()
    bad[j] = good[i] + 1.9 * (good[j] - good[i]) / np.linalg.norm(good[j] - good[i])
    with pytest.raises(bd.BDError) as e:
        s.set_state(bad)
    assert e.value.code == -3
    assert np.array_equal(s.state(want_tri=False)["xy"], good)
    st = s.step(5)
    assert st["steps_done"] == 5
    out = s.state(want_tri=False)
    assert len(cKDTree(out["xy"]).query_pairs(2.0 * (1 - 1e-12))) == 0
    s.close()


def test_one_step_parity_full_size_c3():
    # 2^20 disks at area fraction 0.5 (the paper's lattice start) with 5 % of
    # them moved next to a neighbour: one step of the short-range law with the
    # Delaunay overlap correction against the oracle's step
    n = CFG.n
    L = workloads.box_side(n, CFG.rho)
    xy = workloads.near_contact_state(n, L, CFG.a, seed=5, rho=CFG.rho, frac=0.05)
    _, sp, th = workloads.initial_state(CFG)
    s = bd.System(bd.params_from_config(CFG), xy, sp, th, stream=stream())
    st = s.step(1)
    out = s.state()
    op = ostep.Params(L=L, a=CFG.a, law=CFG.law, eps=CFG.eps, kappa=CFG.kappa, r_cut=CFG.r_cut, D=CFG.D,
                      Dr=CFG.Dr, v0=CFG.v0, dt=CFG.dt, seed=CFG.seed)
    import os
    ref = ostep.step(xy, th, sp, 0, op, threads=max(1, os.cpu_count() or 1))
    assert not ref["rejected"] and ref["corr_iters"] >= 1
    assert np.max(np.abs(out["xy"] - ref["xy"])) <= 1e-5 * CFG.a
    assert st["corr_iters"] == ref["corr_iters"]
    assert np.array_equal(geometry.edges(out["tri"]), geometry.edges(ref["tris"]))
