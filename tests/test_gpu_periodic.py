"""GPU parity of the periodic box (Sec. 2.1: minimum image, re-entry at the
opposite side; Sec. 4.1: the triangulation of the flat torus) through the C
ABI (bd_params.boundary = BD_BOUNDARY_PERIODIC), against the FP64 oracle.

Starts are RSA configurations translated by a seeded offset modulo L, so that
disks, pairs and triangles straddle the box edges.  Tolerances as for walls:
forces within 1e-5 of the RMS force, positions within 1e-5 a after a step,
the torus edge set (vertex pairs with their image shifts) exact."""
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
from oracle import periodic, verlet  # noqa: E402
from oracle import step as ostep  # noqa: E402

POS_TOL = 1e-5
FORCE_TOL = 1e-5
C2 = workloads.CONFIGS["c2"]
C3 = workloads.CONFIGS["c3"]


def stream():
    return torch.cuda.current_stream().cuda_stream


def start(n, rho, seed, near_contact=False):
    L = float(np.float32(workloads.box_side(n, rho)))
    if near_contact:
        xy = workloads.near_contact_state(n, L, 1.0, seed=seed, rho=rho)
    else:
        xy = workloads.initial_positions(n, L, 1.0, rho, seed=seed)
    off = np.random.default_rng(seed + 1000).uniform(0, L, 2)
    return periodic.wrap(xy + off, L), L


def system(cfg, xy, L, sp, th, precision=None, v0=None):
    p = bd.make_params(len(xy), L=L, a=cfg.a, law=cfg.law, alpha=cfg.alpha, n_species=cfg.n_species,
                       eps=cfg.eps, kappa=cfg.kappa, r_cut=cfg.r_cut, skin=cfg.skin, D=cfg.D, Dr=cfg.Dr,
                       v0=cfg.v0 if v0 is None else v0, dt=cfg.dt, seed=cfg.seed,
                       precision=cfg.precision if precision is None else precision,
                       boundary=bd.BOUNDARY_PERIODIC)
    return bd.System(p, xy, sp, th, stream=stream())


def oparams(cfg, L, **kw):
    return ostep.Params(L=L, a=cfg.a, law=cfg.law, alpha=cfg.alpha, eps=cfg.eps, kappa=cfg.kappa,
                        r_cut=cfg.r_cut, D=cfg.D, Dr=cfg.Dr, v0=cfg.v0, dt=cfg.dt, seed=cfg.seed,
                        periodic=True, **kw)


def species_theta(n, seed):
    rng = np.random.default_rng(seed)
    sp = rng.permutation(np.arange(n) % 2).astype(np.uint8)
    th = rng.uniform(0, 2 * math.pi, n).astype(np.float32)
    return sp, th


def rel_force_error(F, ref, allow=None):
    """Largest per-disk force error over the RMS force; with allow (per disk),
    the part of each error within its minimum-image allowance is forgiven."""
    scale = math.sqrt(float(np.mean(np.sum(ref ** 2, axis=1))))
    e = np.linalg.norm(F - ref, axis=1)
    if allow is not None:
        e = np.maximum(0.0, e - allow)
    return float(np.max(e)) / scale


def image_allowance(xy, sp, A, L):
    """Per disk, the force change of its pairs whose minimum image is ambiguous
    at FP32 resolution.  A pair component within delta = 4 ulp_FP32(L) of L/2
    sits at the discontinuity of the minimum-image convention (Sec. 2.1): FP32
    coordinates cannot tell the two images apart there, and either is a valid
    evaluation.  Found by sorting on each coordinate (no O(N^2) pass)."""
    xy = np.asarray(xy, dtype=np.float64)
    n = len(xy)
    T = oforces.species_table(A)
    delta = 4.0 * float(np.spacing(np.float32(L)))
    out = np.zeros(n)
    for c in (0, 1):
        order = np.argsort(xy[:, c])
        xs = xy[order, c]
        for sgn in (1.0, -1.0):
            # partners at x_i + sgn L/2 (mod L), within delta
            tgt = np.mod(xy[:, c] + sgn * L / 2.0, L)
            cand = [[] for _ in range(n)]
            for shift in (0.0, -L, L):     # windows that cross 0 or L
                lo = np.searchsorted(xs, tgt + shift - delta)
                hi = np.searchsorted(xs, tgt + shift + delta)
                for i in np.nonzero(hi > lo)[0]:
                    cand[i].extend(order[lo[i]:hi[i]].tolist())
            for i in range(n):
                for j in set(cand[i]):
                    if j == i:
                        continue
                    d = xy[j] - xy[i]
                    d = d - L * np.rint(d / L)
                    alt = d.copy()
                    alt[c] = d[c] - L * np.sign(d[c])
                    f = lambda v: v / np.linalg.norm(v) ** 3    # noqa: E731
                    out[i] += abs(T[sp[i], sp[j]]) * np.linalg.norm(f(alt) - f(d))
    return out


def gpu_keys(s):
    st = s.state()
    return periodic.edge_keys(st["tri"].astype(np.int64), s.tri_shifts()), st


@pytest.mark.parametrize("n,precision", [(3001, 0), (1500, 1), (700, 0)])
def test_long_range_forces_minimum_image(n, precision):
    xy, L = start(n, C2.rho, seed=n)
    sp, th = species_theta(n, 1)
    s = system(C2, xy, L, sp, th, precision=precision)
    F = s.forces()
    grid = s.state(want_tri=False)["xy"]
    ref = oforces.long_range_numpy(grid, sp, C2.alpha, L=L)
    err = rel_force_error(F, ref, None if precision else image_allowance(grid, sp, C2.alpha, L))
    assert err <= (1e-12 if precision else FORCE_TOL), err
    s.close()


@pytest.mark.parametrize("variant,tiles", [(0, 3), (2, 1), (2, 5), (3, 2), (3, 7)])
@pytest.mark.parametrize("n", [700, 3001])
def test_long_range_force_variants_periodic(monkeypatch, variant, tiles, n):
    # the one-sided sweep and the symmetric sweep's periodic form (minimum
    # images; at n = 700 the box is small, so most tiles take the per-pair
    # minimum image, with and without inert slots), at the start and after
    # steps in which disks re-entered across the edges
    monkeypatch.setenv("BD_FORCE_VARIANT", str(variant))
    monkeypatch.setenv("BD_FORCE_TILES", str(tiles))
    xy, L = start(n, C2.rho, seed=n + 11)
    sp, th = species_theta(n, 3)
    s = system(C2, xy, L, sp, th)
    assert s.tuning()["variant"] == variant and s.tuning()["tiles_per_item"] == tiles
    for k in range(2):
        F = s.forces()
        grid = s.state(want_tri=False)["xy"]
        err = rel_force_error(F, oforces.long_range_numpy(grid, sp, C2.alpha, L=L),
                              image_allowance(grid, sp, C2.alpha, L))
        assert err <= FORCE_TOL, (k, err)
        assert np.array_equal(s.forces(), F)
        s.step(40)
    s.close()


def test_long_range_forces_periodic_full_size_every_disk(monkeypatch):
    # N = 1e5 in a periodic box, the symmetric sweep's periodic form, every
    # disk against the oracle's C loop
    monkeypatch.setenv("BD_FORCE_VARIANT", "3")
    monkeypatch.setenv("BD_FORCE_TILES", "2")
    cfg = workloads.CONFIGS["n1e5"]
    xy, sp, th = workloads.initial_state(cfg)
    L = float(np.float32(cfg.L))
    p = bd.params_from_config(cfg)
    p.box_L = L
    p.boundary = bd.BOUNDARY_PERIODIC
    s = bd.System(p, xy, sp, th, stream=torch.cuda.current_stream().cuda_stream)
    F = s.forces()
    grid = s.state(want_tri=False)["xy"]
    ref = oforces.long_range(grid, sp, cfg.alpha, threads=max(1, min(16, os.cpu_count() or 1)), L=L)
    assert rel_force_error(F, ref, image_allowance(grid, sp, cfg.alpha, L)) <= FORCE_TOL
    s.close()


def test_torus_triangulation_at_init_and_after_steps():
    n = 2000
    xy, L = start(n, C2.rho, seed=5)
    sp, th = species_theta(n, 2)
    s = system(C2, xy, L, sp, th)
    keys, st = gpu_keys(s)
    assert st["n_tri"] == 2 * n
    assert np.array_equal(keys, periodic.edge_keys(*periodic.delaunay_torus(st["xy"], L)))
    for _ in range(5):
        s.step(20)
        keys, st = gpu_keys(s)
        x = st["xy"]
        assert np.all((x >= 0) & (x < L))
        assert len(periodic.close_pairs(x, 2.0, L)) == 0
        assert np.array_equal(keys, periodic.edge_keys(*periodic.delaunay_torus(x, L)))
    s.close()


@pytest.mark.parametrize("n,seed", [(1200, 3), (4000, 4)])
def test_one_step_parity_long_range(n, seed):
    xy, L = start(n, 0.35, seed=seed, near_contact=True)
    sp, th = species_theta(n, seed)
    s = system(C2, xy, L, sp, th)
    x0 = s.state(want_tri=False)["xy"]
    st = s.step(1)
    keys, out = gpu_keys(s)
    ref = ostep.step(x0, th.astype(np.float64), sp, 0, oparams(C2, L))
    assert not ref["rejected"] and ref["corr_iters"] >= 1
    assert st["corr_iters"] == ref["corr_iters"]
    err = float(np.max(np.abs(periodic.min_image(out["xy"] - ref["xy"], L))))
    assert err <= POS_TOL, err
    assert float(np.max(np.abs(out["theta"] - ref["theta"]))) <= 1e-5
    assert np.array_equal(keys, periodic.edge_keys(*periodic.delaunay_torus(out["xy"], L)))
    assert np.array_equal(keys, periodic.edge_keys(*ref["tris"]))
    s.close()


def test_trajectory_crosses_the_edges():
    # strong self-propulsion drives disks across the box edges many times;
    # every 10 steps the GPU state is fed to the oracle for one step
    n = 800
    xy, L = start(n, 0.3, seed=9)
    sp, th = species_theta(n, 9)
    cfg = C2
    s = system(cfg, xy, L, sp, th, v0=500.0)
    p = oparams(cfg, L)
    p.v0 = 500.0
    for k in range(6):
        s.step(10)
        before = s.state(want_tri=False)
        s.step(1)
        keys, after = gpu_keys(s)
        ref = ostep.step(before["xy"], before["theta"].astype(np.float64), sp, before["step"], p)
        assert not ref["rejected"]
        assert float(np.max(np.abs(periodic.min_image(after["xy"] - ref["xy"], L)))) <= POS_TOL
        assert np.array_equal(keys, periodic.edge_keys(*periodic.delaunay_torus(after["xy"], L)))
    s.close()


def test_short_range_lists_forces_and_step():
    n = 6000
    xy, L = start(n, C3.rho, seed=11)
    sp = np.zeros(n, np.uint8)
    th = np.random.default_rng(11).uniform(0, 2 * math.pi, n).astype(np.float32)
    s = system(C3, xy, L, sp, th)
    F = s.forces()
    grid = s.state(want_tri=False)["xy"]
    lists = s.neighbors()
    ref_lists = verlet.build(grid, C3.r_cut, C3.skin, L=L)
    for i in range(0, n, 5):
        assert np.array_equal(np.sort([int(v) for v in lists[i]]), ref_lists[i])
    ref = oforces.short_range(grid, C3.eps, C3.kappa, 2.0, C3.r_cut, L=L)
    assert rel_force_error(F, ref) <= FORCE_TOL
    # one step from a near-contact start
    xy2, _ = start(n, C3.rho, seed=12, near_contact=True)
    s2 = system(C3, xy2, L, sp, th)
    x0 = s2.state(want_tri=False)["xy"]
    st = s2.step(1)
    keys, out = gpu_keys(s2)
    r = ostep.step(x0, th.astype(np.float64), sp, 0, oparams(C3, L))
    assert not r["rejected"] and st["corr_iters"] == r["corr_iters"]
    assert float(np.max(np.abs(periodic.min_image(out["xy"] - r["xy"], L)))) <= POS_TOL
    assert np.array_equal(keys, periodic.edge_keys(*r["tris"]))
    s.close()
    s2.close()


def test_verlet_list_correction_periodic():
    n = 5000
    xy, L = start(n, C3.rho, seed=13, near_contact=True)
    sp = np.zeros(n, np.uint8)
    th = np.random.default_rng(13).uniform(0, 2 * math.pi, n).astype(np.float32)
    p = bd.make_params(n, L=L, law=C3.law, eps=C3.eps, kappa=C3.kappa, r_cut=C3.r_cut, skin=C3.skin,
                       D=C3.D, Dr=C3.Dr, v0=C3.v0, dt=C3.dt, seed=C3.seed, boundary=bd.BOUNDARY_PERIODIC)
    p.overlap_mode = bd.OVERLAP_VERLET
    s = bd.System(p, xy, sp, th, stream=stream())
    x0 = s.state(want_tri=False)["xy"]
    st = s.step(1)
    out = s.state(want_tri=False)
    r = ostep.step(x0, th.astype(np.float64), sp, 0, oparams(C3, L), pairs_from="allpairs")
    assert not r["rejected"] and st["corr_iters"] == r["corr_iters"] >= 1
    assert float(np.max(np.abs(periodic.min_image(out["xy"] - r["xy"], L)))) <= POS_TOL
    assert len(periodic.close_pairs(out["xy"], 2.0, L)) == 0
    s.close()


def test_set_state_across_the_edge_repairs_the_torus_triangulation():
    n = 1000
    xy, L = start(n, 0.3, seed=15)
    sp, th = species_theta(n, 15)
    s = system(C2, xy, L, sp, th)
    cur = s.state(want_tri=False)["xy"]
    # move every disk by a small random step; many cross an edge
    new = cur + np.random.default_rng(3).normal(0, 0.05, cur.shape)
    for _ in range(100):
        bad = periodic.close_pairs(periodic.wrap(new, L), 2.0, L)
        if len(bad) == 0:
            break
        new[bad[:, 0]] = cur[bad[:, 0]]      # both ends back where they were (no overlap there)
        new[bad[:, 1]] = cur[bad[:, 1]]
    # disks just right of x = 0 step across it (they re-enter at the right edge)
    crossed = 0
    for i in np.nonzero(cur[:, 0] < 0.5)[0]:
        trial = new.copy()
        trial[i] = [-0.02, cur[i, 1]]
        if len(periodic.close_pairs(periodic.wrap(trial, L), 2.0, L)) == 0:
            new, crossed = trial, crossed + 1
    assert crossed >= 1
    s.set_state(new)
    keys, st = gpu_keys(s)
    x = st["xy"]
    assert np.max(np.abs(periodic.min_image(x - new, L))) <= 1e-9
    assert np.all((x >= 0) & (x < L))
    assert np.array_equal(keys, periodic.edge_keys(*periodic.delaunay_torus(x, L)))
    s.close()


def test_periodic_argument_errors():
    xy, L = start(10, 0.3, seed=1)
    with pytest.raises(bd.BDError) as e:
        system(C2, xy, L, np.zeros(10, np.uint8), np.zeros(10, np.float32))
    assert e.value.code == -10
    n = 500
    xy, L = start(n, 0.3, seed=2)
    s = system(C2, xy, L, np.zeros(n, np.uint8), np.zeros(n, np.float32))
    with pytest.raises(bd.BDError) as e:
        s.rollout(2)
    assert e.value.code == -10
    s.close()
