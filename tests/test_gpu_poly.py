"""GPU parity of polydisperse disks (Sec. 2.3's extension to radii that do not
differ too much) through the C ABI (bd_init_radii): short-range forces with
the mixed length scale, one step of each law and overlap mode against the
oracle's step, runs that never leave an overlapping pair, and the argument
checks (radius ratio above sqrt(2) with the Delaunay correction, radii
outside (0, a], overlapping starts)."""
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
from oracle import geometry, periodic  # noqa: E402
from oracle import step as ostep  # noqa: E402
from scipy.spatial import cKDTree  # noqa: E402

POS_TOL = 1e-5
ALPHA = (0.05, 0.2, -0.1, 0.05)


def stream():
    return torch.cuda.current_stream().cuda_stream


def overlaps(xy, radii, L=None):
    if L is not None:
        return len(periodic.close_pairs(xy, 2.0 * float(radii.max()), L, radii=radii))
    n = 0
    for i, j in cKDTree(xy).query_pairs(2.0 * float(radii.max())):
        if math.hypot(*(xy[j] - xy[i])) < radii[i] + radii[j]:
            n += 1
    return n


def setup(n, ratio, seed, law, rho=0.3, near=0.3, periodic_box=False, verlet=False, dt=None):
    radii = workloads.poly_radii(n, 1.0, ratio, seed)
    L = workloads.box_side(n, rho)
    xy = workloads.poly_positions(radii, L, seed, near_frac=near)
    sp = (np.arange(n) % 2).astype(np.uint8)
    th = workloads.initial_state(workloads.CONFIGS["c2"], n=n)[2]
    short = law == bd.LAW_SHORT
    p = bd.make_params(n, L=L, a=1.0, law=law, alpha=ALPHA, n_species=2, D=1.0, Dr=0.5 if not short else 0.2,
                       v0=1.0 if not short else 0.5, dt=(dt or (1e-4 if not short else 5e-5)), seed=seed,
                       boundary=bd.BOUNDARY_PERIODIC if periodic_box else bd.BOUNDARY_WALLS)
    if verlet:
        p.overlap_mode = bd.OVERLAP_VERLET
    op = ostep.Params(L=float(np.float32(L)) if periodic_box else L, a=1.0, law=law, alpha=ALPHA, eps=p.eps,
                      kappa=p.kappa, r_cut=p.r_cut, D=p.D, Dr=p.Dr, v0=p.v0, dt=p.dt, seed=seed,
                      periodic=periodic_box, radii=radii)
    return radii, L, xy, sp, th, p, op


def test_short_range_forces_mix_radii():
    radii, L, xy, sp, th, p, op = setup(3000, 1.6, 1, bd.LAW_SHORT, rho=0.45, near=0.2, verlet=True)
    s = bd.System(p, xy, sp, th, stream=stream(), radii=radii)
    F = s.forces()
    grid = s.state(want_tri=False)["xy"]
    ref = oforces.short_range(grid, p.eps, p.kappa, 2.0, p.r_cut, radii=radii)
    scale = math.sqrt(float(np.mean(np.sum(ref ** 2, axis=1))))
    assert float(np.max(np.linalg.norm(F - ref, axis=1))) / scale <= 1e-5


@pytest.mark.parametrize("law,ratio,seed", [(bd.LAW_LONG, 1.35, 2), (bd.LAW_SHORT, 1.4, 3), (bd.LAW_NONE, 1.41, 4)])
def test_one_step_parity_delaunay(law, ratio, seed):
    radii, L, xy, sp, th, p, op = setup(4000, ratio, seed, law)
    s = bd.System(p, xy, sp, th, stream=stream(), radii=radii)
    st = s.step(1)
    out = s.state()
    ref = ostep.step(xy, th, sp, 0, op, threads=max(1, os.cpu_count() or 1))
    assert not ref["rejected"] and ref["corr_iters"] >= 1
    assert np.max(np.abs(out["xy"] - ref["xy"])) <= POS_TOL
    assert st["corr_iters"] == ref["corr_iters"]
    assert np.array_equal(geometry.edges(out["tri"]), geometry.edges(ref["tris"]))
    assert overlaps(out["xy"], radii) == 0


def test_one_step_parity_verlet_wide_ratio():
    # the Verlet-list correction tests every listed pair: radii ratio 2 is allowed
    radii, L, xy, sp, th, p, op = setup(5000, 2.0, 5, bd.LAW_SHORT, rho=0.4, verlet=True)
    s = bd.System(p, xy, sp, th, stream=stream(), radii=radii)
    st = s.step(1)
    out = s.state(want_tri=False)
    ref = ostep.step(xy, th, sp, 0, op, pairs_from="allpairs")
    assert not ref["rejected"] and ref["corr_iters"] >= 1
    assert np.max(np.abs(out["xy"] - ref["xy"])) <= POS_TOL
    assert st["corr_iters"] == ref["corr_iters"]
    assert overlaps(out["xy"], radii) == 0


def test_one_step_parity_periodic():
    radii, L, xy, sp, th, p, op = setup(3000, 1.3, 6, bd.LAW_LONG, periodic_box=True)
    s = bd.System(p, xy, sp, th, stream=stream(), radii=radii)
    st = s.step(1)
    out = s.state()
    ref = ostep.step(xy, th, sp, 0, op)
    assert not ref["rejected"] and ref["corr_iters"] >= 1
    d = out["xy"] - ref["xy"]
    d -= s.L * np.round(d / s.L)
    assert np.max(np.abs(d)) <= POS_TOL
    assert st["corr_iters"] == ref["corr_iters"]
    assert overlaps(out["xy"], radii, s.L) == 0


@pytest.mark.parametrize("law", [bd.LAW_LONG, bd.LAW_SHORT])
def test_runs_keep_every_pair_apart(law):
    radii, L, xy, sp, th, p, op = setup(6000, 1.41, 7, law, rho=0.35, dt=1e-3)
    s = bd.System(p, xy, sp, th, stream=stream(), radii=radii)
    for _ in range(5):
        st = s.step(10)
        assert st["steps_done"] == 10
        out = s.state()
        assert overlaps(out["xy"], radii) == 0
        assert np.all(out["xy"] >= radii[:, None] - 1e-9) and np.all(out["xy"] <= L - radii[:, None] + 1e-9)
        assert np.array_equal(geometry.edges(out["tri"]), geometry.edges(geometry.delaunay(out["xy"], L, 1.0)))


def test_set_state_checks_own_radii():
    radii, L, xy, sp, th, p, op = setup(2000, 1.3, 8, bd.LAW_NONE, near=0.0)
    s = bd.System(p, xy, sp, th, stream=stream(), radii=radii)
    cur = s.state()["xy"]
    tree = cKDTree(cur)
    # a disk smaller than the largest radius, near the left wall: moved to just
    # over its own radius from the wall (closer than the largest radius a = 1)
    cand = [i for i in np.argsort(cur[:, 0] - radii) if radii[i] < 0.95 and cur[i, 0] - radii[i] < 0.6]
    moved_one = False
    for i in cand[:20]:
        trial = cur.copy()
        trial[i, 0] = radii[i] + 1e-6
        nb = [j for j in tree.query_ball_point(trial[i], 2.5) if j != i]
        if any(math.hypot(*(trial[j] - trial[i])) < radii[i] + radii[j] + 1e-3 for j in nb):
            continue
        s.set_state(trial)
        assert abs(s.state()["xy"][i, 0] - trial[i, 0]) <= 1e-9 and trial[i, 0] < 1.0
        cur = trial
        moved_one = True
        # ... but not closer than its own radius
        bad = trial.copy()
        bad[i, 0] = radii[i] - 0.01
        with pytest.raises(bd.BDError) as e:
            s.set_state(bad)
        assert e.value.code == -3
        assert abs(s.state()["xy"][i, 0] - trial[i, 0]) <= 1e-9   # the state kept
        break
    assert moved_one


def test_arguments():
    radii, L, xy, sp, th, p, op = setup(500, 1.3, 9, bd.LAW_LONG)
    wide = radii.copy()
    wide[0] = 0.6                   # ratio 1.67 > sqrt(2) with the Delaunay correction
    with pytest.raises(bd.BDError) as e:
        bd.System(p, xy, sp, th, stream=stream(), radii=wide)
    assert e.value.code == -10
    big = radii.copy()
    big[3] = 1.01                   # above the largest radius a
    with pytest.raises(bd.BDError) as e:
        bd.System(p, xy, sp, th, stream=stream(), radii=big)
    assert e.value.code == -1
    touch = xy.copy()
    touch[1] = touch[0] + [radii[0] + radii[1] - 1e-3, 0.0]
    with pytest.raises(bd.BDError) as e:
        bd.System(p, touch, sp, th, stream=stream(), radii=radii)
    assert e.value.code in (-3,)
    s = bd.System(p, xy, sp, th, stream=stream(), radii=radii)
    with pytest.raises(bd.BDError) as e:
        s.rollout(3)
    assert e.value.code == -10
