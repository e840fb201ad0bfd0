"""GPU tests of the triangulation repair (Sec. 4.3), the predicates' FP32
filters near degeneracy, and the device loops' error exits, through the C ABI.

* Inverted triangles: Fig. 5's move (one repair flip, then Lawson flips to the
  Delaunay triangulation), Fig. 6's move (two crossed edges: the predicate
  finds no repair flip, the move is reverted), and noisy steps large enough to
  invert triangles, each step compared with the oracle's.
* Near-degenerate inputs: vertices moved to within 1e-9 of the line through
  two neighbours, and points on a circle perturbed by 1e-9 .. 1e-6; the
  device's triangulation must equal the oracle's exact Delaunay triangulation,
  and the count of tests the FP32 filters left to the exact path shows which
  side of the filter each case fell on.
* Error exits: a correction-pass cap, a flip-round cap and a timed-out grid
  barrier (a barrier made to wait for one block more than the launch has)
  each return their status, leave the state of the step's start, and the
  handle steps normally afterwards.
"""
from dataclasses import replace

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1703_02484_gb300 as bd  # noqa: E402
from paper_1703_02484_gb300 import workloads  # noqa: E402
from oracle import geometry, overlap  # noqa: E402
from oracle import step as ostep  # noqa: E402
from scipy.spatial import cKDTree  # noqa: E402

POS_TOL = 1e-5


def stream():
    return torch.cuda.current_stream().cuda_stream


def oracle_params(cfg, L, dt=None):
    return ostep.Params(L=L, a=cfg.a, law=cfg.law, alpha=cfg.alpha, eps=cfg.eps, kappa=cfg.kappa,
                        r_cut=cfg.r_cut, D=cfg.D, Dr=cfg.Dr, v0=cfg.v0,
                        dt=cfg.dt if dt is None else dt, seed=cfg.seed)


def edges_of(tri):
    return geometry.edges(np.asarray(tri))


def no_overlap(xy, a):
    return len(cKDTree(xy).query_pairs(2 * a * (1 - 1e-12))) == 0


# ---------------------------------------------------------------- radius a != 1

def test_radius_half_one_step_parity():
    # the ghost ring, the overlap distance and the triangulation all follow a
    cfg = replace(workloads.CONFIGS["c2"], a=0.5)
    n = 3000
    L = workloads.box_side(n, cfg.rho, cfg.a)
    xy = workloads.near_contact_state(n, L, cfg.a, seed=6)
    _, sp, th = workloads.initial_state(cfg, n=n)
    p = bd.params_from_config(cfg, n=n)
    p.box_L = L
    s = bd.System(p, xy, sp, th, stream=stream())
    assert s.L == pytest.approx(L, rel=1e-15)
    st = s.step(1)
    out = s.state()
    ref = ostep.step(xy, th, sp, 0, oracle_params(cfg, L))
    assert not ref["rejected"] and ref["corr_iters"] >= 1
    assert np.max(np.abs(out["xy"] - ref["xy"])) <= POS_TOL * cfg.a
    assert st["corr_iters"] == ref["corr_iters"]
    assert np.array_equal(edges_of(out["tri"]), edges_of(ref["tris"]))
    assert np.array_equal(edges_of(out["tri"]), edges_of(geometry.delaunay(out["xy"], L, cfg.a)))
    assert no_overlap(out["xy"], cfg.a)


# ---------------------------------------------------------- Figs. 5 and 6

def _figure_system(points, a=0.25, L=30.0, offset=10.0):
    xy = np.array(points, dtype=np.float64) + offset
    p = bd.make_params(len(xy), L=L, a=a)
    return bd.System(p, xy, stream=stream()), xy


def test_fig5_inverted_triangle_repaired_on_device(golden):
    g = golden("fig5_one_flip.json")
    names = list(g["points"])
    s, xy = _figure_system([g["points"][k] for k in names])
    L, a = s.L, 0.25
    moved = xy.copy()
    moved[names.index("b")] = np.array(g["b_moved"], dtype=np.float64) + 10.0
    s.set_state(moved)
    st = s.last_stats()
    # the move inverts triangle (b, c, d); one repair flip (edge cd -> ab)
    # removes it, Lawson flips finish the Delaunay triangulation
    assert st["inverted"] >= 1 and st["repair_flips"] >= 1, st
    out = s.state()
    assert np.array_equal(out["xy"], moved)
    assert np.array_equal(edges_of(out["tri"]), edges_of(geometry.delaunay(moved, L, a)))
    # the disks' own triangles are the figure's final ones
    real = {frozenset(t) for t in out["tri"].tolist() if max(t) < len(xy)}
    want = {frozenset(names.index(v) for v in t) for t in g["final_triangles"]}
    assert want <= real
    print("fig5:", {k: st[k] for k in ("inverted", "repair_flips", "flips", "exact_tests")})


def test_fig6_two_crossings_reverted_on_device(golden):
    # f crosses two edges: the predicate finds no repair flip, so the move is
    # detected and reverted (Sec. 4.3, Fig. 6)
    g = golden("fig6_two_flips.json")
    names = list(g["points"])
    s, xy = _figure_system([g["points"][k] for k in names])
    before = s.state()
    moved = xy.copy()
    moved[names.index("f")] = np.array(g["f_moved"], dtype=np.float64) + 10.0
    with pytest.raises(bd.BDError) as e:
        s.set_state(moved)
    assert e.value.code == -4
    st = s.last_stats()
    assert st["inverted"] >= 1 and st["fail_phase"] == 2 and st["repair_flips"] == 0, st
    after = s.state()
    assert np.array_equal(after["xy"], before["xy"])
    assert np.array_equal(after["tri"], before["tri"])
    # a shorter move of f, across edge be only (be meets y = 0 at x = 3.5, ce
    # at x = 4.5), is repaired by one flip
    ok = xy.copy()
    ok[names.index("f")] = np.array([4.0, 0.0]) + 10.0
    s.set_state(ok)
    st = s.last_stats()
    assert st["inverted"] >= 1 and st["repair_flips"] >= 1, st
    assert np.array_equal(edges_of(s.state()["tri"]), edges_of(geometry.delaunay(ok, s.L, 0.25)))


def _noisy_case(rho, dt, seed):
    # sparse starts have slivers; large steps invert some of them
    cfg = replace(workloads.CONFIGS["c2"], rho=rho, dt=dt)
    n = 3000
    L = workloads.box_side(n, rho)
    xy = workloads.initial_positions(n, L, cfg.a, rho, seed)
    _, sp, th = workloads.initial_state(cfg, n=n)
    p = bd.params_from_config(cfg, n=n)
    s = bd.System(p, xy, sp, th, stream=stream())
    before = s.state()
    st, code = s.step(1, raise_on_error=False)
    ref = ostep.step(xy, th, sp, 0, oracle_params(cfg, L))
    out = s.state()
    print("rho %.2f dt %.2f seed %d:" % (rho, dt, seed), {k: st[k] for k in
          ("inverted", "repair_flips", "flips", "corr_iters", "fail_phase", "exact_tests")}, "oracle rejected",
          ref["rejected"])
    if code == 0:
        assert not ref["rejected"]
        assert np.max(np.abs(out["xy"] - ref["xy"])) <= POS_TOL * cfg.a
        assert st["corr_iters"] == ref["corr_iters"]
        assert np.array_equal(edges_of(out["tri"]), edges_of(ref["tris"]))
        assert no_overlap(out["xy"], cfg.a)
    else:
        # a reversal (Sec. 4.3 first criterion, which the oracle shares) or an
        # inversion the predicate cannot repair: the step is undone
        assert code == -4 and st["fail_phase"] in (1, 2, 3)
        if st["fail_phase"] == 1:
            assert ref["rejected"]
        assert np.array_equal(out["xy"], before["xy"]) and np.array_equal(out["tri"], before["tri"])
    return st, code


def test_noisy_steps_that_invert_triangles_match_oracle():
    # each step against the oracle's; across the cases, inverted triangles
    # were met and repaired in steps that completed
    repaired = 0
    for rho, dt, seed in [(0.05, 0.1, 1), (0.02, 0.1, 3), (0.02, 0.12, 4), (0.05, 0.1, 7)]:
        st, code = _noisy_case(rho, dt, seed)
        if code == 0 and st["inverted"] > 0 and st["repair_flips"] > 0:
            repaired += 1
    assert repaired >= 2


# ------------------------------------------------- predicates near degeneracy

def _collinear_moves(xy, tri, n, q, delta, rng, want=40):
    """Move vertex v of far-apart triangles (u, v, w) onto the line through u
    and w (its midpoint, offset by delta along the normal toward v; delta = 0
    exactly on the line in grid units).  Skips a move that overlaps a disk or
    reverses a triangulation edge (Sec. 4.3 first criterion, exact)."""
    moved = xy.copy()
    used = np.zeros(n, bool)
    E = overlap.real_edges(tri, n)
    tree = cKDTree(xy)
    count = 0
    for t in rng.permutation(len(tri)):
        if count >= want:
            break
        tt = tri[t]
        if max(tt) >= n:
            continue
        for k in range(3):
            v, u, w = int(tt[k]), int(tt[(k + 1) % 3]), int(tt[(k + 2) % 3])
            if np.hypot(*(xy[w] - xy[u])) < 4.6:
                continue
            if used[[u, v, w]].any():
                continue
            near = tree.query_ball_point(xy[v], 12.0)
            if used[near].any():
                continue
            U = np.rint(xy[u] / q).astype(np.int64)
            W = np.rint(xy[w] / q).astype(np.int64)
            if delta == 0.0:
                if np.any((W - U) % 2):
                    continue
                m = ((U + W) // 2).astype(np.float64) * q
            else:
                d = xy[w] - xy[u]
                nrm = np.array([-d[1], d[0]]) / np.hypot(*d)
                if np.dot(xy[v] - xy[u], nrm) < 0:
                    nrm = -nrm
                m = 0.5 * (xy[u] + xy[w]) + delta * nrm
            trial = moved.copy()
            trial[v] = m
            nb = [j for j in tree.query_ball_point(m, 2.0 * 1.001) if j != v]
            if nb:
                continue
            if len(overlap.reversed_edges(moved, trial, E)):
                continue
            moved = trial
            used[near] = True
            count += 1
            break
    return moved, count


@pytest.mark.parametrize("delta", [0.0, 1e-9, -1e-9, 1e-7, -1e-7])
def test_near_collinear_moves_decided_exactly(delta):
    cfg = workloads.CONFIGS["c5"]
    n = 2500
    xy0, sp, th = workloads.initial_state(cfg, n=n)
    p = bd.params_from_config(cfg, n=n)
    p.law = bd.LAW_NONE
    s = bd.System(p, xy0, sp, th, stream=stream())
    q, L = s.geometry()
    start = s.state()
    moved, count = _collinear_moves(start["xy"], start["tri"], n, q, delta, np.random.default_rng(11))
    assert count >= 10
    code = 0
    try:
        s.set_state(moved)
    except bd.BDError as e:
        code = e.code
    st = s.last_stats()
    print("delta %g: %d moves" % (delta, count), {k: st[k] for k in
          ("inverted", "repair_flips", "flips", "exact_tests", "fail_phase")})
    # every orientation test of a flattened triangle is inside the filter's bound
    assert st["exact_tests"] >= count
    if code == 0:
        out = s.state()
        # positions are rounded to the grid (q); the oracle triangulates those
        assert np.max(np.abs(out["xy"] - moved)) <= q
        assert np.array_equal(edges_of(out["tri"]), edges_of(geometry.delaunay(out["xy"], L, cfg.a)))
    else:
        # an inversion the predicate cannot repair (Fig. 6's case) is reverted
        assert code == -4 and st["fail_phase"] in (2, 3)
        out = s.state()
        assert np.array_equal(out["xy"], start["xy"]) and np.array_equal(out["tri"], start["tri"])
    if delta < 0:
        # v crossed the line: the flattened triangles inverted
        assert st["inverted"] >= count


def test_clear_moves_decided_by_filter():
    # the same kind of moves kept 0.05 off the line: the filters decide them
    cfg = workloads.CONFIGS["c5"]
    n = 2500
    xy0, sp, th = workloads.initial_state(cfg, n=n)
    p = bd.params_from_config(cfg, n=n)
    p.law = bd.LAW_NONE
    s = bd.System(p, xy0, sp, th, stream=stream())
    q, L = s.geometry()
    start = s.state()
    moved, count = _collinear_moves(start["xy"], start["tri"], n, q, 0.05, np.random.default_rng(11))
    assert count >= 10
    s.set_state(moved)
    st = s.last_stats()
    assert st["exact_tests"] == 0, st
    out = s.state()
    assert np.max(np.abs(out["xy"] - moved)) <= q
    assert np.array_equal(edges_of(out["tri"]), edges_of(geometry.delaunay(out["xy"], L, cfg.a)))


def _ring(nring, R, c, scale, rng):
    th = 2 * np.pi * np.arange(nring) / nring
    d = rng.uniform(-1, 1, nring) * 10.0 ** rng.uniform(np.log10(scale[0]), np.log10(scale[1]), nring)
    return np.stack([c + (R + d) * np.cos(th), c + (R + d) * np.sin(th)], axis=1)


@pytest.mark.parametrize("R,scale", [(100.0, (1e-9, 1e-6)), (60.0, (1e-8, 1e-7))])
def test_near_cocircular_ring_flips_decided_exactly(R, scale):
    # disks on a circle, radii perturbed by 1e-9 .. 1e-6: every in-circle test
    # inside the ring is near zero; new perturbations re-triangulate the disk
    # by Lawson flips decided on the exact path
    nring = int(2 * np.pi * R / 2.2)
    L = 2 * R + 40.0
    c = L / 2
    rng = np.random.default_rng(int(R))
    xy0 = _ring(nring, R, c, scale, rng)
    p = bd.make_params(nring, L=L)
    s = bd.System(p, xy0, stream=stream())
    grid0 = s.state()["xy"]
    assert np.array_equal(edges_of(s.state()["tri"]), edges_of(geometry.delaunay(grid0, L)))
    for k in range(3):
        xy1 = _ring(nring, R, c, scale, rng)
        s.set_state(xy1)
        st = s.last_stats()
        out = s.state()
        P = geometry.with_ghosts(out["xy"], L)
        ref = geometry.delaunay(out["xy"], L)
        assert geometry.general_position(P, ref)
        print("ring R=%g round %d:" % (R, k), {kk: st[kk] for kk in ("flips", "flip_rounds", "exact_tests")})
        assert st["flips"] > 0 and st["exact_tests"] > 0
        assert np.array_equal(edges_of(out["tri"]), edges_of(ref))


# ------------------------------------------------------------ error exits (a9)

def _near_contact_system(n=3000, seed=1, **over):
    cfg = workloads.CONFIGS["c2"]
    L = workloads.box_side(n, cfg.rho)
    xy = workloads.near_contact_state(n, L, cfg.a, seed=seed)
    _, sp, th = workloads.initial_state(cfg, n=n)
    p = bd.params_from_config(cfg, n=n)
    for k, v in over.items():
        setattr(p, k, v)
    return cfg, L, xy, sp, th, bd.System(p, xy, sp, th, stream=stream())


def _assert_start_kept(s, before):
    after = s.state()
    assert np.array_equal(after["xy"], before["xy"])
    assert np.array_equal(after["theta"], before["theta"])
    assert np.array_equal(after["tri"], before["tri"])
    assert after["step"] == before["step"]


def test_correction_pass_cap_exit():
    # this start needs two passes of Algorithm 2 (the oracle's count)
    cfg, L, xy, sp, th, s = _near_contact_system(max_corr_iters=1)
    ref = ostep.step(xy, th, sp, 0, oracle_params(cfg, L))
    assert ref["corr_iters"] == 2
    before = s.state()
    st, code = s.step(3, raise_on_error=False)
    assert code == -5 and st["fail_phase"] == 5 and st["steps_done"] == 0
    _assert_start_kept(s, before)
    s.set_loop_caps(max_corr_iters=1000)
    st = s.step(1)
    out = s.state()
    assert st["corr_iters"] == 2
    assert np.max(np.abs(out["xy"] - ref["xy"])) <= POS_TOL
    assert np.array_equal(edges_of(out["tri"]), edges_of(ref["tris"]))


def test_flip_round_cap_exit():
    cfg = replace(workloads.CONFIGS["c2"], dt=0.01)
    n = 4000
    xy, sp, th = workloads.initial_state(cfg, n=n)
    p = bd.params_from_config(cfg, n=n)
    free = bd.System(p, xy, sp, th, stream=stream())
    st0 = free.step(1)
    # more flip rounds than Lawson sequences (one after the move and one after
    # each correction pass): some sequence took two rounds or more
    assert st0["flip_rounds"] > st0["corr_iters"] + 1 and st0["inverted"] == 0, st0
    want = free.state()
    p.max_flip_rounds = 1
    s = bd.System(p, xy, sp, th, stream=stream())
    before = s.state()
    st, code = s.step(1, raise_on_error=False)
    assert code == -6 and st["fail_phase"] == 4
    _assert_start_kept(s, before)
    s.set_loop_caps(max_flip_rounds=4096)
    s.step(1)
    out = s.state()
    assert np.max(np.abs(out["xy"] - want["xy"])) <= POS_TOL
    assert np.array_equal(edges_of(out["tri"]), edges_of(want["tri"]))


@pytest.mark.parametrize("hold", [1, 3])
def test_barrier_timeout_exit(hold):
    cfg, L, xy, sp, th, s = _near_contact_system()
    cfg, L, xy, sp, th, free = _near_contact_system()
    free.step(2)
    want = free.state()
    before = s.state()
    s.set_wait_limit(0.05, hold_barrier=hold)
    st, code = s.step(2, raise_on_error=False)
    assert code == -7 and st["steps_done"] == 0
    _assert_start_kept(s, before)
    # bd_set_state under a hold of its first barrier (a repair that finds
    # little to flip may not reach a later one): refused, state kept
    s.set_wait_limit(0.05, hold_barrier=1)
    with pytest.raises(bd.BDError) as e:
        s.set_state(before["xy"] + 0.001)
    assert e.value.code == -7
    _assert_start_kept(s, before)
    s.set_wait_limit(2.0, hold_barrier=0)
    st = s.step(2)
    assert st["steps_done"] == 2
    out = s.state()
    assert np.max(np.abs(out["xy"] - want["xy"])) <= POS_TOL
    assert np.array_equal(edges_of(out["tri"]), edges_of(want["tri"]))


def test_barrier_timeout_exit_verlet_correction():
    # Algorithm 2 over the Verlet lists runs in its own persistent kernel
    cfg = workloads.CONFIGS["c3"]
    n = 6000
    L = workloads.box_side(n, cfg.rho)
    xy = workloads.near_contact_state(n, L, cfg.a, seed=3, rho=cfg.rho)
    _, sp, th = workloads.initial_state(cfg, n=n)
    p = bd.params_from_config(cfg, n=n)
    p.overlap_mode = bd.OVERLAP_VERLET
    s = bd.System(p, xy, sp, th, stream=stream())
    free = bd.System(p, xy, sp, th, stream=stream())
    free.step(1)
    want = free.state(want_tri=False)
    before = s.state(want_tri=False)
    s.set_wait_limit(0.05, hold_barrier=1)
    st, code = s.step(1, raise_on_error=False)
    assert code == -7
    after = s.state(want_tri=False)
    assert np.array_equal(after["xy"], before["xy"]) and after["step"] == before["step"]
    s.set_wait_limit(2.0, hold_barrier=0)
    s.step(1)
    assert np.max(np.abs(s.state(want_tri=False)["xy"] - want["xy"])) <= POS_TOL


def test_wait_limit_arguments():
    _, _, _, _, _, s = _near_contact_system(n=300)
    for sec, hold in ((0.0, 0), (100.0, 0), (1.0, -1), (float("nan"), 0)):
        with pytest.raises(bd.BDError):
            s.set_wait_limit(sec, hold)
    with pytest.raises(bd.BDError):
        s.set_loop_caps(0, 10)
