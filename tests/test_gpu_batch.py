"""GPU tests of batched replicas: R systems of different size, box and law
advanced by one launch sequence per step."""
from dataclasses import replace

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1703_02484_gb300 as bd  # noqa: E402
from paper_1703_02484_gb300 import workloads  # noqa: E402
from oracle import geometry  # noqa: E402
from oracle import step as ostep  # noqa: E402
from scipy.spatial import cKDTree  # noqa: E402


def stream():
    return torch.cuda.current_stream().cuda_stream


def small_batch(R=6, seed=11):
    cfgs = workloads.batch_configs(R, seed=seed, n_lo=300, n_hi=3000)
    params, xys, sps, ths = [], [], [], []
    for r, cfg in enumerate(cfgs):
        xy, sp, th = workloads.initial_state(cfg, seed=seed + 100 * r)
        p = bd.params_from_config(cfg)
        p.replica = r
        params.append(p)
        xys.append(xy)
        sps.append(sp)
        ths.append(th)
    return cfgs, params, xys, sps, ths


def test_batch_matches_replicas_run_alone():
    cfgs, params, xys, sps, ths = small_batch()
    b = bd.System(params, np.concatenate(xys), np.concatenate(sps), np.concatenate(ths),
                  stream=stream())
    assert b.R == len(cfgs)
    for r, cfg in enumerate(cfgs):
        rep = b.replica(r)
        assert np.array_equal(geometry.edges(rep["tri"]),
                              geometry.edges(geometry.delaunay(rep["xy"], rep["L"])))
    st = b.step(6)
    assert st["steps_done"] == 6
    for r, cfg in enumerate(cfgs):
        alone = bd.System(params[r], xys[r], sps[r], ths[r], stream=stream())
        alone.step(6)
        a = alone.state()
        rep = b.replica(r)
        # same arithmetic per replica; only the all-pairs chunking (summation
        # order) may differ
        assert np.max(np.abs(rep["xy"] - a["xy"])) <= 1e-8
        assert np.array_equal(geometry.edges(rep["tri"]), geometry.edges(a["tri"]))
        assert len(cKDTree(rep["xy"]).query_pairs(2.0 * (1 - 1e-12))) == 0


def test_batch_one_step_parity_with_oracle():
    cfgs, params, xys, sps, ths = small_batch(R=4, seed=21)
    for r, cfg in enumerate(cfgs):
        L = workloads.box_side(cfg.n, cfg.rho)
        xys[r] = workloads.near_contact_state(cfg.n, L, 1.0, seed=7 + r, rho=cfg.rho)
    b = bd.System(params, np.concatenate(xys), np.concatenate(sps), np.concatenate(ths),
                  stream=stream())
    b.step(1)
    for r, cfg in enumerate(cfgs):
        rep = b.replica(r)
        op = ostep.Params(L=rep["L"], a=1.0, law=cfg.law, alpha=cfg.alpha, eps=cfg.eps,
                          kappa=cfg.kappa, r_cut=cfg.r_cut, D=cfg.D, Dr=cfg.Dr, v0=cfg.v0,
                          dt=cfg.dt, seed=cfg.seed, replica=r)
        ref = ostep.step(xys[r], ths[r], sps[r], 0, op)
        assert np.max(np.abs(rep["xy"] - ref["xy"])) <= 1e-5
        assert np.array_equal(geometry.edges(rep["tri"]), geometry.edges(ref["tris"]))


def test_full_batched_workload_runs_clean():
    cfgs = workloads.batch_configs(256)
    params = []
    for r, cfg in enumerate(cfgs):
        p = bd.params_from_config(cfg)
        p.replica = r
        p.seed = 3 + 1000 * r          # RSA placement seed per replica
        params.append(p)
    b = bd.System(params, stream=stream())   # library RSA starts
    tune = b.tuning()
    assert tune["n_items"] > 0 and tune["tiles_per_item"] >= 1
    st = b.step(10)
    assert st["steps_done"] == 10 and st["rejected"] == 0
    rng = np.random.default_rng(0)
    for r in rng.choice(256, 12, replace=False):
        rep = b.replica(int(r))
        assert len(cKDTree(rep["xy"]).query_pairs(2.0 * (1 - 1e-12))) == 0
        assert np.array_equal(geometry.edges(rep["tri"]),
                              geometry.edges(geometry.delaunay(rep["xy"], rep["L"])))


def test_batch_mixes_walls_and_periodic_replicas():
    # replicas with walls and with a periodic box in one handle: each advances
    # as it does alone (the periodic sweep serves both kinds in a batch)
    from oracle import periodic
    cfgs, params, xys, sps, ths = small_batch(R=4, seed=21)
    for r in (1, 3):
        L = float(np.float32(workloads.box_side(params[r].n, cfgs[r].rho)))
        params[r].box_L = L
        params[r].boundary = bd.BOUNDARY_PERIODIC
        xys[r] = periodic.wrap(xys[r] + np.array([0.3 * L, 0.7 * L]), L)
    b = bd.System(params, np.concatenate(xys), np.concatenate(sps), np.concatenate(ths), stream=stream())
    st = b.step(8)
    assert st["steps_done"] == 8
    shifts = b.tri_shifts()
    off = 0
    for r in range(4):
        rep = b.replica(r)
        alone = bd.System(params[r], xys[r], sps[r], ths[r], stream=stream())
        alone.step(8)
        a = alone.state()
        L = rep["L"]
        d = rep["xy"] - a["xy"]
        if params[r].boundary:
            d = periodic.min_image(d, L)
            sh = shifts[off:off + len(rep["tri"])]
            assert np.array_equal(periodic.edge_keys(rep["tri"].astype(np.int64), sh),
                                  periodic.edge_keys(*periodic.delaunay_torus(rep["xy"], L)))
        else:
            assert np.array_equal(geometry.edges(rep["tri"]), geometry.edges(a["tri"]))
        assert float(np.max(np.abs(d))) <= 1e-8
        off += len(rep["tri"])
        alone.close()
    b.close()


def test_batch_step_per_replica_counters():
    # bd_batch_step: each replica's correction passes and Lawson flips equal
    # those of the same replica run alone
    cfgs, params, xys, sps, ths = small_batch(R=4, seed=17)
    b = bd.System(params, np.concatenate(xys), np.concatenate(sps), np.concatenate(ths), stream=stream())
    per = b.batch_step(6)
    assert len(per) == 4 and all(p["steps_done"] == 6 for p in per)
    tot_flips = 0
    for r in range(4):
        alone = bd.System(params[r], xys[r], sps[r], ths[r], stream=stream())
        st = alone.step(6)
        assert per[r]["corr_iters"] == st["corr_iters"], (r, per[r], st)
        assert per[r]["flips"] == st["flips"], (r, per[r], st)
        tot_flips += st["flips"]
        alone.close()
    assert tot_flips > 0
    b.close()


def test_batch_step_per_replica_counters_verlet_correction():
    # Algorithm 2 over the Verlet lists (no triangulation): each replica's
    # correction passes counted on the device equal its passes run alone; no
    # triangulation, so no inverted triangles and no flips
    R = 4
    cfgs = [replace(workloads.CONFIGS["c3"], n=int(n), rho=0.45, seed=5) for n in (900, 1500, 2200, 700)]
    params, xys, sps, ths = [], [], [], []
    for r, cfg in enumerate(cfgs):
        L = workloads.box_side(cfg.n, cfg.rho)
        xy = workloads.near_contact_state(cfg.n, L, cfg.a, seed=40 + r, rho=cfg.rho)
        _, sp, th = workloads.initial_state(cfg)
        p = bd.params_from_config(cfg)
        p.replica = r
        p.overlap_mode = bd.OVERLAP_VERLET
        params.append(p)
        xys.append(xy)
        sps.append(sp)
        ths.append(th)
    b = bd.System(params, np.concatenate(xys), np.concatenate(sps), np.concatenate(ths), stream=stream())
    per = b.batch_step(5)
    assert len(per) == R and all(p["steps_done"] == 5 for p in per)
    tot = 0
    for r in range(R):
        alone = bd.System(params[r], xys[r], sps[r], ths[r], stream=stream())
        st = alone.step(5)
        assert per[r]["corr_iters"] == st["corr_iters"], (r, per[r], st)
        assert per[r]["inverted"] == st["inverted"] == 0
        assert per[r]["flips"] == st["flips"] == 0
        tot += st["corr_iters"]
        alone.close()
    assert tot > 0
    b.close()


def test_single_replica_batch_step_counters():
    # a batch of one replica keeps no per-replica device counters: its counters
    # are the call's own
    cfgs, params, xys, sps, ths = small_batch(R=1, seed=23)
    b = bd.System(params, xys[0], sps[0], ths[0], stream=stream())
    per = b.batch_step(4)
    alone = bd.System(params[0], xys[0], sps[0], ths[0], stream=stream())
    st = alone.step(4)
    assert per[0]["corr_iters"] == st["corr_iters"] and per[0]["flips"] == st["flips"]
    assert per[0]["steps_done"] == 4
