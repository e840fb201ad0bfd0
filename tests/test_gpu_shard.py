"""GPU tests of force sharding (one system's all-pairs sweep shared among
ranks, bd_set_force_shard / bd_step_begin / bd_step_end) emulated on one GPU:
the ranks' partial forces add up to the whole force, and ranks that advance
the same state with the summed forces stay bit-identical -- the correction's
displacement sums are order-independent, which also makes repeated runs
bit-identical.  The exchange itself (an all-reduce over the ranks) is
covered with gloo ranks on the CPU (test_multirank_gloo.py)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1703_02484_gb300 as bd  # noqa: E402
from paper_1703_02484_gb300 import workloads  # noqa: E402
from oracle import geometry  # noqa: E402


def stream():
    return torch.cuda.current_stream().cuda_stream


def make(n=20000, seed=3, monkeypatch=None):
    cfg = workloads.CONFIGS["c2"]
    L = workloads.box_side(n, cfg.rho)
    xy = workloads.near_contact_state(n, L, cfg.a, seed=seed)
    _, sp, th = workloads.initial_state(cfg, n=n)
    return bd.System(bd.params_from_config(cfg, n=n), xy, sp, th, stream=stream())


@pytest.fixture
def fixed_sweep(monkeypatch):
    # the same sweep shape on every handle (the autotuner times candidates)
    monkeypatch.setenv("BD_FORCE_VARIANT", "3")
    monkeypatch.setenv("BD_FORCE_TILES", "8")


def test_partial_forces_add_up(fixed_sweep):
    whole = make()
    F = torch.empty(2 * whole.force_slots(), dtype=torch.float64, device="cuda")
    whole.step_begin(F.data_ptr())
    ref = F.clone()
    world = 3
    tot = torch.zeros_like(F)
    parts = []
    for r in range(world):
        h = make()
        h.set_force_shard(r, world)
        h.step_begin(F.data_ptr())
        parts.append(F.clone())
        tot += F
        h.close()
    scale = float(torch.sqrt(torch.mean(ref.view(-1, 2).pow(2).sum(1))))
    assert float((tot - ref).abs().max()) <= 1e-10 * scale
    # every rank did a share of the work
    assert all(float(p.abs().max()) > 0 for p in parts)


def test_sharded_ranks_stay_identical(fixed_sweep):
    world = 3
    ranks = [make() for _ in range(world)]
    for r, h in enumerate(ranks):
        h.set_force_shard(r, world)
    whole = make()
    F = torch.empty(2 * whole.force_slots(), dtype=torch.float64, device="cuda")
    tot = torch.empty_like(F)
    corr = 0
    for step in range(12):
        tot.zero_()
        for h in ranks:
            h.step_begin(F.data_ptr())
            tot += F
        sts = [h.step_end(tot.data_ptr()) for h in ranks]
        corr += sts[0]["corr_iters"]
        st = whole.step(1)
        outs = [h.state() for h in ranks]
        for o in outs[1:]:
            assert np.array_equal(o["xy"], outs[0]["xy"]) and np.array_equal(o["tri"], outs[0]["tri"])
        w = whole.state()
        assert np.max(np.abs(outs[0]["xy"] - w["xy"])) <= 1e-9
        assert np.array_equal(geometry.edges(outs[0]["tri"]), geometry.edges(w["tri"]))
        assert sts[0]["corr_iters"] == st["corr_iters"]
    assert corr > 0
    assert outs[0]["step"] == 12


def test_repeated_runs_are_bit_identical(fixed_sweep):
    a, b = make(seed=8), make(seed=8)
    sa, sb = a.step(25), b.step(25)
    assert sa["corr_iters"] == sb["corr_iters"] > 0
    oa, ob = a.state(), b.state()
    assert np.array_equal(oa["xy"], ob["xy"]) and np.array_equal(oa["tri"], ob["tri"])


def test_shard_arguments(fixed_sweep):
    h = make(n=3000)
    for r, w in ((0, 0), (-1, 2), (2, 2)):
        with pytest.raises(bd.BDError) as e:
            h.set_force_shard(r, w)
        assert e.value.code == -1
    h.set_force_shard(1, 2)
    with pytest.raises(bd.BDError) as e:
        h.step(1)
    assert e.value.code == -10
    h.set_force_shard(0, 1)           # the whole sweep again: bd_step works
    assert h.step(1)["steps_done"] == 1
