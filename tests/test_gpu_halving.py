"""GPU parity of repeating a rejected move with a lower dt (Sec. 4.3) through
the C ABI (bd_params.max_dt_halvings), against the FP64 oracle's halving.

Case: the two closest disks of an RSA start attract each other strongly
enough that a whole move, and a half move, make them pass through each other;
quarter moves do not (tests/test_oracle_halving.py pins the oracle on it)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1703_02484_gb300 as bd  # noqa: E402
from oracle import geometry, overlap  # noqa: E402
from oracle import step as ostep  # noqa: E402
from test_oracle_halving import attracting_pair_case  # noqa: E402

POS_TOL = 1e-5


def stream():
    return torch.cuda.current_stream().cuda_stream


def gpu_system(xy, sp, th, p, H, precision=0):
    params = bd.make_params(len(xy), L=p.L, a=p.a, law=bd.LAW_LONG, alpha=p.alpha, n_species=2,
                            D=p.D, Dr=p.Dr, v0=p.v0, dt=p.dt, seed=p.seed, precision=precision,
                            max_dt_halvings=H)
    return bd.System(params, xy, sp, th.astype(np.float32), stream=stream())


@pytest.mark.parametrize("depth_ok,precision", [(2, 0), (2, 1), (3, 1)])
def test_halved_step_matches_oracle(depth_ok, precision):
    xy, sp, th, (i, j), r, p = attracting_pair_case(depth_ok=depth_ok)
    s = gpu_system(xy, sp, th, p, H=depth_ok + 1, precision=precision)
    x0 = s.state(want_tri=False)["xy"]          # the start on the position grid
    st = s.step(1)
    out = s.state()
    p.max_halvings = depth_ok + 1
    ref = ostep.step(x0, th, sp, 0, p)
    assert not ref["rejected"] and st["rejected"] == 0 and st["steps_done"] == 1
    assert st["halvings"] == ref["halvings"] and st["substeps"] == ref["substeps"]
    err = float(np.max(np.abs(out["xy"] - ref["xy"])))
    assert err <= POS_TOL * p.a, err
    assert np.max(np.abs(out["theta"] - ref["theta"])) <= 1e-5
    assert out["step"] == 1
    # the maintained triangulation is the Delaunay triangulation of the result
    assert np.array_equal(geometry.edges(out["tri"]), geometry.edges(geometry.delaunay(out["xy"], p.L)))
    assert len(overlap.close_pairs(out["xy"], 2.0 * p.a)) == 0
    s.close()


def test_fp32_deeper_halving_structure():
    # depth 3 in FP32: the pair closes at ~1e4 a per unit time and collides in
    # every piece, which multiplies the FP32 rounding of its ~6e4 force (a few
    # 1e-7 relative) from piece to piece; the FP64 path above checks the
    # positions of this case, here the pieces, the halvings and the outcome
    xy, sp, th, (i, j), r, p = attracting_pair_case(depth_ok=3)
    s = gpu_system(xy, sp, th, p, H=4, precision=0)
    x0 = s.state(want_tri=False)["xy"]
    st = s.step(1)
    out = s.state()
    p.max_halvings = 4
    ref = ostep.step(x0, th, sp, 0, p)
    assert st["rejected"] == 0 and not ref["rejected"]
    assert st["halvings"] == ref["halvings"] and st["substeps"] == ref["substeps"]
    others = np.ones(len(xy), bool)
    others[[i, j]] = False
    assert float(np.max(np.abs(out["xy"][others] - ref["xy"][others]))) <= POS_TOL * p.a
    assert float((x0[j] - x0[i]) @ (out["xy"][j] - out["xy"][i])) > 0
    assert np.array_equal(geometry.edges(out["tri"]), geometry.edges(geometry.delaunay(out["xy"], p.L)))
    assert len(overlap.close_pairs(out["xy"], 2.0 * p.a)) == 0
    s.close()


def test_too_few_halvings_rejects_and_keeps_the_state():
    xy, sp, th, _, r, p = attracting_pair_case(depth_ok=3)
    s = gpu_system(xy, sp, th, p, H=2)
    before = s.state()
    st, code = s.step(1, raise_on_error=False)
    assert code == -4 and st["rejected"] == 1 and st["steps_done"] == 0
    assert st["halvings"] >= 2
    after = s.state()
    assert np.array_equal(after["xy"], before["xy"]) and np.array_equal(after["theta"], before["theta"])
    assert np.array_equal(after["tri"], before["tri"]) and after["step"] == before["step"]
    # no halving at all: the plain rejection of Sec. 4.3
    s0 = gpu_system(xy, sp, th, p, H=0)
    st0, code0 = s0.step(1, raise_on_error=False)
    assert code0 == -4 and st0["halvings"] == 0 and st0["fail_phase"] in (1, 2, 3)
    s.close()
    s0.close()


def test_steps_after_a_halved_step_follow_the_oracle():
    # a multi-step call: the first step is halved, the rest are whole steps
    # (or halved again); each step of the GPU trajectory is checked against
    # the oracle started from the GPU's state before it
    xy, sp, th, _, r, p = attracting_pair_case(depth_ok=2)
    p.max_halvings = 4
    s = gpu_system(xy, sp, th, p, H=4)
    cur = s.state(want_tri=False)
    x, t = cur["xy"], cur["theta"].astype(np.float64)
    st = s.step(4)
    assert st["steps_done"] == 4 and st["halvings"] >= 3
    s2 = gpu_system(xy, sp, th, p, H=4)
    for k in range(4):
        s2.step(1)
        g = s2.state(want_tri=False)
        ref = ostep.step(x, t, sp, k, p)
        assert not ref["rejected"]
        assert float(np.max(np.abs(g["xy"] - ref["xy"]))) <= POS_TOL * p.a
        x, t = g["xy"], g["theta"].astype(np.float64)
    # one 4-step call and four 1-step calls give the same trajectory
    assert np.array_equal(s.state(want_tri=False)["xy"], x)
    s.close()
    s2.close()


def test_batched_handles_refuse_halving():
    xy, sp, th, _, r, p = attracting_pair_case()
    params = [bd.make_params(len(xy), L=p.L, law=bd.LAW_LONG, alpha=p.alpha, n_species=2,
                             max_dt_halvings=2) for _ in range(2)]
    with pytest.raises(bd.BDError) as e:
        bd.System(params, stream=stream())
    assert e.value.code == -10
