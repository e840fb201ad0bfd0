"""bd_forces_noalloc: the all-pairs force for callers that cannot allocate.

Some users cannot let this library call cudaMalloc (their device memory is
owned by a host framework's allocator, or their loop cannot afford the
synchronisation an allocation implies).  These tests give the entry point
caller-owned device buffers and call it twice in a row (the shared static
scratch keeps the first call's contents).  Both results are checked against
the force the regular entry point bd_compute_forces returns for the same
disks and against the oracle's FP64 sum, within the force tolerance of the
other GPU tests, at sizes up to the documented maximum n = 65536 (where the
scratch is full); a smaller call after the largest one shows that what the
larger call left in the scratch does not leak into the result.  This file is
collected last, so a run that stops at the first failure has run every other
test first."""
import math
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1703_02484_gb300 as bd  # noqa: E402
from paper_1703_02484_gb300 import binding, workloads  # noqa: E402
from oracle import forces as oforces  # noqa: E402

FORCE_TOL = 1e-5
MAX_N = 65536


def _rel(F, ref):
    scale = math.sqrt(float(np.mean(np.sum(ref ** 2, axis=1))))
    return float(np.max(np.linalg.norm(F - ref, axis=1))) / scale


def _inputs(n):
    cfg = workloads.CONFIGS["c2"]
    xy, sp, th = workloads.initial_state(cfg, n=n)
    return cfg, xy, sp, th


def _noalloc(n, xy, sp, alpha, calls=2):
    stream = torch.cuda.current_stream()
    d_xy = torch.from_numpy(np.ascontiguousarray(xy)).cuda()
    d_sp = torch.from_numpy(sp.astype(np.uint8)).cuda()
    outs = []
    for _ in range(calls):
        d_F = torch.full((n, 2), float("nan"), dtype=torch.float64, device="cuda")
        binding.forces_noalloc(n, d_xy.data_ptr(), d_sp.data_ptr(), alpha, d_F.data_ptr(),
                               stream.cuda_stream)
        torch.cuda.synchronize()
        outs.append(d_F.cpu().numpy())
    return outs


@pytest.mark.parametrize("n", [5000, 777, MAX_N])
def test_noalloc_matches_compute_forces_and_oracle_twice(n):
    cfg, xy, sp, th = _inputs(n)
    s = bd.System(bd.params_from_config(cfg, n=n), xy, sp, th,
                  stream=torch.cuda.current_stream().cuda_stream)
    ref = s.forces()                               # existing entry point
    grid = s.state(want_tri=False)["xy"]           # the same (grid-rounded) positions
    s.close()
    exact = oforces.long_range(grid, sp, cfg.alpha, threads=max(1, os.cpu_count() or 1))
    outs = _noalloc(n, grid, sp, cfg.alpha)
    for F in outs:
        assert np.all(np.isfinite(F))
        assert _rel(F, ref) <= FORCE_TOL
        assert _rel(F, exact) <= FORCE_TOL
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_smaller_call_after_full_scratch():
    # the largest size fills the scratch (three j chunks of partial forces);
    # a smaller call afterwards must not pick up any of it
    cfg, xy, sp, _ = _inputs(MAX_N)
    _noalloc(MAX_N, xy, sp, cfg.alpha, calls=1)
    n = 1500
    cfg, xy2, sp2, _ = _inputs(n)
    F = _noalloc(n, xy2, sp2, cfg.alpha, calls=1)[0]
    assert _rel(F, oforces.long_range_numpy(xy2, sp2, cfg.alpha)) <= FORCE_TOL


def test_noalloc_rejects_bad_arguments():
    cfg = workloads.CONFIGS["c2"]
    d = torch.zeros(64, dtype=torch.float64, device="cuda")
    with pytest.raises(bd.BDError) as e:
        binding.forces_noalloc(MAX_N + 1, d.data_ptr(), d.data_ptr(), cfg.alpha, d.data_ptr())
    assert e.value.code == -1
    # a double* that is 8 bytes off a 16-byte boundary: refused, not read
    with pytest.raises(bd.BDError) as e:
        binding.forces_noalloc(4, d.data_ptr() + 8, d.data_ptr(), cfg.alpha, d.data_ptr() + 128)
    assert e.value.code == -1
    with pytest.raises(bd.BDError) as e:
        binding.forces_noalloc(4, d.data_ptr(), d.data_ptr(), cfg.alpha, d.data_ptr() + 136)
    assert e.value.code == -1
