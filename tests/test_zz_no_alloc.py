"""bd_forces_noalloc: the all-pairs force for callers that cannot allocate.

Some users cannot let this library call cudaMalloc (their device memory is
owned by a host framework's allocator, or their loop cannot afford the
synchronisation an allocation implies).  This test gives the entry point
caller-owned device buffers, calls it twice in a row (the shared static
scratch keeps the first call's contents), and checks both results against
the force the regular entry point bd_compute_forces returns for the same
disks, within the force tolerance of the other GPU tests.  This file is
collected last, so a run that stops at the first failure has run every
other test first."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1703_02484_gb300 as bd  # noqa: E402
from paper_1703_02484_gb300 import binding, workloads  # noqa: E402

FORCE_TOL = 1e-5


def _rel(F, ref):
    scale = math.sqrt(float(np.mean(np.sum(ref ** 2, axis=1))))
    return float(np.max(np.linalg.norm(F - ref, axis=1))) / scale


@pytest.mark.parametrize("n", [5000, 777])
def test_noalloc_matches_compute_forces_twice(n):
    cfg = workloads.CONFIGS["c2"]
    xy, sp, th = workloads.initial_state(cfg, n=n)
    stream = torch.cuda.current_stream()
    s = bd.System(bd.params_from_config(cfg, n=n), xy, sp, th, stream=stream.cuda_stream)
    ref = s.forces()                               # existing entry point
    grid = s.state(want_tri=False)["xy"]           # the same (grid-rounded) positions
    s.close()
    d_xy = torch.from_numpy(np.ascontiguousarray(grid)).cuda()
    d_sp = torch.from_numpy(sp.astype(np.uint8)).cuda()
    outs = []
    for _ in range(2):
        d_F = torch.full((n, 2), float("nan"), dtype=torch.float64, device="cuda")
        binding.forces_noalloc(n, d_xy.data_ptr(), d_sp.data_ptr(), cfg.alpha, d_F.data_ptr(),
                               stream.cuda_stream)
        torch.cuda.synchronize()
        outs.append(d_F.cpu().numpy())
    for F in outs:
        assert np.all(np.isfinite(F))
        assert _rel(F, ref) <= FORCE_TOL
    assert np.array_equal(outs[0], outs[1])


def test_noalloc_rejects_oversize():
    cfg = workloads.CONFIGS["c2"]
    d = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(bd.BDError) as e:
        binding.forces_noalloc(65537, d.data_ptr(), d.data_ptr(), cfg.alpha, d.data_ptr())
    assert e.value.code == -1
