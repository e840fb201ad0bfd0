"""GPU parity of the step's noise (Sec. 2.4) through the C ABI: the device's
Philox4x32-10 words, bit for bit, and its clamped Box-Muller normals (the
FP32 and FP64 forms the step uses) against the oracle, for counters with all
four words set (disk id, step low and high words, stream tag)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1703_02484_gb300 import binding  # noqa: E402
from oracle import noise, philox  # noqa: E402


@pytest.mark.parametrize("seed,replica", [(0, 0), (100, 3), (0xFFFFFFFFFFFFFFFF, 7), (0x0123456789ABCDEF, 255)])
def test_device_philox_words_and_normals(seed, replica):
    rng = np.random.default_rng(seed & 0xFFFF)
    n = 1 << 17
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:8, 1:] = 0                         # a few counters with words 1-3 zero
    ctr[8:16, 3] = philox.substep_tag(5)    # the tag of a halved piece
    words, z32, z64 = binding.noise_sample(seed, replica, ctr)
    k0, k1 = philox.stream_key(seed, replica)
    ref = np.stack(philox.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], k0, k1), axis=1)
    assert np.array_equal(words, ref.astype(np.uint32))
    u = noise.uniforms([ref[:, k].astype(np.uint64) for k in range(4)])
    a0, a1 = noise.box_muller(u[0], u[1])
    b0, _ = noise.box_muller(u[2], u[3])
    zr = np.stack([noise.clamp(a0), noise.clamp(a1), noise.clamp(b0)], axis=1)
    # the FP64 form: the device's log / sincospi against numpy's, a few ulp
    assert np.max(np.abs(z64 - zr)) <= 1e-12
    # the FP32 form: u rounded to FP32 (absolute error <= 2^-25 near 1), then
    # FP32 log, sqrt and sincospi.  r = sqrt(-2 ln u) has dr/du = -1/(u r), so
    # near u = 1 (r small) the rounding of u costs up to 2^-25 / r
    ra = np.sqrt(-2.0 * np.log(u[0]))
    rb = np.sqrt(-2.0 * np.log(u[2]))
    tol = 4e-6 + (2.0 ** -24) / np.stack([ra, ra, rb], axis=1)
    assert np.all(np.abs(z32.astype(np.float64) - zr) <= tol)
    # the truncation is exercised: about 0.27 % of normals lie beyond 3
    assert np.sum(np.abs(zr) == 3.0) > 100 and np.all(np.abs(z32) <= 3.0)


def test_noise_sample_step_layout_matches_oracle_stream():
    # counters laid out as the step lays them out: (disk, step lo, step hi, tag)
    ids = np.arange(5000, dtype=np.uint64)
    step = (1 << 33) + 12345
    ctr = np.stack([ids, np.full_like(ids, step & 0xFFFFFFFF), np.full_like(ids, step >> 32),
                    np.zeros_like(ids)], axis=1).astype(np.uint32)
    words, _, z64 = binding.noise_sample(77, 2, ctr)
    ref = np.stack(philox.draw(ids, step, 77, 2), axis=1)
    assert np.array_equal(words, ref.astype(np.uint32))
    x, y, t, _ = noise.normals(ids, step, 77, 2)
    assert np.max(np.abs(z64 - np.stack([x, y, t], axis=1))) <= 1e-12
