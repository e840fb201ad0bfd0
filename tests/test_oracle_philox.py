"""Pins for the oracle's Philox4x32-10 and its stream layout.

The pin is cuRAND's own Philox4_32_10 host generator (run as a library, on
the CPU).  Seeded with s and started at offset o (curandSetGeneratorOffset),
its output block b is the ten-round Philox block of key (s mod 2^32, s >> 32)
and counter (B >> 16 mod 2^32, B >> 48, B mod 65536, 0) with B = b + o/4 (the
host generator lays its stream out as 65536 subsequences).  A wrong
multiplier, a swapped hi/lo half, a missing key bump or a transposed counter
word changes every output word; an offset of 2^52 sets counter word 1 to 4.  Word
3 (the stream tag) is 0 in every cuRAND host block; a tag that changes every
word pins that it enters at all, and the GPU test (test_gpu_noise.py)
compares the library's device generator with this one over counters with all
four words set."""
import ctypes
import os

import numpy as np
import pytest

from oracle import noise, philox

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    for p in ("/usr/local/cuda/lib64/libcurand.so", "libcurand.so", "libcurand.so.10"):
        try:
            return ctypes.CDLL(p)
        except OSError:
            continue
    pytest.skip("libcurand not available")


def curand_blocks(seed, nblocks):
    lib = _curand()
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(4 * nblocks, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p),
                                  ctypes.c_size_t(out.size)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out.reshape(nblocks, 4)


@pytest.mark.parametrize("seed", [0, 1, 100, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host(seed):
    nb = 3 * 65536 + 17
    ref = curand_blocks(seed, nb)
    b = np.arange(nb, dtype=np.uint64)
    k0, k1 = seed & 0xFFFFFFFF, seed >> 32
    got = np.stack(philox.philox4x32_10(b >> np.uint64(16), 0, b & np.uint64(0xFFFF), 0, k0, k1),
                   axis=1)
    assert np.array_equal(got, ref)


def test_philox_matches_curand_host_with_offset():
    # offset o = 2^52 + 4 * 123457: block b is counter B = b + o/4 = b + 2^50 +
    # 123457, so counter word 1 (B >> 48) is 4 and word 0 carries the rest
    lib = _curand()
    seed = 0x00C0FFEE12345678
    off = (1 << 52) + 4 * 123457
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(off)) == 0
        nb = 2 * 65536 + 5
        ref = np.zeros(4 * nb, dtype=np.uint32)
        assert lib.curandGenerate(gen, ref.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(ref.size)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    B = np.arange(nb, dtype=np.uint64) + np.uint64(off // 4)
    c0 = (B >> np.uint64(16)) & np.uint64(0xFFFFFFFF)
    c1 = B >> np.uint64(48)
    assert np.all(c1 == 4)
    got = np.stack(philox.philox4x32_10(c0, c1, B & np.uint64(0xFFFF), 0, seed & 0xFFFFFFFF, seed >> 32), axis=1)
    assert np.array_equal(got, ref.reshape(nb, 4))


def test_tag_word_enters():
    a = np.stack(philox.draw(np.arange(1000), 5, seed=7, tag=0), axis=1)
    b = np.stack(philox.draw(np.arange(1000), 5, seed=7, tag=philox.substep_tag(2)), axis=1)
    assert not np.any(a == b)


def test_stream_layout_words_distinct():
    a = np.stack(philox.draw(np.arange(1000), 5, seed=7), axis=1)
    b = np.stack(philox.draw(np.arange(1000), 6, seed=7), axis=1)
    c = np.stack(philox.draw(np.arange(1000), 5, seed=7, replica=1), axis=1)
    assert not np.any(np.all(a == b, axis=1))
    assert not np.any(np.all(a == c, axis=1))


def test_uniform_words():
    w = np.concatenate(philox.draw(np.arange(200000), 3, seed=11))
    u = (w.astype(np.float64) + 0.5) / 2.0 ** 32
    hist, _ = np.histogram(u, bins=64, range=(0, 1))
    exp = len(u) / 64
    chi2 = float(np.sum((hist - exp) ** 2 / exp))
    assert chi2 < 120.0   # 63 dof, p ~ 1e-5
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / len(u))
