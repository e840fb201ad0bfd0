"""Philox4x32-10 counter-based generator -- oracle (test infrastructure).

Written from the definition in Salmon, Moraes, Dror & Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC'11): a 128-bit counter is mixed with a 64-bit
key by ten rounds; each round multiplies counter words 0 and 2 by fixed
32-bit constants, keeps the 64-bit products' high and low halves, and xors the
high halves with the other two counter words and the round key; the key is
bumped by two Weyl constants between rounds.

The paper draws its noise with cuRAND's XORWOW (Sec. 5); Philox is used
here so that every random number is a pure function of
(seed, particle, step) and the GPU and the oracle can draw identical streams
independently.  Stream layout (both sides implement it on their own):
    key     = (seed mod 2^32, (seed >> 32) xor replica)
    counter = (particle id, step mod 2^32, step >> 32, tag)
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)

TAG_NOISE = 0


def substep_tag(node: int) -> int:
    """Counter word 3 of the noise of one piece of a step that was redone with
    a lower dt (Sec. 4.3).  Pieces are numbered as a binary heap: node 1 is
    the whole step, nodes 2k and 2k+1 the two halves of node k.  The whole
    step keeps TAG_NOISE; node k >= 2 uses TAG_NOISE + 256 k."""
    node = int(node)
    return TAG_NOISE if node <= 1 else (TAG_NOISE + 256 * node) & 0xFFFFFFFF


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.  Inputs are uint32-valued arrays or scalars
    (broadcast together); returns four uint32 arrays."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK for v in (c0, c1, c2, c3))
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    c0, c1, c2, c3 = (v.copy() for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK
    k1 = np.asarray(k1, dtype=np.uint64) & MASK
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0          # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return tuple(v.astype(np.uint32) for v in (c0, c1, c2, c3))


def stream_key(seed: int, replica: int = 0):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, ((seed >> 32) ^ int(replica)) & 0xFFFFFFFF


def draw(ids, step: int, seed: int, replica: int = 0, tag: int = TAG_NOISE):
    """Four uint32 words per particle id for time step `step`."""
    k0, k1 = stream_key(seed, replica)
    step = int(step)
    return philox4x32_10(np.asarray(ids, dtype=np.uint64), step & 0xFFFFFFFF,
                         (step >> 32) & 0xFFFFFFFF, tag, k0, k1)
