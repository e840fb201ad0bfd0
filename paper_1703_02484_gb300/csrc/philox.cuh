// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) for the per-particle
// noise of Eq. (integration) (Sec. 2.2, Sec. 2.4) and the seeded placement.
// Ten rounds of: multiply counter words 0 and 2 by fixed odd constants, keep
// both halves of each 64-bit product, xor the high halves with the other two
// counter words and the round key; the key advances by two Weyl increments
// between rounds.  Stream layout:
//   key     = (seed mod 2^32, (seed >> 32) xor replica)
//   counter = (particle id, step mod 2^32, step >> 32, tag)
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define BD_PHX_HD __host__ __device__ __forceinline__
#else
#define BD_PHX_HD inline
#endif

namespace bdrng {

struct U4 {
  uint32_t x, y, z, w;
};

BD_PHX_HD void mulhilo(uint32_t a, uint32_t b, uint32_t &hi, uint32_t &lo) {
#if defined(__CUDA_ARCH__)
  lo = a * b;
  hi = __umulhi(a, b);
#else
  uint64_t p = (uint64_t)a * (uint64_t)b;
  lo = (uint32_t)p;
  hi = (uint32_t)(p >> 32);
#endif
}

BD_PHX_HD U4 philox(U4 c, uint32_t k0, uint32_t k1) {
  const uint32_t MA = 0xD2511F53u, MB = 0xCD9E8D57u;
  const uint32_t KA = 0x9E3779B9u, KB = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t h0, l0, h1, l1;
    mulhilo(MA, c.x, h0, l0);
    mulhilo(MB, c.z, h1, l1);
    U4 n;
    n.x = h1 ^ c.y ^ k0;
    n.y = l1;
    n.z = h0 ^ c.w ^ k1;
    n.w = l0;
    c = n;
    k0 += KA;
    k1 += KB;
  }
  return c;
}

enum : uint32_t { TAG_NOISE = 0u, TAG_PLACE = 0x504C4143u, TAG_LATTICE = 0x4C415454u };

BD_PHX_HD U4 draw(uint32_t particle, int64_t step, uint64_t seed, uint32_t replica, uint32_t tag) {
  U4 c;
  c.x = particle;
  c.y = (uint32_t)((uint64_t)step & 0xFFFFFFFFull);
  c.z = (uint32_t)((uint64_t)step >> 32);
  c.w = tag;
  return philox(c, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32) ^ replica);
}

}  // namespace bdrng
