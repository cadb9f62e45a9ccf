// philox.cuh -- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11), written from its published definition:
// ten rounds of two 32x32 -> 64-bit multiplications with the Philox multipliers,
// the key bumped by the Weyl constants after each round.  One device copy for
// every user in the library: the channel's Gaussian samples and the random
// keys of Algorithm 4's fill.
#pragma once

#include <cstdint>

namespace ldpc {

// c: counter in, output block out; key (k0, k1)
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    const uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
}

// the same with a 64-bit key (low word first)
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint64_t seed) {
  philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
}

}  // namespace ldpc
