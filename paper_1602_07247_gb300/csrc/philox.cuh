// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror and Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of two
// 32 x 32 -> 64-bit multiplications with the published multipliers and Weyl
// key increments.  Used by the event simulator and by the random shift of
// reconstructed positions.
#pragma once

#include <cstdint>

namespace ants {

__device__ __forceinline__ void philox10(uint32_t k0, uint32_t k1, uint32_t c[4])
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// uniform in (0, 1) from the top 24 bits of a word
__device__ __forceinline__ float u01(uint32_t x) { return ((float)(x >> 8) + 0.5f) * (1.0f / 16777216.0f); }
__device__ __forceinline__ double u01d(uint32_t x) { return ((double)(x >> 8) + 0.5) * (1.0 / 16777216.0); }

}  // namespace ants
