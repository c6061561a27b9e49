// Philox-4x64-10 counter-based generator (Salmon, Moraes, Dror, Shaw:
// "Parallel random numbers: as easy as 1, 2, 3", SC'11), device version.
// Ten rounds of two 64x64->128 multiplications with the published
// multipliers and Weyl key increments; the key is bumped between rounds.
#pragma once

#include <cstdint>

namespace kadabra {

struct U64x4 {
    unsigned long long v[4];
};

__device__ __forceinline__ U64x4 philox4x64_10(unsigned long long c0, unsigned long long c1,
                                               unsigned long long c2, unsigned long long c3,
                                               unsigned long long k0, unsigned long long k1)
{
    constexpr unsigned long long kMul0 = 0xD2E7470EE14C6C93ULL;
    constexpr unsigned long long kMul1 = 0xCA5A826395121157ULL;
    constexpr unsigned long long kWeyl0 = 0x9E3779B97F4A7C15ULL;
    constexpr unsigned long long kWeyl1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long hi0 = __umul64hi(kMul0, c0), lo0 = kMul0 * c0;
        const unsigned long long hi1 = __umul64hi(kMul1, c2), lo1 = kMul1 * c2;
        const unsigned long long n0 = hi1 ^ c1 ^ k0;
        const unsigned long long n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += kWeyl0;
        k1 += kWeyl1;
    }
    U64x4 out;
    out.v[0] = c0;
    out.v[1] = c1;
    out.v[2] = c2;
    out.v[3] = c3;
    return out;
}

// Draw `k` of sample `idx` on stream `tag` under `seed`:
// counter (idx, k, tag, 0), key (seed, 0).
__device__ __forceinline__ U64x4 sample_draw(unsigned long long seed, unsigned int tag,
                                             unsigned long long idx, unsigned long long k)
{
    return philox4x64_10(idx, k, tag, 0ULL, seed, 0ULL);
}

}  // namespace kadabra
