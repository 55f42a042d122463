// seed.cuh -- the device-seeded deviation vectors of chs_ensemble_init:
// SplitMix64 (Steele, Lea and Flood 2014) read at a given position of the
// stream of `seed`, mapped to [-1, 1) by its top 53 bits.
#pragma once

#include <stdint.h>

namespace chs {

// The finaliser applied to the state seed + m * 0x9e3779b97f4a7c15, i.e. the
// m-th output of the stream seeded with `seed`.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t m)
{
    uint64_t z = seed + m * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// 2 u - 1 with u = (top 53 bits of the m-th output) / 2^53, each operation
// rounded on its own (no contraction), as a plain sequential program rounds it.
__device__ __forceinline__ double seed_uniform(uint64_t seed, uint64_t m)
{
    const uint64_t z = splitmix64_at(seed, m);
    return __dsub_rn(__dmul_rn(2.0, __dmul_rn((double)(z >> 11), 0x1.0p-53)), 1.0);
}

}  // namespace chs
