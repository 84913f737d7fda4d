// D step of DFC-LRR (Algorithm 1, Section 2.2): a uniformly random partition
// of the n columns of M into t blocks.  Host code only; the solve uses it when
// the caller passes no permutation or no block offsets.
//
// Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", OOPSLA 2014, with the 64-bit mixing
// constants of Vigna's public-domain reference), state advanced by the golden
// gamma 0x9e3779b97f4a7c15 and output mix64(state).  Uniform integers in
// [0, k) by rejection of the top 2^64 mod k values (no modulo bias).
// Permutation: Durstenfeld's form of the Fisher-Yates shuffle, i = n-1 .. 1
// swapping position i with a uniform position in [0, i], applied to the
// identity.  Blocks: offsets[i] = floor(i n / t), so block sizes are
// floor(n/t) or ceil(n/t) (the paper's equal split, l = n/t).
#include <cstdint>

#include "dfc_lrr.h"
#include "kernels.cuh"

namespace lrr {
namespace {

inline uint64_t splitmix64(uint64_t& state) {
    state += 0x9e3779b97f4a7c15ULL;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

// uniform in [0, k), k >= 1
inline uint64_t uniform_below(uint64_t& state, uint64_t k) {
    // values >= limit would make the residues of the last partial period more likely
    const uint64_t limit = UINT64_MAX - (UINT64_MAX % k + 1) % k;
    uint64_t x = splitmix64(state);
    while (x > limit) x = splitmix64(state);
    return x % k;
}

}  // namespace

void draw_partition(int64_t n, int t, uint64_t seed, int64_t* perm, int64_t* offsets) {
    if (perm) {
        for (int64_t j = 0; j < n; ++j) perm[j] = j;
        uint64_t state = seed;
        for (int64_t i = n - 1; i >= 1; --i) {
            const int64_t j = (int64_t)uniform_below(state, (uint64_t)i + 1);
            const int64_t tmp = perm[i];
            perm[i] = perm[j];
            perm[j] = tmp;
        }
    }
    if (offsets)
        for (int i = 0; i <= t; ++i) offsets[i] = (int64_t)(((__int128)i * n) / t);
}

}  // namespace lrr

extern "C" LRR_API int dfc_partition(int64_t n, int32_t t, uint64_t seed, int64_t* perm, int64_t* offsets) {
    if (n < 1 || t < 1 || t > n || (!perm && !offsets)) return LRR_ERR_INVALID;
    lrr::draw_partition(n, t, seed, perm, offsets);
    return LRR_OK;
}
