// K = P#/d as machine words (host code).
//
// The generator computes K mod p as a running product of K's prime factors
// packed into words: below 2^31 for the lazily reduced 32-bit Montgomery
// product (a chain of such products by words below 2^31 stays below 2p) and
// below 2^64 for the 64-bit one.  Fewer words mean fewer multiplications per
// prime, so the factors are packed first fit, largest first (for 953#/210:
// 45 words below 2^31, against 48 when the factors are packed in order and a
// lower bound of 43 from the total number of bits).
#pragma once
#include <stdint.h>

#include <algorithm>
#include <vector>

namespace cs {

// Words below `limit` whose product is the product of qK (qK: primes, any
// order).  First fit decreasing: a word takes a factor while the product stays
// below the limit.
inline std::vector<unsigned __int128> pack_factor_words(const std::vector<uint32_t> &qK,
                                                        unsigned __int128 limit) {
    std::vector<uint32_t> q(qK);
    std::sort(q.begin(), q.end(), [](uint32_t a, uint32_t b) { return a > b; });
    std::vector<unsigned __int128> bins;
    for (uint32_t f : q) {
        bool placed = false;
        for (auto &b : bins)
            if (b * f < limit) {
                b *= f;
                placed = true;
                break;
            }
        if (!placed) bins.push_back(f);
    }
    return bins;
}

inline void pack_k_words(const std::vector<uint32_t> &qK, std::vector<uint32_t> &w32, std::vector<uint64_t> &w64) {
    w32.clear();
    w64.clear();
    for (auto b : pack_factor_words(qK, (unsigned __int128)1 << 31)) w32.push_back((uint32_t)b);
    for (auto b : pack_factor_words(qK, (unsigned __int128)1 << 64)) w64.push_back((uint64_t)b);
}

}  // namespace cs
