// The m-classes the three-gap walk takes per large-prime chunk (host code).
//
// Rows are the m coprime to d, so a walk can skip every m that shares a factor
// with a divisor Q of d.  Tiers, from the chunks whose primes have the most hits
// per prime to those with the fewest:
//   class items mod 210 (or 30): every class of m mod Q coprime to Q is a work
//     item of its own, 8/35 (4/15) of the hits, when a class still has at least
//     class_item_hits expected hits per prime;
//   m = 1, 5 (mod 6) as two walkers of one item (6 | d), a third of the hits,
//     from class_min_hits expected hits per prime;
//   the odd m (2 | d), one walker, half of the hits;
//   every m (odd d).
// Class residues are offsets of m - M_start mod Q.
#pragma once
#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "cs_internal.h"

namespace cs {

// Class items mod Q: one class per residue c of m mod Q with gcd(c, Q) = 1.
inline MClasses class_items(uint32_t Q, uint64_t M_start) {
    MClasses mc = EVERY_M;
    mc.Q = Q;
    mc.n = 0;
    const uint32_t ms = (uint32_t)(M_start % Q);
    for (uint32_t c = 1; c < Q; c++)
        if (std::gcd(c, Q) == 1) mc.item_off[mc.n++] = (uint8_t)((c + Q - ms) % Q);
    mc.items = mc.n;
    mc.off[0] = mc.item_off[0];
    return mc;
}

struct ClassTiers {
    MClasses mcls = EVERY_M;         // classes of the chunks with many hits (mod 6, else mod 2)
    MClasses mcls_light = EVERY_M;   // classes of the other chunks (the odd m when 2 | d)
    std::vector<MClasses> fine;      // class-item candidates, finest first
    uint32_t m_classes = 0;          // cs_tuning.m_classes
    double hits_scale = 0;           // M_inc * S: expected hits of a prime p are hits_scale / p
    double split_min_hits = 48.0;
    double class_item_hits = 64.0;

    // chunks whose low end is lo walk the two classes mod 6 (or the one mod 2)
    bool split(uint64_t lo) const {
        if (mcls.Q == 1) return false;
        if (m_classes == 2) return true;
        return hits_scale / (double)std::max<uint64_t>(lo, 1) >= split_min_hits;
    }
    // the classes a chunk whose primes start above lo walks
    MClasses for_chunk(uint64_t lo) const {
        if (m_classes == 3) return fine.empty() ? EVERY_M : fine[0];
        if (m_classes == 0)
            for (const MClasses &mc : fine)
                if (hits_scale / ((double)std::max<uint64_t>(lo, 1) * mc.Q) >= class_item_hits) return mc;
        return split(lo) ? mcls : mcls_light;
    }
};

// Tiers for a plan: three_gap = the three-gap walk is used and SL > 0 (the
// one-solve-per-hit walk and SL = 0 take every m); t.m_classes <= 3.
inline ClassTiers class_tiers(bool three_gap, uint64_t d, uint64_t M_start, uint64_t M_inc, uint64_t S,
                              const cs_tuning &t) {
    ClassTiers ct;
    ct.m_classes = t.m_classes;
    ct.hits_scale = (double)M_inc * (double)S;
    if (t.class_min_hits) ct.split_min_hits = (double)t.class_min_hits;
    if (t.class_item_hits) ct.class_item_hits = (double)t.class_item_hits;
    if (three_gap && t.m_classes != 1) {
        const uint32_t m6 = (uint32_t)(M_start % 6), m2 = (uint32_t)(M_start % 2);
        if (d % 2 == 0) ct.mcls_light = ct.mcls = MClasses{2, 1, {(1 + 2 - m2) % 2, 0}, 0, {}};
        if (d % 6 == 0) ct.mcls = MClasses{6, 2, {(1 + 6 - m6) % 6, (5 + 6 - m6) % 6}, 0, {}};
        // class items mod 210 and 30 by default; mod 6 and 2 too when forced everywhere
        for (uint32_t Q : {210u, 30u, 6u, 2u})
            if (d % Q == 0 && (Q > 6 || t.m_classes == 3)) ct.fine.push_back(class_items(Q, M_start));
    }
    return ct;
}

}  // namespace cs
