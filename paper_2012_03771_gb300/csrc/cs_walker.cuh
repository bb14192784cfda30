// The walker of one prime for the three-gap walk's one-walker chunks (odd m,
// or every m for odd d; one segment per prime), computed ahead of the walk by
// the preparation kernel k_tg_prep.  (Computed inside the 64-bit residue
// kernel right after K mod p instead, it made that kernel 80 registers wide and
// the two together 22% slower than apart.)
//
// With r' = Q r mod p, the two steps of the walk come from one run of
// Euclid's algorithm on (p, r') (tg_steps / tg_steps_w), and the class's first
// hit from the step basis in O(1) (first_hit32 / first_hit_w / first_hit64):
// the same work, in the same order and arithmetic, as the walk kernel does for
// an item it prepares itself, so the results and the solver statistics are
// identical.  The descriptor: d0 = {first m - M_start (NO_WALKER when no hit
// falls in the range), v at that m, d_a, u_b}, d1 = {steps of m a Q, b Q,
// clamped to M_inc}.
#pragma once
#include <stdint.h>

#include "cs_arith.cuh"
#include "cs_errors.h"

namespace cs {

constexpr uint32_t NO_WALKER = 0xffffffffu;

// v + k r mod p for a small k (v, r < p, 2p fits in UT)
template <class UT>
__device__ __forceinline__ UT add_times(UT v, UT r, uint32_t k, UT p) {
    for (; k; k--) {
        v += r;
        if (v >= p) v -= p;
    }
    return v;
}

// pp: the prime; r = K mod p; vv = (r M_start + SL) mod p; w = 2 SL > 0; M =
// M_inc; Q <= 2 and off0 < Q: the class of m walked.  Adds the solver's work to
// solves / levels and ERR_SOLVER_LIMIT to err when a run exceeds max_iter.
template <class UT>
__device__ __forceinline__ void prep_walker(UT pp, UT r, UT vv, UT w, uint64_t M, uint32_t Q, uint32_t off0,
                                            uint32_t max_iter, unsigned long long &solves,
                                            unsigned long long &levels, unsigned long long &err, uint4 &d0,
                                            uint2 &d1) {
    uint32_t it = 0;
    UT ma_ = 0, da_ = 0, mb_ = 0, ub_ = 0;
    uint64_t first = 0;
    // the class's first m is m = off0 (mod Q): v advances by r per m
    const uint32_t dd = off0;
    UT vk = add_times(vv, r, dd, pp);
    const UT rq = add_times(r, r, Q - 1, pp);
    bool ok;
    if constexpr (sizeof(UT) == 8) {
        if (w >= 1024) {
            uint64_t a64, b64;
            uint32_t da32, ub32;
            ok = tg_steps_w(pp, rq, (uint32_t)w, a64, da32, b64, ub32, it, max_iter);
            ma_ = a64; mb_ = b64; da_ = da32; ub_ = ub32;
        } else {
            ok = tg_steps<UT>(pp, rq, w, ma_, da_, mb_, ub_, it, max_iter);
        }
    } else {
        ok = tg_steps<UT>(pp, rq, w, ma_, da_, mb_, ub_, it, max_iter);
    }
    if (!ok) err |= ERR_SOLVER_LIMIT;
    solves += 2 + (vk > w);
    if (ok && vk > w) {
        if constexpr (sizeof(UT) == 4) {
            uint32_t y;
            first = (uint64_t)first_hit32(pp, rcp_rn((float)pp), w, ma_, da_, mb_, ub_, vk, y) * Q;
            vk = y;
        } else {
            const bool narrow_ab = w >= 1024 && ((uint64_t)ma_ | (uint64_t)mb_) < (1ull << 31);
            if (narrow_ab) {
                uint32_t y;
                first = first_hit_w(pp, rcp_rn(u64_to_f((uint64_t)pp)), (uint32_t)w, (uint32_t)ma_,
                                    (uint32_t)da_, (uint32_t)mb_, (uint32_t)ub_, vk, y) * Q;
                vk = (UT)y;
            } else {
                uint64_t y;
                first = first_hit64(pp, w, ma_, da_, mb_, ub_, vk, y) * Q;
                vk = (UT)y;
            }
        }
    }
    levels += it;
    const uint64_t mf = dd + first;
    const uint64_t sa = (uint64_t)ma_ * Q, sb = (uint64_t)mb_ * Q;
    d0 = make_uint4(ok && mf < M ? (uint32_t)mf : NO_WALKER, (uint32_t)vk, (uint32_t)da_, (uint32_t)ub_);
    d1 = make_uint2((uint32_t)(sa < M ? sa : M), (uint32_t)(sb < M ? sb : M));
}

}  // namespace cs
