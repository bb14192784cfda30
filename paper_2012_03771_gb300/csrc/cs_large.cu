// Large-prime kernel (primes T < p <= L), Section 3.2 "Large Prime Optimization".
//
// For a fixed p with r = K mod p, p divides a number of the interval around
// N = m K iff v(m) = (r m + SL) mod p <= 2 SL (Eq. modeq), and then x = SL - v.
// Each thread walks one prime over m in [M_start, M_start + M_inc):
//
//   LARGE_PAPER      as in the paper: from the current m, one G solve
//                    (Section 3.3) finds the next m whose v is in the window,
//                    the hit is recorded, m advances by one and the next solve
//                    starts there.
//   LARGE_THREE_GAP  the first m with r*m mod p in [p - 2SL, p - 1] (a step
//                    that lowers v by at most 2SL) and in [1, 2SL] (a step that
//                    raises it), i.e. G of those two windows; by the
//                    three-distance theorem the next hit after any hit is one of
//                    those steps or their sum (cf. Franke and Kleinjung,
//                    "Continued fractions and lattice sieving", SHARCS 2005), so
//                    after the first hit every further hit costs O(1).
//
// Each hit on a coprime m and a stored x clears one bit of the device bitset
// with a 32-bit atomic AND and counts one enumerated factor.
#include <atomic>
#include <new>
#include <vector>

#include "cs_arith.cuh"
#include "cs_internal.h"
#include "cs_walker.cuh"

namespace cs {

namespace {

constexpr int LARGE_THREADS = 256;

struct LargeArgs {
    DevPlan pl;
    const void *p, *r, *v;
    const unsigned long long *count;
    uint64_t cap;
    uint32_t n_seg;      // m-segments per prime (work items = primes x n_seg)
    uint64_t p_lo, p_hi; // walk only p_lo < p <= p_hi (v == NULL: shared cache chunk)
    MClasses mc;         // three-gap walk: m-classes walked (Q = 1: every m)
    // one-walker chunks: walkers prepared by k_tg_prep, per prime i
    // {first m - M_start (or NO_WALKER), v there, d_a, u_b} and {steps of m a, b}
    const uint4 *desc0;
    const uint2 *desc1;
};

// v0 = (r * M_start + SL) mod p, for primes from a shared residue cache
__device__ __forceinline__ uint32_t start_v(uint32_t r, uint64_t M_start, uint32_t SL, uint32_t p) {
    return (uint32_t)(((uint64_t)r * (M_start % p) + SL) % p);
}
__device__ __forceinline__ uint64_t start_v(uint64_t r, uint64_t M_start, uint32_t SL, uint64_t p) {
    return (uint64_t)(((unsigned __int128)r * (M_start % p) + SL) % p);
}

// (r * m + v) mod p for m < 2^31
__device__ __forceinline__ uint32_t advance(uint32_t v, uint32_t r, uint64_t m, uint32_t p) {
    return (uint32_t)(((uint64_t)r * m + v) % p);
}
__device__ __forceinline__ uint64_t advance(uint64_t v, uint64_t r, uint64_t m, uint64_t p) {
    return (uint64_t)(((unsigned __int128)r * m + v) % p);
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct Counters {
    // per lane and launch: F and hits stay far below 2^32 (at most a few million)
    uint32_t F = 0, hits = 0;
    unsigned long long solves = 0, levels = 0, err = 0;
};

// One hit of prime p at m = M_start + moff, raw offset z = x + SL = 2SL - v
// for v = (r m + SL) mod p <= 2SL.  Branch-free up to the atomic: the row and
// column tests are bit lookups in small tables (coprime-m mask, stored-x
// mask, each interleaved with its per-word prefix counts) that stay in L1.
// The prime is read (from the chunk's array, entry idx) only when N + x can be
// a sieving prime itself (K below 2^64).
// The fields of a plan that a hit reads, held in registers by the multi-job
// walk (its plan descriptors sit in shared memory, which the walkers' queue
// stores would otherwise make it reload at every hit); the one-chunk walk reads
// them from its kernel parameters.
struct HitView {
    const uint2 *row_tab, *col_tab;
    uint64_t *bits;
    uint32_t wpr, SL;
    int small_n, compact;
    uint64_t M_start, K64;
    const uint32_t *cls_word, *cmask, *cprefix;
    uint32_t n_cls, S32;
};
__device__ __forceinline__ HitView hit_view(const DevPlan &p) {
    return HitView{p.row_tab, p.col_tab, p.bits, p.wpr, p.SL, p.small_n, p.compact, p.M_start, p.K64,
                   p.cls_word, p.cmask, p.cprefix, p.n_cls, p.S32};
}

// BKT: the stored hit becomes a record in this CTA's region for its band of
// rows (slot from the CTA's per-band counter bkt_s in shared memory, one plain
// store); a full region clears directly.
// rt = row_tab[moff >> 5] {coprime-m mask, rows before}, ct = col_tab[z >> 5]
// {stored-x mask, columns before}: loaded by the caller, the walk one step
// ahead so that the loads are in flight while the previous hit is recorded.
// ROWS: m is known to be a row, and its row index is row_in (rt unused; the
// class-item walk with Q = d, literal layout).
template <class UT, class PV = DevPlan, bool BKT = false, bool ROWS = false>
__device__ __forceinline__ void record_hit_rc(const PV &pl, uint64_t moff, uint32_t z, uint2 rt, uint2 ct,
                                              const UT *Pp, uint32_t idx, Counters &c, uint32_t *bkt_s = nullptr,
                                              uint32_t row_in = 0) {
    const uint32_t ms = (uint32_t)moff;                  // bit of m in its 32-m word: ms mod 32
    // m coprime to d, x coprime to K
    bool ok = ROWS ? bit_of(ct.x, z) != 0 : (bit_of(rt.x, ms) & bit_of(ct.x, z)) != 0;
    if (pl.small_n) {
        unsigned __int128 n = (unsigned __int128)(pl.M_start + moff) * pl.K64 + z - pl.SL;
        ok = ok && n != (unsigned __int128)Pp[idx];      // N + x is p itself
    }
    const uint32_t row_below = ROWS ? 0u : __popc(bits_below(rt.x, ms));
    const uint32_t row = ROWS ? row_in : rt.y + row_below;
    uint32_t col = ct.y + __popc(bits_below(ct.x, z));
    bool store = ok;                                     // F counts every stored x coprime to K
    if (!ROWS && pl.compact && ok) {
        // the row's class keeps only x with gcd(N + x, d) = 1; class of the
        // first row of this 32-m word, plus the rows before m in the word
        uint32_t cls = __ldg(&pl.cls_word[moff >> 5]) + row_below;
        while (cls >= pl.n_cls) cls -= pl.n_cls;
        const uint32_t ccw = __ldg(&pl.cmask[(size_t)cls * pl.S32 + (z >> 5)]);
        col = __ldg(&pl.cprefix[(size_t)cls * pl.S32 + (z >> 5)]) + __popc(bits_below(ccw, z));
        store = bit_of(ccw, z) != 0;
    }
    // 32-bit view of the row's words: column col is bit (col mod 32) of word col >> 5
    if (store) {
        bool direct = true;
        if constexpr (BKT) {
            const uint32_t band = row >> pl.band_log;
            const uint32_t slot = atomicAdd(bkt_s + band, 1u);
            if (slot < pl.region_cap) {
                pl.bkt[((uint64_t)band * pl.n_regions + blockIdx.x) * pl.region_cap + slot] =
                    (row & ((1u << pl.band_log) - 1)) * (64 * pl.wpr) + col;
                direct = false;
            }
        }
        if (direct)
            atomicAnd(reinterpret_cast<unsigned int *>(pl.bits) + (uint64_t)row * (2 * pl.wpr) + (col >> 5),
                      ~bit_at(col));
    }
    c.F += ok;
}
template <class UT, class PV = DevPlan, bool BKT = false>
__device__ __forceinline__ void record_hit_z(const PV &pl, uint64_t moff, uint32_t z, const UT *Pp,
                                             uint32_t idx, Counters &c, uint32_t *bkt_s = nullptr) {
    record_hit_rc<UT, PV, BKT>(pl, moff, z, __ldg(&pl.row_tab[moff >> 5]), __ldg(&pl.col_tab[z >> 5]), Pp, idx, c,
                               bkt_s);
}
template <class UT>
__device__ __forceinline__ void record_hit(const DevPlan &pl, uint64_t moff, UT v, const UT *Pp, uint32_t idx,
                                           Counters &c) {
    record_hit_z<UT>(pl, moff, 2 * pl.SL - (uint32_t)v, Pp, idx, c);
}

template <class UT, class ST>
__global__ void __launch_bounds__(LARGE_THREADS) k_large(const LargeArgs a) {
    const DevPlan &pl = a.pl;
    const UT *Pp = reinterpret_cast<const UT *>(a.p);
    const UT *Rp = reinterpret_cast<const UT *>(a.r);
    const UT *Vp = reinterpret_cast<const UT *>(a.v);
    const uint64_t n = min((uint64_t)*a.count, a.cap);
    const UT w = (UT)(2 * pl.SL);
    const uint64_t M = pl.M_inc;
    const uint32_t max_iter = 4 * 8 * sizeof(UT) + 8;
    const uint32_t n_seg = a.n_seg;
    Counters c;
    if (M == 0) return;

    // work item = (prime, m-segment); consecutive items share a prime
    for (uint64_t item = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; item < n * n_seg;
         item += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t i = item / n_seg;
        const uint32_t sg = (uint32_t)(item - i * n_seg);
        const uint64_t m_lo = M * sg / n_seg, m_hi = M * (sg + 1) / n_seg;
        if (m_lo >= m_hi) continue;
        const uint64_t Mseg = m_hi - m_lo;      // walk m_lo + [0, Mseg)
        const UT p = Pp[i], r = Rp[i];
        if ((uint64_t)p <= a.p_lo || (uint64_t)p > a.p_hi) continue;
        UT v = Vp ? Vp[i] : start_v(r, pl.M_start, pl.SL, p);
        if (m_lo) v = advance(v, r, m_lo, p);
        uint32_t it = 0;
        {
            uint64_t m = 0;
            while (true) {
                if (v <= w) {
                    c.hits++;
                    record_hit<UT>(pl, m_lo + m, v, Pp, (uint32_t)i, c);
                    if (++m >= Mseg) break;
                    v += r;
                    if (v >= p) v -= p;
                    continue;
                }
                UT t, y;
                c.solves++;
                if (!g_solve<UT, ST>(p, r, (UT)(p - v), w, t, y, it, max_iter)) {
                    c.err |= ERR_SOLVER_LIMIT;
                    break;
                }
                if ((uint64_t)t >= Mseg - m) break;
                m += t;
                v = (UT)(v + y - p);
            }
        }
        c.levels += it;
    }

    const unsigned long long F = warp_sum(c.F), hits = warp_sum(c.hits);
    c.solves = warp_sum(c.solves);
    c.levels = warp_sum(c.levels);
    for (int o = 16; o; o >>= 1) c.err |= __shfl_xor_sync(0xffffffffu, c.err, o);
    if ((threadIdx.x & 31) == 0) {
        if (F) atomicAdd(pl.stats + ST_F_LARGE, F);
        if (c.solves) atomicAdd(pl.stats + ST_SOLVES, c.solves);
        if (c.levels) atomicAdd(pl.stats + ST_LEVELS, c.levels);
        if (hits) atomicAdd(pl.stats + ST_HITS_ALL, hits);
        if (c.err) atomicOr(pl.stats + ST_ERROR, c.err);
    }
}

// Three-gap walk with persistent lanes.  A warp prepares 32 work items at a
// time (one fused solve each: the two steps and the first hits of the item's
// m-segment) into a queue in shared memory; every lane then steps its own
// walker and, when its segment is exhausted, takes the next prepared walker
// from the queue, so that lanes stay busy although walkers have different
// numbers of hits.
//
// m-classes: rows are the m coprime to d, so when Q | d (Q = 6 or 2) the m that
// share a factor with Q can never be rows.  An item then walks only the NC
// classes m = c (mod Q) with gcd(c, Q) = 1, each as its own walker over
// j in m = m_c + Q j: v steps by r' = Q r mod p per unit of j, the two step
// windows are solved for r' (steps of Q j' in m), and each class needs its own
// first hit.  The walk visits a third of the hits (Q = 6) or half of them
// (Q = 2).  Class items (NC = 1, mc.items classes, Q = 30 or 210): each work
// item is one class of one (prime, m-segment), so the finer classes (4/15 or
// 8/35 of the hits) cost one Euclid run per class walker.  The two steps come from one run of Euclid's algorithm on (p, r')
// (tg_steps, the same answers as G for the two step windows); in the 32-bit
// walk the first hits follow from the two step vectors, a basis of the lattice
// of (j, r' j mod p) (first_hit32; first_hit64 in the 64-bit walk).
// A prepared walker: after its first hit v and the steps of v are at most
// 2SL < 2^22, so 32 bits hold them for both prime widths; the prime itself is
// referenced by its index in the chunk's arrays.
template <class MT>
struct TGItem {
    MT moff, end;                  // current m - M_start, end of the segment
    uint32_t v, idx, da, ub;       // v = (r m + SL) mod p, prime index, steps of v
    MT ma, mb;                     // steps of m (clamped to M_inc)
};

// three-gap steps per lane between queue checks, class walkers (class items
// and the two walkers mod 6): their m-segments hold nearly the same number of
// hits (about the walked hits per item, 128), so the lanes of a warp finish
// their walkers at nearly the same time and waiting for them costs little,
// while each queue check costs its ballots and branches.  large_1019 walk: 720
// ms at 8 steps, 689 at 16, 656 at 48, 625 at 128, 617-618 at 256 and more;
// search_953 (fewer hits per item): 4.14, 4.08, 4.13, 4.10, 4.20-4.48 ms.
#ifndef CS_TG_STEPS
#define CS_TG_STEPS 128
#endif
// one-walker items (odd m or every m; the light chunks, a few hits per walker):
// four steps measured best of 2, 3, 4, 6, 8
#ifndef CS_TG_STEPS_ALL_M
#define CS_TG_STEPS_ALL_M 4
#endif
constexpr int TG_STEPS = CS_TG_STEPS;               // class walks (long walkers)
constexpr int TG_STEPS_ALL_M = CS_TG_STEPS_ALL_M;   // one-walker items (the light chunks)
constexpr int TG_WARPS = LARGE_THREADS / 32;

// the same for k < 2^31 in one reduction (fr = rcp_rn(p) for 32-bit p)
__device__ __forceinline__ uint32_t mul_add_mod(uint32_t v, uint32_t r, uint32_t k, uint32_t p, float fr) {
    int64_t rem;
    udiv64_est((uint64_t)r * k + v, p, fr, rem);     // quotient <= k
    return (uint32_t)rem;
}
__device__ __forceinline__ uint64_t mul_add_mod(uint64_t v, uint64_t r, uint32_t k, uint64_t p, float) {
    return advance(v, r, k, p);
}

// resident CTAs per SM the 32-bit walk is compiled for: three (85 registers)
// measured 7% faster than four (64 registers, with spills) on a GB300
#ifndef CS_TG_MIN_BLOCKS
#define CS_TG_MIN_BLOCKS 3
#endif
// the same for the 64-bit walk (primes above 2^30): three CTAs (80 registers,
// a few spills) measured 19% faster than one (136-154 registers) on L = 1e11
#ifndef CS_TG_MIN_BLOCKS_WIDE
#define CS_TG_MIN_BLOCKS_WIDE 3
#endif

// One warp's share of a walk: the batches first, first + n_warps, ... of 32
// work items of the chunk that `a` describes, prepared into the warp's queue q
// and walked by its lanes until the share is done and the queue is empty;
// then the warp's counters go to the plan's statistics.  item_off: the class
// residues of class items (shared memory).
// CI: 0 = m-class walkers, 1 = class items, 2 = class items mod Q = d in the
// literal layout, whose rows follow from the walker's steps: every walked m is
// a row, and a step of k Q in m passes k phi(Q) rows.
// PRE: the walkers come prepared by k_tg_prep (one-walker items, one segment).
template <class UT, class ST, class MT, int NC, int CI, bool JOBS = false, bool BKT = false, bool PRE = false>
__device__ __forceinline__ void walk_warp(const LargeArgs &a, TGItem<MT> *q, const uint8_t *item_off,
                                          uint64_t first, uint64_t n_warps, uint32_t *bkt_s = nullptr) {
    static_assert(!CI || NC == 1, "class items walk one class per item");
    static_assert(!PRE || (NC == 1 && !CI && !JOBS), "prepared walkers: one-walker items");
    constexpr int QCAP = 32 * (NC + 1);   // a refill adds at most 32 NC walkers
    const uint32_t n_cls_items = CI ? a.mc.items : 1;
    const DevPlan &pl = a.pl;
    // the hit path's plan fields: kernel parameters, or registers for the multi-job walk
    [[maybe_unused]] const HitView hv = JOBS ? hit_view(pl) : HitView{};
    const UT *Pp = reinterpret_cast<const UT *>(a.p);
    const UT *Rp = reinterpret_cast<const UT *>(a.r);
    const UT *Vp = reinterpret_cast<const UT *>(a.v);
    const uint64_t n = min((uint64_t)*a.count, a.cap);
    const UT w = (UT)(2 * pl.SL);
    const uint64_t M = pl.M_inc;
    const uint32_t Q = a.mc.Q;
    const uint32_t max_iter = 4 * 8 * sizeof(UT) + 8;
    const uint32_t n_seg = a.n_seg;
    const unsigned lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1;
    const uint64_t n_items = n * n_seg * n_cls_items;
    // any step >= M ends a walker (its segment is at most M long); two clamped
    // steps still add up below 2^32
    const uint64_t cap_step = M;
    const uint64_t seg_len = (M + n_seg - 1) / n_seg;
    Counters c;
    if (M == 0) return;

    uint64_t batch = first;            // next batch of 32 items to prepare
    uint32_t qhead = 0, qcount = 0;    // warp-uniform ring state
    bool active = false;
    // walker: m offset, segment end, raw offset z = 2SL - v, and the three steps
    // precomputed: down (v >= d_a, z <= 2SL - d_a): m += a, z += d_a; up
    // (v <= 2SL - u_b, z >= u_b): m += b, z -= u_b; else m += a + b,
    // z += d_a - u_b
    MT moff = 0, end = 0, ma = 0, mb = 0, mab = 0;
    uint32_t z = 0, idx = 0, da = 0, ub = 0, wmda = 0, nub = 0, dmu = 0;
    // the current hit's row and column table words (loaded one step ahead)
    const uint2 *row_tab = JOBS ? hv.row_tab : pl.row_tab;
    const uint2 *col_tab = JOBS ? hv.col_tab : pl.col_tab;
    uint2 rt = make_uint2(0, 0), ct = make_uint2(0, 0);
    constexpr bool ROWS = CI == 2;
    uint32_t row = 0, ra = 0, rb = 0, rab = 0;   // ROWS: row of the current hit, rows per step

    while (true) {
        // refill: prepare 32 items when the queue can take their walkers
        if (qcount + 32 * NC <= QCAP && batch * 32 < n_items) {
            const uint64_t item = batch * 32 + lane;
            batch += n_warps;
            bool push[NC];
            MT first_m[NC];
            UT first_v[NC];
            TGItem<MT> e;
#pragma unroll
            for (int k = 0; k < NC; k++) push[k] = false;
            if (PRE && item < n_items) {
                const uint4 d = a.desc0[item];
                const uint2 st = a.desc1[item];
                push[0] = d.x != NO_WALKER;
                first_m[0] = (MT)d.x;
                first_v[0] = (UT)d.y;
                e.end = (MT)M;
                e.idx = (uint32_t)item;
                e.da = d.z;
                e.ub = d.w;
                e.ma = (MT)st.x;
                e.mb = (MT)st.y;
            } else if (!PRE && item < n_items) {
                uint64_t i = item, m_lo = 0, m_hi = M;
                uint32_t off0 = a.mc.off[0];               // NC = 1: the class walked
                if constexpr (CI) {
                    // consecutive items are the classes of one (prime, segment)
                    i = n_items >> 32 ? item / n_cls_items : (uint32_t)item / n_cls_items;
                    off0 = item_off[item - i * n_cls_items];
                }
                if (n_seg > 1) {
                    // segments of seg_len m (the last one shorter), segment-major:
                    // the items in flight at one time share a segment, so that
                    // their bit clears fall in one band of rows, which stays in L2
                    const uint64_t ps = i;
                    const uint32_t sg = n_items >> 32 ? (uint32_t)(ps / n) : (uint32_t)ps / (uint32_t)n;
                    i = ps - (uint64_t)sg * n;
                    m_lo = (uint64_t)sg * seg_len;
                    m_hi = min(M, m_lo + seg_len);
                }
                const UT pp = Pp[i], r = Rp[i];
                bool ok = m_lo < m_hi && (uint64_t)pp > a.p_lo && (uint64_t)pp <= a.p_hi;
                UT vv = ok ? (Vp ? Vp[i] : start_v(r, pl.M_start, pl.SL, pp)) : (UT)0;
                if (ok && m_lo) {
                    if constexpr (sizeof(UT) == 4) {
                        // (r m_lo + v) mod p: quotient below m_lo + 1 < 2^31
                        int64_t rm;
                        udiv64_est((uint64_t)r * m_lo + vv, pp, rcp_rn((float)pp), rm);
                        vv = (UT)rm;
                    } else {
                        vv = advance(vv, r, m_lo, pp);
                    }
                }
                uint32_t it = 0;
                UT ma_ = 0, da_ = 0, mb_ = 0, ub_ = 0;
                uint64_t first[NC];
                UT vk[NC];
                uint32_t dk[NC];
#pragma unroll
                for (int k = 0; k < NC; k++) {
                    first[k] = 0;
                    vk[k] = vv;
                    dk[k] = 0;
                }
                if (ok && w == 0) {
                    // SL = 0 (Q = 1, NC = 1): every p-th m; v stays 0
                    ma_ = pp;
                    if (vv > w) {
                        UT t, y;
                        c.solves++;
                        ok = g_solve<UT, ST>(pp, r, (UT)(pp - vv), w, t, y, it, max_iter);
                        if (!ok) c.err |= ERR_SOLVER_LIMIT;
                        first[0] = t;
                        vk[0] = (UT)(vv + y - pp);
                    }
                } else if (ok) {
                    // class k starts at the first m_lo + dk with m = c_k (mod Q)
                    const uint32_t lo_res = (Q == 1 || m_lo == 0) ? 0u : (uint32_t)m_lo % Q;   // m_lo < M_inc < 2^31
                    const float fq = rcp_rn((float)pp);
                    // r' = Q r mod p (Q <= 6 by additions, class items Q <= 210 by one reduction)
                    const bool big_q = CI && Q > 6;
                    const UT rq = big_q ? mul_add_mod((UT)0, r, Q, pp, fq) : add_times(r, r, Q - 1, pp);
#pragma unroll
                    for (int k = 0; k < NC; k++) {
                        uint32_t dd = (NC == 1 ? off0 : a.mc.off[k]) + Q - lo_res;
                        if (dd >= Q) dd -= Q;
                        dk[k] = dd;
                        vk[k] = big_q ? mul_add_mod(vv, r, dd, pp, fq) : add_times(vv, r, dd, pp);
                    }
                    // the two steps from one run of Euclid's algorithm on (p, r');
                    // for 64-bit primes and 2SL >= 1024 mostly in 32-bit steps
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
                    if (!ok) c.err |= ERR_SOLVER_LIMIT;
                    uint32_t n_first = 0;
#pragma unroll
                    for (int k = 0; k < NC; k++) n_first += vk[k] > w;
                    c.solves += 2 + n_first;
                    if constexpr (sizeof(UT) == 4) {
                        // each walker's first hit from the step basis, without a solve
#pragma unroll
                        for (int k = 0; k < NC; k++) {
                            if (ok && vk[k] > w) {
                                uint32_t y;
                                first[k] = (uint64_t)first_hit32(pp, fq, w, ma_, da_, mb_, ub_, vk[k], y) * Q;
                                vk[k] = y;
                            }
                        }
                    } else if (ok && n_first) {
                        // 64-bit (p < 2^40, 2SL <= 2^21): the same with 64-bit
                        // products (first_hit_w) when both steps are below 2^31 and
                        // 2SL >= 1024, else with 128-bit ones (first_hit64)
                        const bool narrow_ab = w >= 1024 && ((uint64_t)ma_ | (uint64_t)mb_) < (1ull << 31);
                        const float fp = rcp_rn(u64_to_f((uint64_t)pp));
#pragma unroll
                        for (int k = 0; k < NC; k++) {
                            if (vk[k] > w) {
                                if (narrow_ab) {
                                    uint32_t y;
                                    first[k] = first_hit_w(pp, fp, (uint32_t)w, (uint32_t)ma_, (uint32_t)da_,
                                                           (uint32_t)mb_, (uint32_t)ub_, vk[k], y) * Q;
                                    vk[k] = (UT)y;
                                } else {
                                    uint64_t y;
                                    first[k] = first_hit64(pp, w, ma_, da_, mb_, ub_, vk[k], y) * Q;
                                    vk[k] = (UT)y;
                                }
                            }
                        }
                    }
                }
                c.levels += it;
                if (ok) {
#pragma unroll
                    for (int k = 0; k < NC; k++) {
                        const uint64_t mf = m_lo + dk[k] + first[k];
                        push[k] = mf < m_hi;
                        first_m[k] = (MT)mf;
                        first_v[k] = vk[k];
                    }
                    const uint64_t sa = (uint64_t)ma_ * Q, sb = (uint64_t)mb_ * Q;
                    e.end = (MT)m_hi;
                    e.idx = (uint32_t)i;
                    e.da = (uint32_t)da_;
                    e.ub = (uint32_t)ub_;
                    e.ma = (MT)(sa < cap_step ? sa : cap_step);
                    e.mb = (MT)(sb < cap_step ? sb : cap_step);
                }
            }
            uint32_t tail = qhead + qcount;
#pragma unroll
            for (int k = 0; k < NC; k++) {
                const unsigned pm = __ballot_sync(0xffffffffu, push[k]);
                if (push[k]) {
                    TGItem<MT> ek = e;
                    ek.moff = first_m[k];
                    ek.v = (uint32_t)first_v[k];
                    q[(tail + __popc(pm & lt_mask)) % QCAP] = ek;
                }
                tail += __popc(pm);
            }
            qcount = tail - qhead;
            __syncwarp();
        }
        // hand queued items to idle lanes
        const unsigned idle = __ballot_sync(0xffffffffu, !active);
        if (idle && qcount) {
            const uint32_t rank = __popc(idle & lt_mask);
            const uint32_t take = min((uint32_t)__popc(idle), qcount);
            if (!active && rank < take) {
                const TGItem<MT> e = q[(qhead + rank) % QCAP];
                moff = e.moff; end = e.end; z = (uint32_t)w - e.v; idx = e.idx; da = e.da; ub = e.ub;
                ma = e.ma; mb = e.mb;
                mab = ma + mb;                       // ma, mb <= M_inc < 2^31
                wmda = (uint32_t)w - da;
                nub = 0u - ub;
                dmu = da - ub;                       // both wrap; z ends in [0, 2SL]
                rt = __ldg(&row_tab[moff >> 5]);
                ct = __ldg(&col_tab[z >> 5]);
                if constexpr (ROWS) {
                    // steps are multiples of Q (a clamped one ends the walker)
                    row = rt.y + __popc(bits_below(rt.x, (uint32_t)moff));
                    ra = (uint32_t)ma / Q * n_cls_items;
                    rb = (uint32_t)mb / Q * n_cls_items;
                    rab = ra + rb;
                }
                active = true;
            }
            qhead = (qhead + take) % QCAP;
            qcount -= take;
            __syncwarp();
        }
        const unsigned act = __ballot_sync(0xffffffffu, active);
        if (!act) {
            if (qcount == 0 && batch * 32 >= n_items) break;
            continue;
        }
        // up to TG_STEPS three-distance steps per active lane between queue
        // checks (each step as selects)
        constexpr int STEPS = NC == 1 && !CI ? TG_STEPS_ALL_M : TG_STEPS;
        int u = 0;
        for (; u < STEPS && active; u++) {
            const bool down = z <= wmda;
            const bool up = z >= ub;
            const uint32_t zn = z + (down ? da : (up ? nub : dmu));
            const MT step = down ? ma : (up ? mb : mab);
            active = step < end - moff;
            const MT mn = moff + step;
            // the next hit's table words, in flight while this one is recorded
            uint2 rtn = rt, ctn = ct;
            if (active) {
                if constexpr (!ROWS) rtn = __ldg(&row_tab[mn >> 5]);
                ctn = __ldg(&col_tab[zn >> 5]);
            }
            if constexpr (JOBS)
                record_hit_rc<UT>(hv, (uint64_t)moff, z, rt, ct, Pp, idx, c);
            else
                record_hit_rc<UT, DevPlan, BKT, ROWS>(pl, (uint64_t)moff, z, rt, ct, Pp, idx, c, bkt_s, row);
            if constexpr (ROWS) row += down ? ra : (up ? rb : rab);
            rt = rtn;
            ct = ctn;
            z = zn;
            moff = mn;
        }
        c.hits += u;                                 // one hit per step taken
    }

    const unsigned long long F = warp_sum(c.F), hits = warp_sum(c.hits);
    c.solves = warp_sum(c.solves);
    c.levels = warp_sum(c.levels);
    for (int o = 16; o; o >>= 1) c.err |= __shfl_xor_sync(0xffffffffu, c.err, o);
    if (lane == 0) {
        if (F) atomicAdd(pl.stats + ST_F_LARGE, F);
        if (c.solves) atomicAdd(pl.stats + ST_SOLVES, c.solves);
        if (c.levels) atomicAdd(pl.stats + ST_LEVELS, c.levels);
        if (hits) atomicAdd(pl.stats + ST_HITS_ALL, hits);
        if (c.err) atomicOr(pl.stats + ST_ERROR, c.err);
    }
}

template <class UT, class ST, class MT, int NC, int CI = 0, bool BKT = false, bool PRE = false>
__global__ void __launch_bounds__(LARGE_THREADS, sizeof(UT) == 4 ? CS_TG_MIN_BLOCKS : CS_TG_MIN_BLOCKS_WIDE) k_large_tg(const LargeArgs a) {
    constexpr int QCAP = 32 * (NC + 1);
    __shared__ TGItem<MT> queue[TG_WARPS][QCAP];
    __shared__ uint8_t item_off[CI ? MAX_CLASS_ITEMS : 1];   // class items: residue of each class
    extern __shared__ uint32_t bkt_s[];                      // BKT: records in this CTA's region per band
    const DevPlan &pl = a.pl;
    if constexpr (CI) {
        if (threadIdx.x == 0) {
#pragma unroll
            for (uint32_t k = 0; k < MAX_CLASS_ITEMS; k++) item_off[k] = a.mc.item_off[k];
        }
    }
    if constexpr (BKT)
        for (uint32_t b = threadIdx.x; b < pl.n_bands; b += LARGE_THREADS)
            bkt_s[b] = pl.bkt_cnt[(uint64_t)b * pl.n_regions + blockIdx.x];
    if constexpr (CI || BKT) __syncthreads();
    walk_warp<UT, ST, MT, NC, CI, false, BKT, PRE>(a, queue[threadIdx.x >> 5], item_off,
                                              (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5,
                                              ((uint64_t)gridDim.x * blockDim.x) >> 5, bkt_s);
    if constexpr (BKT) {
        // the region counts for the next launch (slots past the region's end were cleared directly)
        __syncthreads();
        for (uint32_t b = threadIdx.x; b < pl.n_bands; b += LARGE_THREADS)
            pl.bkt_cnt[(uint64_t)b * pl.n_regions + blockIdx.x] = min(bkt_s[b], pl.region_cap);
    }
}

// Walker preparation for the one-walker chunks (odd m, or every m; one
// segment per prime): per prime, the class's first v, the two steps from one
// Euclid run and the first hit, exactly as the walk prepares an item, written
// as a descriptor that the walk reads instead.  The Euclid runs are serial
// chains of float-estimate divisions (one per step, about a dozen steps per
// prime); the walk kernel, with its queue and hit path, holds 80 registers and
// keeps 24 warps per SM, too few to hide them, while this kernel keeps one
// prime per thread and many more warps.  Solver statistics and errors are
// counted here.
constexpr int PREP_THREADS = 256;
template <class UT, class ST>
__global__ void __launch_bounds__(PREP_THREADS) k_tg_prep(const LargeArgs a, uint4 *desc0, uint2 *desc1) {
    const DevPlan &pl = a.pl;
    const UT *Pp = reinterpret_cast<const UT *>(a.p);
    const UT *Rp = reinterpret_cast<const UT *>(a.r);
    const UT *Vp = reinterpret_cast<const UT *>(a.v);
    const uint64_t n = min((uint64_t)*a.count, a.cap);
    const UT w = (UT)(2 * pl.SL);
    const uint64_t M = pl.M_inc;
    const uint32_t Q = a.mc.Q, off0 = a.mc.off[0];
    const uint32_t max_iter = 4 * 8 * sizeof(UT) + 8;
    unsigned long long solves = 0, levels = 0, err = 0;
    const uint64_t stride = (uint64_t)gridDim.x * PREP_THREADS;
    for (uint64_t i = blockIdx.x * (uint64_t)PREP_THREADS + threadIdx.x; i < n; i += stride) {
        const UT pp = Pp[i], r = Rp[i];
        uint4 d0 = make_uint4(NO_WALKER, 0, 0, 0);
        uint2 d1 = make_uint2(0, 0);
        if ((uint64_t)pp > a.p_lo && (uint64_t)pp <= a.p_hi) {
            const UT vv = Vp ? Vp[i] : start_v(r, pl.M_start, pl.SL, pp);
            prep_walker<UT>(pp, r, vv, w, M, Q, off0, max_iter, solves, levels, err, d0, d1);
        }
        desc0[i] = d0;
        desc1[i] = d1;
    }
    solves = warp_sum(solves);
    levels = warp_sum(levels);
    for (int o = 16; o; o >>= 1) err |= __shfl_xor_sync(0xffffffffu, err, o);
    if ((threadIdx.x & 31) == 0) {
        if (solves) atomicAdd(pl.stats + ST_SOLVES, solves);
        if (levels) atomicAdd(pl.stats + ST_LEVELS, levels);
        if (err) atomicOr(pl.stats + ST_ERROR, err);
    }
}

// Clears the bucketed records: each CTA takes whole regions one at a time from
// a shared counter (bkt_cnt[n_bands * n_regions]) in band-major order, so that
// the regions in work at one time belong to one or two consecutive bands,
// whose words stay in L2 while their clears land (a fixed stride instead lets
// the CTAs with small regions run ahead into later bands; a warp per region
// keeps about ten bands in work, which with bands above 4 MB no longer fit).
// The records are read once, with loads marked evict-first so that they do
// not push the bands' words out of L2.  Regions start on 16-byte boundaries
// (region_cap is a multiple of 4): each thread loads two 16-byte groups of
// records before their eight clears.
constexpr int APPLY_THREADS = 256;
__global__ void __launch_bounds__(APPLY_THREADS) k_apply_buckets(const DevPlan pl) {
    uint32_t *bits = reinterpret_cast<uint32_t *>(pl.bits);
    const uint32_t n_reg = pl.n_bands * pl.n_regions;
    const uint64_t band_words = (uint64_t)(2 * pl.wpr) << pl.band_log;
    __shared__ uint32_t q_s;
    for (;;) {
        __syncthreads();                                 // every thread has read the last q_s
        if (threadIdx.x == 0) q_s = atomicAdd(pl.bkt_cnt + n_reg, 1u);
        __syncthreads();
        const uint32_t q = q_s;
        if (q >= n_reg) break;
        const uint32_t n = min(pl.bkt_cnt[q], pl.region_cap);
        if (threadIdx.x == 0 && n) atomicAdd(pl.stats + ST_RECORDS, (unsigned long long)n);
        const uint32_t *src = pl.bkt + (uint64_t)q * pl.region_cap;
        const uint4 *src4 = reinterpret_cast<const uint4 *>(src);
        uint32_t *dst = bits + (q / pl.n_regions) * band_words;
        const uint32_t n4 = n / 4;
        uint32_t i = threadIdx.x;
        for (; i + APPLY_THREADS < n4; i += 2 * APPLY_THREADS) {
            const uint4 a = __ldcs(src4 + i), b = __ldcs(src4 + i + APPLY_THREADS);
            atomicAnd(dst + (a.x >> 5), ~bit_at(a.x));
            atomicAnd(dst + (a.y >> 5), ~bit_at(a.y));
            atomicAnd(dst + (a.z >> 5), ~bit_at(a.z));
            atomicAnd(dst + (a.w >> 5), ~bit_at(a.w));
            atomicAnd(dst + (b.x >> 5), ~bit_at(b.x));
            atomicAnd(dst + (b.y >> 5), ~bit_at(b.y));
            atomicAnd(dst + (b.z >> 5), ~bit_at(b.z));
            atomicAnd(dst + (b.w >> 5), ~bit_at(b.w));
        }
        if (i < n4) {
            const uint4 a = __ldcs(src4 + i);
            atomicAnd(dst + (a.x >> 5), ~bit_at(a.x));
            atomicAnd(dst + (a.y >> 5), ~bit_at(a.y));
            atomicAnd(dst + (a.z >> 5), ~bit_at(a.z));
            atomicAnd(dst + (a.w >> 5), ~bit_at(a.w));
        }
        for (uint32_t k = 4 * n4 + threadIdx.x; k < n; k += APPLY_THREADS) {
            const uint32_t r = __ldcs(src + k);
            atomicAnd(dst + (r >> 5), ~bit_at(r));
        }
    }
}

// resident CTAs per SM the multi-job walk is compiled for: its hit path keeps
// the plan's fields in registers, which at three CTAs per SM would spill
#ifndef CS_TG_JOBS_MIN_BLOCKS
#define CS_TG_JOBS_MIN_BLOCKS 2
#endif
template <class UT, class ST, class MT, int NC, int CI = 0>
__global__ void __launch_bounds__(LARGE_THREADS, CS_TG_JOBS_MIN_BLOCKS)
    k_large_tg_jobs(const LargeArgs *jobs, uint32_t n_jobs) {
    constexpr int QCAP = 32 * (NC + 1);
    __shared__ TGItem<MT> queue[TG_WARPS][QCAP];
    __shared__ LargeArgs job[TG_WARPS];
    const unsigned lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const uint64_t warp_id = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    static_assert(sizeof(LargeArgs) % 4 == 0, "copied as 32-bit words");
    constexpr uint32_t WORDS = sizeof(LargeArgs) / 4;
    uint64_t dealt = 0;                 // batches of the jobs before j
    for (uint32_t j = 0; j < n_jobs; j++) {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(jobs + j);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&job[wib]);
        for (uint32_t k = lane; k < WORDS; k += 32) dst[k] = __ldg(src + k);
        __syncwarp();
        const LargeArgs &a = job[wib];
        const uint64_t n = min((uint64_t)*a.count, a.cap);
        const uint64_t batches = (n * a.n_seg * (CI ? a.mc.items : 1) + 31) / 32;
        const uint64_t first = (warp_id + n_warps - dealt % n_warps) % n_warps;
        walk_warp<UT, ST, MT, NC, CI, true>(a, queue[wib], a.mc.item_off, first, n_warps);
        dealt += batches;
        __syncwarp();
    }
}

template <class UT, class ST>
__global__ void k_modsolve(const uint64_t *p, const uint64_t *K, const uint64_t *L,
                           const uint64_t *R, uint64_t *m, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        UT t, y;
        uint32_t it = 0;
        const UT pp = (UT)p[i];
        const UT kk = (UT)(K[i] % p[i]);
        bool ok = kk != 0 && g_solve<UT, ST>(pp, kk, (UT)L[i], (UT)(R[i] - L[i]), t, y, it,
                                             4 * 8 * sizeof(UT) + 8);
        m[i] = ok ? (uint64_t)t : ~0ull;
    }
}

}  // namespace

bool prep_eligible(const DevPlan &pl, int mode, uint32_t n_seg, MClasses mc) {
    return mode != LARGE_PAPER && pl.SL > 0 && (n_seg <= 1) && !mc.items && mc.n == 1 && mc.Q <= 2 &&
           mc.off[0] < mc.Q;
}

cudaError_t launch_tg_prep(const DevPlan &pl, bool narrow, const void *p, const void *r, const void *v,
                           const unsigned long long *count, uint64_t cap, uint64_t p_lo, uint64_t p_hi,
                           MClasses mc, uint4 *desc0, uint2 *desc1, cudaStream_t stream) {
    LargeArgs a{pl, p, r, v, count, cap, 1, p_lo, p_hi, mc, nullptr, nullptr};
    void (*kern)(const LargeArgs, uint4 *, uint2 *) =
        narrow ? k_tg_prep<uint32_t, int32_t> : k_tg_prep<uint64_t, int64_t>;
    // one wave of resident CTAs, looked up once per width
    static std::atomic<int> resident[2];
    std::atomic<int> &cached = resident[narrow ? 1 : 0];
    int per_sm = cached.load(std::memory_order_relaxed);
    if (per_sm == 0) {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PREP_THREADS, 0) != cudaSuccess ||
            per_sm <= 0)
            per_sm = 1;
        cached.store(per_sm, std::memory_order_relaxed);
    }
    kern<<<sm_count() * per_sm, PREP_THREADS, 0, stream>>>(a, desc0, desc1);
    return cudaGetLastError();
}

cudaError_t launch_large(const DevPlan &pl, bool narrow, int mode, const void *p, const void *r,
                         const void *v, const unsigned long long *count, uint64_t cap, uint32_t n_seg,
                         int grid, cudaStream_t stream, uint64_t p_lo, uint64_t p_hi, MClasses mc,
                         const uint4 *desc0, const uint2 *desc1) {
    const bool items_ok = mc.items == mc.n && mc.n <= MAX_CLASS_ITEMS && mc.Q <= 256;
    if (mc.Q == 0 || mc.n < 1 || mc.n > mc.Q || (mc.items ? !items_ok : mc.n > 2) || pl.SL == 0) mc = EVERY_M;
    // walk kernel: 0 = one walker per item, 1 = two classes per item, 2 = class
    // items, 3 = class items mod Q = d with rows from the steps (32-bit primes,
    // literal layout)
    int kind = mc.items ? 2 : mc.n == 2 ? 1 : 0;
    if (kind == 2 && narrow && mode != LARGE_PAPER && !pl.compact && mc.Q == pl.d) kind = 3;
    // 4 = one walker per item, prepared by k_tg_prep
    const bool pre = desc0 && desc1 && kind == 0 && prep_eligible(pl, mode, n_seg, mc);
    if (pre) kind = 4;
    LargeArgs a{pl, p, r, v, count, cap, n_seg ? n_seg : 1, p_lo, p_hi, mc, pre ? desc0 : nullptr,
                pre ? desc1 : nullptr};
    // bucketed hits: three-gap walk only (the paper's walk clears directly)
    const int bkt = (pl.bucket && mode != LARGE_PAPER) ? 1 : 0;
    if (!bkt) a.pl.bucket = 0;
    const size_t dyn = bkt ? (size_t)pl.n_bands * sizeof(uint32_t) : 0;
    void (*walk)(const LargeArgs) = nullptr;
    if (narrow) {
        walk = kind == 4 ? (bkt ? k_large_tg<uint32_t, int32_t, uint32_t, 1, 0, true, true>
                                : k_large_tg<uint32_t, int32_t, uint32_t, 1, 0, false, true>)
             : kind == 3 ? (bkt ? k_large_tg<uint32_t, int32_t, uint32_t, 1, 2, true>
                                : k_large_tg<uint32_t, int32_t, uint32_t, 1, 2>)
             : kind == 2 ? (bkt ? k_large_tg<uint32_t, int32_t, uint32_t, 1, 1, true>
                                : k_large_tg<uint32_t, int32_t, uint32_t, 1, 1>)
             : kind == 1 ? (bkt ? k_large_tg<uint32_t, int32_t, uint32_t, 2, 0, true>
                                : k_large_tg<uint32_t, int32_t, uint32_t, 2>)
                         : (bkt ? k_large_tg<uint32_t, int32_t, uint32_t, 1, 0, true>
                                : k_large_tg<uint32_t, int32_t, uint32_t, 1>);
    } else {
        walk = kind == 4 ? (bkt ? k_large_tg<uint64_t, int64_t, uint32_t, 1, 0, true, true>
                                : k_large_tg<uint64_t, int64_t, uint32_t, 1, 0, false, true>)
             : kind == 2 ? (bkt ? k_large_tg<uint64_t, int64_t, uint32_t, 1, 1, true>
                                : k_large_tg<uint64_t, int64_t, uint32_t, 1, 1>)
             : kind == 1 ? (bkt ? k_large_tg<uint64_t, int64_t, uint32_t, 2, 0, true>
                                : k_large_tg<uint64_t, int64_t, uint32_t, 2>)
                         : (bkt ? k_large_tg<uint64_t, int64_t, uint32_t, 1, 0, true>
                                : k_large_tg<uint64_t, int64_t, uint32_t, 1>);
    }
    // the three-gap walk's lanes are persistent: by default one wave of
    // resident CTAs (a partial last wave left SMs idle: 3% slower measured);
    // the paper's walk takes eight CTAs per SM
    if (grid <= 0) {
        grid = sm_count() * 8;
        if (mode != LARGE_PAPER) {
            // looked up once per [narrow][kind][bucketed] (the bucket counters,
            // at most 16 KB, do not change the occupancy bound by registers)
            static std::atomic<int> resident[2][5][2];
            std::atomic<int> &cached = resident[narrow ? 1 : 0][kind][bkt];
            int per_sm = cached.load(std::memory_order_relaxed);
            if (per_sm == 0) {
                cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, walk, LARGE_THREADS,
                                                                              bkt ? 4 * BKT_MAX_BANDS : 0);
                if (e != cudaSuccess || per_sm <= 0) per_sm = -1;
                cached.store(per_sm, std::memory_order_relaxed);
            }
            if (per_sm > 0) grid = sm_count() * per_sm;
        }
    }
    // every walking CTA owns a region per band
    if (bkt && (uint32_t)grid > pl.n_regions) grid = (int)pl.n_regions;
    // m - M_start < M_inc < 2^31: 32-bit m offsets in both widths
    if (mode == LARGE_PAPER) {
        if (narrow)
            k_large<uint32_t, int32_t><<<grid, LARGE_THREADS, 0, stream>>>(a);
        else
            k_large<uint64_t, int64_t><<<grid, LARGE_THREADS, 0, stream>>>(a);
    } else {
        walk<<<grid, LARGE_THREADS, dyn, stream>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_apply_buckets(const DevPlan &pl, cudaStream_t stream) {
    if (!pl.bucket || pl.n_bands == 0) return cudaSuccess;
    // four CTAs per SM, each on one region at a time: the regions in work span
    // about 1.3 bands (152 x 3 regions per band)
    k_apply_buckets<<<sm_count() * 4, APPLY_THREADS, 0, stream>>>(pl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the region counts and the apply's region counter back to 0
    return cudaMemsetAsync(pl.bkt_cnt, 0, ((size_t)pl.n_bands * pl.n_regions + 1) * sizeof(uint32_t), stream);
}

struct WalkJobs {
    // one group per walk kernel: [narrow][kind]
    LargeArgs *d_jobs[2][3] = {{nullptr, nullptr, nullptr}, {nullptr, nullptr, nullptr}};
    uint32_t n_jobs[2][3] = {{0, 0, 0}, {0, 0, 0}};
};

namespace {
// MClasses as launch_large normalises them, and the walk kernel they select
int walk_kind(MClasses &mc, uint32_t SL) {
    const bool items_ok = mc.items == mc.n && mc.n <= MAX_CLASS_ITEMS && mc.Q <= 256;
    if (mc.Q == 0 || mc.n < 1 || mc.n > mc.Q || (mc.items ? !items_ok : mc.n > 2) || SL == 0) mc = EVERY_M;
    return mc.items ? 2 : mc.n == 2 ? 1 : 0;
}
}  // namespace

cudaError_t walk_jobs_create(const std::vector<WalkJob> &jobs, WalkJobs **out) {
    *out = nullptr;
    std::vector<LargeArgs> g[2][3];
    for (const WalkJob &j : jobs) {
        MClasses mc = j.mc;
        const int kind = walk_kind(mc, j.pl.SL);
        g[j.narrow ? 1 : 0][kind].push_back(
            LargeArgs{j.pl, j.p, j.r, nullptr, j.count, j.cap, j.n_seg ? j.n_seg : 1, j.p_lo, j.p_hi, mc});
        g[j.narrow ? 1 : 0][kind].back().pl.bucket = 0;      // the job walks clear directly
    }
    WalkJobs *wj = new (std::nothrow) WalkJobs();
    if (!wj) return cudaErrorMemoryAllocation;
    for (int nw = 0; nw < 2; nw++)
        for (int k = 0; k < 3; k++) {
            if (g[nw][k].empty()) continue;
            const size_t bytes = g[nw][k].size() * sizeof(LargeArgs);
            cudaError_t e = cudaMalloc(&wj->d_jobs[nw][k], bytes);
            if (e == cudaSuccess) e = cudaMemcpy(wj->d_jobs[nw][k], g[nw][k].data(), bytes, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                walk_jobs_destroy(wj);
                return e;
            }
            wj->n_jobs[nw][k] = (uint32_t)g[nw][k].size();
        }
    *out = wj;
    return cudaSuccess;
}

cudaError_t walk_jobs_launch(const WalkJobs *wj, cudaStream_t stream) {
    for (int nw = 0; nw < 2; nw++)
        for (int k = 0; k < 3; k++) {
            if (!wj->n_jobs[nw][k]) continue;
            void (*kern)(const LargeArgs *, uint32_t);
            if (nw) {
                kern = k == 2 ? k_large_tg_jobs<uint32_t, int32_t, uint32_t, 1, 1>
                     : k == 1 ? k_large_tg_jobs<uint32_t, int32_t, uint32_t, 2>
                              : k_large_tg_jobs<uint32_t, int32_t, uint32_t, 1>;
            } else {
                kern = k == 2 ? k_large_tg_jobs<uint64_t, int64_t, uint32_t, 1, 1>
                     : k == 1 ? k_large_tg_jobs<uint64_t, int64_t, uint32_t, 2>
                              : k_large_tg_jobs<uint64_t, int64_t, uint32_t, 1>;
            }
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, LARGE_THREADS, 0) != cudaSuccess ||
                per_sm <= 0)
                per_sm = 1;
            kern<<<sm_count() * per_sm, LARGE_THREADS, 0, stream>>>(wj->d_jobs[nw][k], wj->n_jobs[nw][k]);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
    return cudaSuccess;
}

uint64_t walk_jobs_launches(const WalkJobs *wj) {
    uint64_t n = 0;
    for (int nw = 0; nw < 2; nw++)
        for (int k = 0; k < 3; k++) n += wj->n_jobs[nw][k] ? 1 : 0;
    return n;
}

void walk_jobs_destroy(WalkJobs *wj) {
    if (!wj) return;
    for (int nw = 0; nw < 2; nw++)
        for (int k = 0; k < 3; k++)
            if (wj->d_jobs[nw][k]) cudaFree(wj->d_jobs[nw][k]);
    delete wj;
}

cudaError_t launch_modsolve(const uint64_t *p, const uint64_t *K, const uint64_t *L,
                            const uint64_t *R, uint64_t *m, uint64_t n, int narrow,
                            cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    if (narrow)
        k_modsolve<uint32_t, int32_t><<<(unsigned)blocks, 256, 0, stream>>>(p, K, L, R, m, n);
    else
        k_modsolve<uint64_t, int64_t><<<(unsigned)blocks, 256, 0, stream>>>(p, K, L, R, m, n);
    return cudaGetLastError();
}

}  // namespace cs
