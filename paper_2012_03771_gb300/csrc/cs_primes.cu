// Sieving-prime source: a segmented sieve of Eratosthenes over odd numbers,
// fused with the cached residue r = K mod p of Section 3.1 (Space-Time
// Tradeoff).  The paper treats prime generation up to P_limit as a small
// one-time cost (Runtime section); here it runs on the device so that the
// primes never cross the host boundary.
//
// One CTA sieves one segment of SEG odd numbers in shared memory at a time
// (grid-stride over segments).  The multiples of 3..31 come from tabulated
// period masks; those of the other base primes q <= sqrt(hi) are marked with
// shared-memory atomics: small q cooperatively by a warp, large q one per
// thread.  Each warp then scans its share of the segment, queues the
// primes it finds in shared memory and, 32 at a time, computes K mod p with
// Montgomery multiplication over K's prime factors packed into machine words,
// and appends the entries to the output with one atomic per 32 primes.
#include <atomic>

#include "cs_arith.cuh"
#include "cs_internal.h"

namespace cs {

namespace {

// odd numbers per segment (maximum), and the base primes marked by a whole
// warp (below) or one thread each (above): a warp's lanes on multiples of one
// q >= 1024 fall on few shared-memory banks, one q per lane spreads them
// (1024 measured best of 128 to 16384)
#ifndef CS_GEN_SEG_LOG
#define CS_GEN_SEG_LOG 17
#endif
#ifndef CS_WARP_COOP_Q
#define CS_WARP_COOP_Q 1024
#endif
// grid of the generator: CTAs per SM, and segments per CTA it is sized for
#ifndef CS_GEN_GRID_PER_SM
#define CS_GEN_GRID_PER_SM 8
#endif
#ifndef CS_GEN_SEGS_PER_CTA
#define CS_GEN_SEGS_PER_CTA 1
#endif
// 1: grid of the resident CTAs and segments sized for whole waves of them
#ifndef CS_GEN_ONE_WAVE
#define CS_GEN_ONE_WAVE 1
#endif
constexpr uint32_t SEG = 1u << CS_GEN_SEG_LOG;
constexpr uint32_t SEG_MIN = 1u << 12;      // smallest segment: 8 warps x 16-word batches
constexpr uint32_t SEG_WORDS = SEG / 32;
constexpr uint32_t GEN_THREADS = 256;
constexpr uint32_t GEN_WARPS = GEN_THREADS / 32;
constexpr uint32_t WARP_COOP_Q = CS_WARP_COOP_Q;
constexpr uint32_t BATCH = 16;              // words scanned per warp step (lanes 0..15)
constexpr uint32_t QCAP = BATCH * 32 + 32;  // per-warp queue (odd indices within the segment)

// SMALL: tile records; LARGE32/64: (p, r, v0) of one plan; LIST: p only;
// PR32/64: (p, r) for a residue cache shared by plans with the same K
enum Kind { KIND_SMALL = 0, KIND_LARGE32 = 1, KIND_LARGE64 = 2, KIND_LIST = 3, KIND_PR32 = 4, KIND_PR64 = 5 };

struct GenArgs {
    uint64_t i_begin, i_end;      // odd indices [i_begin, i_end): numbers 2i+1
    uint64_t n_seg;
    uint32_t seg;                 // odd numbers per segment (multiple of SEG_MIN, <= SEG)
    bool emit_two;                // 2 is in range
    const uint32_t *base;         // odd base primes, ascending
    uint32_t n_base;
    // residue parameters
    const uint32_t *kch32;
    uint32_t n_kch32;
    const uint64_t *kch64;
    uint32_t n_kch64;
    uint64_t M_start;
    uint32_t SL;
    // outputs
    void *o0, *o1, *o2;
    uint64_t cap;
    unsigned long long *count;
    unsigned long long *err;
};

__device__ __forceinline__ uint32_t kmodp32(uint32_t p, uint32_t pinv, uint32_t r1, uint32_t r2,
                                            const uint32_t *kch, uint32_t n) {
    if (n == 0) return 1u % p;
    uint32_t acc = mont32_rpow(n, r1, r2, p, pinv);     // R^n: cancels the n factors R^-1
    // the factor words are below 2^31, so the running product stays below 2p;
    // four words per 16-byte load when the word array is aligned
    uint32_t i = 0;
    if ((reinterpret_cast<uintptr_t>(kch) & 15) == 0) {
        const uint4 *k4 = reinterpret_cast<const uint4 *>(kch);
        for (; i + 4 <= n; i += 4) {
            const uint4 w = __ldg(&k4[i / 4]);
            acc = mont32_mul_lazy(acc, w.x, p, pinv);
            acc = mont32_mul_lazy(acc, w.y, p, pinv);
            acc = mont32_mul_lazy(acc, w.z, p, pinv);
            acc = mont32_mul_lazy(acc, w.w, p, pinv);
        }
    }
    for (; i < n; i++) acc = mont32_mul_lazy(acc, __ldg(&kch[i]), p, pinv);
    return acc >= p ? acc - p : acc;
}

// K mod p for 64-bit p from R^2 mod p: the product of the n factor words
// starts at R^n mod p, which cancels their n factors R^-1
__device__ __forceinline__ uint64_t kmodp64(uint64_t p, uint64_t pinv, uint64_t r2,
                                            const uint64_t *kch, uint32_t n) {
    if (n == 0) return 1ull % p;
    uint64_t acc = mont64_rpow2(n, r2, p, pinv);
    for (uint32_t i = 0; i < n; i++) acc = mont64_mul(acc, __ldg(&kch[i]), p, pinv);
    return acc;
}

template <int KIND>
__device__ __forceinline__ void emit(const GenArgs &a, uint64_t p, bool valid, unsigned lane) {
    // residue work for this lane's prime
    uint32_t e0 = 0, e1 = 0, e2 = 0, e3 = 0;
    uint64_t w0 = 0, w1 = 0;
    if (valid) {
        if (KIND == KIND_SMALL) {
            uint32_t p32 = (uint32_t)p;
            if (p32 == 2) {
                // only when P < 2, so K = 1 and r = 1
                e0 = 2; e1 = 0; e2 = 1; e3 = (uint32_t)((a.M_start + a.SL) & 1);
            } else {
                uint32_t pinv = mont32_neg_inv(p32);
                uint32_t r1 = mont32_r1(p32), r2 = mont32_r2(p32);
                uint32_t r = kmodp32(p32, pinv, r1, r2, a.kch32, a.n_kch32);
                uint32_t rt = mont32_mul(r, r2, p32, pinv);
                uint32_t ms = (uint32_t)(a.M_start % p32);
                uint32_t v = mont32_mul(rt, ms, p32, pinv) + a.SL % p32;
                e0 = p32; e1 = pinv; e2 = rt; e3 = v >= p32 ? v - p32 : v;
            }
        } else if (KIND == KIND_LARGE32) {
            uint32_t p32 = (uint32_t)p;
            uint32_t pinv = mont32_neg_inv(p32);
            uint32_t r2 = mont32_r2_fast(p32);
            uint32_t r1 = mont32_mul(r2, 1u, p32, pinv);         // R mod p
            uint32_t r = kmodp32(p32, pinv, r1, r2, a.kch32, a.n_kch32);
            uint32_t rt = mont32_mul(r, r2, p32, pinv);
            e0 = p32; e1 = r; e2 = mont32_affine(rt, a.M_start, a.SL, r2, p32, pinv);   // SL < p
        } else if (KIND == KIND_LARGE64) {
            w0 = p;                                               // residues: k_large_res
        } else if (KIND == KIND_PR32) {
            uint32_t p32 = (uint32_t)p;
            uint32_t pinv = mont32_neg_inv(p32);
            e0 = p32;
            const uint32_t r2 = mont32_r2_fast(p32);
            e1 = kmodp32(p32, pinv, mont32_mul(r2, 1u, p32, pinv), r2, a.kch32, a.n_kch32);
        } else if (KIND == KIND_PR64) {
            uint64_t pinv = mont64_neg_inv(p);
            w0 = p;
            w1 = kmodp64(p, pinv, mont64_r2_fast(p, rcp_rn(u64_to_f(p))), a.kch64, a.n_kch64);
        } else {
            w0 = p;
        }
    }
    unsigned mask = __ballot_sync(0xffffffffu, valid);
    unsigned n = __popc(mask);
    if (n == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(a.count, (unsigned long long)n);
    base = __shfl_sync(0xffffffffu, base, 0);
    unsigned rank = __popc(mask & ((1u << lane) - 1));
    if (!valid) return;
    uint64_t slot = base + rank;
    if (slot >= a.cap) {
        atomicOr(a.err, (unsigned long long)ERR_PRIME_OVERFLOW);
        return;
    }
    if (KIND == KIND_SMALL) {
        reinterpret_cast<SmallPrime *>(a.o0)[slot] = SmallPrime{e0, e1, e2, e3};
    } else if (KIND == KIND_LARGE32) {
        reinterpret_cast<uint32_t *>(a.o0)[slot] = e0;
        reinterpret_cast<uint32_t *>(a.o1)[slot] = e1;
        reinterpret_cast<uint32_t *>(a.o2)[slot] = e2;
    } else if (KIND == KIND_LARGE64) {
        reinterpret_cast<uint64_t *>(a.o0)[slot] = w0;
    } else if (KIND == KIND_PR32) {
        reinterpret_cast<uint32_t *>(a.o0)[slot] = e0;
        reinterpret_cast<uint32_t *>(a.o1)[slot] = e1;
    } else if (KIND == KIND_PR64) {
        reinterpret_cast<uint64_t *>(a.o0)[slot] = w0;
        reinterpret_cast<uint64_t *>(a.o1)[slot] = w1;
    } else {
        reinterpret_cast<uint64_t *>(a.o0)[slot] = w0;
    }
}

// Residues of the 64-bit large primes the generator wrote (o0): r = K mod p
// (Section 3.1) into o1 and v = (r M_start + SL) mod p into o2, RES_ILP primes
// per thread, every resident warp on the chains of 64-bit Montgomery products
// (9% faster than inside the sieve kernel on L = 1e11).  The 32-bit residues stay in
// the sieve kernel, where they fill issue slots that its barriers and marking
// phases leave idle (split out, the generator took 3.06 instead of 2.57 ms per
// sieve on L = 1e9).
constexpr uint32_t RES_THREADS = 256;
// primes per thread, whose Montgomery chains interleave (each chain is a
// sequence of dependent multiplications, so one chain alone leaves issue slots
// idle between them); on L = 1e11, generation and residues took 441 ms with
// one, 420 with two, 426 with three and 427 with four (the wide multiplies'
// pipe is then about 80% busy)
#ifndef CS_RES_ILP
#define CS_RES_ILP 2
#endif
constexpr int RES_ILP = CS_RES_ILP;
__global__ void __launch_bounds__(RES_THREADS) k_large_res(const GenArgs a) {
    const uint64_t n = min((uint64_t)*a.count, a.cap);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t *P = reinterpret_cast<const uint64_t *>(a.o0);
    for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < n; i0 += RES_ILP * stride) {
        uint64_t p[RES_ILP], pinv[RES_ILP], r2[RES_ILP], acc[RES_ILP];
        float fp[RES_ILP];
#pragma unroll
        for (int k = 0; k < RES_ILP; k++) {
            const uint64_t i = i0 + k * stride;
            p[k] = i < n ? P[i] : P[i0];                     // the extra chains repeat a valid prime
            pinv[k] = mont64_neg_inv(p[k]);
            fp[k] = rcp_rn(u64_to_f(p[k]));
            r2[k] = mont64_r2_fast(p[k], fp[k]);
        }
        // K mod p: R^n from R^2, then the n factor words (the same control flow for every chain)
        const uint32_t nw = a.n_kch64;
        if (nw == 0) {
#pragma unroll
            for (int k = 0; k < RES_ILP; k++) acc[k] = 1ull % p[k];
        } else {
#pragma unroll
            for (int k = 0; k < RES_ILP; k++) acc[k] = mont64_rpow2(nw, r2[k], p[k], pinv[k]);
            for (uint32_t w = 0; w < nw; w++) {
                const uint64_t f = __ldg(&a.kch64[w]);
#pragma unroll
                for (int k = 0; k < RES_ILP; k++) acc[k] = mont64_mul(acc[k], f, p[k], pinv[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < RES_ILP; k++) {
            const uint64_t i = i0 + k * stride;
            const uint64_t rt = mont64_mul(acc[k], r2[k], p[k], pinv[k]);
            // M_start < 2^40: below p, or a quotient below 2^20 for p >= 2^20
            const uint64_t ms = a.M_start < p[k] ? a.M_start
                              : p[k] >= (1ull << 20) ? mod_q20(a.M_start, p[k], fp[k]) : a.M_start % p[k];
            const uint64_t v = mont64_mul(rt, ms, p[k], pinv[k]) + a.SL;
            if (i < n) {
                reinterpret_cast<uint64_t *>(a.o1)[i] = acc[k];
                reinterpret_cast<uint64_t *>(a.o2)[i] = v >= p[k] ? v - p[k] : v;
            }
        }
    }
}

// n mod q with 32-bit arithmetic when n fits (all segments below 2^32)
__device__ __forceinline__ uint32_t first_rem(uint64_t n, uint32_t q) {
    return (n >> 32) == 0 ? (uint32_t)n % q : (uint32_t)(n % q);
}

// Pre-sieve of the odd multiples of 3..31 (half of all marks, and the ones
// whose lanes collide on the same shared-memory word): the masks of one period
// of T = 3*5*7, 11*13, 17*19, 23*29 and 31 odd indices are tabulated in shared
// memory, and word w of a segment, whose first odd index I = i0 + 32 w has
// I mod T = s, ORs in table entry s.  Bit b of that entry is set when the odd
// number 2(I + b) + 1 has a factor q | T, i.e. I + b = (q - 1)/2 (mod q).
constexpr int PRE_N = 5;
constexpr uint32_t PRE_MAX_Q = 31;
__device__ __constant__ uint32_t c_pre_T[PRE_N] = {105, 143, 323, 667, 31};
__device__ __constant__ uint32_t c_pre_off[PRE_N + 1] = {0, 105, 248, 571, 1238, 1269};
constexpr uint32_t PRE_WORDS = 1269;

__device__ __forceinline__ uint32_t pre_mask(uint32_t T, uint32_t s) {
    const uint32_t qs[10] = {3, 5, 7, 11, 13, 17, 19, 23, 29, 31};
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < 10; k++) {
        const uint32_t q = qs[k];
        if (T % q) continue;
        const uint32_t h = (q - 1) / 2;
        for (uint32_t b = (h + q - s % q) % q; b < 32; b += q) m |= 1u << b;
    }
    return m;
}

template <int KIND>
__global__ void __launch_bounds__(GEN_THREADS) k_gen(const GenArgs a) {
    __shared__ uint32_t comp[SEG_WORDS];          // bit set = composite (or out of range)
    __shared__ uint32_t queue[GEN_WARPS][QCAP];
    __shared__ uint32_t pre[PRE_WORDS];           // pre-sieve tables
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t e = threadIdx.x; e < PRE_WORDS; e += GEN_THREADS) {
        int t = 0;
        while (e >= c_pre_off[t + 1]) t++;
        pre[e] = pre_mask(c_pre_T[t], e - c_pre_off[t]);
    }
    __syncthreads();

    if (a.emit_two && blockIdx.x == 0 && warp == 0) emit<KIND>(a, 2, lane == 0, lane);

    // first base index with q >= WARP_COOP_Q (base is ascending)
    uint32_t big0 = 0;
    {
        uint32_t hi = a.n_base;
        while (big0 < hi) {
            uint32_t mid = (big0 + hi) / 2;
            if (__ldg(&a.base[mid]) < WARP_COOP_Q) big0 = mid + 1; else hi = mid;
        }
    }

    for (uint64_t s = blockIdx.x; s < a.n_seg; s += gridDim.x) {
        const uint64_t i0 = a.i_begin + s * a.seg;
        const uint64_t i1 = min(i0 + a.seg, a.i_end);
        const uint32_t seg_words = a.seg / 32;
        const uint32_t len = (uint32_t)(i1 - i0);
        const uint64_t n_first = 2 * i0 + 1;
        const uint64_t n_last = 2 * (i1 - 1) + 1;
        // the tables apply when no q <= 31 lies in the segment itself
        const bool pre_ok = n_first > PRE_MAX_Q;
        uint32_t ph[PRE_N], step[PRE_N];
#pragma unroll
        for (int t = 0; t < PRE_N; t++) {
            const uint32_t T = c_pre_T[t];
            ph[t] = pre_ok ? first_rem(i0 + 32ull * threadIdx.x, T) : 0;
            step[t] = (32u * GEN_THREADS) % T;
        }
        for (uint32_t w = threadIdx.x; w < seg_words; w += GEN_THREADS) {
            uint32_t v = 0;
            uint32_t lo = w * 32;
            if (lo + 32 > len) v = lo >= len ? 0xffffffffu : (0xffffffffu << (len - lo));
            if (pre_ok) {
#pragma unroll
                for (int t = 0; t < PRE_N; t++) {
                    v |= pre[c_pre_off[t] + ph[t]];
                    ph[t] += step[t];
                    if (ph[t] >= c_pre_T[t]) ph[t] -= c_pre_T[t];
                }
            }
            comp[w] = v;
        }
        __syncthreads();
        if (i0 == 0 && threadIdx.x == 0) atomicOr(&comp[0], 1u);   // 1 is not prime

        // mark odd multiples of the base primes, starting at max(q^2, first in segment)
        for (uint32_t b = warp; b < a.n_base; b += GEN_WARPS) {
            const uint32_t q = __ldg(&a.base[b]);
            if ((uint64_t)q * q > n_last) break;
            if (q >= WARP_COOP_Q) break;
            if (pre_ok && q <= PRE_MAX_Q) continue;          // in the pre-sieve
            uint64_t start = (uint64_t)q * q;
            if (start < n_first) {
                const uint32_t rem = first_rem(n_first, q);
                start = rem ? n_first + (q - rem) : n_first;
                if ((start & 1) == 0) start += q;
            }
            for (uint64_t idx = (start - n_first) / 2 + (uint64_t)lane * q; idx < len; idx += 32ull * q)
                atomicOr(&comp[idx >> 5], 1u << (idx & 31));
        }
        // large base primes: one per thread (at most SEG / q + 1 marks each)
        {
            for (uint32_t b = big0 + threadIdx.x; b < a.n_base; b += GEN_THREADS) {
                const uint32_t q = __ldg(&a.base[b]);
                if ((uint64_t)q * q > n_last) break;
                uint64_t start = (uint64_t)q * q;
                if (start < n_first) {
                    const uint32_t rem = first_rem(n_first, q);
                    start = rem ? n_first + (q - rem) : n_first;
                    if ((start & 1) == 0) start += q;
                }
                for (uint64_t idx = (start - n_first) / 2; idx < len; idx += q)
                    atomicOr(&comp[idx >> 5], 1u << (idx & 31));
            }
        }
        __syncthreads();

        // extract: each warp owns a contiguous run of words
        const uint32_t wpw = seg_words / GEN_WARPS;
        uint32_t qlen = 0;
        for (uint32_t w0 = warp * wpw; w0 < (warp + 1) * wpw; w0 += BATCH) {
            uint32_t w = w0 + lane;
            uint32_t primes = lane < BATCH ? ~comp[w] : 0u;
            uint32_t c = __popc(primes);
            uint32_t incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (unsigned)o) incl += t;
            }
            uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
            uint32_t pos = qlen + incl - c;
            while (primes) {
                uint32_t bit = __ffs(primes) - 1;
                primes &= primes - 1;
                queue[warp][pos++] = w * 32 + bit;
            }
            qlen += total;
            __syncwarp();
            uint32_t done = 0;
            while (qlen - done >= 32) {
                uint32_t idx = queue[warp][done + lane];
                emit<KIND>(a, 2 * (i0 + idx) + 1, true, lane);
                done += 32;
            }
            __syncwarp();
            // move the remainder (< 32 entries) to the front
            uint32_t rest = qlen - done;
            uint32_t keep = lane < rest ? queue[warp][done + lane] : 0;
            __syncwarp();
            if (lane < rest) queue[warp][lane] = keep;
            qlen = rest;
            __syncwarp();
        }
        {
            bool valid = lane < qlen;
            uint32_t idx = valid ? queue[warp][lane] : 0;
            emit<KIND>(a, 2 * (i0 + idx) + 1, valid, lane);
        }
        __syncthreads();
    }
}

// CTAs of k_gen<KIND> resident at once on the device (occupancy API, once per kind)
template <int KIND>
int gen_resident() {
    static std::atomic<int> cached{0};
    int n = cached.load(std::memory_order_relaxed);
    if (n == 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gen<KIND>, GEN_THREADS, 0) != cudaSuccess ||
            per_sm <= 0)
            per_sm = CS_GEN_GRID_PER_SM;
        n = sm_count() * per_sm;
        cached.store(n, std::memory_order_relaxed);
    }
    return n;
}

GenArgs make_args(uint64_t lo, uint64_t hi, const uint32_t *base, uint32_t n_base, int resident) {
    GenArgs a{};
    a.base = base;
    a.n_base = n_base;
    if (hi <= lo || hi < 2) {
        a.n_seg = 0;
        return a;
    }
    a.i_begin = (lo + 1) / 2;
    a.i_end = (hi + 1) / 2;
    const uint64_t odds = a.i_end > a.i_begin ? a.i_end - a.i_begin : 0;
    uint32_t seg = SEG_MIN;
#if CS_GEN_ONE_WAVE
    // segment size: the range split evenly over whole waves of the resident
    // CTAs (k segments each), in multiples of SEG_MIN within [SEG_MIN, SEG], so
    // that no CTA waits on a partly filled last wave
    {
        const uint64_t res = (uint64_t)(resident > 0 ? resident : 1);
        const uint64_t k = (odds + res * SEG - 1) / (res * SEG);               // segments per CTA
        const uint64_t per = k ? (odds + res * k - 1) / (res * k) : 0;          // odds per segment
        const uint64_t sz = (per + SEG_MIN - 1) / SEG_MIN * SEG_MIN;
        seg = (uint32_t)(sz < SEG_MIN ? SEG_MIN : (sz > SEG ? SEG : sz));
    }
#else
    // segment size: enough segments for every CTA of the grid to get
    // CS_GEN_SEGS_PER_CTA of them, within [SEG_MIN, SEG]
    uint64_t want = odds / ((uint64_t)sm_count() * CS_GEN_GRID_PER_SM * CS_GEN_SEGS_PER_CTA);
    while (seg < SEG && seg < want) seg *= 2;
    (void)resident;
#endif
    a.seg = seg;
    a.n_seg = odds ? (odds + seg - 1) / seg : 0;
    a.emit_two = lo < 2 && hi >= 2;
    return a;
}

int gen_grid(uint64_t n_seg, int resident) {
#if CS_GEN_ONE_WAVE
    uint64_t g = (uint64_t)(resident > 0 ? resident : 1);
#else
    uint64_t g = (uint64_t)sm_count() * CS_GEN_GRID_PER_SM;
    (void)resident;
#endif
    if (n_seg < g) g = n_seg;
    return (int)(g ? g : 1);
}

}  // namespace

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

uint64_t l2_bytes() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrL2CacheSize, dev);
        if (n <= 0) n = 1 << 20;
    }
    return (uint64_t)n;
}

cudaError_t launch_gen_small(const DevPlan &pl, uint64_t lo, uint64_t hi, const uint32_t *base,
                             uint32_t n_base, SmallPrime *out, uint64_t cap,
                             unsigned long long *count, cudaStream_t stream) {
    const int res = gen_resident<KIND_SMALL>();
    GenArgs a = make_args(lo, hi, base, n_base, res);
    if (a.n_seg == 0 && !a.emit_two) return cudaSuccess;
    a.kch32 = pl.kch32; a.n_kch32 = pl.n_kch32;
    a.M_start = pl.M_start; a.SL = pl.SL;
    a.o0 = out; a.cap = cap; a.count = count; a.err = pl.stats + ST_ERROR;
    k_gen<KIND_SMALL><<<gen_grid(a.n_seg, res), GEN_THREADS, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gen_large(const DevPlan &pl, bool narrow, uint64_t lo, uint64_t hi,
                             const uint32_t *base, uint32_t n_base, void *p_out, void *r_out,
                             void *v_out, uint64_t cap, unsigned long long *count,
                             cudaStream_t stream) {
    const int res = narrow ? gen_resident<KIND_LARGE32>() : gen_resident<KIND_LARGE64>();
    GenArgs a = make_args(lo, hi, base, n_base, res);
    if (a.n_seg == 0 && !a.emit_two) return cudaSuccess;
    a.kch32 = pl.kch32; a.n_kch32 = pl.n_kch32;
    a.kch64 = pl.kch64; a.n_kch64 = pl.n_kch64;
    a.M_start = pl.M_start; a.SL = pl.SL;
    a.o0 = p_out; a.o1 = r_out; a.o2 = v_out;
    a.cap = cap; a.count = count; a.err = pl.stats + ST_ERROR;
    if (narrow) {
        k_gen<KIND_LARGE32><<<gen_grid(a.n_seg, res), GEN_THREADS, 0, stream>>>(a);
    } else {
        // residues of the primes written: one wave of resident CTAs over the count
        static std::atomic<int> res_per_sm{0};
        int per_sm = res_per_sm.load(std::memory_order_relaxed);
        if (per_sm == 0) {
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_large_res, RES_THREADS, 0) != cudaSuccess ||
                per_sm <= 0)
                per_sm = 4;
            res_per_sm.store(per_sm, std::memory_order_relaxed);
        }
        k_gen<KIND_LARGE64><<<gen_grid(a.n_seg, res), GEN_THREADS, 0, stream>>>(a);
        k_large_res<<<sm_count() * per_sm, RES_THREADS, 0, stream>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_gen_pr(const DevPlan &kp, bool narrow, uint64_t lo, uint64_t hi, const uint32_t *base,
                          uint32_t n_base, void *p_out, void *r_out, uint64_t cap,
                          unsigned long long *count, unsigned long long *err, cudaStream_t stream) {
    const int res = narrow ? gen_resident<KIND_PR32>() : gen_resident<KIND_PR64>();
    GenArgs a = make_args(lo, hi, base, n_base, res);
    if (a.n_seg == 0 && !a.emit_two) return cudaSuccess;
    a.kch32 = kp.kch32; a.n_kch32 = kp.n_kch32;
    a.kch64 = kp.kch64; a.n_kch64 = kp.n_kch64;
    a.o0 = p_out; a.o1 = r_out;
    a.cap = cap; a.count = count; a.err = err;
    if (narrow)
        k_gen<KIND_PR32><<<gen_grid(a.n_seg, res), GEN_THREADS, 0, stream>>>(a);
    else
        k_gen<KIND_PR64><<<gen_grid(a.n_seg, res), GEN_THREADS, 0, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_gen_list(uint64_t lo, uint64_t hi, const uint32_t *base, uint32_t n_base,
                            uint64_t *out, uint64_t cap, unsigned long long *count,
                            unsigned long long *err, cudaStream_t stream) {
    const int res = gen_resident<KIND_LIST>();
    GenArgs a = make_args(lo, hi, base, n_base, res);
    if (a.n_seg == 0 && !a.emit_two) return cudaSuccess;
    a.o0 = out; a.cap = cap; a.count = count; a.err = err;
    k_gen<KIND_LIST><<<gen_grid(a.n_seg, res), GEN_THREADS, 0, stream>>>(a);
    return cudaGetLastError();
}

namespace {
__global__ void k_kmodp(const uint64_t *p, uint64_t n, uint64_t *r, const uint32_t *kch32,
                        uint32_t n32, const uint64_t *kch64, uint32_t n64) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t q = p[i];
        if (q < (1ull << 31)) {
            uint32_t q32 = (uint32_t)q;
            uint32_t pinv = mont32_neg_inv(q32);
            r[i] = kmodp32(q32, pinv, mont32_r1(q32), mont32_r2(q32), kch32, n32);
        } else {
            uint64_t pinv = mont64_neg_inv(q);
            r[i] = kmodp64(q, pinv, mont64_r2_fast(q, rcp_rn(u64_to_f(q))), kch64, n64);
        }
    }
}
}  // namespace

cudaError_t launch_kmodp(const DevPlan &pl, const uint64_t *p, uint64_t n, uint64_t *r,
                         cudaStream_t stream) {
    if (n == 0) return cudaSuccess;
    uint64_t blocks = (n + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    k_kmodp<<<(unsigned)blocks, 256, 0, stream>>>(p, n, r, pl.kch32, pl.n_kch32, pl.kch64,
                                                   pl.n_kch64);
    return cudaGetLastError();
}

}  // namespace cs
