// Host side of the C ABI: parameter validation, the row / column maps, K's
// factor words, device memory and the order of kernel launches for one sieve.
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/combsieve.h"
#include "cs_arith.cuh"
#include "cs_internal.h"
#include "cs_words.h"
#include "cs_classes.h"

using namespace cs;

namespace {

thread_local std::string g_err;

cs_status fail(cs_status code, const std::string &msg) {
    g_err = msg;
    return code;
}

cs_status cuda_fail(cudaError_t e, const char *what) {
    return fail(e == cudaErrorMemoryAllocation ? CS_ENOMEM : CS_EDEVICE,
                std::string(what) + ": " + cudaGetErrorString(e));
}

#define CS_CUDA(call)                                  \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

constexpr uint64_t MAX_P = 1ull << 20;
constexpr uint64_t MAX_SL = 1ull << 20;
constexpr uint64_t MAX_L = 1ull << 40;
constexpr uint64_t MAX_M = 1ull << 40;
constexpr uint64_t MAX_T = 1ull << 30;
constexpr uint64_t NARROW_LIMIT = 1ull << 30;

std::vector<uint32_t> primes_upto(uint64_t n) {
    std::vector<uint32_t> out;
    if (n < 2) return out;
    std::vector<uint8_t> comp(n + 1, 0);
    for (uint64_t i = 2; i <= n; i++) {
        if (comp[i]) continue;
        out.push_back((uint32_t)i);
        for (uint64_t j = i * i; j <= n; j += i) comp[j] = 1;
    }
    return out;
}

uint64_t isqrt_u64(uint64_t n) {
    uint64_t r = (uint64_t)sqrt((double)n);
    while (r * r > n) r--;
    while ((r + 1) * (r + 1) <= n) r++;
    return r;
}

// Upper bound on the number of primes in any interval of length y (y >= 2):
// pi(x + y) - pi(x) <= 2y / log y (Montgomery and Vaughan, "The large sieve",
// Mathematika 20, 1973), plus slack.
uint64_t primes_in_interval_bound(uint64_t y) {
    if (y < 64) return 64;
    return (uint64_t)(2.0 * (double)y / log((double)y)) + 1024;
}

// pi(x) < 1.25506 x / log x for x > 1 (Rosser and Schoenfeld, 1962), plus slack.
uint64_t prime_count_bound(uint64_t x) {
    if (x < 64) return 64;
    return (uint64_t)(1.25506 * (double)x / log((double)x)) + 1024;
}

enum KernelClass { KC_GEN_SMALL = 0, KC_TILE, KC_GEN_LARGE, KC_LARGE, KC_FINAL, KC_APPLY, KC_PREP, KC_N };

// Device memory of plain plans: a library-owned stream-ordered pool per device
// that keeps up to POOL_KEEP bytes of freed plan memory for the next plan
// (cudaMalloc / cudaFree of a plan's ~100 MB took about a millisecond per
// plan), and a stream on which plans return their buffers.
constexpr uint64_t POOL_KEEP = 1ull << 30;
struct PlanPool {
    cudaMemPool_t pool = nullptr;
    cudaStream_t free_stream = nullptr;
    cudaStream_t upload_stream = nullptr;   // plans' allocations and table uploads
};
std::mutex g_pool_mu;
PlanPool g_plan_pools[64];

cudaError_t plan_pool(PlanPool **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    PlanPool &pp = g_plan_pools[dev];
    if (!pp.pool) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if ((e = cudaMemPoolCreate(&pool, &props)) != cudaSuccess) return e;
        uint64_t keep = POOL_KEEP;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        cudaStream_t fs = nullptr, us = nullptr;
        if ((e = cudaStreamCreateWithFlags(&fs, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&us, cudaStreamNonBlocking)) != cudaSuccess) {
            if (fs) cudaStreamDestroy(fs);
            cudaMemPoolDestroy(pool);
            return e;
        }
        pp.pool = pool;
        pp.free_stream = fs;
        pp.upload_stream = us;
    }
    *out = &pp;
    return cudaSuccess;
}

}  // namespace

struct cs_plan_s {
    // parameters
    uint32_t P = 0;
    uint64_t d = 0, M_start = 0, M_inc = 0, L = 0;
    uint32_t SL = 0;
    cs_tuning tune{};
    // derived
    uint64_t M_c = 0, W = 0, wpr = 0, S = 0, S32 = 0, T = 0, small_hi = 0;
    bool narrow = true, wheel = true;
    int mode = LARGE_THREE_GAP;
    uint32_t layout = 0;
    // compact layout, host copies: classes' widths and raw offsets of columns
    uint32_t n_cls = 1, cls0 = 0, Wc_max = 0;
    std::vector<uint32_t> cW_h, craw_h;
    std::vector<uint64_t> m_of_row;
    std::vector<int64_t> x_of_col;
    std::vector<std::pair<uint64_t, uint64_t>> chunks;    // large-prime ranges (lo, hi]
    std::vector<uint32_t> chunk_seg;                      // m-segments per prime, per chunk
    std::vector<MClasses> chunk_mc;                       // m-classes each chunk walks
    MClasses mcls = EVERY_M;                              // classes of the chunks with many hits
    MClasses mcls_light = EVERY_M;                        // classes of the other chunks
    uint64_t split_chunks = 0;                            // chunks that walk mcls
    uint32_t item_mod = 0, item_classes = 0;              // finest class items walked
    uint64_t item_chunks = 0;                             // chunks that walk class items
    uint64_t large_cap = 0, small_cap = 0, est_cost = 0;
    std::vector<uint8_t> apply_after;                     // bucketed hits: apply after this chunk's walk
    uint64_t apply_launches = 0, bucket_bytes = 0;
    int large_grid = 0;
    uint64_t h2d = 0, dev_bytes = 0;
    // device
    DevPlan dp{};
    TileConfig tc{};
    std::vector<void *> allocs;
    uint32_t *d_base = nullptr;
    uint32_t n_base = 0;
    SmallPrime *d_small = nullptr;
    void *d_lp = nullptr, *d_lr = nullptr, *d_lv = nullptr;
    uint4 *d_desc0 = nullptr;             // walkers prepared by k_tg_prep (one-walker chunks)
    uint2 *d_desc1 = nullptr;
    unsigned long long *d_counts = nullptr;   // [0] small count, [1..] per-chunk counts
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool sieved = false;
    cs_status sticky = CS_OK;
    // stream-ordered allocation (plans built by the request server): device
    // buffers come from cudaMallocAsync on alloc_stream and go back with
    // cudaFreeAsync, so building or freeing a plan does not wait for other work
    cudaStream_t alloc_stream = nullptr;
    bool async_alloc = false;
    PlanPool *pool = nullptr;             // plain plans: the device's plan pool
    bool built = false;                   // build_plan finished
    // host-side fault injection for tests: the fail_alloc_at-th device
    // allocation of the build fails as if the device were out of memory
    // (environment CS_FAIL_ALLOC_AT; 0 = off)
    uint64_t fail_alloc_at = 0, n_allocs = 0;
    // stream of the plan's allocations and uploads: the server's, else the
    // device pool's (set up by the first dalloc)
    cudaStream_t upload_stream() { return async_alloc ? alloc_stream : pool->upload_stream; }
    // tables to upload, staged in one host arena (256-byte aligned parts) and
    // sent with one allocation and one copy by flush_uploads, which then sets
    // each destination pointer
    std::vector<uint8_t> staging;
    std::vector<std::function<void(uint8_t *)>> pending;
    // residue cache: large primes come from these cache chunks (indices)
    cs_cache_t cache = nullptr;
    std::vector<size_t> cache_idx;
    // profiling
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev[KC_N];
    size_t prof_used[KC_N] = {};

    ~cs_plan_s() {
        // a plan that failed while being built: its allocations and upload are
        // ordered on the upload stream, so let them finish before the frees
        if (!built && !allocs.empty()) cudaStreamSynchronize(upload_stream());
        if (done) cudaEventDestroy(done);
        for (int k = 0; k < KC_N; k++)
            for (auto &e : prof_ev[k]) {
                cudaEventDestroy(e.first);
                cudaEventDestroy(e.second);
            }
        for (void *p : allocs) {
            if (async_alloc)
                cudaFreeAsync(p, alloc_stream);
            else if (pool)
                cudaFreeAsync(p, pool->free_stream);   // back to the pool: the plan's work is done
            else
                cudaFree(p);
        }
        // the pool can hand the memory to the next plan once the frees ran
        if (pool && !allocs.empty() && !async_alloc) cudaStreamSynchronize(pool->free_stream);
    }

    template <class T>
    cs_status dalloc(T **p, size_t count) {
        size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
        if (fail_alloc_at && ++n_allocs == fail_alloc_at)
            return fail(CS_ENOMEM, "device allocation failed (injected by CS_FAIL_ALLOC_AT)");
        cudaError_t e;
        if (async_alloc) {
            e = cudaMallocAsync((void **)p, bytes, alloc_stream);
        } else {
            if (!pool && (e = plan_pool(&pool)) != cudaSuccess) return cuda_fail(e, "memory pool");
            e = cudaMallocFromPoolAsync((void **)p, bytes, pool->pool, upload_stream());
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc");
        allocs.push_back(*p);
        dev_bytes += bytes;
        return CS_OK;
    }
    template <class D, class T>
    void stage(D **dst, const std::vector<T> &v) {
        const size_t off = (staging.size() + 255) & ~(size_t)255;
        staging.resize(off + std::max<size_t>(v.size(), 1) * sizeof(T));
        if (!v.empty()) memcpy(staging.data() + off, v.data(), v.size() * sizeof(T));
        pending.push_back([dst, off](uint8_t *base) { *dst = reinterpret_cast<D *>(base + off); });
        h2d += v.size() * sizeof(T);
    }
    cs_status flush_uploads() {
        if (pending.empty()) return CS_OK;
        uint8_t *base = nullptr;
        cs_status s = dalloc(&base, staging.size());
        if (s) return s;
        // one copy on the upload stream, which the plan builder synchronises
        // before the arena goes away and before any kernel reads the tables (a
        // plain cudaMemcpy from pageable memory may return before its DMA lands
        // and is ordered only on the legacy stream)
        cudaError_t e = cudaMemcpyAsync(base, staging.data(), staging.size(), cudaMemcpyHostToDevice,
                                        upload_stream());
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy H2D");
        for (auto &f : pending) f(base);
        pending.clear();
        return CS_OK;
    }
};

namespace {

// factor d over the primes <= P; returns false if d is not squarefree or has a
// prime factor above P
bool split_primes(uint32_t P, uint64_t d, std::vector<uint32_t> &qK, std::vector<uint32_t> &qd) {
    std::vector<uint32_t> pr = primes_upto(P);
    uint64_t rest = d;
    for (uint32_t q : pr) {
        if (rest % q == 0) {
            rest /= q;
            if (rest % q == 0) return false;
            qd.push_back(q);
        } else {
            qK.push_back(q);
        }
    }
    return rest == 1;
}

cs_status check_params(uint32_t P, uint64_t d, uint64_t M_start, uint64_t M_inc, uint32_t SL, uint64_t L,
                       std::vector<uint32_t> &qK, std::vector<uint32_t> &qd) {
    if (d == 0 || P > MAX_P) return fail(CS_EINVAL, "d must be >= 1 and P <= 2^20");
    if (SL > MAX_SL) return fail(CS_EINVAL, "SL must be <= 2^20");
    if (L > MAX_L) return fail(CS_EINVAL, "L must be <= 2^40");
    if (M_start < 1 || M_start > MAX_M || M_inc > MAX_M - M_start)
        return fail(CS_EINVAL, "need 1 <= M_start and M_start + M_inc <= 2^40");
    if (M_inc >= (1ull << 31)) return fail(CS_EINVAL, "M_inc must be < 2^31");
    if (!split_primes(P, d, qK, qd)) return fail(CS_EINVAL, "d must be squarefree and divide P#");
    // every N + x >= 2: M_start*K - SL >= 2 (only K < 2^64 can fail it)
    unsigned __int128 K = 1;
    for (uint32_t q : qK) {
        K *= q;
        if (K > (unsigned __int128)UINT64_MAX) return CS_OK;
    }
    if ((unsigned __int128)M_start * K < (unsigned __int128)SL + 2) return fail(CS_EINVAL, "need M_start*K - SL >= 2");
    return CS_OK;
}

// tuning fields left at 0 may be set from the environment
void env_tuning(cs_tuning &t) {
    auto get = [](const char *n) -> uint64_t {
        const char *v = getenv(n);
        return v ? strtoull(v, nullptr, 10) : 0;
    };
    if (!t.threshold) t.threshold = get("CS_THRESHOLD");
    if (!t.tile_rows) t.tile_rows = (uint32_t)get("CS_TILE_ROWS");
    if (!t.large_mode) t.large_mode = (uint32_t)get("CS_LARGE_MODE");
    if (!t.large_grid) t.large_grid = (uint32_t)get("CS_LARGE_GRID");
    if (!t.m_classes) t.m_classes = (uint32_t)get("CS_M_CLASSES");
    if (!t.item_hits) t.item_hits = (uint32_t)get("CS_ITEM_HITS");
    if (!t.class_min_hits) t.class_min_hits = (uint32_t)get("CS_CLASS_MIN_HITS");
    if (!t.class_item_hits) t.class_item_hits = (uint32_t)get("CS_CLASS_ITEM_HITS");
    if (!t.chunk_numbers) t.chunk_numbers = get("CS_CHUNK_NUMBERS");
    if (!t.hit_buckets) t.hit_buckets = (uint32_t)get("CS_HIT_BUCKETS");
    if (!t.band_rows_log) t.band_rows_log = (uint32_t)get("CS_BAND_ROWS_LOG");
    if (!t.bucket_records) t.bucket_records = get("CS_BUCKET_RECORDS");
    if (!t.walk_prep) t.walk_prep = (uint32_t)get("CS_WALK_PREP");
}

cs_status build_plan(cs_plan_s *pl, uint32_t P, uint64_t d, uint64_t M_start, uint64_t M_inc,
                     uint32_t SL, uint64_t L, const cs_tuning *tune, cs_cache_t cache) {
    std::vector<uint32_t> qK, qd;
    cs_status sv = check_params(P, d, M_start, M_inc, SL, L, qK, qd);
    if (sv) return sv;

    pl->P = P; pl->d = d; pl->M_start = M_start; pl->M_inc = M_inc; pl->SL = SL; pl->L = L;
    if (tune) pl->tune = *tune;
    env_tuning(pl->tune);
    if (const char *fa = getenv("CS_FAIL_ALLOC_AT")) pl->fail_alloc_at = strtoull(fa, nullptr, 10);
    pl->wheel = !pl->tune.no_wheel;

    // K as 32- and 64-bit factor words; K itself when it fits in 64 bits
    std::vector<uint32_t> kch32;
    std::vector<uint64_t> kch64;
    k_factor_words(qK, kch32, kch64);
    bool k_fits = kch64.size() <= 1;
    uint64_t K64 = kch64.empty() ? 1 : kch64[0];
    if (k_fits) {
        unsigned __int128 lo = (unsigned __int128)M_start * K64;
        if (lo < (unsigned __int128)SL + 2) return fail(CS_EINVAL, "need M_start*K - SL >= 2");
    }
    bool small_n = false;
    if (k_fits) {
        unsigned __int128 lowest = (unsigned __int128)M_start * K64 - SL;
        small_n = lowest <= (unsigned __int128)std::max<uint64_t>(L, P);
    }

    // columns: x in [-SL, SL] with gcd(|x|, K) = 1 (x = 0 only for K = 1)
    const uint64_t S = 2ull * SL + 1, S32 = (S + 31) / 32;
    std::vector<uint8_t> stored(S, 1);
    for (uint32_t q : qK) {
        // multiples of q in [-SL, SL] (x = 0 included)
        int64_t first = -(int64_t)(SL / q) * q;
        for (int64_t x = first; x <= (int64_t)SL; x += q) stored[x + SL] = 0;
    }
    std::vector<uint32_t> col_mask(S32, 0), col_prefix(S32, 0), raw_of_col;
    for (uint64_t z = 0; z < S; z++)
        if (stored[z]) {
            col_mask[z >> 5] |= 1u << (z & 31);
            raw_of_col.push_back((uint32_t)z);
            pl->x_of_col.push_back((int64_t)z - SL);
        }
    for (uint64_t w = 0, c = 0; w < S32; w++) {
        col_prefix[w] = (uint32_t)c;
        c += __builtin_popcount(col_mask[w]);
    }
    const uint64_t W = raw_of_col.size();
    uint64_t wpr = (W + 63) / 64;

    // rows: m coprime to d
    std::vector<uint32_t> moff_of_row;
    std::vector<uint32_t> row_mask((M_inc + 31) / 32, 0), row_prefix((M_inc + 31) / 32, 0);
    {
        std::vector<uint64_t> rem(qd.size());
        for (size_t i = 0; i < qd.size(); i++) rem[i] = M_start % qd[i];
        for (uint64_t k = 0; k < M_inc; k++) {
            bool ok = true;
            for (size_t i = 0; i < qd.size(); i++) {
                if (rem[i] == 0) ok = false;
                if (++rem[i] == qd[i]) rem[i] = 0;
            }
            if (ok) {
                row_mask[k >> 5] |= 1u << (k & 31);
                moff_of_row.push_back((uint32_t)k);
                pl->m_of_row.push_back(M_start + k);
            }
        }
    }
    const uint64_t M_c = moff_of_row.size();
    for (uint64_t w = 0, c = 0; w < row_mask.size(); w++) {
        row_prefix[w] = (uint32_t)c;
        c += __builtin_popcount(row_mask[w]);
    }

    // wheel tables: for each q | d, pattern[k] = bits i < 32 with (k + i) % q == 0
    std::vector<uint32_t> wq, wkmod, woff, wpat;
    if (pl->wheel) {
        for (uint32_t q : qd) {
            uint64_t km = 1;
            for (uint32_t f : qK) km = km * f % q;
            wq.push_back(q);
            wkmod.push_back((uint32_t)km);
            woff.push_back((uint32_t)wpat.size());
            for (uint32_t k = 0; k < q; k++) {
                uint32_t b = 0;
                for (uint32_t i = 0; i < 32; i++)
                    if ((k + i) % q == 0) b |= 1u << i;
                wpat.push_back(b);
            }
        }
    }

    // compact layout: per residue class rho of m mod d, the literal columns
    // that the wheel keeps (gcd(rho K + x, d) = 1)
    pl->layout = pl->tune.layout;
    std::vector<uint32_t> cmask, cprefix;
    if (pl->layout > 1) return fail(CS_EINVAL, "layout must be 0 or 1");
    if (pl->layout == 1) {
        if (!pl->wheel) return fail(CS_EINVAL, "the compact layout needs the wheel");
        if (k_fits && (unsigned __int128)M_start * K64 - SL <= (unsigned __int128)P)
            return fail(CS_EINVAL, "the compact layout needs N + x above the primes of d");
        uint64_t phi = 1;
        for (uint32_t q : qd) phi *= (q - 1);
        if (phi > 4096) return fail(CS_EINVAL, "the compact layout needs phi(d) <= 4096");
        std::vector<uint64_t> res;
        for (uint64_t rho = 0; rho < d; rho++) {
            bool ok = true;
            for (uint32_t q : qd) ok = ok && rho % q != 0;
            if (ok) res.push_back(rho);
        }
        pl->n_cls = (uint32_t)res.size();
        cmask.assign((size_t)pl->n_cls * S32, 0);
        cprefix.assign((size_t)pl->n_cls * S32, 0);
        pl->cW_h.assign(pl->n_cls, 0);
        std::vector<std::vector<uint32_t>> lists(pl->n_cls);
        for (uint32_t k = 0; k < pl->n_cls; k++) {
            uint32_t *cm = &cmask[(size_t)k * S32];
            for (uint64_t w = 0; w < S32; w++) cm[w] = col_mask[w];
            for (size_t qi = 0; qi < qd.size(); qi++) {
                const uint64_t q = qd[qi], kq = wkmod[qi];
                // z = x + SL with q | rho K + x:  z = SL - rho K (mod q)
                uint64_t z = ((SL % q) + q - (res[k] % q) * kq % q) % q;
                for (; z < S; z += q) cm[z >> 5] &= ~(1u << (z & 31));
            }
            uint32_t c = 0;
            for (uint64_t w = 0; w < S32; w++) {
                cprefix[(size_t)k * S32 + w] = c;
                uint32_t bits = cm[w];
                while (bits) {
                    uint32_t b = __builtin_ctz(bits);
                    bits &= bits - 1;
                    lists[k].push_back((uint32_t)(32 * w + b));
                }
                c += __builtin_popcount(cm[w]);
            }
            pl->cW_h[k] = c;
            pl->Wc_max = std::max(pl->Wc_max, c);
        }
        pl->craw_h.assign((size_t)pl->n_cls * std::max<uint32_t>(pl->Wc_max, 1), 0);
        for (uint32_t k = 0; k < pl->n_cls; k++)
            std::copy(lists[k].begin(), lists[k].end(), pl->craw_h.begin() + (size_t)k * std::max<uint32_t>(pl->Wc_max, 1));
        if (M_c) {
            const uint64_t r0 = pl->m_of_row[0] % d;
            pl->cls0 = (uint32_t)(std::lower_bound(res.begin(), res.end(), r0) - res.begin());
        }
        wpr = (pl->Wc_max + 63) / 64;
    }

    // small / large threshold and work split
    pl->mode = pl->tune.large_mode == 1 ? LARGE_PAPER : LARGE_THREE_GAP;
    uint64_t T = pl->tune.threshold;
    if (T) {
        if (T < 2ull * SL || T > MAX_T)
            return fail(CS_EINVAL, "threshold must satisfy 2*SL <= T <= 2^30");
    } else {
        uint64_t mult = pl->mode == LARGE_PAPER ? 100 : 8;
        T = std::min<uint64_t>(std::max<uint64_t>(mult * S, 1u << 16), MAX_T);
    }
    // the large-prime walk needs p > 2*SL (at most one hit per interval)
    T = std::max<uint64_t>({T, 2ull * SL, (uint64_t)P, 2});
    pl->T = T;
    pl->small_hi = std::min<uint64_t>(T, L);
    pl->narrow = L < NARROW_LIMIT;

    // large primes in chunks of (T, L]: geometric (factor 2) so that the hits
    // per prime, about M_inc * S / p, vary at most 2x inside a chunk, capped at
    // chunk_numbers wide; a chunk's primes are split into n_seg m-segments of
    // about HITS_PER_ITEM expected hits each
    const uint64_t chunk = pl->tune.chunk_numbers ? pl->tune.chunk_numbers : (1ull << 27);
    // m-classes per chunk (cs_classes.h): class items mod 210 or 30 for the
    // primes with the most hits, then m = 1, 5 (mod 6), then the odd m
    if (pl->tune.m_classes > 3) return fail(CS_EINVAL, "m_classes must be 0, 1, 2 or 3");
    const ClassTiers tiers = class_tiers(pl->mode == LARGE_THREE_GAP && SL > 0, d, M_start, M_inc, S, pl->tune);
    pl->mcls = tiers.mcls;
    pl->mcls_light = tiers.mcls_light;
    const double HITS_PER_ITEM = pl->tune.item_hits ? (double)pl->tune.item_hits : 128.0;
    auto classes_for = [&](uint64_t lo) -> MClasses { return tiers.for_chunk(lo); };
    // walked hits per item: a class (class items) or the item's n classes
    auto segs_for = [&](uint64_t lo) {
        double hits = (double)M_inc * (double)S / (double)std::max<uint64_t>(lo, 1);
        const MClasses mc = classes_for(lo);
        hits *= (double)(mc.items ? 1 : mc.n) / (double)mc.Q;
        double seg = std::min<double>(std::max(1.0, std::ceil(hits / HITS_PER_ITEM)), (double)std::max<uint64_t>(M_inc, 1));
        return (uint32_t)std::min(seg, 65536.0);
    };
    auto add_chunk = [&](uint64_t lo, uint64_t hi) {
        const MClasses mc = classes_for(lo);
        pl->chunks.push_back({lo, hi});
        pl->chunk_seg.push_back(segs_for(lo));
        pl->chunk_mc.push_back(mc);
        if (mc.items) {
            pl->item_chunks++;
            if (mc.Q > pl->item_mod) {
                pl->item_mod = mc.Q;
                pl->item_classes = mc.items;
            }
        } else {
            pl->split_chunks += mc.Q == pl->mcls.Q && mc.n == pl->mcls.n && pl->mcls.Q > 1;
        }
    };
    uint64_t widest = 0;
    if (cache) {
        // the cache's chunks that overlap (T, L]; the walk skips primes outside
        ResidueCacheView cv;
        cache_view(cache, &cv);
        if (cv.P != P || cv.d != d) return fail(CS_EINVAL, "cache was built for another P or d");
        if (L > cv.L_max) return fail(CS_EINVAL, "cache does not reach L");
        pl->cache = cache;
        for (size_t k = 0; k < cv.n_chunks; k++) {
            const CacheChunk &ch = cv.chunks[k];
            if (ch.hi <= T || ch.lo >= L) continue;
            const uint64_t lo = std::max(ch.lo, T), hi = std::min(ch.hi, L);
            add_chunk(lo, hi);
            pl->cache_idx.push_back(k);
        }
        pl->large_cap = 0;
    } else {
        for (uint64_t lo = T; lo < L;) {
            uint64_t hi = std::min<uint64_t>({L, lo + std::max<uint64_t>(lo, 1), lo + chunk});
            // a chunk ends below 2^30 when the next one starts above: it keeps the
            // 32-bit kernels
            if (lo < NARROW_LIMIT - 1 && hi >= NARROW_LIMIT) hi = NARROW_LIMIT - 1;
            add_chunk(lo, hi);
            widest = std::max(widest, hi - lo);
            lo = hi;
        }
        pl->large_cap = pl->chunks.empty() ? 0 : primes_in_interval_bound(widest);
    }
    // one segment count and one class choice per chunk (and one cache index
    // for cached plans): cs_sieve indexes all of them by chunk
    const size_t n_chunks = pl->chunks.size();
    if (pl->chunk_seg.size() != n_chunks || pl->chunk_mc.size() != n_chunks ||
        (pl->cache && pl->cache_idx.size() != n_chunks))
        return fail(CS_EDEVICE, "internal: large-prime chunk tables disagree");
    pl->small_cap = pl->small_hi > P ? prime_count_bound(pl->small_hi) : 0;
    pl->large_grid = (int)pl->tune.large_grid;   // 0: the launcher picks (one wave of resident CTAs)

    // tile shape: up to 32 rows of raw offsets in shared memory
    int dev = 0, optin = 0;
    CS_CUDA(cudaGetDevice(&dev));
    CS_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const uint64_t budget = (std::min<uint64_t>((uint64_t)optin, 200 * 1024) - tile_stage_bytes()) / 4;   // words
    std::vector<uint32_t> chunk_tab;
    uint32_t TR = pl->tune.tile_rows;
    if (TR && (TR > 32 || (TR & (TR - 1)))) return fail(CS_EINVAL, "tile_rows must be 1..32, a power of 2");
    auto words_of = [&](uint64_t j0, uint64_t j1) -> uint64_t {
        if (j1 <= j0) return 1;
        uint64_t z0 = raw_of_col[j0], z1 = raw_of_col[j1 - 1] + 1;
        return (z1 - (z0 & ~31ull) + 31) / 32;
    };
    uint64_t full_words = W ? words_of(0, W) : 1;
    if (!TR) {
        TR = 32;
        while (TR > 1 && (uint64_t)(TR + 1) * full_words > budget) TR /= 2;
    }
    uint64_t max_words_per_chunk = budget / (TR + 1);
    if (max_words_per_chunk < 64) return fail(CS_EINVAL, "tile_rows too large for shared memory");
    if (pl->layout == 1 && (uint64_t)(TR + 1) * full_words > budget)
        return fail(CS_EINVAL, "the compact layout needs the interval's tile in one piece (smaller SL or tile_rows)");
    uint32_t max_words = 1;
    if (W == 0) {
        chunk_tab = {0, 0, 0, 0};
    } else {
        uint64_t j0 = 0;
        while (j0 < W) {
            uint64_t j1 = std::min<uint64_t>(W, j0 + 64);
            while (j1 < W) {
                uint64_t nj = std::min<uint64_t>(W, j1 + 64);
                if (words_of(j0, nj) > max_words_per_chunk) break;
                j1 = nj;
            }
            uint64_t z0 = raw_of_col[j0], z1 = raw_of_col[j1 - 1] + 1;
            chunk_tab.insert(chunk_tab.end(), {(uint32_t)j0, (uint32_t)j1, (uint32_t)z0, (uint32_t)z1});
            max_words = std::max<uint32_t>(max_words, (uint32_t)words_of(j0, j1));
            j0 = j1;
        }
    }

    pl->M_c = M_c; pl->W = W; pl->wpr = wpr; pl->S = S; pl->S32 = S32;
    CS_CUDA(prepare_tile(optin));

    // relative cost, for ordering instances in a batch: tile pairs, walk hits,
    // large primes (each weighted by its measured per-unit time on a GB300)
    {
        auto pi = [](double x) { return x < 3 ? 0.0 : x / std::log(x); };
        const double Td = (double)T, Ld = (double)std::max<uint64_t>(L, 2);
        const double small = (double)M_c * std::max(0.0, pi((double)pl->small_hi) - pi((double)P));
        double hits = 0, large = 0;
        if (L > T && T > 2) {
            hits = (double)M_inc * (double)S * std::log(std::log(Ld) / std::log(Td));
            large = pi(Ld) - pi(Td);
        }
        // per-unit times measured on search_953: 7.4 ps per (row, small prime)
        // pair, ~7 ps per walk hit, ~150 ps per large prime (generation, K mod p
        // and the walk's solves), ~5 us per kernel launch
        pl->est_cost = (uint64_t)(small * 7.4 + hits * 7.0 + large * (cache ? 60.0 : 150.0) +
                                  5e6 * (3.0 + 2.0 * (double)pl->chunks.size()));
    }

    // device memory and tables
    DevPlan &dp = pl->dp;

    // the walk's stored hits through per-band regions (cs_buckets.h): by
    // default for bitsets of 256 MiB and more, whose scattered clears would go
    // to DRAM (4.77 GB bitset: 12% less time per sieve)
    dp.bucket = 0;
    {
        if (pl->tune.hit_buckets > 2) return fail(CS_EINVAL, "hit_buckets must be 0, 1 or 2");
        if (pl->tune.walk_prep > 2) return fail(CS_EINVAL, "walk_prep must be 0, 1 or 2");
        if (pl->tune.band_rows_log > 20) return fail(CS_EINVAL, "band_rows_log must be at most 20");
        // a region per band for every CTA of the walk's grid (three per SM)
        const BucketLayout b = bucket_layout(pl->tune.hit_buckets, pl->tune.band_rows_log,
                                             pl->tune.bucket_records, pl->mode == LARGE_THREE_GAP,
                                             !pl->chunks.empty(), M_c, wpr, l2_bytes(), (uint64_t)sm_count() * 3);
        if (b.bad_band_log)
            return fail(CS_EINVAL, "band_rows_log gives records above 32 bits or more than 4096 bands");
        if (b.on) {
            dp.bucket = 1;
            dp.band_log = b.band_log;
            dp.n_bands = (uint32_t)b.n_bands;
            dp.n_regions = (uint32_t)b.n_regions;
            dp.region_cap = (uint32_t)b.cap;
            pl->apply_after = apply_groups(pl->chunks, M_c, W, b);
            for (uint8_t f : pl->apply_after) pl->apply_launches += f;
        }
    }
    dp.M_start = M_start; dp.M_inc = M_inc; dp.M_c = M_c;
    dp.SL = SL; dp.S = (uint32_t)S; dp.S32 = (uint32_t)S32;
    dp.W = (uint32_t)W; dp.wpr = (uint32_t)wpr;
    dp.P = P; dp.L = L; dp.T = T; dp.d = d;
    dp.small_n = small_n; dp.K64 = K64;
    cs_status s;
    // the read-only tables go up together (one allocation, one copy)
    pl->stage(&dp.kch32, kch32);
    pl->stage(&dp.kch64, kch64);
    dp.n_kch32 = (uint32_t)kch32.size();
    dp.n_kch64 = (uint32_t)kch64.size();
    pl->stage(&dp.col_mask, col_mask);
    pl->stage(&dp.col_prefix, col_prefix);
    pl->stage(&dp.raw_of_col, raw_of_col);
    pl->stage(&dp.moff_of_row, moff_of_row);
    pl->stage(&dp.row_mask, row_mask);
    pl->stage(&dp.row_prefix, row_prefix);
    {
        // the same tables interleaved as {mask, prefix} pairs for the walk's lookups
        std::vector<uint2> ct(S32), rt(row_mask.size());
        for (uint64_t w = 0; w < S32; w++) ct[w] = make_uint2(col_mask[w], col_prefix[w]);
        for (size_t w = 0; w < row_mask.size(); w++) rt[w] = make_uint2(row_mask[w], row_prefix[w]);
        pl->stage(&dp.col_tab, ct);
        pl->stage(&dp.row_tab, rt);
    }
    pl->stage(&dp.qd, wq);
    pl->stage(&dp.qd_kmod, wkmod);
    pl->stage(&dp.qd_pat_off, woff);
    pl->stage(&dp.qd_pat, wpat);
    dp.n_qd = (uint32_t)wq.size();
    dp.compact = pl->layout == 1;
    dp.n_cls = pl->n_cls;
    dp.cls0 = pl->cls0;
    dp.Wc_max = pl->Wc_max;
    if (dp.compact) {
        // class of the first row in each 32-m word of the row mask
        std::vector<uint32_t> cls_word(row_mask.size(), 0);
        for (size_t w = 0; w < row_mask.size(); w++) cls_word[w] = (uint32_t)((pl->cls0 + row_prefix[w]) % pl->n_cls);
        pl->stage(&dp.cls_word, cls_word);
        pl->stage(&dp.cmask, cmask);
        pl->stage(&dp.cprefix, cprefix);
        pl->stage(&dp.craw, pl->craw_h);
        pl->stage(&dp.cW, pl->cW_h);
    }
    uint64_t *d_bits; uint32_t *d_cnt; unsigned long long *d_stats;
    if ((s = pl->dalloc(&d_bits, M_c * wpr))) return s;
    if ((s = pl->dalloc(&d_cnt, M_c))) return s;
    if ((s = pl->dalloc(&d_stats, ST_COUNT))) return s;
    dp.bits = d_bits; dp.counts = d_cnt; dp.stats = d_stats;
    if (dp.bucket) {
        const uint64_t before = pl->dev_bytes;
        const uint64_t n_reg = (uint64_t)dp.n_bands * dp.n_regions;
        if ((s = pl->dalloc(&dp.bkt, n_reg * dp.region_cap))) return s;
        if ((s = pl->dalloc(&dp.bkt_cnt, n_reg + 1))) return s;   // + the apply's region counter
        pl->bucket_bytes = pl->dev_bytes - before;
    }

    // base primes (odd) <= sqrt(L) for the segmented generator
    std::vector<uint32_t> base;
    for (uint32_t q : primes_upto(isqrt_u64(std::max<uint64_t>(L, T)) + 1))
        if (q != 2) base.push_back(q);
    pl->stage(&pl->d_base, base);
    pl->n_base = (uint32_t)base.size();

    pl->stage(&pl->tc.chunk, chunk_tab);
    pl->tc.rows = TR;
    pl->tc.n_chunks = (uint32_t)(chunk_tab.size() / 4);
    pl->tc.max_words = max_words;
    if ((s = pl->flush_uploads())) return s;

    if ((s = pl->dalloc(&pl->d_small, pl->small_cap))) return s;
    if ((s = pl->dalloc(&pl->d_counts, 1 + pl->chunks.size()))) return s;
    if (!pl->chunks.empty() && !pl->cache) {
        size_t el = pl->narrow ? 4 : 8;
        uint8_t *a, *b, *c;
        if ((s = pl->dalloc(&a, pl->large_cap * el))) return s;
        if ((s = pl->dalloc(&b, pl->large_cap * el))) return s;
        if ((s = pl->dalloc(&c, pl->large_cap * el))) return s;
        pl->d_lp = a; pl->d_lr = b; pl->d_lv = c;
        bool any_prep = false;
        for (size_t k = 0; k < pl->chunks.size(); k++)
            any_prep = any_prep || prep_eligible(pl->dp, pl->mode, pl->chunk_seg[k], pl->chunk_mc[k]);
        if (any_prep && pl->tune.walk_prep != 1) {
            if ((s = pl->dalloc(&pl->d_desc0, pl->large_cap))) return s;
            if ((s = pl->dalloc(&pl->d_desc1, pl->large_cap))) return s;
        }
    }
    CS_CUDA(cudaEventCreateWithFlags(&pl->done, cudaEventDisableTiming));
    CS_CUDA(cudaStreamSynchronize(pl->upload_stream()));
    std::vector<uint8_t>().swap(pl->staging);   // the copy has landed
    pl->built = true;
    return CS_OK;
}

cs_status wait_plan(cs_plan_t pl) {
    if (!pl->sieved) return fail(CS_ESTATE, "cs_sieve has not been called on this plan");
    if (pl->sticky) return pl->sticky;
    cudaError_t e = cudaEventSynchronize(pl->done);
    if (e != cudaSuccess) {
        pl->sticky = cuda_fail(e, "cudaEventSynchronize");
        return pl->sticky;
    }
    return CS_OK;
}

struct Prof {
    cs_plan_t pl;
    cudaStream_t st;
    bool on;
    cudaEvent_t end_ev = nullptr;
    int cls = -1;
    cs_status begin(int k) {
        if (!on) return CS_OK;
        auto &v = pl->prof_ev[k];
        size_t i = pl->prof_used[k]++;
        if (i == v.size()) {
            cudaEvent_t a, b;
            CS_CUDA(cudaEventCreate(&a));
            CS_CUDA(cudaEventCreate(&b));
            v.push_back({a, b});
        }
        CS_CUDA(cudaEventRecord(v[i].first, st));
        end_ev = v[i].second;
        return CS_OK;
    }
    cs_status end() {
        if (!on) return CS_OK;
        CS_CUDA(cudaEventRecord(end_ev, st));
        return CS_OK;
    }
};

}  // namespace

namespace cs {

void k_factor_words(const std::vector<uint32_t> &qK, std::vector<uint32_t> &w32, std::vector<uint64_t> &w64) {
    pack_k_words(qK, w32, w64);
}


cs_status plan_create(uint32_t P, uint64_t d, uint64_t M_start, uint64_t M_inc, uint32_t SL,
                      uint64_t L, const cs_tuning *tune, cudaStream_t alloc_stream, bool async_alloc,
                      cs_cache_t cache, cs_plan_t *out) {
    if (!out) return fail(CS_EINVAL, "out is NULL");
    *out = nullptr;
    cs_plan_s *pl = new (std::nothrow) cs_plan_s();
    if (!pl) return fail(CS_ENOMEM, "host allocation failed");
    pl->alloc_stream = alloc_stream;
    pl->async_alloc = async_alloc;
    cs_status s;
    try {
        s = build_plan(pl, P, d, M_start, M_inc, SL, L, tune, cache);
    } catch (const std::bad_alloc &) {
        s = fail(CS_ENOMEM, "host allocation failed");
    }
    if (s) {
        delete pl;
        return s;
    }
    *out = pl;
    g_err.clear();
    return CS_OK;
}

void plan_set_sieved(cs_plan_t pl, bool sieved) { pl->sieved = sieved; }
cs_cache_t plan_cache(cs_plan_t pl) { return pl->cache; }
bool plan_profiled(cs_plan_t pl) { return pl->tune.profile != 0; }
cudaEvent_t plan_done_event(cs_plan_t pl) { return pl->done; }
cs_status set_error(cs_status code, const char *msg) { return fail(code, msg); }
cs_status validate_params(uint32_t P, uint64_t d, uint64_t M_start, uint64_t M_inc, uint32_t SL, uint64_t L) {
    std::vector<uint32_t> qK, qd;
    return check_params(P, d, M_start, M_inc, SL, L, qK, qd);
}

}  // namespace cs

namespace cs {

cs_status plan_sieve_head(cs_plan_t pl, cudaStream_t st) {
    if (pl->sticky) return pl->sticky;
    pl->stream = st;
    const DevPlan &dp = pl->dp;
    Prof prof{pl, st, pl->tune.profile != 0};
    for (int k = 0; k < KC_N; k++) pl->prof_used[k] = 0;
    CS_CUDA(cudaMemsetAsync(dp.stats, 0, ST_COUNT * sizeof(unsigned long long), st));
    CS_CUDA(cudaMemsetAsync(pl->d_counts, 0, (1 + pl->chunks.size()) * sizeof(unsigned long long), st));
    if (dp.bucket)
        CS_CUDA(cudaMemsetAsync(dp.bkt_cnt, 0, ((size_t)dp.n_bands * dp.n_regions + 1) * sizeof(uint32_t), st));
    cs_status s;
    if (pl->small_hi > pl->P) {
        if ((s = prof.begin(KC_GEN_SMALL))) return s;
        CS_CUDA(launch_gen_small(dp, pl->P, pl->small_hi, pl->d_base, pl->n_base, pl->d_small,
                                 pl->small_cap, pl->d_counts, st));
        if ((s = prof.end())) return s;
    }
    if ((s = prof.begin(KC_TILE))) return s;
    CS_CUDA(launch_tile(dp, pl->tc, pl->d_small, pl->d_counts, pl->small_cap, st));
    return prof.end();
}

bool plan_walk_jobs(cs_plan_t pl, std::vector<WalkJob> &out) {
    if (!pl->cache || pl->mode != LARGE_THREE_GAP || pl->tune.profile || pl->tune.large_grid) return false;
    ResidueCacheView cv;
    cache_view(pl->cache, &cv);
    for (size_t c = 0; c < pl->chunks.size(); c++) {
        const CacheChunk &ch = cv.chunks[pl->cache_idx[c]];
        out.push_back(WalkJob{pl->dp, ch.narrow, ch.p, ch.r, ch.count, ch.cap, pl->chunk_seg[c], pl->T, pl->L,
                              pl->chunk_mc[c]});
    }
    return true;
}

cs_status plan_sieve_tail(cs_plan_t pl, cudaStream_t st) {
    Prof prof{pl, st, pl->tune.profile != 0};
    cs_status s;
    if ((s = prof.begin(KC_FINAL))) return s;
    CS_CUDA(launch_final(pl->dp, st));
    if ((s = prof.end())) return s;
    // inside a stream capture the completion event becomes an event-record node
    // of the graph, so that it is recorded each time the graph runs
    cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
    CS_CUDA(cudaStreamIsCapturing(st, &capst));
    if (capst == cudaStreamCaptureStatusActive)
        CS_CUDA(cudaEventRecordWithFlags(pl->done, st, cudaEventRecordExternal));
    else
        CS_CUDA(cudaEventRecord(pl->done, st));
    pl->sieved = true;
    return CS_OK;
}

}  // namespace cs

extern "C" {

cs_status cs_plan(uint32_t P, uint64_t d, uint64_t M_start, uint64_t M_inc, uint32_t SL,
                  uint64_t L, const cs_tuning *tune, cs_plan_t *out) {
    return cs::plan_create(P, d, M_start, M_inc, SL, L, tune, nullptr, false, nullptr, out);
}

cs_status cs_plan_cached(uint32_t P, uint64_t d, uint64_t M_start, uint64_t M_inc, uint32_t SL,
                         uint64_t L, const cs_tuning *tune, cs_cache_t cache, cs_plan_t *out) {
    if (!cache) return fail(CS_EINVAL, "cache is NULL");
    return cs::plan_create(P, d, M_start, M_inc, SL, L, tune, nullptr, false, cache, out);
}


cs_status cs_sieve(cs_plan_t pl, void *stream) {
    if (!pl) return fail(CS_EINVAL, "plan is NULL");
    if (pl->sticky) return pl->sticky;
    cudaStream_t st = (cudaStream_t)stream;
    const DevPlan &dp = pl->dp;
    cs_status s;
    if ((s = cs::plan_sieve_head(pl, st))) return s;
    Prof prof{pl, st, pl->tune.profile != 0};
    // bucketed hits: the records of a group of chunks are cleared after its last walk
    auto apply = [&](size_t c) -> cs_status {
        if (!dp.bucket || !pl->apply_after[c]) return CS_OK;
        cs_status r;
        if ((r = prof.begin(KC_APPLY))) return r;
        CS_CUDA(launch_apply_buckets(dp, st));
        return prof.end();
    };
    cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
    CS_CUDA(cudaStreamIsCapturing(st, &capst));
    if (pl->cache) {
        ResidueCacheView cv;
        cache_view(pl->cache, &cv);
        for (size_t c = 0; c < pl->chunks.size(); c++) {
            const CacheChunk &ch = cv.chunks[pl->cache_idx[c]];
            if (!ch.filled && capst != cudaStreamCaptureStatusActive)
                return fail(CS_ESTATE, "the residue cache has not been filled (cs_cache_fill)");
            CS_CUDA(cudaStreamWaitEvent(st, ch.ready, 0));
            if ((s = prof.begin(KC_LARGE))) return s;
            CS_CUDA(launch_large(dp, ch.narrow, pl->mode, ch.p, ch.r, nullptr, ch.count, ch.cap,
                                 pl->chunk_seg[c], pl->large_grid, st, pl->T, pl->L, pl->chunk_mc[c]));
            if ((s = prof.end())) return s;
            if ((s = apply(c))) return s;
        }
    }
    for (size_t c = 0; c < pl->chunks.size() && !pl->cache; c++) {
        unsigned long long *cnt = pl->d_counts + 1 + c;
        // 32-bit entries and kernels for every chunk below 2^30, also in a plan
        // whose L is above (its buffers hold 64-bit entries, so 32-bit ones fit)
        const bool narrow = pl->narrow || pl->chunks[c].second < NARROW_LIMIT;
        if ((s = prof.begin(KC_GEN_LARGE))) return s;
        CS_CUDA(launch_gen_large(dp, narrow, pl->chunks[c].first, pl->chunks[c].second,
                                 pl->d_base, pl->n_base, pl->d_lp, pl->d_lr, pl->d_lv,
                                 pl->large_cap, cnt, st));
        if ((s = prof.end())) return s;
        const bool pre = pl->d_desc0 && prep_eligible(dp, pl->mode, pl->chunk_seg[c], pl->chunk_mc[c]);
        if (pre) {
            if ((s = prof.begin(KC_PREP))) return s;
            CS_CUDA(launch_tg_prep(dp, narrow, pl->d_lp, pl->d_lr, pl->d_lv, cnt, pl->large_cap, 0, ~0ull,
                                   pl->chunk_mc[c], pl->d_desc0, pl->d_desc1, st));
            if ((s = prof.end())) return s;
        }
        if ((s = prof.begin(KC_LARGE))) return s;
        CS_CUDA(launch_large(dp, narrow, pl->mode, pl->d_lp, pl->d_lr, pl->d_lv, cnt,
                             pl->large_cap, pl->chunk_seg[c], pl->large_grid, st, 0, ~0ull,
                             pl->chunk_mc[c], pre ? pl->d_desc0 : nullptr, pre ? pl->d_desc1 : nullptr));
        if ((s = prof.end())) return s;
        if ((s = apply(c))) return s;
    }
    return cs::plan_sieve_tail(pl, st);
}

cs_status cs_sync(cs_plan_t pl) {
    if (!pl) return fail(CS_EINVAL, "plan is NULL");
    cs_status s = wait_plan(pl);
    if (s) return s;
    unsigned long long err = 0;
    CS_CUDA(cudaMemcpy(&err, pl->dp.stats + ST_ERROR, sizeof(err), cudaMemcpyDeviceToHost));
    if (pl->cache) {
        ResidueCacheView cv;
        cache_view(pl->cache, &cv);
        unsigned long long cerr = 0;
        CS_CUDA(cudaMemcpy(&cerr, cv.err, sizeof(cerr), cudaMemcpyDeviceToHost));
        err |= cerr;
    }
    const char *msg = nullptr;
    const cs_status st = status_of_device_errors(err, &msg);
    return st ? fail(st, msg) : CS_OK;
}

cs_status cs_info(cs_plan_t pl, cs_info_t *out) {
    if (!pl || !out) return fail(CS_EINVAL, "NULL argument");
    memset(out, 0, sizeof(*out));
    out->M_c = pl->M_c;
    out->W = pl->W;
    out->words_per_row = pl->wpr;
    out->bitset_bytes = pl->M_c * pl->wpr * 8;
    out->S = pl->S;
    out->threshold = pl->T;
    out->tile_rows = pl->tc.rows;
    out->large_mode = (uint32_t)pl->mode;
    out->narrow = pl->narrow;
    out->wheel = pl->wheel;
    out->n_large_chunks = pl->chunks.size();
    // per large-prime chunk: the walk, and without a cache the generator (and,
    // for 64-bit primes, the residue kernel)
    // (and the walker preparation of the one-walker chunks)
    uint64_t large_launches = 0;
    for (size_t c = 0; c < pl->chunks.size(); c++) {
        const auto &ch = pl->chunks[c];
        large_launches += pl->cache ? 1 : (pl->narrow || ch.second < NARROW_LIMIT) ? 2 : 3;
        large_launches += pl->d_desc0 && prep_eligible(pl->dp, pl->mode, pl->chunk_seg[c], pl->chunk_mc[c]);
    }
    out->launches_per_sieve = (pl->small_hi > pl->P ? 1 : 0) + (pl->M_c && pl->W ? 1 : 0) +
                              (pl->M_c ? 1 : 0) + large_launches + (pl->dp.bucket ? pl->apply_launches : 0);
    out->h2d_bytes = pl->h2d;
    out->device_bytes = pl->dev_bytes;
    out->est_cost = pl->est_cost;
    out->layout = pl->layout;
    out->n_classes = pl->n_cls;
    out->m_mod = pl->mcls.Q;
    out->m_walked = pl->mcls.n;
    out->split_chunks = pl->split_chunks;
    out->item_mod = pl->item_mod;
    out->item_classes = pl->item_classes;
    out->item_chunks = pl->item_chunks;
    out->hit_buckets = pl->dp.bucket ? 1 : 0;
    out->n_bands = pl->dp.bucket ? pl->dp.n_bands : 0;
    out->bucket_bytes = pl->bucket_bytes;
    out->apply_launches = pl->dp.bucket ? pl->apply_launches : 0;
    out->prep_chunks = 0;
    for (size_t c = 0; c < pl->chunks.size() && pl->d_desc0; c++)
        out->prep_chunks += prep_eligible(pl->dp, pl->mode, pl->chunk_seg[c], pl->chunk_mc[c]);
    if (pl->layout == 1) out->W = pl->Wc_max;
    return CS_OK;
}

cs_status cs_fetch_bitset(cs_plan_t pl, uint64_t *host, size_t n_words) {
    if (!pl) return fail(CS_EINVAL, "plan is NULL");
    const uint64_t need = pl->M_c * pl->wpr;
    if (need && !host) return fail(CS_EINVAL, "host is NULL");
    if (n_words < need) return fail(CS_ESIZE, "host buffer smaller than M_c * words_per_row");
    cs_status s = wait_plan(pl);
    if (s) return s;
    if (need) {
        CS_CUDA(cudaMemcpyAsync(host, pl->dp.bits, need * 8, cudaMemcpyDeviceToHost, pl->stream));
        CS_CUDA(cudaStreamSynchronize(pl->stream));
    }
    return CS_OK;
}

cs_status cs_fetch_rows(cs_plan_t pl, uint64_t row0, uint64_t n_rows, uint64_t *host, size_t n_words) {
    if (!pl) return fail(CS_EINVAL, "plan is NULL");
    if (row0 > pl->M_c || n_rows > pl->M_c - row0) return fail(CS_EINVAL, "row range beyond M_c");
    const uint64_t need = n_rows * pl->wpr;
    if (need && !host) return fail(CS_EINVAL, "host is NULL");
    if (n_words < need) return fail(CS_ESIZE, "host buffer smaller than n_rows * words_per_row");
    cs_status s = wait_plan(pl);
    if (s) return s;
    if (need) {
        CS_CUDA(cudaMemcpyAsync(host, pl->dp.bits + row0 * pl->wpr, need * 8, cudaMemcpyDeviceToHost, pl->stream));
        CS_CUDA(cudaStreamSynchronize(pl->stream));
    }
    return CS_OK;
}

cs_status cs_counts(cs_plan_t pl, uint32_t *per_row, size_t n_rows, uint64_t *F, uint64_t *hash) {
    if (!pl) return fail(CS_EINVAL, "plan is NULL");
    if (per_row && n_rows < pl->M_c) return fail(CS_ESIZE, "per_row smaller than M_c");
    cs_status s = wait_plan(pl);
    if (s) return s;
    unsigned long long st[ST_COUNT];
    CS_CUDA(cudaMemcpyAsync(st, pl->dp.stats, sizeof(st), cudaMemcpyDeviceToHost, pl->stream));
    if (per_row && pl->M_c)
        CS_CUDA(cudaMemcpyAsync(per_row, pl->dp.counts, pl->M_c * 4, cudaMemcpyDeviceToHost, pl->stream));
    CS_CUDA(cudaStreamSynchronize(pl->stream));
    if (F) *F = st[ST_F_SMALL] + st[ST_F_LARGE];
    if (hash) *hash = st[ST_HASH];
    return CS_OK;
}

cs_status cs_stats(cs_plan_t pl, cs_stats_t *out) {
    if (!pl || !out) return fail(CS_EINVAL, "NULL argument");
    cs_status s = wait_plan(pl);
    if (s) return s;
    unsigned long long st[ST_COUNT];
    unsigned long long cnt[1];
    CS_CUDA(cudaMemcpy(st, pl->dp.stats, sizeof(st), cudaMemcpyDeviceToHost));
    CS_CUDA(cudaMemcpy(cnt, pl->d_counts, sizeof(cnt), cudaMemcpyDeviceToHost));
    std::vector<unsigned long long> lc(pl->chunks.size());
    if (!lc.empty())
        CS_CUDA(cudaMemcpy(lc.data(), pl->d_counts + 1, lc.size() * 8, cudaMemcpyDeviceToHost));
    memset(out, 0, sizeof(*out));
    out->F_small = st[ST_F_SMALL];
    out->F_large = st[ST_F_LARGE];
    out->F = out->F_small + out->F_large;
    out->solves = st[ST_SOLVES];
    out->levels = st[ST_LEVELS];
    out->hits_all = st[ST_HITS_ALL];
    out->n_small_primes = std::min<uint64_t>(cnt[0], pl->small_cap);
    for (auto c : lc) out->n_large_primes += c;
    out->survivors = st[ST_SURVIVORS];
    out->hash = st[ST_HASH];
    out->bucket_records = st[ST_RECORDS];
    return CS_OK;
}

cs_status cs_rows(cs_plan_t pl, uint64_t *m_of_row, size_t n) {
    if (!pl) return fail(CS_EINVAL, "plan is NULL");
    if (n < pl->M_c) return fail(CS_ESIZE, "buffer smaller than M_c");
    if (pl->M_c) memcpy(m_of_row, pl->m_of_row.data(), pl->M_c * 8);
    return CS_OK;
}

cs_status cs_columns(cs_plan_t pl, int64_t *x_of_col, size_t n) {
    if (!pl) return fail(CS_EINVAL, "plan is NULL");
    if (n < pl->W) return fail(CS_ESIZE, "buffer smaller than W");
    if (pl->W) memcpy(x_of_col, pl->x_of_col.data(), pl->W * 8);
    return CS_OK;
}

cs_status cs_row_columns(cs_plan_t pl, uint64_t row, int64_t *x_of_col, size_t n, uint64_t *n_cols) {
    if (!pl || !n_cols) return fail(CS_EINVAL, "NULL argument");
    if (row >= pl->M_c) return fail(CS_EINVAL, "row beyond M_c");
    if (pl->layout == 0) {
        *n_cols = pl->W;
        if (n < pl->W) return fail(CS_ESIZE, "buffer smaller than the row's columns");
        if (pl->W) memcpy(x_of_col, pl->x_of_col.data(), pl->W * 8);
        return CS_OK;
    }
    const uint32_t k = (uint32_t)((pl->cls0 + row) % pl->n_cls);
    const uint32_t w = pl->cW_h[k];
    *n_cols = w;
    if (n < w) return fail(CS_ESIZE, "buffer smaller than the row's columns");
    const uint32_t *raw = &pl->craw_h[(size_t)k * std::max<uint32_t>(pl->Wc_max, 1)];
    for (uint32_t j = 0; j < w; j++) x_of_col[j] = (int64_t)raw[j] - pl->SL;
    return CS_OK;
}

const void *cs_device_bitset(cs_plan_t pl) { return pl ? (const void *)pl->dp.bits : nullptr; }

cs_status cs_kernel_times(cs_plan_t pl, double ms[7], uint64_t launches[7]) {
    if (!pl || !ms || !launches) return fail(CS_EINVAL, "NULL argument");
    if (!pl->tune.profile) return fail(CS_ESTATE, "plan was built without profile = 1");
    cs_status s = wait_plan(pl);
    if (s) return s;
    for (int k = 0; k < KC_N; k++) {
        double tot = 0;
        for (size_t i = 0; i < pl->prof_used[k]; i++) {
            float t = 0;
            CS_CUDA(cudaEventElapsedTime(&t, pl->prof_ev[k][i].first, pl->prof_ev[k][i].second));
            tot += t;
        }
        ms[k] = tot;
        launches[k] = pl->prof_used[k];
    }
    return CS_OK;
}

cs_status cs_destroy(cs_plan_t pl) {
    if (!pl) return CS_OK;
    if (pl->sieved && pl->done) cudaEventSynchronize(pl->done);
    delete pl;
    return CS_OK;
}

const char *cs_last_error(void) { return g_err.c_str(); }

cs_status cs_primes(uint64_t lo, uint64_t hi, uint64_t *out, uint64_t cap, uint64_t *count,
                    void *stream) {
    if (hi > MAX_L) return fail(CS_EINVAL, "hi must be <= 2^40");
    if (!count) return fail(CS_EINVAL, "count is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    *count = 0;
    if (hi <= lo || hi < 2) return CS_OK;
    std::vector<uint32_t> base;
    for (uint32_t q : primes_upto(isqrt_u64(hi) + 1))
        if (q != 2) base.push_back(q);
    uint32_t *d_base = nullptr;
    unsigned long long *d_cnt = nullptr;
    CS_CUDA(cudaMalloc(&d_base, std::max<size_t>(base.size(), 1) * 4));
    cudaError_t e = cudaMalloc(&d_cnt, 16);
    if (e == cudaSuccess && !base.empty())
        e = cudaMemcpyAsync(d_base, base.data(), base.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, 16, st);
    if (e == cudaSuccess) e = launch_gen_list(lo, hi, d_base, (uint32_t)base.size(), out, cap, d_cnt, d_cnt + 1, st);
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_cnt, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_base);
    cudaFree(d_cnt);
    if (e != cudaSuccess) return cuda_fail(e, "cs_primes");
    *count = h[0];
    if (h[1] || h[0] > cap) return fail(CS_EOVERFLOW, "more primes than cap");
    return CS_OK;
}

cs_status cs_k_mod_p(uint32_t P, uint64_t d, const uint64_t *p, uint64_t n, uint64_t *r, void *stream) {
    if (d == 0 || P > MAX_P) return fail(CS_EINVAL, "bad P or d");
    std::vector<uint32_t> qK, qd;
    if (!split_primes(P, d, qK, qd)) return fail(CS_EINVAL, "d must be squarefree and divide P#");
    std::vector<uint32_t> kch32;
    std::vector<uint64_t> kch64;
    k_factor_words(qK, kch32, kch64);
    cudaStream_t st = (cudaStream_t)stream;
    uint32_t *d32 = nullptr;
    uint64_t *d64 = nullptr;
    CS_CUDA(cudaMalloc(&d32, std::max<size_t>(kch32.size(), 1) * 4));
    cudaError_t e = cudaMalloc(&d64, std::max<size_t>(kch64.size(), 1) * 8);
    if (e == cudaSuccess && !kch32.empty())
        e = cudaMemcpyAsync(d32, kch32.data(), kch32.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !kch64.empty())
        e = cudaMemcpyAsync(d64, kch64.data(), kch64.size() * 8, cudaMemcpyHostToDevice, st);
    DevPlan dp{};
    dp.kch32 = d32; dp.n_kch32 = (uint32_t)kch32.size();
    dp.kch64 = d64; dp.n_kch64 = (uint32_t)kch64.size();
    if (e == cudaSuccess) e = launch_kmodp(dp, p, n, r, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d32);
    cudaFree(d64);
    if (e != cudaSuccess) return cuda_fail(e, "cs_k_mod_p");
    return CS_OK;
}

cs_status cs_modsolve(const uint64_t *p, const uint64_t *K, const uint64_t *L, const uint64_t *R,
                      uint64_t *m, uint64_t n, int narrow, void *stream) {
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = launch_modsolve(p, K, L, R, m, n, narrow, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "cs_modsolve");
    return CS_OK;
}

}  // extern "C"
