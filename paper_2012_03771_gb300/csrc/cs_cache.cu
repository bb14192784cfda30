// Residue cache: device-resident primes and r = K mod p for one K = P#/d.
//
// Section 3.1 caches K mod p so that every m costs one word-sized product.
// Searches with the same K but other m-ranges, intervals or limits (Section 5:
// many m-ranges per P#/d) can share more than that: the whole list of
// (p, K mod p) up to a limit.  The cache keeps that list in HBM on a fixed grid
// of chunks; plans walk the chunks that overlap their own (T, L].
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/combsieve.h"
#include "cs_internal.h"

using namespace cs;

struct cs_cache_s {
    uint32_t P = 0;
    uint64_t d = 0, L_max = 0;
    DevPlan kp{};                      // only kch32 / kch64 are used
    std::vector<void *> allocs;
    uint32_t *base = nullptr;          // odd primes <= sqrt(L_max), ascending
    uint32_t n_base = 0;
    std::vector<CacheChunk> chunks;
    unsigned long long *err = nullptr;
    uint64_t bytes = 0;
    std::mutex mu;

    ~cs_cache_s() {
        for (auto &c : chunks)
            if (c.ready) cudaEventDestroy(c.ready);
        for (void *p : allocs) cudaFree(p);
    }
    cs_status alloc(void **p, size_t bytes_) {
        cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes_, 8));
        if (e != cudaSuccess) return set_error(e == cudaErrorMemoryAllocation ? CS_ENOMEM : CS_EDEVICE, "cudaMalloc (cache)");
        allocs.push_back(*p);
        bytes += bytes_;
        return CS_OK;
    }
};

namespace {

// Host-to-device copy that has landed when it returns: on a private stream,
// synchronised (a plain cudaMemcpy from pageable memory may return before its
// DMA completes and is ordered only on the legacy default stream).
cudaError_t upload_now(void *dst, const void *src, size_t bytes) {
    cudaStream_t st;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    e = src ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) : cudaMemsetAsync(dst, 0, bytes, st);
    cudaError_t e2 = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    return e != cudaSuccess ? e : e2;
}

constexpr uint64_t GRID0 = 1ull << 16;
constexpr uint64_t GRID_MAX_WIDTH = 1ull << 27;
constexpr uint64_t NARROW = 1ull << 30;

// pi(x) bounds of P. Dusart (2010): x/ln x (1 + 1/ln x + 2/ln^2 x) <= pi(x) for
// x >= 88789 and pi(x) <= x/ln x (1 + 1/ln x + 2.51/ln^2 x) for x >= 355991.
double pi_upper(double x) {
    if (x < 355991.0) return x < 2 ? 0 : 1.26 * x / log(x) + 16;   // Rosser-Schoenfeld for small x
    double l = log(x);
    return x / l * (1 + 1 / l + 2.51 / (l * l));
}
double pi_lower(double x) {
    if (x < 355991.0) return 0;
    double l = log(x);
    return x / l * (1 + 1 / l + 2 / (l * l));
}

uint64_t chunk_cap(uint64_t lo, uint64_t hi) {
    double c = pi_upper((double)hi) - pi_lower((double)lo);
    double mv = hi - lo >= 64 ? 2.0 * (double)(hi - lo) / log((double)(hi - lo)) : 64.0;   // Montgomery-Vaughan
    return (uint64_t)(std::min(c, mv) * 1.01) + 4096;
}

std::vector<uint32_t> small_primes(uint64_t n) {
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

uint64_t isqrt_ceil(uint64_t n) {
    uint64_t r = (uint64_t)sqrt((double)n);
    while (r * r > n) r--;
    while ((r + 1) * (r + 1) <= n) r++;
    return r + 1;
}

cs_status cuda_err(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return CS_OK;
    return set_error(e == cudaErrorMemoryAllocation ? CS_ENOMEM : CS_EDEVICE, what);
}

}  // namespace

namespace cs {

std::mutex &cache_mutex(cs_cache_t c) { return c->mu; }

bool cache_view(cs_cache_t c, ResidueCacheView *out) {
    if (!c) return false;
    out->P = c->P;
    out->d = c->d;
    out->L_max = c->L_max;
    out->chunks = c->chunks.data();
    out->n_chunks = c->chunks.size();
    out->err = c->err;
    return true;
}

cs_status cache_extend(cs_cache_t c, uint64_t L) {
    if (L > (1ull << 40)) return set_error(CS_EINVAL, "cache limit must be <= 2^40");
    uint64_t lo = c->chunks.empty() ? 0 : c->chunks.back().hi;
    while (lo < L) {
        uint64_t hi = lo == 0 ? GRID0 : lo + std::min(lo, GRID_MAX_WIDTH);
        CacheChunk ch;
        ch.lo = lo;
        ch.hi = hi;
        ch.narrow = hi < NARROW;
        ch.cap = chunk_cap(lo, hi);
        const size_t el = ch.narrow ? 4 : 8;
        cs_status s;
        if ((s = c->alloc(&ch.p, ch.cap * el))) return s;
        if ((s = c->alloc(&ch.r, ch.cap * el))) return s;
        void *cnt;
        if ((s = c->alloc(&cnt, 8))) return s;
        ch.count = static_cast<unsigned long long *>(cnt);
        if ((s = cuda_err(cudaEventCreateWithFlags(&ch.ready, cudaEventDisableTiming), "cudaEventCreate"))) return s;
        c->chunks.push_back(ch);
        lo = hi;
    }
    if (L > c->L_max) {
        // base primes up to sqrt of the new limit
        std::vector<uint32_t> base;
        for (uint32_t q : small_primes(isqrt_ceil(std::max<uint64_t>(c->chunks.back().hi, 4))))
            if (q != 2) base.push_back(q);
        void *b;
        cs_status s;
        if ((s = c->alloc(&b, base.size() * 4))) return s;
        if (!base.empty() && (s = cuda_err(upload_now(b, base.data(), base.size() * 4), "upload")))
            return s;
        c->base = static_cast<uint32_t *>(b);
        c->n_base = (uint32_t)base.size();
        c->L_max = c->chunks.back().hi;
    }
    return CS_OK;
}

cs_status cache_new(uint32_t P, uint64_t d, uint64_t L_max, cs_cache_t *out) {
    if (!out) return set_error(CS_EINVAL, "out is NULL");
    *out = nullptr;
    if (d == 0 || P > (1u << 20)) return set_error(CS_EINVAL, "bad P or d");
    if (L_max > (1ull << 40)) return set_error(CS_EINVAL, "cache limit must be <= 2^40");
    std::vector<uint32_t> pr = small_primes(P), qK;
    uint64_t rest = d;
    for (uint32_t q : pr) {
        if (rest % q == 0) {
            rest /= q;
            if (rest % q == 0) return set_error(CS_EINVAL, "d must be squarefree and divide P#");
        } else {
            qK.push_back(q);
        }
    }
    if (rest != 1) return set_error(CS_EINVAL, "d must be squarefree and divide P#");
    std::vector<uint32_t> kch32;
    std::vector<uint64_t> kch64;
    k_factor_words(qK, kch32, kch64);

    cs_cache_s *c = new (std::nothrow) cs_cache_s();
    if (!c) return set_error(CS_ENOMEM, "host allocation failed");
    c->P = P;
    c->d = d;
    cs_status s = CS_OK;
    void *k32, *k64, *err;
    if (!s) s = c->alloc(&k32, kch32.size() * 4);
    if (!s) s = c->alloc(&k64, kch64.size() * 8);
    if (!s) s = c->alloc(&err, 8);
    if (!s && !kch32.empty()) s = cuda_err(upload_now(k32, kch32.data(), kch32.size() * 4), "upload");
    if (!s && !kch64.empty()) s = cuda_err(upload_now(k64, kch64.data(), kch64.size() * 8), "upload");
    if (!s) s = cuda_err(upload_now(err, nullptr, 8), "memset");
    if (s) { delete c; return s; }
    c->kp.kch32 = static_cast<uint32_t *>(k32);
    c->kp.n_kch32 = (uint32_t)kch32.size();
    c->kp.kch64 = static_cast<uint64_t *>(k64);
    c->kp.n_kch64 = (uint32_t)kch64.size();
    c->err = static_cast<unsigned long long *>(err);
    s = cache_extend(c, std::max<uint64_t>(L_max, 2));
    if (s) { delete c; return s; }
    *out = c;
    return CS_OK;
}

cs_status cache_fill_upto(cs_cache_t c, uint64_t L, cudaStream_t st, bool only_missing) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cs_status s = cuda_err(cudaStreamIsCapturing(st, &cap), "cudaStreamIsCapturing");
    if (s) return s;
    for (auto &ch : c->chunks) {
        if (L && ch.lo >= L) break;
        if (only_missing && ch.filled) continue;
        if ((s = cuda_err(cudaMemsetAsync(ch.count, 0, 8, st), "cudaMemsetAsync"))) return s;
        if ((s = cuda_err(launch_gen_pr(c->kp, ch.narrow, ch.lo, ch.hi, c->base, c->n_base, ch.p, ch.r, ch.cap,
                                        ch.count, c->err, st), "launch_gen_pr")))
            return s;
        if ((s = cuda_err(cudaEventRecord(ch.ready, st), "cudaEventRecord"))) return s;
        // an event recorded inside a capture only orders work inside that graph
        ch.filled = cap != cudaStreamCaptureStatusActive;
    }
    return CS_OK;
}

}  // namespace cs

extern "C" {

cs_status cs_cache_create(uint32_t P, uint64_t d, uint64_t L_max, cs_cache_t *out) {
    return cache_new(P, d, L_max, out);
}

cs_status cs_cache_fill(cs_cache_t c, void *stream) {
    if (!c) return set_error(CS_EINVAL, "cache is NULL");
    std::lock_guard<std::mutex> lk(c->mu);
    return cache_fill_upto(c, 0, (cudaStream_t)stream, false);
}

cs_status cs_cache_info(cs_cache_t c, uint64_t *n_chunks, uint64_t *device_bytes, uint64_t *n_primes) {
    if (!c) return set_error(CS_EINVAL, "cache is NULL");
    if (n_chunks) *n_chunks = c->chunks.size();
    if (device_bytes) *device_bytes = c->bytes;
    if (n_primes) {
        cs_status s = cuda_err(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
        if (s) return s;
        uint64_t tot = 0;
        for (auto &ch : c->chunks) {
            unsigned long long v = 0;
            if ((s = cuda_err(cudaMemcpy(&v, ch.count, 8, cudaMemcpyDeviceToHost), "cudaMemcpy"))) return s;
            tot += v;
        }
        unsigned long long e = 0;
        if ((s = cuda_err(cudaMemcpy(&e, c->err, 8, cudaMemcpyDeviceToHost), "cudaMemcpy"))) return s;
        if (e) return set_error(CS_EOVERFLOW, "a cache chunk overflowed");
        *n_primes = tot;
    }
    return CS_OK;
}

cs_status cs_cache_destroy(cs_cache_t c) {
    if (!c) return CS_OK;
    cudaDeviceSynchronize();
    delete c;
    return CS_OK;
}

}  // extern "C"
