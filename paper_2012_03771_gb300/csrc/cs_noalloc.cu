// Prime generation without device allocation: cs_primes_static.
//
// cs_primes allocates two small device buffers per call (the base primes and
// the counters).  This variant keeps them in a fixed file-scope device array
// instead, for callers that cannot allocate device memory.  The array is
// loaded with the library on every GPU that loads it and stays resident until
// the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/combsieve.h"
#include "cs_internal.h"

namespace {

// Layout of the scratch array (32-bit words):
//   [0, 4)                      counters: uint64 prime count, uint64 error flags
//   [BITMAP_OFF, + BITMAP_WORDS) sieve of the odd numbers <= 2^20 (bit set = composite)
//   [BASE_OFF, + BASE_CAP)      odd base primes <= sqrt(hi), ascending, then
//                               0xffffffff sentinels up to BASE_CAP
constexpr uint32_t LIMIT_MAX = 1u << 20;                 // sqrt(2^40)
constexpr uint32_t BITMAP_OFF = 64;
constexpr uint32_t BITMAP_WORDS = (LIMIT_MAX / 2 + 1 + 31) / 32 + 1;
constexpr uint32_t BASE_OFF = BITMAP_OFF + BITMAP_WORDS + 63 & ~63u;
constexpr uint32_t BASE_CAP = 82048;                     // > 82024 odd primes below 2^20
constexpr uint32_t SCRATCH_WORDS = BASE_OFF + BASE_CAP;  // about 385 KiB

static __device__ __align__(256) uint32_t g_cs_scratch[SCRATCH_WORDS];

constexpr int BASE_THREADS = 1024;

// Odd primes <= limit (limit <= 2^20) into the base list, in ascending order,
// followed by sentinels; one block.
__global__ void __launch_bounds__(BASE_THREADS) k_base_primes(uint32_t *scratch, uint32_t limit) {
    uint32_t *bm = scratch + BITMAP_OFF;
    uint32_t *base = scratch + BASE_OFF;
    const uint32_t n_odd = (limit + 1) / 2;               // odd numbers 1, 3, ..., <= limit
    const uint32_t n_words = (n_odd + 31) / 32;
    for (uint32_t w = threadIdx.x; w < n_words; w += BASE_THREADS) bm[w] = 0;
    __syncthreads();
    if (threadIdx.x == 0) atomicOr(&bm[0], 1u);           // 1 is not prime
    // mark odd multiples q^2, q^2 + 2q, ... of every odd q with q^2 <= limit
    for (uint32_t q = 3; q * q <= limit; q += 2) {
        for (uint32_t v = q * q + 2 * q * threadIdx.x; v <= limit; v += 2 * q * BASE_THREADS)
            atomicOr(&bm[(v / 2) >> 5], 1u << ((v / 2) & 31));
    }
    __syncthreads();
    // ordered compaction: each thread owns a contiguous run of words
    __shared__ uint32_t sums[BASE_THREADS];
    const uint32_t per = (n_words + BASE_THREADS - 1) / BASE_THREADS;
    const uint32_t w0 = threadIdx.x * per, w1 = min(w0 + per, n_words);
    uint32_t cnt = 0;
    for (uint32_t w = w0; w < w1; w++) {
        uint32_t valid = 32 * w + 32 <= n_odd ? 0xffffffffu : (n_odd > 32 * w ? (1u << (n_odd - 32 * w)) - 1 : 0u);
        cnt += __popc(~bm[w] & valid);
    }
    sums[threadIdx.x] = cnt;
    __syncthreads();
    for (uint32_t o = 1; o < BASE_THREADS; o <<= 1) {
        uint32_t t = threadIdx.x >= o ? sums[threadIdx.x - o] : 0;
        __syncthreads();
        sums[threadIdx.x] += t;
        __syncthreads();
    }
    uint32_t pos = sums[threadIdx.x] - cnt;
    for (uint32_t w = w0; w < w1; w++) {
        uint32_t valid = 32 * w + 32 <= n_odd ? 0xffffffffu : (n_odd > 32 * w ? (1u << (n_odd - 32 * w)) - 1 : 0u);
        uint32_t pr = ~bm[w] & valid;
        while (pr) {
            uint32_t b = __ffs(pr) - 1;
            pr &= pr - 1;
            if (pos < BASE_CAP) base[pos] = 2 * (32 * w + b) + 1;
            pos++;
        }
    }
    __syncthreads();
    const uint32_t total = sums[BASE_THREADS - 1];
    for (uint32_t i = total + threadIdx.x; i < BASE_CAP; i += BASE_THREADS) base[i] = 0xffffffffu;
}

std::mutex g_mu;
uint32_t *g_ptr[256];   // device address of g_cs_scratch, per device ordinal

cs_status scratch_for_current_device(uint32_t **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 256) return CS_EDEVICE;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_cs_scratch);
        if (e != cudaSuccess || !p) return CS_EDEVICE;
        g_ptr[dev] = static_cast<uint32_t *>(p);
    }
    *out = g_ptr[dev];
    return CS_OK;
}

uint64_t isqrt_floor(uint64_t n) {
    uint64_t r = 0;
    for (int b = 31; b >= 0; b--) {
        uint64_t t = r | (1ull << b);
        if (t * t <= n) r = t;
    }
    return r;
}

// errors go through the library's error text, like those of cs_primes
cs_status cuda_error(cudaError_t e, const char *what) {
    return cs::set_error(CS_EDEVICE, (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}

}  // namespace

extern "C" cs_status cs_primes_static(uint64_t lo, uint64_t hi, uint64_t *out, uint64_t cap,
                                      uint64_t *count, void *stream) {
    if (!count) return cs::set_error(CS_EINVAL, "cs_primes_static: count is NULL");
    *count = 0;
    if (hi > (1ull << 40)) return cs::set_error(CS_EINVAL, "cs_primes_static: hi above 2^40");
    if (hi <= lo || hi < 2) return CS_OK;
    uint32_t *scratch = nullptr;
    cs_status s = scratch_for_current_device(&scratch);
    if (s) return cs::set_error(s, "cs_primes_static: no device address for the static scratch");
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t limit = (uint32_t)isqrt_floor(hi) + 1;   // <= 2^20 + 1, odd part <= 2^20
    const uint32_t lim = limit > LIMIT_MAX ? LIMIT_MAX : limit;
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(scratch);
    cudaError_t e = cudaMemsetAsync(ctr, 0, 16, st);            // count and error start at zero
    if (e == cudaSuccess) {
        k_base_primes<<<1, BASE_THREADS, 0, st>>>(scratch, lim);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cs::launch_gen_list(lo, hi, scratch + BASE_OFF, BASE_CAP, out, cap, ctr, ctr + 1, st);
    unsigned long long h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, ctr, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "cs_primes_static");
    *count = h[0];
    if (h[1] || h[0] > cap) return cs::set_error(CS_EOVERFLOW, "cs_primes_static: more primes than cap");
    return CS_OK;
}
