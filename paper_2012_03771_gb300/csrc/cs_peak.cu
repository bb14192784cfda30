// Micro-benchmarks for the measured peaks of the roofline.  The paper has no
// counterpart; its cost model counts cycles of a CPU instead.
//
// cs_issue_rate: the integer issue rate, against which the integer-bound
// kernels (the large-prime walk, the residues K mod p) are placed.
//
// Every thread runs CHAINS independent dependency chains of integer
// operations, UNROLL steps per loop iteration, so that the schedulers always
// have independent instructions to issue:
//   MIX_ALU  per step and chain: x = (x + y) ^ c       (add and logic op)
//   MIX_FMA  per step and chain: x = x * y + z          (integer multiply-add)
//   MIX_BOTH per step and chain: x = (x * y + z) ^ c    (one of each)
// The operation count is what the source states (ops_per_step x steps x
// threads); the loop's own counter, compare and branch add 3 instructions per
// UNROLL steps and are not counted, so the measured rate is at most about 1%
// below the true instruction rate.
#include <cuda_runtime.h>

#include "../../include/combsieve.h"
#include "cs_arith.cuh"
#include "cs_internal.h"

namespace cs {

namespace {

constexpr int PEAK_THREADS = 256;
constexpr int CHAINS = 8;
constexpr int UNROLL = 32;

template <int MIX>
__global__ void __launch_bounds__(PEAK_THREADS) k_issue(uint32_t iters, uint32_t seed, uint32_t *sink) {
    const uint32_t tid = blockIdx.x * PEAK_THREADS + threadIdx.x;
    uint32_t x[CHAINS];
    const uint32_t y = seed * 2654435761u + tid, z = seed ^ 0x9e3779b9u;
#pragma unroll
    for (int k = 0; k < CHAINS; k++) x[k] = tid * (2u * k + 1u) + seed;
    for (uint32_t it = 0; it < iters; it++) {
#pragma unroll
        for (int u = 0; u < UNROLL; u++) {
#pragma unroll
            for (int k = 0; k < CHAINS; k++) {
                const uint32_t c = 0x01000193u * (uint32_t)(u * CHAINS + k + 1);
                if (MIX == 0) x[k] = (x[k] + y) ^ c;
                else if (MIX == 1) x[k] = x[k] * y + z;
                else x[k] = (x[k] * y + z) ^ c;
            }
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < CHAINS; k++) acc ^= x[k];
    sink[tid] = acc;
}

// cs_atomic_rate: 32-bit atomic ANDs of one bit each at pseudo-random words of
// a region, the access pattern of the walk's bit clears (one per stored hit,
// scattered over the bitset).  Word and bit come from the SplitMix64
// finaliser of (thread, step), so every word index is below n_words.
__global__ void __launch_bounds__(PEAK_THREADS) k_scatter_clear(uint32_t *buf, uint64_t n_words, uint32_t ops,
                                                                 uint64_t seed) {
    const uint64_t t = blockIdx.x * (uint64_t)PEAK_THREADS + threadIdx.x;
    for (uint32_t k = 0; k < ops; k++) {
        const uint64_t h = mix64(seed + t * kHashStep + k);
        atomicAnd(buf + (h >> 5) % n_words, ~(1u << (h & 31)));
    }
}

}  // namespace

}  // namespace cs

extern "C" cs_status cs_issue_rate(int mix, uint32_t iters, uint32_t *sink, uint64_t sink_words, void *stream,
                                   double *thread_ops, float *ms) {
    using namespace cs;
    if (!thread_ops || !ms || !sink || mix < 0 || mix > 2 || iters == 0)
        return set_error(CS_EINVAL, "cs_issue_rate: bad argument");
    void (*kern)(uint32_t, uint32_t, uint32_t *) =
        mix == 0 ? k_issue<0> : mix == 1 ? k_issue<1> : k_issue<2>;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, PEAK_THREADS, 0) != cudaSuccess || per_sm <= 0)
        return set_error(CS_EDEVICE, "cs_issue_rate: occupancy query failed");
    const uint64_t blocks = (uint64_t)sm_count() * per_sm;
    if (blocks * PEAK_THREADS > sink_words) return set_error(CS_ESIZE, "cs_issue_rate: sink smaller than the grid");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) {
        kern<<<(unsigned)blocks, PEAK_THREADS, 0, st>>>(iters / 8 + 1, 1u, sink);   // warm-up
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    if (e == cudaSuccess) {
        kern<<<(unsigned)blocks, PEAK_THREADS, 0, st>>>(iters, 2u, sink);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return set_error(CS_EDEVICE, cudaGetErrorString(e));
    const double ops_per_step = mix == 1 ? 1.0 : 2.0;
    *thread_ops = ops_per_step * CHAINS * UNROLL * (double)iters * (double)blocks * PEAK_THREADS;
    return CS_OK;
}

extern "C" cs_status cs_atomic_rate(uint32_t *region, uint64_t n_words, uint32_t ops_per_thread, void *stream,
                                    double *clears, float *ms) {
    using namespace cs;
    if (!region || !clears || !ms || n_words == 0 || ops_per_thread == 0)
        return set_error(CS_EINVAL, "cs_atomic_rate: bad argument");
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_scatter_clear, PEAK_THREADS, 0) != cudaSuccess ||
        per_sm <= 0)
        return set_error(CS_EDEVICE, "cs_atomic_rate: occupancy query failed");
    const uint64_t blocks = (uint64_t)sm_count() * per_sm;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    if (e == cudaSuccess) {
        k_scatter_clear<<<(unsigned)blocks, PEAK_THREADS, 0, st>>>(region, n_words, ops_per_thread / 8 + 1, 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(a, st);
    if (e == cudaSuccess) {
        k_scatter_clear<<<(unsigned)blocks, PEAK_THREADS, 0, st>>>(region, n_words, ops_per_thread, 2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(b, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (e != cudaSuccess) return set_error(CS_EDEVICE, cudaGetErrorString(e));
    *clears = (double)ops_per_thread * (double)blocks * PEAK_THREADS;
    return CS_OK;
}
