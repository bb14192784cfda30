// Per-row survivor counts and the bitset checksum.
//
// One warp per row: popcount of the row's words and the position-dependent
// checksum  sum_{i,w} mix64(word[i][w] + (i*wpr + w) * 0x9E3779B97F4A7C15)
// mod 2^64 (mix64 = SplitMix64 finaliser).  A sum is order-independent, so the
// reduction needs no fixed order to be deterministic.
#include "cs_arith.cuh"
#include "cs_internal.h"

namespace cs {

namespace {

constexpr int FIN_THREADS = 256;

__global__ void __launch_bounds__(FIN_THREADS) k_final(const DevPlan pl) {
    const unsigned lane = threadIdx.x & 31;
    const uint64_t warp_global = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long h = 0, surv = 0;
    for (uint64_t row = warp_global; row < pl.M_c; row += n_warps) {
        const uint64_t *w = pl.bits + row * pl.wpr;
        uint32_t cnt = 0;
        for (uint32_t k = lane; k < pl.wpr; k += 32) {
            const uint64_t word = w[k];
            cnt += __popcll(word);
            h += mix64(word + (row * pl.wpr + k) * kHashStep);
        }
        for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0) pl.counts[row] = cnt;
        surv += cnt;
    }
    for (int o = 16; o; o >>= 1) h += __shfl_xor_sync(0xffffffffu, h, o);
    __shared__ unsigned long long sh[FIN_THREADS / 32], ss[FIN_THREADS / 32];
    if (lane == 0) {
        sh[threadIdx.x >> 5] = h;
        ss[threadIdx.x >> 5] = surv;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long th = 0, ts = 0;
        for (int i = 0; i < FIN_THREADS / 32; i++) {
            th += sh[i];
            ts += ss[i];
        }
        if (th) atomicAdd(pl.stats + ST_HASH, th);
        if (ts) atomicAdd(pl.stats + ST_SURVIVORS, ts);
    }
}

}  // namespace

cudaError_t launch_final(const DevPlan &pl, cudaStream_t stream) {
    if (pl.M_c == 0) return cudaSuccess;
    uint64_t blocks = (pl.M_c + FIN_THREADS / 32 - 1) / (FIN_THREADS / 32);
    uint64_t cap = (uint64_t)sm_count() * 16;
    if (blocks > cap) blocks = cap;
    k_final<<<(unsigned)blocks, FIN_THREADS, 0, stream>>>(pl);
    return cudaGetLastError();
}

}  // namespace cs
