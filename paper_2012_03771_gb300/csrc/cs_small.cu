// Small-prime tile sieve (primes P < p <= T) fused with row initialisation,
// the wheel of d's primes and the column compression.
//
// Section 3.1 keeps the composite status of all offsets of all coprime m in
// one array and loops p outside, m inside, with N mod p = (m mod p)(K mod p).
// Here one CTA owns a tile of up to 32 rows (coprime m) and one span of raw
// offsets z = x + SL in shared memory, runs every small prime over it, and
// writes each output word of the [m][x coprime to K] bitset exactly once:
//
//   1. tile <- stored-column mask & wheel (x with q | N + x, q | d, cleared;
//      N + x = q itself is kept).
//   2. for each small prime (lanes = rows, all lanes of a warp on the same
//      prime): v = (r*m + SL) mod p = v0 + r*(m - M_start) (Montgomery), then
//      clear z = 2SL - v, 2SL - v - p, ... >= 0 (x = SL - v - k p >= -SL), i.e.
//      the x with p | N + x, counting each stored one as an enumerated factor.
//   3. gather the stored columns with warp ballots and store 128-byte runs.
#include "cs_arith.cuh"
#include "cs_internal.h"

namespace cs {

namespace {

constexpr int TILE_THREADS = 1024;
constexpr int SP_STAGE = 1024;      // small-prime records staged in shared memory at a time
constexpr int TILE_WARPS = TILE_THREADS / 32;

struct TileArgs {
    DevPlan pl;
    TileConfig tc;
    const SmallPrime *sp;
    const unsigned long long *n_sp;
    uint64_t sp_cap;
};

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v) {
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Bulk asynchronous copies global -> shared (the 1-D form of the tensor memory
// accelerator), whose completion is counted in bytes on an mbarrier.
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// the one arrival of this phase, announcing `bytes` to come, then the copy
// (16-byte aligned addresses, a multiple of 16 bytes)
__device__ __forceinline__ void bulk_to_shared(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"((unsigned long long)__cvta_generic_to_global(src)), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// waits for the phase with the given parity; false after max_tries polls
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t max_tries) {
    for (uint32_t t = 0; t < max_tries; t++) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred q;\n mbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n selp.u32 %0, 1, 0, q;\n}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
constexpr uint32_t STAGE_WAIT_TRIES = 1u << 20;
constexpr int SP_HALF = SP_STAGE / 2;   // records per staging buffer (two buffers)

__global__ void __launch_bounds__(TILE_THREADS) k_tile(const TileArgs a) {
    extern __shared__ __align__(128) uint32_t smem[];
    const DevPlan &pl = a.pl;
    const uint32_t TR = a.tc.rows;
    const unsigned lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    const uint32_t chunk = blockIdx.x % a.tc.n_chunks;
    const uint64_t row0 = (uint64_t)(blockIdx.x / a.tc.n_chunks) * TR;
    const uint32_t j0 = __ldg(&a.tc.chunk[4 * chunk + 0]);
    const uint32_t j1 = __ldg(&a.tc.chunk[4 * chunk + 1]);
    const uint32_t z0 = __ldg(&a.tc.chunk[4 * chunk + 2]);
    const uint32_t z1 = __ldg(&a.tc.chunk[4 * chunk + 3]);
    const uint32_t zb = z0 & ~31u;
    const uint32_t nw = (z1 - zb + 31) / 32;
    const uint32_t nrows = (uint32_t)min((uint64_t)TR, pl.M_c - row0);
    uint32_t *tile = smem;               // TR x nw
    uint32_t *mask = smem + TR * nw;     // nw

    for (uint32_t w = threadIdx.x; w < nw; w += TILE_THREADS) {
        uint32_t g = zb / 32 + w;
        mask[w] = g < pl.S32 ? __ldg(&pl.col_mask[g]) : 0u;
    }
    __syncthreads();

    // 1. rows start as the stored columns minus the wheel of d's primes; one
    //    pass per prime q | d with the pattern phase advanced incrementally.
    //    Rows are split into word ranges so that every warp has work when a
    //    tile has fewer rows than the CTA has warps.
    {
        const uint32_t parts = nrows ? max(1u, TILE_WARPS / nrows) : 1u;
        const uint32_t span = ((nw + parts - 1) / parts + 31) & ~31u;       // words per part
        for (uint32_t t = warp; t < nrows * parts; t += TILE_WARPS) {
            const uint32_t r = t / parts, w0 = (t % parts) * span, w1 = min(nw, w0 + span);
            const uint64_t m = pl.M_start + __ldg(&pl.moff_of_row[row0 + r]);
            for (uint32_t w = w0 + lane; w < w1; w += 32) tile[r * nw + w] = mask[w];
            for (uint32_t qi = 0; qi < pl.n_qd; qi++) {
                const uint32_t q = __ldg(&pl.qd[qi]);
                const uint32_t *pat = pl.qd_pat + __ldg(&pl.qd_pat_off[qi]);
                // phase of word w: (N - SL + zb + 32 w) mod q, N = m*K
                const uint32_t nq = (uint32_t)((m % q) * __ldg(&pl.qd_kmod[qi]) % q);
                uint32_t k = (uint32_t)(((uint64_t)nq + q - pl.SL % q + (zb + 32 * (w0 + lane)) % q) % q);
                const uint32_t step = 1024u % q;
                __syncwarp();
                for (uint32_t w = w0 + lane; w < w1; w += 32) {
                    tile[r * nw + w] &= ~__ldg(&pat[k]);
                    k += step;
                    if (k >= q) k -= q;
                }
            }
        }
    }
    __syncthreads();
    if (pl.small_n) {
        // N + x = q for a prime q | d: prime, so it stays a survivor
        for (uint32_t t = threadIdx.x; t < nrows * pl.n_qd; t += TILE_THREADS) {
            const uint32_t r = t / pl.n_qd, qi = t % pl.n_qd;
            const uint64_t m = pl.M_start + __ldg(&pl.moff_of_row[row0 + r]);
            const unsigned __int128 lowest = (unsigned __int128)m * pl.K64 - pl.SL;   // N - SL
            const uint64_t q = __ldg(&pl.qd[qi]);
            if ((unsigned __int128)q < lowest) continue;
            const unsigned __int128 z = (unsigned __int128)q - lowest;
            if (z >= z1 || z < z0) continue;
            const uint32_t zz = (uint32_t)z - zb;
            if (mask[zz >> 5] & (1u << (zz & 31))) atomicOr(&tile[r * nw + (zz >> 5)], 1u << (zz & 31));
        }
    }
    __syncthreads();

    // 2. small primes: lane -> row (lane % TR), prime (lane / TR) of this warp's
    //    group; the prime records come into two shared-memory buffers by bulk
    //    asynchronous copies, the next one loading while the current one is
    //    used, so that the inner loop reads them with shared-memory latency
    unsigned long long F = 0;
    {
        const uint32_t stage_off = ((TR + 1) * a.tc.max_words + 3) & ~3u;      // 16-byte aligned
        SmallPrime *stage = reinterpret_cast<SmallPrime *>(smem + stage_off);
        uint64_t *bars = reinterpret_cast<uint64_t *>(stage + 2 * SP_HALF);
        const uint64_t n = min((uint64_t)*a.n_sp, a.sp_cap);
        const uint32_t n_st = (uint32_t)((n + SP_HALF - 1) / SP_HALF);
        auto issue = [&](uint32_t st) {             // one thread
            const uint32_t cnt = (uint32_t)min((uint64_t)SP_HALF, n - (uint64_t)st * SP_HALF);
            bulk_to_shared(stage + (st & 1) * SP_HALF, a.sp + (uint64_t)st * SP_HALF, cnt * sizeof(SmallPrime),
                           &bars[st & 1]);
        };
        if (threadIdx.x == 0) {
            mbar_init(&bars[0]);
            mbar_init(&bars[1]);
            mbar_init_fence();
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (n_st > 0) issue(0);
            if (n_st > 1) issue(1);
        }
        const uint32_t pp = 32 / TR;
        const uint32_t r = lane % TR, sub = lane / TR;
        const bool row_ok = r < nrows;
        const uint32_t moff = row_ok ? __ldg(&pl.moff_of_row[row0 + r]) : 0u;
        unsigned __int128 lowest = 0;
        if (pl.small_n) lowest = (unsigned __int128)(pl.M_start + moff) * pl.K64 - pl.SL;
        const uint32_t two_sl = 2 * pl.SL;
        bool failed = false;                       // a wait gave up: no more copies, no more waits
        uint32_t issued = n_st < 2 ? n_st : 2;     // stages whose copies were issued
        uint32_t fail_st = n_st;                   // first stage whose wait gave up
        for (uint32_t st = 0; st < n_st; st++) {
            const uint32_t cn = (uint32_t)min((uint64_t)SP_HALF, n - (uint64_t)st * SP_HALF);
            const SmallPrime *buf = stage + (st & 1) * SP_HALF;
            const bool ok = !failed && mbar_wait(&bars[st & 1], (st >> 1) & 1, STAGE_WAIT_TRIES);
            for (uint32_t base = warp * pp; ok && base < cn; base += TILE_WARPS * pp) {
                const uint32_t i = base + sub;
                if (!row_ok || i >= cn) continue;
                const SmallPrime e = buf[i];
                uint32_t v;
                if (e.p == 2) {
                    v = (e.v0 + moff) & 1u;
                } else {
                    v = e.v0 + mont32_mul(e.rt, moff, e.p, e.pinv);
                    if (v >= e.p) v -= e.p;
                }
                if (v > two_sl) continue;
                int32_t z = (int32_t)(two_sl - v);
                if ((uint32_t)z >= z1) z -= (int32_t)(((uint32_t)z - z1) / e.p + 1) * (int32_t)e.p;
                for (; z >= (int32_t)z0; z -= (int32_t)e.p) {
                    const uint32_t zz = (uint32_t)z - zb;
                    const uint32_t bit = 1u << (zz & 31);
                    if (!(mask[zz >> 5] & bit)) continue;
                    if (pl.small_n && lowest + (unsigned)z == (unsigned __int128)e.p) continue;
                    atomicAnd(&tile[r * nw + (zz >> 5)], ~bit);
                    F++;
                }
            }
            // every thread is done with this buffer before it is loaded again
            const bool was_failed = failed;
            failed = __syncthreads_or(!ok) != 0;
            if (failed && !was_failed) fail_st = st;
            if (!failed && st + 2 < n_st) {
                if (threadIdx.x == 0) issue(st + 2);
                issued = st + 3;
            }
        }
        if (failed) {
            // let the copies still in flight (stages fail_st .. issued - 1, at
            // most two) land, with the same bound, before the CTA exits
            if (threadIdx.x == 0) {
                for (uint32_t st = fail_st; st < issued; st++) mbar_wait(&bars[st & 1], (st >> 1) & 1, STAGE_WAIT_TRIES);
                atomicOr(pl.stats + ST_ERROR, (unsigned long long)ERR_STAGE_TIMEOUT);
            }
        }
    }
    __syncthreads();

    // 3. compress the stored columns [j0, j1) of each row into the output words
    //    (compact layout: the row's class columns, one chunk covers the row)
    //    Each row's columns are split into runs of 1024 (32 output words) over
    //    several warps when the tile has fewer rows than warps.
    const bool last_chunk = chunk + 1 == a.tc.n_chunks;
    const uint32_t jend = last_chunk ? 64 * pl.wpr : j1;      // pad the row with zeros
    const uint32_t cparts = nrows ? max(1u, TILE_WARPS / nrows) : 1u;
    const uint32_t cspan = ((jend - j0 + cparts - 1) / cparts + 1023) & ~1023u;   // columns per part
    for (uint32_t t = warp; t < nrows * cparts; t += TILE_WARPS) {
        const uint32_t r = t / cparts;
        const uint32_t ja = j0 + (t % cparts) * cspan, jz = min(jend, ja + cspan);
        uint32_t *out = reinterpret_cast<uint32_t *>(pl.bits + (row0 + r) * pl.wpr);
        const uint32_t *raw = pl.raw_of_col;
        uint32_t jlim = min(pl.W, j1);
        if (pl.compact) {
            const uint32_t cls = (uint32_t)((pl.cls0 + row0 + r) % pl.n_cls);
            raw = pl.craw + (size_t)cls * pl.Wc_max;
            jlim = __ldg(&pl.cW[cls]);
        }
        uint32_t keep = 0;
        uint32_t k = (ja - j0) / 32;
        for (uint32_t jb = ja; jb < jz; jb += 32, k++) {
            const uint32_t j = jb + lane;
            uint32_t bit = 0;
            if (j < jlim) {
                const uint32_t zz = __ldg(&raw[j]) - zb;
                bit = (tile[r * nw + (zz >> 5)] >> (zz & 31)) & 1u;
            }
            const uint32_t word = __ballot_sync(0xffffffffu, bit);
            const uint32_t kk = k & 31;
            if (lane == kk) keep = word;
            if (kk == 31 || jb + 32 >= jz) {
                const uint32_t first = j0 / 32 + (k - kk);
                if (lane <= kk) out[first + lane] = keep;
            }
        }
    }

    F = warp_sum(F);
    if (lane == 0 && F) atomicAdd(pl.stats + ST_F_SMALL, F);
}

}  // namespace

cudaError_t launch_tile(const DevPlan &pl, const TileConfig &tc, const SmallPrime *sp,
                        const unsigned long long *n_sp, uint64_t sp_cap, cudaStream_t stream) {
    if (pl.M_c == 0 || pl.W == 0) return cudaSuccess;
    const uint64_t row_blocks = (pl.M_c + tc.rows - 1) / tc.rows;
    const uint64_t blocks = row_blocks * tc.n_chunks;
    const size_t smem = (size_t)(tc.rows + 1) * tc.max_words * sizeof(uint32_t) + tile_stage_bytes();
    TileArgs a{pl, tc, sp, n_sp, sp_cap};
    if (blocks > 0x7fffffffull) return cudaErrorInvalidValue;
    k_tile<<<(unsigned)blocks, TILE_THREADS, smem, stream>>>(a);
    return cudaGetLastError();
}

// two staging buffers, their two mbarriers, and up to 12 bytes of alignment
size_t tile_stage_bytes() { return SP_STAGE * sizeof(SmallPrime) + 2 * sizeof(uint64_t) + 16; }

cudaError_t prepare_tile(int max_dynamic_smem) {
    // raise the kernel's dynamic shared-memory limit once, outside any launch
    // sequence (so that cs_sieve itself enqueues launches only)
    return cudaFuncSetAttribute(k_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, max_dynamic_smem);
}

}  // namespace cs
