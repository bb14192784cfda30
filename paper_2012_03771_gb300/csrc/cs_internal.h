// Internal interfaces between the host orchestration (cs_api.cu) and the
// kernel translation units.  Not part of the public C ABI.
#pragma once
#include <vector>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/combsieve.h"
#include "cs_buckets.h"
#include "cs_errors.h"

namespace cs {

// device statistics, one uint64 each (index into Plan::d_stats)
enum Stat {
    ST_F_SMALL = 0,     // enumerated factors found by the small-prime tile sieve
    ST_F_LARGE,         // enumerated factors found by the large-prime walk
    ST_SOLVES,          // G solves (Eq. modeq) issued by the large-prime walk
    ST_LEVELS,          // passes through the solver's case analysis
    ST_HITS_ALL,        // large-prime hits before the coprime-m / stored-x filters
    ST_N_SMALL,         // small sieving primes generated
    ST_N_LARGE,         // large sieving primes generated
    ST_HASH,            // bitset checksum (sum of mix64 terms, mod 2^64)
    ST_ERROR,           // bit flags, see Err
    ST_SURVIVORS,       // total survivors (sum of per-row counts)
    ST_RECORDS,         // bucketed hit records cleared by the apply kernel
    ST_COUNT = 16
};


// layout of one small sieving prime (p <= T < 2^31), for the tile sieve
struct SmallPrime {
    uint32_t p;
    uint32_t pinv;   // -p^-1 mod 2^32 (p odd); unused for p = 2
    uint32_t rt;     // (K mod p) * 2^32 mod p: Montgomery form of r
    uint32_t v0;     // (r * M_start + SL) mod p
};

// everything a kernel needs about one sieve instance (device pointers)
struct DevPlan {
    uint64_t M_start, M_inc, M_c;
    uint32_t SL, S, S32;          // S = 2 SL + 1 raw offsets, S32 = ceil(S/32) raw words
    uint32_t W, wpr;              // stored columns, uint64 words per row
    uint64_t P, L, T;             // primorial bound, sieve limit, small/large threshold
    uint64_t d;                   // K = P# / d
    int small_n;                  // N + x may equal a sieving prime or a prime of d
    uint64_t K64;                 // K when it fits in 64 bits (small_n only)
    // K's prime factors packed into words: products below 2^31 / 2^64
    const uint32_t *kch32;
    uint32_t n_kch32;
    const uint64_t *kch64;
    uint32_t n_kch64;
    // columns
    const uint32_t *col_mask;     // S32 words: bit z set iff raw offset z = x + SL is stored
    const uint32_t *col_prefix;   // S32 words: stored columns before word
    const uint32_t *raw_of_col;   // W entries: raw offset of column j
    // rows
    const uint2 *col_tab;         // S32 pairs {col_mask, col_prefix}: one load per lookup
    const uint2 *row_tab;         // ceil(M_inc/32) pairs {row_mask, row_prefix}
    const uint32_t *moff_of_row;  // M_c entries: m - M_start
    const uint32_t *row_mask;     // ceil(M_inc/32) words: bit k set iff m = M_start + k is a row
    const uint32_t *row_prefix;   // ceil(M_inc/32) words: rows before word
    // wheel (primes of d)
    const uint32_t *qd;           // n_qd primes
    uint32_t n_qd;
    const uint32_t *qd_kmod;      // K mod q
    const uint32_t *qd_pat_off;   // offset of q's pattern table in qd_pat
    const uint32_t *qd_pat;       // pattern[k]: bits i < 32 with (k + i) % q == 0
    // compact layout: per residue class of m mod d (ascending), the stored
    // columns are the literal ones the wheel does not clear
    int compact;
    uint32_t n_cls, cls0;         // classes, class of row 0 (row i has class (cls0 + i) % n_cls)
    const uint32_t *cmask;        // n_cls x S32: stored raw offsets of the class
    const uint32_t *cprefix;      // n_cls x S32: stored columns before each word
    const uint32_t *craw;         // n_cls x Wc_max: raw offset of each column of the class
    const uint32_t *cW;           // n_cls: columns of the class
    const uint32_t *cls_word;     // ceil(M_inc/32): class of the first row at or after m = M_start + 32 w
    uint32_t Wc_max;
    // bucketed hits (bitsets larger than L2): a stored hit of the walk is written
    // as a record to the walking CTA's region for its band of rows, and
    // k_apply_buckets clears the records band after band; regions are band-major
    int bucket;                   // 1: the three-gap walk buckets its stored hits
    uint32_t band_log;            // rows per band = 2^band_log
    uint32_t n_bands;             // at most BKT_MAX_BANDS (a walking CTA counts its regions in shared memory)
    uint32_t n_regions;           // regions per band (walk CTAs; the walk grid is at most this)
    uint32_t region_cap;          // records per region; hits beyond it are cleared directly
    uint32_t *bkt;                // n_bands x n_regions x region_cap records: (row in band) * 64 wpr + column
    uint32_t *bkt_cnt;            // n_bands x n_regions: records in each region, then the apply's region counter
    // outputs
    uint64_t *bits;               // M_c * wpr words
    uint32_t *counts;             // M_c
    unsigned long long *stats;    // ST_COUNT
};

// ---- kernel launchers (each enqueues on `stream`; no synchronisation) ----

// Primes p with lo < p <= hi, written as small-prime entries.
cudaError_t launch_gen_small(const DevPlan &pl, uint64_t lo, uint64_t hi, const uint32_t *base,
                             uint32_t n_base, SmallPrime *out, uint64_t cap,
                             unsigned long long *count, cudaStream_t stream);
// Primes p with lo < p <= hi as (p, r, v0) large-prime entries; narrow: 32-bit fields.
cudaError_t launch_gen_large(const DevPlan &pl, bool narrow, uint64_t lo, uint64_t hi,
                             const uint32_t *base, uint32_t n_base, void *p_out, void *r_out,
                             void *v_out, uint64_t cap, unsigned long long *count,
                             cudaStream_t stream);
// Primes p in (lo, hi] with r = K mod p for the K of kp (kch32/kch64 only),
// for a residue cache; narrow: 32-bit fields (hi < 2^30).
cudaError_t launch_gen_pr(const DevPlan &kp, bool narrow, uint64_t lo, uint64_t hi, const uint32_t *base,
                          uint32_t n_base, void *p_out, void *r_out, uint64_t cap,
                          unsigned long long *count, unsigned long long *err, cudaStream_t stream);
// Plain prime list (uint64) in (lo, hi], no residues (for tests of the generator).
cudaError_t launch_gen_list(uint64_t lo, uint64_t hi, const uint32_t *base, uint32_t n_base,
                            uint64_t *out, uint64_t cap, unsigned long long *count,
                            unsigned long long *err, cudaStream_t stream);
// K mod p for an array of odd primes p > P (tests of the residue kernel).
cudaError_t launch_kmodp(const DevPlan &pl, const uint64_t *p, uint64_t n, uint64_t *r,
                         cudaStream_t stream);

struct TileConfig {
    uint32_t rows;           // rows per tile (1, 2, 4, 8, 16 or 32)
    uint32_t n_chunks;       // column chunks
    const uint32_t *chunk;   // device: per chunk {j0, j1, z0, z1}
    uint32_t max_words;      // raw words of the widest chunk
};
cudaError_t launch_tile(const DevPlan &pl, const TileConfig &tc, const SmallPrime *sp,
                        const unsigned long long *n_sp, uint64_t sp_cap, cudaStream_t stream);
// sets k_tile's dynamic shared-memory limit (called when a plan is built)
cudaError_t prepare_tile(int max_dynamic_smem);
// shared memory the tile kernel uses besides the tile itself
size_t tile_stage_bytes();

enum LargeMode { LARGE_PAPER = 1, LARGE_THREE_GAP = 2 };
// m-classes of the three-gap walk: only m = c (mod Q) for the n classes c with
// gcd(c, Q) = 1 are walked (Q | d, so the others are never rows).  off[k] is
// class k's residue of m - M_start mod Q.  Q = 1, n = 1: every m.
// items = 0: one work item walks all n <= 2 classes (off[0..n)).  items = n
// (class items, Q up to 210, n up to 48): every class is a work item of its
// own, item_off[k] its residue; the prime's walk is then split by class as
// well as by m-segment.
constexpr uint32_t MAX_CLASS_ITEMS = 48;
struct MClasses {
    uint32_t Q, n;
    uint32_t off[2];
    uint32_t items;
    uint8_t item_off[MAX_CLASS_ITEMS];
};
constexpr MClasses EVERY_M = MClasses{1, 1, {0, 0}, 0, {}};
// n_seg: the m-range of every prime is split into n_seg segments walked by
// separate threads (each starts with its own solve), to balance primes with
// many hits against primes with few.
// v may be NULL: then v0 = (r M_start + SL) mod p is computed per prime, and
// only primes with p_lo < p <= p_hi are walked (a residue-cache chunk holds
// primes outside the plan's range).
// desc0/desc1: walkers prepared by launch_tg_prep for this chunk (used when
// prep_eligible; NULL: the walk prepares its items itself).
cudaError_t launch_large(const DevPlan &pl, bool narrow, int mode, const void *p, const void *r,
                         const void *v, const unsigned long long *count, uint64_t cap,
                         uint32_t n_seg, int grid, cudaStream_t stream, uint64_t p_lo = 0,
                         uint64_t p_hi = ~0ull, MClasses mc = EVERY_M, const uint4 *desc0 = nullptr,
                         const uint2 *desc1 = nullptr);
// Walker preparation for one-walker chunks of the three-gap walk (odd m or
// every m, one segment per prime, SL > 0): per prime of the chunk, the first
// hit and the two steps, into desc0/desc1 (cap entries each).
bool prep_eligible(const DevPlan &pl, int mode, uint32_t n_seg, MClasses mc);
cudaError_t launch_tg_prep(const DevPlan &pl, bool narrow, const void *p, const void *r, const void *v,
                           const unsigned long long *count, uint64_t cap, uint64_t p_lo, uint64_t p_hi,
                           MClasses mc, uint4 *desc0, uint2 *desc1, cudaStream_t stream);
cudaError_t launch_final(const DevPlan &pl, cudaStream_t stream);
// Clears the bucketed hits of the walk launches since the last application,
// band after band, and empties the regions.
cudaError_t launch_apply_buckets(const DevPlan &pl, cudaStream_t stream);

// One chunk's three-gap walk as a job of a persistent multi-job launch (the
// arguments launch_large takes, primes from a residue-cache chunk).
struct WalkJob {
    DevPlan pl;
    bool narrow;
    const void *p, *r;
    const unsigned long long *count;
    uint64_t cap;
    uint32_t n_seg;
    uint64_t p_lo, p_hi;
    MClasses mc;
};
// The jobs grouped by walk kernel, in device memory; walk_jobs_launch enqueues
// one persistent launch per kernel that has jobs (each job's walk in its
// order within the group).
struct WalkJobs;
cudaError_t walk_jobs_create(const std::vector<WalkJob> &jobs, WalkJobs **out);
cudaError_t walk_jobs_launch(const WalkJobs *wj, cudaStream_t stream);
uint64_t walk_jobs_launches(const WalkJobs *wj);
void walk_jobs_destroy(WalkJobs *wj);

// K's prime factors qK packed into factor words below 2^31 (the generator's
// lazily reduced Montgomery product) and below 2^64, first fit with the
// largest factors first: K = product of either list.
void k_factor_words(const std::vector<uint32_t> &qK, std::vector<uint32_t> &w32, std::vector<uint64_t> &w64);

// batch of G solves (tests of the solver)
cudaError_t launch_modsolve(const uint64_t *p, const uint64_t *K, const uint64_t *L,
                            const uint64_t *R, uint64_t *m, uint64_t n, int narrow,
                            cudaStream_t stream);

int sm_count();
uint64_t l2_bytes();   // L2 size of the current device

// ---- residue cache (cs_cache.cu) ----
// Primes and K mod p for one K = P#/d, on a fixed grid of chunks of (0, L_max]:
// (0, 2^16], then chunks that double in width up to 2^27, then 2^27 wide.
struct CacheChunk {
    uint64_t lo, hi;                   // primes lo < p <= hi
    bool narrow;                       // hi < 2^30: 32-bit p and r
    void *p = nullptr, *r = nullptr;   // cap entries each
    unsigned long long *count = nullptr;
    uint64_t cap = 0;
    cudaEvent_t ready = nullptr;       // recorded after the chunk's generation
    bool filled = false;               // a generation has been enqueued since the last capture
};
struct ResidueCacheView {
    uint32_t P;
    uint64_t d, L_max;
    CacheChunk *chunks;
    size_t n_chunks;
    unsigned long long *err;           // device error flags of the cache's generation
};
bool cache_view(cs_cache_t cache, ResidueCacheView *out);
// Enqueues the generation of every chunk with lo < L (all if L = 0) on stream
// (only the chunks never filled, if only_missing); inside a stream capture the
// chunks are marked not filled for later plain use.
cs_status cache_fill_upto(cs_cache_t cache, uint64_t L, cudaStream_t stream, bool only_missing);
std::mutex &cache_mutex(cs_cache_t cache);
// Extends the grid (and allocates) so that it covers L.
cs_status cache_extend(cs_cache_t cache, uint64_t L);
cs_status cache_new(uint32_t P, uint64_t d, uint64_t L_max, cs_cache_t *out);

// ---- plan internals used by the batch and server runtime (cs_runtime.cu) ----
// Builds a plan; with async_alloc its device memory is stream-ordered on
// alloc_stream (cudaMallocAsync / cudaFreeAsync).
// A cached three-gap plan's sieve in three phases, for batches that run the
// walks of all their plans in persistent multi-job launches: the head
// (statistics reset, small primes, tile sieve), the walk jobs (one per large
// prime chunk; false if the plan does not qualify), the tail (counts and
// checksum, completion event).
cs_status plan_sieve_head(cs_plan_t pl, cudaStream_t stream);
bool plan_walk_jobs(cs_plan_t pl, std::vector<WalkJob> &out);
cs_status plan_sieve_tail(cs_plan_t pl, cudaStream_t stream);
cs_status plan_create(uint32_t P, uint64_t d, uint64_t M_start, uint64_t M_inc, uint32_t SL,
                      uint64_t L, const cs_tuning *tune, cudaStream_t alloc_stream, bool async_alloc,
                      cs_cache_t cache, cs_plan_t *out);
cs_cache_t plan_cache(cs_plan_t pl);
void plan_set_sieved(cs_plan_t pl, bool sieved);
bool plan_profiled(cs_plan_t pl);
cudaEvent_t plan_done_event(cs_plan_t pl);
cs_status set_error(cs_status code, const char *msg);
// parameter checks of cs_plan, without device work
cs_status validate_params(uint32_t P, uint64_t d, uint64_t M_start, uint64_t M_inc, uint32_t SL, uint64_t L);

}  // namespace cs
