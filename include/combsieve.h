/*
 * combsieve.h -- C ABI of the GB300 Combined Sieve.
 *
 * The Combined Sieve (S. Troisi, "Combined Sieve Algorithm for Prime Gaps",
 * arXiv:2012.03771) sieves many intervals [N - SL, N + SL], N = m*K, at once,
 * for K = P#/d and every multiplier m in a range that is coprime to d.  This
 * library runs the whole sieve on one GPU (sm_103a) and keeps the result, a
 * composite bitset laid out as [m][x coprime to K], in device memory.
 *
 * Output definition (the sieve's contract; a CPU oracle implements the same):
 *   K      = P#/d, the product of the primes q <= P that do not divide d
 *            (Section 2, "Primorials").
 *   rows   = m in [M_start, M_start + M_inc) with gcd(m, d) = 1, ascending
 *            (Section 3: m sharing a factor with d are skipped).  M_c rows.
 *   cols   = x in [-SL, SL] with gcd(|x|, K) = 1, ascending; x = 0 is a column
 *            only when K = 1.  W columns.
 *   layout = words_per_row = ceil(W/64) uint64 words per row, row-major;
 *            column j is bit (j & 63) of word (j >> 6); padding bits are 0.
 *   bit    = 1 (survivor) iff no sieving prime p, P < p <= L, divides N + x
 *            with N + x != p, and (wheel on, the default) no prime q | d
 *            divides N + x with N + x != q.
 *   F      = enumerated factors: the number of (p, row, col) with p | N + x,
 *            N + x != p (the wheel is not counted).
 *   hash   = sum over rows i, words w of mix64(word + (i*wpr + w)*0x9E3779B97F4A7C15)
 *            mod 2^64; mix64 is the SplitMix64 finaliser.
 *
 * Parameter limits (violations return CS_EINVAL): 1 <= d, d squarefree with
 * every prime factor <= P; P <= 2^20; SL <= 2^20; L <= 2^40; 1 <= M_start;
 * M_start + M_inc <= 2^40; M_inc < 2^31; M_start*K - SL >= 2 (every N + x >= 2).
 *
 * Errors: every call returns a cs_status (0 = CS_OK, negative = error) and
 * never throws; cs_last_error() gives a message for the calling thread.  A
 * device error inside cs_sieve is sticky for that plan.
 *
 * Threads: a plan may be used by one thread at a time; distinct plans are
 * independent.  All device work of a plan is enqueued on the stream given to
 * cs_sieve; the caller may overlap several plans on several streams.
 */
#ifndef COMBSIEVE_H
#define COMBSIEVE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cs_plan_s *cs_plan_t;
typedef struct cs_batch_s *cs_batch_t;
typedef struct cs_server_s *cs_server_t;
typedef struct cs_cache_s *cs_cache_t;
typedef int cs_status;

#define CS_OK 0
#define CS_EINVAL (-1)     /* parameter outside the limits above, or a bad argument */
#define CS_ENOMEM (-2)     /* host or device allocation failed */
#define CS_EDEVICE (-3)    /* a CUDA call failed; see cs_last_error() */
#define CS_ETIMEOUT (-4)   /* a bounded device wait gave up */
#define CS_ESTATE (-5)     /* call out of order, e.g. fetching before cs_sieve */
#define CS_ESIZE (-6)      /* caller buffer too small */
#define CS_EOVERFLOW (-7)  /* an internal device buffer overflowed (result invalid) */
#define CS_EAGAIN (-8)     /* admission refused (no free slot or memory) */

/* Tuning knobs.  A zeroed struct (or NULL) selects the defaults.  None of
 * them changes the output; they only move work between kernels. */
typedef struct {
    uint64_t threshold;      /* T: primes P < p <= T take the small-prime tile
                                sieve, T < p <= L the large-prime walk (Section
                                3.2's threshold, "naively p > 10 S").  Must be
                                >= 2*SL and <= 2^30 when given.  0 = automatic. */
    uint32_t tile_rows;      /* rows per small-prime tile: 1, 2, 4, 8, 16 or 32; 0 = auto */
    uint32_t large_mode;     /* 1 = one G solve per hit, as in Section 3.2;
                                2 = three-gap stepping (two extra solves per prime,
                                then O(1) per hit); 0 = automatic (2) */
    uint32_t no_wheel;       /* 1 = do not clear x with q | N + x for primes q | d */
    uint32_t large_grid;     /* CTAs of the large-prime kernel; 0 = automatic */
    uint64_t chunk_numbers;  /* width of one large-prime chunk of (T, L]; 0 = automatic */
    uint32_t profile;        /* 1 = time each kernel with CUDA events (cs_kernel_times) */
    uint32_t layout;         /* 0 = columns x coprime to K (the same for every row);
                                1 = compact: row m keeps only the x with gcd(m K + x, d) = 1
                                (the x the wheel would clear are not stored), so its columns
                                depend on m mod d (cs_row_columns).  Needs the wheel, no
                                N + x small enough to be a prime of d, phi(d) <= 4096 and an
                                interval whose tile fits in one piece (SL up to about 3.7e5).
                                F and the per-row counts are the same in both layouts. */
    uint32_t m_classes;      /* three-gap walk over m (the m sharing a factor with d are never
                                rows): 0 = automatic (chunks whose primes have at least
                                class_item_hits expected hits per class of m mod 210, else mod 30,
                                walk the m coprime to that modulus, one work item per class,
                                when it divides d; chunks whose primes have at least 48
                                expected hits walk only the m = 1, 5 (mod 6) when 6 | d, the
                                other chunks the odd m when 2 | d); 1 = every m; 2 = the
                                classes mod 6 (else mod 2) in every chunk; 3 = class items
                                mod 210 (else 30, 6, 2: the largest that divides d) in every
                                chunk */
    uint32_t item_hits;      /* three-gap walk: expected walked hits per work item (prime,
                                m-segment); 0 = automatic (128) */
    uint32_t class_min_hits; /* m_classes = 0: expected hits per prime (every m) from which a
                                chunk walks only the m-classes; 0 = automatic (48) */
    uint32_t class_item_hits;/* m_classes = 0: expected hits of one class of m mod Q (Q = 210
                                or 30) per prime from which a chunk walks class items mod Q;
                                0 = automatic (64) */
    uint32_t hit_buckets;    /* three-gap walk's stored hits: 1 = cleared directly, one atomic AND
                                each; 2 = written as records to the walk CTA's region for their
                                band of rows (a slot taken with a shared-memory atomic, one plain
                                store) and cleared band after band by an apply kernel, each band's
                                words staying in L2 meanwhile (a region that is full clears
                                directly); 0 = automatic (2 when the bitset is at least 256 MiB) */
    uint32_t band_rows_log;  /* hit buckets: rows per band = 2^band_rows_log (at most 2^20);
                                0 = automatic (bands of at most a fifth of L2, at most 4096
                                bands) */
    uint64_t bucket_records; /* hit buckets: records per (CTA, band) region, rounded up to a
                                multiple of 4; 0 = automatic (up to 8 GiB of regions, twice the
                                bitset at most) */
    uint32_t walk_prep;      /* one-walker chunks of the three-gap walk (odd m or every m, one
                                segment per prime, in a plan without a residue cache): 2 = each
                                prime's first hit and steps computed by a preparation kernel
                                into a 24-byte walker descriptor that the walk reads; 1 = the
                                walk prepares its items itself; 0 = automatic (2) */
} cs_tuning;

typedef struct {
    uint64_t M_c;              /* rows */
    uint64_t W;                /* columns (layout 1: the widest row's) */
    uint64_t words_per_row;    /* ceil(W / 64) */
    uint64_t bitset_bytes;     /* M_c * words_per_row * 8 */
    uint64_t S;                /* 2*SL + 1 */
    uint64_t threshold;        /* effective T */
    uint32_t tile_rows;
    uint32_t large_mode;
    uint32_t narrow;           /* 1: all large primes < 2^30 (32-bit kernels); with 0 the
                                  chunks below 2^30 still take the 32-bit kernels */
    uint32_t wheel;
    uint64_t n_large_chunks;
    uint64_t launches_per_sieve;  /* kernels one cs_sieve launches */
    uint64_t h2d_bytes;        /* bytes uploaded by cs_plan */
    uint64_t device_bytes;     /* device memory held by the plan */
    uint64_t est_cost;         /* relative device cost estimate (about picoseconds on a
                                  GB300), used to order instances in a batch */
    uint32_t layout;           /* 0 literal, 1 compact */
    uint32_t n_classes;        /* compact: residue classes of m mod d (phi(d)), else 1 */
    uint32_t m_mod;            /* Q of the m-classes of the chunks with many hits per prime
                                  (1: every m is walked) */
    uint32_t m_walked;         /* classes of m mod Q those chunks walk (1 or 2) */
    uint64_t split_chunks;     /* large-prime chunks that walk those classes (the others walk
                                  the odd m when 2 | d) */
    uint32_t item_mod;         /* finest Q of the chunks that walk class items (0: none) */
    uint32_t item_classes;     /* classes of m mod item_mod they walk (phi(item_mod)) */
    uint64_t item_chunks;      /* large-prime chunks that walk class items */
    uint32_t hit_buckets;      /* 1 = the walk's stored hits go through per-band regions */
    uint32_t n_bands;          /* bands of rows (hit buckets) */
    uint64_t bucket_bytes;     /* device memory of the regions and their counts */
    uint64_t apply_launches;   /* bucket applications per sieve (one per group of chunks) */
    uint64_t prep_chunks;      /* large-prime chunks whose walkers a preparation kernel computes */
} cs_info_t;

typedef struct {
    uint64_t F;                /* enumerated factors (F_small + F_large) */
    uint64_t F_small;
    uint64_t F_large;
    uint64_t solves;           /* G solves of Eq. modeq in the large-prime walk */
    uint64_t levels;           /* passes through G's case analysis */
    uint64_t hits_all;         /* large-prime hits the walk visits, before the coprime-m and
                                  stored-x tests (m outside the walked classes are not visited) */
    uint64_t n_small_primes;
    uint64_t n_large_primes;
    uint64_t survivors;        /* set bits in the bitset */
    uint64_t hash;
    uint64_t bucket_records;   /* hit buckets: stored hits cleared through records (the rest of
                                  F_large, if any, found their region full and cleared directly) */
} cs_stats_t;

/* Builds a sieve instance: validates the parameters, computes the row and
 * column maps and K's factor words on the host, allocates the device bitset and
 * work buffers (owned by the plan) and uploads the tables.  tune may be NULL.
 * On success *out is a new plan; on error *out is NULL.  The device memory
 * comes from a stream-ordered memory pool the library keeps per device (plans
 * built by a request server use the server's). */
cs_status cs_plan(uint32_t P, uint64_t d, uint64_t M_start, uint64_t M_inc, uint32_t SL,
                  uint64_t L, const cs_tuning *tune, cs_plan_t *out);

/* Enqueues the whole sieve on `stream` (a cudaStream_t; NULL = the legacy
 * default stream) and returns without waiting: prime generation (P, L], K mod p
 * (Section 3.1), the small-prime tile sieve, the large-prime walk (Sections
 * 3.2-3.3), per-row counts and the checksum.  May be called again to recompute. */
cs_status cs_sieve(cs_plan_t plan, void *stream);

/* Waits for the last cs_sieve of this plan and returns its device status:
 * CS_OK, CS_EOVERFLOW (an internal buffer overflowed), CS_EDEVICE. */
cs_status cs_sync(cs_plan_t plan);

cs_status cs_info(cs_plan_t plan, cs_info_t *out);

/* Copies the bitset (M_c * words_per_row uint64 words, row-major) to host
 * memory owned by the caller.  n_words must be at least that.  Waits for the
 * plan's last cs_sieve. */
cs_status cs_fetch_bitset(cs_plan_t plan, uint64_t *host, size_t n_words);

/* Rows [row0, row0 + n_rows) of the bitset (n_rows * words_per_row words) to
 * caller-owned host memory, for consumers that need only part of a large
 * bitset.  CS_EINVAL if the range exceeds M_c.  Waits. */
cs_status cs_fetch_rows(cs_plan_t plan, uint64_t row0, uint64_t n_rows, uint64_t *host, size_t n_words);

/* Per-row survivor counts (n_rows >= M_c uint32, may be NULL), F and hash
 * (either may be NULL), copied to caller-owned host memory.  Waits. */
cs_status cs_counts(cs_plan_t plan, uint32_t *per_row, size_t n_rows, uint64_t *F, uint64_t *hash);

/* Device counters of the last cs_sieve.  Waits. */
cs_status cs_stats(cs_plan_t plan, cs_stats_t *out);

/* The plan's row map (m of each row) and column map (x of each column). */
cs_status cs_rows(cs_plan_t plan, uint64_t *m_of_row, size_t n);
cs_status cs_columns(cs_plan_t plan, int64_t *x_of_col, size_t n);

/* Columns of one row: the x values of its bits in order (layout 0: the same
 * for every row, as cs_columns; layout 1: the row's own set).  *n_cols gets
 * the count (at most W); n is the capacity of x_of_col. */
cs_status cs_row_columns(cs_plan_t plan, uint64_t row, int64_t *x_of_col, size_t n, uint64_t *n_cols);

/* Borrowed device pointer to the bitset; valid until cs_destroy. */
const void *cs_device_bitset(cs_plan_t plan);

/* Kernel timings of the last cs_sieve (profile = 1 only), in milliseconds,
 * per kernel class: [0] small-prime generation, [1] tile sieve, [2] large-prime
 * generation, [3] large-prime walk, [4] counts/checksum, [5] application of the
 * walk's bucketed hits, [6] walker preparation of the one-walker chunks;
 * launches[i] = launches of that class.  Waits. */
cs_status cs_kernel_times(cs_plan_t plan, double ms[7], uint64_t launches[7]);

/* Frees the plan and its device memory (waits for its work first).  The memory
 * goes back to the library's pool, which keeps up to 1 GiB of it for later
 * plans on the device (returned to the device beyond that) until the process
 * exits. */
cs_status cs_destroy(cs_plan_t plan);

/* Message for the last error on the calling thread ("" if none). */
const char *cs_last_error(void);

/* ---- autotuning -------------------------------------------------------------
 * Picks the threshold T (as a multiple of S) and the tile height for a
 * parameter set by timing candidates on the device, on a proxy instance with
 * the same P, d and SL, M_inc clipped to 1e5 and L to 1e9, then the walk's
 * work-item size (item_hits: 32, 64, 128, 256 or 512 expected walked hits per
 * item, which sets how many primes and m-segments the CTAs take at a time)
 * for that threshold and tile height.  The choice is kept
 * per (P, d, SL, ceil(log2 L)) in memory and, if cache_path is not NULL,
 * appended to that text file and read back by later calls (one line per key).
 * *out receives a complete tuning (large_mode = 2).  Validation errors as for
 * cs_plan.  Tuning fields left at 0 in any plan may also be set from the
 * environment: CS_THRESHOLD, CS_TILE_ROWS, CS_LARGE_MODE, CS_LARGE_GRID, CS_M_CLASSES,
 * CS_ITEM_HITS, CS_CLASS_MIN_HITS, CS_CLASS_ITEM_HITS, CS_CHUNK_NUMBERS, CS_HIT_BUCKETS,
 * CS_BAND_ROWS_LOG, CS_BUCKET_RECORDS. */
cs_status cs_autotune(uint32_t P, uint64_t d, uint64_t M_start, uint64_t M_inc, uint32_t SL, uint64_t L,
                      const char *cache_path, cs_tuning *out);

/* ---- residue cache ---------------------------------------------------------
 * Device-resident primes p <= L_max with r = K mod p for one K = P#/d
 * (Section 3.1's cached residue, kept for many searches with the same K).
 * Memory: about 8 bytes per prime below 2^30 and 16 above, plus slack (for
 * L_max = 1e10 about 8 GB).  cs_cache_fill enqueues the generation of all
 * primes on `stream` (a few milliseconds per 1e9 of range).  Plans built with
 * cs_plan_cached read their large primes from the cache instead of generating
 * them: the cache must be filled before their cs_sieve is enqueued (cs_sieve
 * orders itself after the fill with events) and must outlive them.  A batch
 * whose plans use caches fills those caches itself at every cs_batch_run. */
cs_status cs_cache_create(uint32_t P, uint64_t d, uint64_t L_max, cs_cache_t *out);
cs_status cs_cache_fill(cs_cache_t cache, void *stream);
cs_status cs_cache_info(cs_cache_t cache, uint64_t *n_chunks, uint64_t *device_bytes, uint64_t *n_primes);
cs_status cs_cache_destroy(cs_cache_t cache);
/* cs_plan with its large primes taken from `cache` (same P and d, L <= L_max);
 * the output is identical to cs_plan's. */
cs_status cs_plan_cached(uint32_t P, uint64_t d, uint64_t M_start, uint64_t M_inc, uint32_t SL,
                         uint64_t L, const cs_tuning *tune, cs_cache_t cache, cs_plan_t *out);

/* ---- batched execution ---------------------------------------------------
 * Many independent searches of uneven size (Section 5, "Real world searching")
 * share the GPU.  cs_batch_create spreads the plans over n_streams worker
 * streams (0 = 1 when the plans use residue caches, else min(n, 2): each
 * instance fills the GPU, so more concurrent instances mostly cost L2
 * locality), longest estimated cost first onto the least loaded
 * stream, and captures their whole launch sequence once into a CUDA graph;
 * cs_batch_run replays it with one graph launch on `stream`.  The plans stay
 * owned by the caller and must outlive the batch; their results are read with
 * cs_counts / cs_fetch_bitset after cs_batch_sync.  Plans built with
 * profile = 1 are rejected (CS_EINVAL), and so is a plan listed twice. */
cs_status cs_batch_create(const cs_plan_t *plans, int n, int n_streams, cs_batch_t *out);
cs_status cs_batch_run(cs_batch_t batch, void *stream);
cs_status cs_batch_sync(cs_batch_t batch);            /* waits; first plan error, if any */
cs_status cs_batch_info(cs_batch_t batch, uint64_t *n_streams, uint64_t *launches);
cs_status cs_batch_destroy(cs_batch_t batch);

/* ---- served execution (continuous batching) ------------------------------
 * A request server with max_slots streams and a device-memory budget.
 * cs_submit builds the request's plan (stream-ordered allocation on a free
 * slot's stream, so it does not wait for running requests) and starts its
 * sieve; it returns CS_EAGAIN when no slot is free or the plan's device memory
 * would exceed the budget, in which case nothing was kept.  A request's work
 * overlaps on the device with the requests already running.  cs_poll reports
 * completion (and frees the slot); the bitset stays resident, readable through
 * the borrowed plan of cs_server_plan, until cs_release. */
cs_status cs_server_start(uint64_t budget_bytes, int max_slots, const cs_tuning *tune, cs_server_t *out);
cs_status cs_submit(cs_server_t server, uint32_t P, uint64_t d, uint64_t M_start, uint64_t M_inc,
                    uint32_t SL, uint64_t L, uint64_t *ticket);
cs_status cs_poll(cs_server_t server, uint64_t ticket, int *done);
cs_status cs_server_plan(cs_server_t server, uint64_t ticket, cs_plan_t *plan);
cs_status cs_release(cs_server_t server, uint64_t ticket);
cs_status cs_server_usage(cs_server_t server, uint64_t *used_bytes, uint64_t *busy_slots, uint64_t *resident);
cs_status cs_server_stop(cs_server_t server);   /* releases every ticket */

/* ---- single steps of the path, on caller-owned DEVICE buffers ---------- */

/* Primes p with lo < p <= hi (hi <= 2^40), unordered, into out[0 .. cap).
 * *count (host) receives the number found; CS_EOVERFLOW if more than cap.
 * Synchronises `stream`. */
cs_status cs_primes(uint64_t lo, uint64_t hi, uint64_t *out, uint64_t cap, uint64_t *count,
                    void *stream);

/* r[i] = K mod p[i] for K = P#/d (Section 3.1), for odd p[i] > P, p[i] < 2^40.
 * Montgomery arithmetic with R = 2^32 when p < 2^31, else R = 2^64.
 * Synchronises `stream`. */
cs_status cs_k_mod_p(uint32_t P, uint64_t d, const uint64_t *p, uint64_t n, uint64_t *r,
                     void *stream);

/* m[i] = G(p[i], K[i], L[i], R[i]) of Section 3.3 (Eq. modfunc): the smallest
 * m >= 0 with L <= m*K mod p <= R.  Requires 0 <= L <= R < p < 2^40,
 * gcd(K, p) = 1; narrow = 1 uses 32-bit arithmetic and needs p < 2^30.
 * Entries with K = 0 mod p get m = 2^64 - 1.  Synchronises `stream`. */
cs_status cs_modsolve(const uint64_t *p, const uint64_t *K, const uint64_t *L, const uint64_t *R,
                      uint64_t *m, uint64_t n, int narrow, void *stream);

/* ---- measurement -------------------------------------------------------- */

/* Integer issue-rate micro-benchmark: the measured peak for the roofline of
 * the integer-bound kernels.  The paper has no counterpart (its cost model
 * counts CPU cycles).  One launch of every resident thread (one wave, full
 * occupancy), each running 8 independent chains of `iters` x 32 steps:
 *   mix 0: x = (x + y) ^ c          two operations per step (add, logic)
 *   mix 1: x = x * y + z            one integer multiply-add per step
 *   mix 2: x = (x * y + z) ^ c      one multiply-add and one logic op per step
 * after one untimed warm-up launch.  *thread_ops (host) receives the thread-level
 * operations the source states; *ms (host) the launch's duration from CUDA
 * events on `stream`.  sink: device, one uint32 per launched thread (at most
 * 152 x 2048 on a GB300; CS_ESIZE if smaller).  Synchronises `stream`. */
cs_status cs_issue_rate(int mix, uint32_t iters, uint32_t *sink, uint64_t sink_words, void *stream,
                        double *thread_ops, float *ms);

/* Scattered bit clears: every resident thread (one wave) performs
 * ops_per_thread 32-bit atomic ANDs, each clearing one pseudo-random bit of a
 * pseudo-random word of region[0 .. n_words) (device memory owned by the
 * caller, whose contents it changes), after one untimed shorter launch.  The
 * access pattern of the large-prime walk's bit clears, measured over a region
 * of the bitset's size.  *clears (host): atomics of the timed launch; *ms: its
 * duration from CUDA events on `stream`.  Synchronises `stream`. */
cs_status cs_atomic_rate(uint32_t *region, uint64_t n_words, uint32_t ops_per_thread, void *stream,
                         double *clears, float *ms);

/* ---- allocation-free variant -------------------------------------------- */

/* The same prime list as cs_primes, for callers that must not allocate device
 * memory: a process whose device memory is handed out by its own pool sized at
 * start-up (an allocation outside the pool can fail or break its accounting),
 * or a latency-critical loop, where cudaMalloc/cudaFree can synchronise the
 * whole device.  The paper has no counterpart; it is an interface of this
 * library only.
 *
 * Instead of two small per-call device buffers, it uses one file-scope device
 * array of 385 KiB (base primes up to 2^20 and two counters) that every GPU
 * holds from the moment it loads the library until the process exits.  The
 * caller still owns `out` (device, cap uint64 entries) and `count` (host).
 * Limits are those of cs_primes: hi <= 2^40 (CS_EINVAL beyond), CS_EOVERFLOW
 * if more than cap primes.  It calls no allocating routine.
 *
 * The first call on a device looks up that array's device address (once per
 * device, with that device current); make that first call before any stream
 * capture.  All calls share the one array and each call leaves its contents
 * behind (the counters are cleared at the start of every call), so calls that
 * overlap on the GPU -- from two streams or two host threads -- race: issue
 * them one after another.  Every call, not only the first, ends by reading
 * the count back and synchronising `stream` (the caller's stream only, not the
 * device).  Errors set cs_last_error() like those of every other call. */
cs_status cs_primes_static(uint64_t lo, uint64_t hi, uint64_t *out, uint64_t cap, uint64_t *count,
                           void *stream);

#ifdef __cplusplus
}
#endif

#endif /* COMBSIEVE_H */
