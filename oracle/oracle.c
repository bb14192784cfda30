/*
 * Combined Sieve oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct CPU implementation of what the sieve
 * computes.  Only the tests, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs may load it.  It shares no code with the CUDA
 * path (paper_2012_03771_gb300/csrc).
 *
 * It follows the traditional sieve of Section 2.1 ("Sieving"): for every
 * sieving prime p and every interval centre N = m*K, compute r = N mod p and
 * mark N - r + i*p as composite.  N mod p uses the cached K mod p of
 * Section 3.1 (Space-Time Tradeoff): N mod p = ((m mod p) * (K mod p)) mod p.
 * K mod p itself is the plain big-integer remainder (Horner over 64-bit limbs).
 *
 * Output definition (the same one the CUDA path must reproduce bit for bit):
 *   K    = P#/d, the product of the primes q <= P that do not divide d
 *          (Section 2, "Primorials").
 *   rows = m in [M_start, M_start+M_inc) with gcd(m, d) = 1, ascending
 *          (Section 3: only m coprime to d are sieved).
 *   cols = x in [-SL, SL] with gcd(|x|, K) = 1, ascending; x = 0 is a column
 *          only when K = 1.  W = number of columns.
 *   row word layout: ceil(W/64) uint64 words per row, column j is bit (j & 63)
 *          of word (j >> 6); padding bits are 0.
 *   bit(i, j) = 1 (survivor) iff no sieving prime p (P < p <= L) divides N + x
 *          with N + x != p, and (wheel on) no prime q | d divides N + x with
 *          N + x != q.
 *   F    = number of triples (p, row, col) with p | N + x, N + x != p
 *          ("enumerated factors"; the wheel is not counted).
 *   hash = sum over rows i and words w of mix64(word + (i*wpr + w)*0x9E3779B97F4A7C15)
 *          mod 2^64, with mix64 the SplitMix64 finaliser (Steele, Lea and
 *          Flood, 2014).  A position-dependent checksum of the bitset.
 */
#include <errno.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef unsigned __int128 u128;
typedef __int128 i128;

#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)

#define OR_MAX_P (1u << 20)
#define OR_MAX_SL (1u << 20)
#define OR_MAX_L (1ull << 40)
#define OR_MAX_M (1ull << 40)

/* ---------------------------------------------------------------- primes */

/* All primes <= n by the sieve of Eratosthenes; caller frees. */
static uint64_t *simple_primes(uint64_t n, size_t *count) {
    *count = 0;
    if (n < 2) return calloc(1, sizeof(uint64_t));
    uint8_t *comp = calloc(n + 1, 1);
    if (!comp) return NULL;
    size_t c = 0;
    for (uint64_t i = 2; i <= n; i++) {
        if (comp[i]) continue;
        c++;
        for (uint64_t j = i * i; j <= n; j += i) comp[j] = 1;
    }
    uint64_t *out = malloc((c ? c : 1) * sizeof(uint64_t));
    if (!out) { free(comp); return NULL; }
    size_t k = 0;
    for (uint64_t i = 2; i <= n; i++)
        if (!comp[i]) out[k++] = i;
    free(comp);
    *count = c;
    return out;
}

static uint64_t isqrt64(uint64_t n) {
    uint64_t r = (uint64_t)sqrt((double)n);
    while (r * r > n) r--;
    while ((r + 1) * (r + 1) <= n) r++;
    return r;
}

/* --------------------------------------------------------- K = P#/d */

typedef struct {
    uint64_t *limbs;   /* little-endian */
    size_t n;          /* number of limbs, >= 1 */
    uint64_t *qK;      /* primes dividing K */
    size_t nqK;
    uint64_t *qd;      /* primes dividing d */
    size_t nqd;
} kinfo;

static void kinfo_free(kinfo *k) {
    free(k->limbs); free(k->qK); free(k->qd);
    memset(k, 0, sizeof(*k));
}

/* Checks that d is squarefree with all prime factors <= P (so d | P#), then
 * builds K = P#/d as a big integer.  Returns 0 or OR_EINVAL. */
static int kinfo_make(uint32_t P, uint64_t d, kinfo *k) {
    memset(k, 0, sizeof(*k));
    if (d == 0 || P > OR_MAX_P) return OR_EINVAL;
    size_t np;
    uint64_t *pr = simple_primes(P, &np);
    if (!pr) return OR_ENOMEM;
    k->qK = malloc((np + 1) * sizeof(uint64_t));
    k->qd = malloc((np + 1) * sizeof(uint64_t));
    k->limbs = calloc(np + 2, sizeof(uint64_t));
    if (!k->qK || !k->qd || !k->limbs) { free(pr); kinfo_free(k); return OR_ENOMEM; }
    uint64_t rest = d;
    for (size_t i = 0; i < np; i++) {
        uint64_t q = pr[i];
        if (rest % q == 0) {
            rest /= q;
            if (rest % q == 0) { free(pr); kinfo_free(k); return OR_EINVAL; } /* not squarefree */
            k->qd[k->nqd++] = q;
        } else {
            k->qK[k->nqK++] = q;
        }
    }
    free(pr);
    if (rest != 1) { kinfo_free(k); return OR_EINVAL; } /* d does not divide P# */
    /* K = product of qK, schoolbook multiply by one small factor at a time */
    k->limbs[0] = 1;
    k->n = 1;
    for (size_t i = 0; i < k->nqK; i++) {
        u128 carry = 0;
        for (size_t j = 0; j < k->n; j++) {
            u128 t = (u128)k->limbs[j] * k->qK[i] + carry;
            k->limbs[j] = (uint64_t)t;
            carry = t >> 64;
        }
        if (carry) k->limbs[k->n++] = (uint64_t)carry;
    }
    return 0;
}

/* K mod p by Horner's rule over the limbs (the plain big-integer remainder). */
static uint64_t k_mod(const kinfo *k, uint64_t p) {
    u128 r = 0;
    for (size_t i = k->n; i-- > 0;) r = ((r << 64) | k->limbs[i]) % p;
    return (uint64_t)r;
}

static int k_is_one(const kinfo *k) { return k->n == 1 && k->limbs[0] == 1; }

/* ------------------------------------------------------------ validation */

static int validate(const kinfo *k, uint64_t M_start, uint64_t M_inc, uint32_t SL, uint64_t L) {
    if (SL > OR_MAX_SL || L > OR_MAX_L) return OR_EINVAL;
    if (M_start < 1 || M_start > OR_MAX_M || M_inc > OR_MAX_M - M_start) return OR_EINVAL;
    if (M_inc >= (1ull << 31)) return OR_EINVAL;
    /* every N + x must be >= 2: M_start*K - SL >= 2 */
    if (k->n == 1) {
        u128 lo = (u128)M_start * k->limbs[0];
        if (lo < (u128)SL + 2) return OR_EINVAL;
    }
    return 0;
}

int or_validate(uint32_t P, uint64_t d, uint64_t M_start, uint64_t M_inc, uint32_t SL, uint64_t L) {
    kinfo k;
    int rc = kinfo_make(P, d, &k);
    if (rc) return rc;
    rc = validate(&k, M_start, M_inc, SL, L);
    kinfo_free(&k);
    return rc;
}

/* --------------------------------------------------------- rows, columns */

static uint64_t gcd64(uint64_t a, uint64_t b) {
    while (b) { uint64_t t = a % b; a = b; b = t; }
    return a;
}

/* Columns: x in [-SL, SL] with gcd(|x|, K) = 1.  Writes x values ascending to
 * x_of_col (capacity 2*SL+1, may be NULL).  Returns W or a negative error. */
int64_t or_columns(uint32_t P, uint64_t d, uint32_t SL, int64_t *x_of_col) {
    kinfo k;
    int rc = kinfo_make(P, d, &k);
    if (rc) return rc;
    if (SL > OR_MAX_SL) { kinfo_free(&k); return OR_EINVAL; }
    int64_t W = 0;
    int one = k_is_one(&k);
    for (int64_t x = -(int64_t)SL; x <= (int64_t)SL; x++) {
        uint64_t ax = (uint64_t)(x < 0 ? -x : x);
        int keep;
        if (ax == 0) {
            keep = one;
        } else {
            keep = 1;
            for (size_t i = 0; i < k.nqK; i++)
                if (ax % k.qK[i] == 0) { keep = 0; break; }
        }
        if (keep) {
            if (x_of_col) x_of_col[W] = x;
            W++;
        }
    }
    kinfo_free(&k);
    return W;
}

/* Rows: m in [M_start, M_start+M_inc) with gcd(m, d) = 1.  Returns M_c. */
int64_t or_rows(uint64_t d, uint64_t M_start, uint64_t M_inc, uint64_t *m_out) {
    if (d == 0) return OR_EINVAL;
    int64_t c = 0;
    for (uint64_t m = M_start; m < M_start + M_inc; m++)
        if (gcd64(m, d) == 1) {
            if (m_out) m_out[c] = m;
            c++;
        }
    return c;
}

int or_k_mod_p(uint32_t P, uint64_t d, const uint64_t *p, size_t n, uint64_t *r) {
    kinfo k;
    int rc = kinfo_make(P, d, &k);
    if (rc) return rc;
    for (size_t i = 0; i < n; i++) r[i] = p[i] >= 1 ? k_mod(&k, p[i]) : 0;
    kinfo_free(&k);
    return 0;
}

/* ------------------------------------------------------ prime enumeration */

/* Segments of odd numbers; each worker pulls the next segment index. */
#define SEG_ODDS (1u << 19)

typedef struct {
    uint64_t lo, hi;            /* primes p with lo < p <= hi */
    const uint64_t *base;       /* primes <= sqrt(hi) */
    size_t nbase;
    uint64_t next_seg;          /* shared, atomic */
    uint64_t nseg;
} prime_src;

/* Sieves segment s (odd numbers 2*(s0+i)+1) and calls fn for each prime in (lo, hi]. */
typedef void (*prime_fn)(void *ctx, uint64_t p);

static void sieve_segment(const prime_src *src, uint64_t s, uint8_t *flag, prime_fn fn, void *ctx) {
    /* odd index range [i0, i1): number = 2*i + 1 */
    uint64_t i0 = s * SEG_ODDS;
    uint64_t i1 = i0 + SEG_ODDS;
    uint64_t imax = (src->hi - 1) / 2 + 1;   /* numbers 2i+1 <= hi */
    if (i1 > imax) i1 = imax;
    if (i0 >= i1) return;
    memset(flag, 1, i1 - i0);
    if (i0 == 0) flag[0] = 0;              /* 1 is not prime */
    for (size_t b = 0; b < src->nbase; b++) {
        uint64_t q = src->base[b];
        if (q == 2) continue;
        uint64_t q2 = q * q;
        if (q2 > 2 * (i1 - 1) + 1) break;
        /* first odd multiple of q that is >= max(q*q, 2*i0+1) */
        uint64_t start = 2 * i0 + 1;
        if (start < q2) start = q2;
        uint64_t mlt = (start + q - 1) / q * q;
        if ((mlt & 1) == 0) mlt += q;
        for (uint64_t v = mlt; v <= 2 * (i1 - 1) + 1; v += 2 * q) flag[(v - 1) / 2 - i0] = 0;
    }
    if (s == 0 && src->lo < 2 && src->hi >= 2) fn(ctx, 2);
    for (uint64_t i = i0; i < i1; i++) {
        if (!flag[i - i0]) continue;
        uint64_t p = 2 * i + 1;
        if (p > src->lo && p <= src->hi) fn(ctx, p);
    }
}

static int prime_src_init(prime_src *src, uint64_t lo, uint64_t hi) {
    memset(src, 0, sizeof(*src));
    src->lo = lo;
    src->hi = hi;
    if (hi < 2 || hi <= lo) { src->nseg = 0; return 0; }
    uint64_t *base = simple_primes(isqrt64(hi), &src->nbase);
    if (!base) return OR_ENOMEM;
    src->base = base;
    uint64_t imax = (hi - 1) / 2 + 1;
    src->next_seg = (lo / 2) / SEG_ODDS;   /* skip segments entirely below lo */
    src->nseg = (imax + SEG_ODDS - 1) / SEG_ODDS;
    return 0;
}

static void prime_src_free(prime_src *src) { free((void *)src->base); }

static int n_threads(int want) {
    if (want > 0) return want;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

/* ------------------------------------------------------------------ sieve */

typedef struct {
    const kinfo *k;
    uint32_t SL;
    const uint64_t *rows_m;
    size_t n_rows;
    const int64_t *col_of_x;   /* index x + SL -> column or -1 */
    size_t wpr;
    int small_n;               /* N + x may equal a sieving prime */
    prime_src *src;
    /* per worker */
    uint64_t *bits;
    uint64_t *F_rows;
    uint64_t n_hit;
} sieve_job;

static void sieve_one_prime(void *ctx, uint64_t p) {
    sieve_job *j = ctx;
    uint64_t r = k_mod(j->k, p);                 /* cached K mod p (Section 3.1) */
    int hit_any = 0;
    const int64_t SL = j->SL;
    for (size_t i = 0; i < j->n_rows; i++) {
        uint64_t m = j->rows_m[i];
        uint64_t n = (uint64_t)((u128)(m % p) * r % p);   /* N mod p */
        /* x with p | N + x are x = -n (mod p); start at the smallest one >= -SL */
        int64_t x0 = (int64_t)((p - n) % p);
        int64_t x = x0 - (int64_t)p * ((x0 + SL) / (int64_t)p);
        for (; x <= SL; x += (int64_t)p) {
            hit_any = 1;
            int64_t col = j->col_of_x[x + SL];
            if (col < 0) continue;
            if (j->small_n) {
                i128 v = (i128)m * j->k->limbs[0] + x;
                if (v == (i128)p) continue;      /* N + x is the prime p itself */
            }
            j->bits[i * j->wpr + (uint64_t)col / 64] &= ~(1ull << (col % 64));
            j->F_rows[i]++;
        }
    }
    if (hit_any) j->n_hit++;
}

static void *sieve_worker(void *arg) {
    sieve_job *j = arg;
    uint8_t *flag = malloc(SEG_ODDS);
    if (!flag) return (void *)1;
    for (;;) {
        uint64_t s = __atomic_fetch_add(&j->src->next_seg, 1, __ATOMIC_RELAXED);
        if (s >= j->src->nseg) break;
        sieve_segment(j->src, s, flag, sieve_one_prime, j);
    }
    free(flag);
    return NULL;
}

/*
 * Sieves the given rows (each m must be coprime to d) with the primes p,
 * max(P, p_lo) < p <= p_hi, then (wheel != 0) removes multiples of the primes
 * of d.  bits: n_rows * ceil(W/64) words (output).  F_rows: per-row enumerated
 * factors (output).  n_hit_primes: number of primes dividing at least one
 * N + x, |x| <= SL, over the given rows (output, may be NULL).
 */
int or_sieve(uint32_t P, uint64_t d, uint32_t SL, uint64_t p_lo, uint64_t p_hi, int wheel,
             const uint64_t *rows_m, size_t n_rows, uint64_t *bits, uint64_t *F_rows,
             uint64_t *n_hit_primes, int nthreads) {
    kinfo k;
    int rc = kinfo_make(P, d, &k);
    if (rc) return rc;
    if (SL > OR_MAX_SL || p_hi > OR_MAX_L) { kinfo_free(&k); return OR_EINVAL; }
    for (size_t i = 0; i < n_rows; i++) {
        if (gcd64(rows_m[i], d) != 1) { kinfo_free(&k); return OR_EINVAL; }
        if (validate(&k, rows_m[i], 1, SL, p_hi)) { kinfo_free(&k); return OR_EINVAL; }
    }
    const size_t S = 2 * (size_t)SL + 1;
    int64_t *xs = malloc(S * sizeof(int64_t));
    int64_t *col_of_x = malloc(S * sizeof(int64_t));
    if (!xs || !col_of_x) { free(xs); free(col_of_x); kinfo_free(&k); return OR_ENOMEM; }
    int64_t W = or_columns(P, d, SL, xs);
    for (size_t i = 0; i < S; i++) col_of_x[i] = -1;
    for (int64_t c = 0; c < W; c++) col_of_x[xs[c] + SL] = c;
    const size_t wpr = (size_t)(W + 63) / 64;

    /* all stored columns start as survivors; padding bits stay 0 */
    for (size_t i = 0; i < n_rows; i++) {
        if (F_rows) F_rows[i] = 0;
        for (size_t w = 0; w < wpr; w++) {
            uint64_t v = ~0ull;
            int64_t valid = W - (int64_t)(64 * w);
            if (valid < 64) v = valid <= 0 ? 0 : ((1ull << valid) - 1);
            bits[i * wpr + w] = v;
        }
    }

    /* N + x can equal a sieving prime only when K fits in one word */
    int small_n = k.n == 1;

    uint64_t lo = p_lo > P ? p_lo : P;
    prime_src src;
    rc = prime_src_init(&src, lo, p_hi);
    if (rc) { free(xs); free(col_of_x); kinfo_free(&k); return rc; }

    int nt = n_threads(nthreads);
    sieve_job *jobs = calloc(nt, sizeof(sieve_job));
    pthread_t *th = calloc(nt, sizeof(pthread_t));
    int ok = jobs && th;
    for (int t = 0; ok && t < nt; t++) {
        jobs[t] = (sieve_job){&k, SL, rows_m, n_rows, col_of_x, wpr, small_n, &src, NULL, NULL, 0};
        jobs[t].bits = malloc((n_rows * wpr + 1) * sizeof(uint64_t));
        jobs[t].F_rows = calloc(n_rows + 1, sizeof(uint64_t));
        if (!jobs[t].bits || !jobs[t].F_rows) { ok = 0; break; }
        memcpy(jobs[t].bits, bits, n_rows * wpr * sizeof(uint64_t));
    }
    int started = 0;
    for (int t = 0; ok && t < nt; t++) {
        if (pthread_create(&th[t], NULL, sieve_worker, &jobs[t])) { ok = 0; break; }
        started++;
    }
    for (int t = 0; t < started; t++) {
        void *ret = NULL;
        pthread_join(th[t], &ret);
        if (ret) ok = 0;
    }
    uint64_t n_hit = 0;
    if (ok) {
        /* merge: a cell survives only if it survives every worker's primes */
        for (int t = 0; t < nt; t++) {
            for (size_t w = 0; w < n_rows * wpr; w++) bits[w] &= jobs[t].bits[w];
            for (size_t i = 0; i < n_rows; i++) if (F_rows) F_rows[i] += jobs[t].F_rows[i];
            n_hit += jobs[t].n_hit;
        }
    }
    for (int t = 0; jobs && t < nt; t++) { free(jobs[t].bits); free(jobs[t].F_rows); }
    free(jobs);
    free(th);
    prime_src_free(&src);

    if (ok && wheel) {
        /* primes q | d: clear x with q | N + x, unless N + x = q */
        for (size_t qi = 0; qi < k.nqd; qi++) {
            uint64_t q = k.qd[qi];
            uint64_t rq = k_mod(&k, q);
            for (size_t i = 0; i < n_rows; i++) {
                uint64_t m = rows_m[i];
                uint64_t n = (uint64_t)((u128)(m % q) * rq % q);
                int64_t x0 = (int64_t)((q - n) % q);
                int64_t x = x0 - (int64_t)q * ((x0 + (int64_t)SL) / (int64_t)q);
                for (; x <= (int64_t)SL; x += (int64_t)q) {
                    int64_t col = col_of_x[x + SL];
                    if (col < 0) continue;
                    if (k.n == 1) {
                        i128 v = (i128)m * k.limbs[0] + x;
                        if (v == (i128)q) continue;
                    }
                    bits[i * wpr + (uint64_t)col / 64] &= ~(1ull << (col % 64));
                }
            }
        }
    }
    if (n_hit_primes) *n_hit_primes = n_hit;
    free(xs);
    free(col_of_x);
    kinfo_free(&k);
    return ok ? 0 : OR_ENOMEM;
}

/* ------------------------------------------------------- counts and hash */

static uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Checksum of n_rows rows starting at global row index row0. */
uint64_t or_hash(const uint64_t *bits, size_t n_rows, size_t wpr, uint64_t row0) {
    uint64_t h = 0;
    for (size_t i = 0; i < n_rows; i++)
        for (size_t w = 0; w < wpr; w++) {
            uint64_t pos = (row0 + i) * wpr + w;
            h += mix64(bits[i * wpr + w] + pos * 0x9E3779B97F4A7C15ull);
        }
    return h;
}

void or_row_counts(const uint64_t *bits, size_t n_rows, size_t wpr, uint32_t *counts) {
    for (size_t i = 0; i < n_rows; i++) {
        uint32_t c = 0;
        for (size_t w = 0; w < wpr; w++) c += (uint32_t)__builtin_popcountll(bits[i * wpr + w]);
        counts[i] = c;
    }
}

/* ----------------------------------------------------------- prime stats */

typedef struct {
    prime_src *src;
    uint64_t count;
    double log_prod;     /* sum of log(1 - 1/p) */
    double inv_sum;      /* sum of 1/p */
} stats_job;

static void stats_one(void *ctx, uint64_t p) {
    stats_job *j = ctx;
    j->count++;
    j->log_prod += log1p(-1.0 / (double)p);
    j->inv_sum += 1.0 / (double)p;
}

static void *stats_worker(void *arg) {
    stats_job *j = arg;
    uint8_t *flag = malloc(SEG_ODDS);
    if (!flag) return (void *)1;
    for (;;) {
        uint64_t s = __atomic_fetch_add(&j->src->next_seg, 1, __ATOMIC_RELAXED);
        if (s >= j->src->nseg) break;
        sieve_segment(j->src, s, flag, stats_one, j);
    }
    free(flag);
    return NULL;
}

/* Number of primes in (lo, hi], sum of log(1 - 1/p) and sum of 1/p over them. */
int or_prime_stats(uint64_t lo, uint64_t hi, uint64_t *count, double *log_prod, double *inv_sum,
                   int nthreads) {
    if (hi > OR_MAX_L) return OR_EINVAL;
    prime_src src;
    int rc = prime_src_init(&src, lo, hi);
    if (rc) return rc;
    int nt = n_threads(nthreads);
    stats_job *jobs = calloc(nt, sizeof(stats_job));
    pthread_t *th = calloc(nt, sizeof(pthread_t));
    int ok = jobs && th, started = 0;
    for (int t = 0; ok && t < nt; t++) {
        jobs[t].src = &src;
        if (pthread_create(&th[t], NULL, stats_worker, &jobs[t])) { ok = 0; break; }
        started++;
    }
    uint64_t c = 0;
    double lp = 0, is = 0;
    for (int t = 0; t < started; t++) {
        void *ret = NULL;
        pthread_join(th[t], &ret);
        if (ret) ok = 0;
        c += jobs[t].count;
        lp += jobs[t].log_prod;
        is += jobs[t].inv_sum;
    }
    free(jobs);
    free(th);
    prime_src_free(&src);
    if (!ok) return OR_ENOMEM;
    *count = c;
    if (log_prod) *log_prod = lp;
    if (inv_sum) *inv_sum = is;
    return 0;
}

/* Writes the primes in (lo, hi] ascending (single thread); returns the count,
 * or a negative error if more than cap. */
typedef struct { uint64_t *out; size_t cap, n; } list_job;
static void list_one(void *ctx, uint64_t p) {
    list_job *j = ctx;
    if (j->n < j->cap) j->out[j->n] = p;
    j->n++;
}

int64_t or_primes(uint64_t lo, uint64_t hi, uint64_t *out, size_t cap) {
    if (hi > OR_MAX_L) return OR_EINVAL;
    prime_src src;
    int rc = prime_src_init(&src, lo, hi);
    if (rc) return rc;
    uint8_t *flag = malloc(SEG_ODDS);
    if (!flag) { prime_src_free(&src); return OR_ENOMEM; }
    list_job j = {out, cap, 0};
    for (uint64_t s = src.next_seg; s < src.nseg; s++) sieve_segment(&src, s, flag, list_one, &j);
    free(flag);
    prime_src_free(&src);
    if (j.n > cap) return OR_ENOMEM;
    return (int64_t)j.n;
}
