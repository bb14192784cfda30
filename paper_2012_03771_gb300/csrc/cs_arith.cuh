// Integer arithmetic used by the Combined Sieve kernels.
//
// * Montgomery multiplication (P. L. Montgomery, "Modular multiplication
//   without trial division", Math. Comp. 44, 1985) with R = 2^32 and R = 2^64,
//   for the cached residues K mod p of Section 3.1.
// * A stack-free form of the modular-equation solver G(p, K, L, R) of
//   Section 3.3 (Eq. modsol).
// * The SplitMix64 finaliser (Steele, Lea and Flood, 2014) for the bitset
//   checksum.
#pragma once
#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define CS_HD __host__ __device__ __forceinline__
#else
#define CS_HD inline
#endif

namespace cs {

// Bit helpers for 32-bit words, the shift taken mod 32 (one funnel shift on
// the device, where a plain shift needs the mask as a second instruction):
// bit (s mod 32) of x, and x with only its bits below position (s mod 32)
// (shifted to the top, so that their population count is the number of set
// bits below s; 0 for s = 0).
CS_HD uint32_t bit_of(uint32_t x, uint32_t s) {
#if defined(__CUDA_ARCH__)
    return __funnelshift_r(x, 0u, s) & 1u;
#else
    return (x >> (s & 31)) & 1u;
#endif
}
CS_HD uint32_t bits_below(uint32_t x, uint32_t s) {
#if defined(__CUDA_ARCH__)
    return __funnelshift_r(0u, x, s);
#else
    return (s & 31) ? x << (32 - (s & 31)) : 0u;
#endif
}
CS_HD uint32_t bit_at(uint32_t s) {
#if defined(__CUDA_ARCH__)
    return __funnelshift_l(0u, 1u, s);
#else
    return 1u << (s & 31);
#endif
}

CS_HD uint64_t mulhi64(uint64_t a, uint64_t b) {
#if defined(__CUDA_ARCH__)
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// ---------------------------------------------------------------- R = 2^32
// -p^-1 mod 2^32 for odd p, by Newton's iteration x <- x(2 - p x); an odd p is
// its own inverse mod 8, and every step doubles the number of correct bits.
CS_HD uint32_t mont32_neg_inv(uint32_t p) {
    uint32_t x = p;
    x *= 2u - p * x;
    x *= 2u - p * x;
    x *= 2u - p * x;
    x *= 2u - p * x;
    return 0u - x;
}

// a * b * 2^-32 mod p, fully reduced.  Requires odd p < 2^31, a < p, b < 2^32.
CS_HD uint32_t mont32_mul(uint32_t a, uint32_t b, uint32_t p, uint32_t pinv) {
    uint64_t t = (uint64_t)a * b;
    uint32_t m = (uint32_t)t * pinv;
    uint64_t u = t + (uint64_t)m * p;   // divisible by 2^32, u < 2^64
    uint32_t r = (uint32_t)(u >> 32);
    return r >= p ? r - p : r;
}

// a * b * 2^-32 mod p, reduced only below 2p (P. L. Montgomery's REDC without
// the final subtraction): for odd p < 2^31, a < 2p and b < 2^31,
// (a b + m p) / 2^32 < (2p 2^31 + 2^32 p) / 2^32 = 2p and a b + m p < 2^64,
// so a chain of such products by words below 2^31 needs one subtraction at
// its end.
CS_HD uint32_t mont32_mul_lazy(uint32_t a, uint32_t b, uint32_t p, uint32_t pinv) {
    const uint64_t t = (uint64_t)a * b;
    const uint32_t m = (uint32_t)t * pinv;
    return (uint32_t)((t + (uint64_t)m * p) >> 32);
}

// R mod p and R^2 mod p for R = 2^32.
CS_HD uint32_t mont32_r1(uint32_t p) { return (0u - p) % p; }
CS_HD uint32_t mont32_r2(uint32_t p) {
    uint64_t r = mont32_r1(p);
    return (uint32_t)((r * r) % p);
}

// R^2 mod p without a 64-bit division, for odd 2^20 <= p < 2^31 (smaller p
// take the plain remainder): a Barrett-style reduction (P. Barrett, CRYPTO '86)
// of n = 2^64 - 1 whose quotients are estimated with the correctly rounded
// float reciprocal of p.  The first estimate of n / p <= 2^44 is off by less
// than 2^23; its remainder, taken in wrapping 64-bit arithmetic, is exact as a
// signed value; two more estimates bring it into (-p, 2p), and two
// corrections into [0, p).  Then R^2 = n + 1.
CS_HD float rcp_rn(float x) {
#if defined(__CUDA_ARCH__)
    return __frcp_rn(x);
#else
    return 1.0f / x;
#endif
}
// Conversions between 64-bit integers and float through 32-bit halves: on
// this GPU the direct 64-bit conversions issue to the slow FP64 pipe.  The
// value is rounded at most three times (relative error below 2^-22; the
// halves of a magnitude are both non-negative, so they never cancel), and
// f_to_u64 truncates exactly: for x >= 2^32 the part below 2^32 has at most 24
// significant bits.
CS_HD float u64_to_f(uint64_t n) {
    return (float)(uint32_t)(n >> 32) * 4294967296.0f + (float)(uint32_t)n;
}
CS_HD float s64_to_f(int64_t n) {   // magnitude and sign: the halves must not cancel
    const float f = u64_to_f((uint64_t)(n < 0 ? -n : n));
    return n < 0 ? -f : f;
}
CS_HD uint64_t f_to_u64(float x) {   // 0 <= x < 2^64
    const float hi = floorf(x * 2.3283064365386963e-10f);
    return ((uint64_t)(uint32_t)hi << 32) + (uint32_t)(x - hi * 4294967296.0f);
}

CS_HD uint32_t mont32_r2_fast(uint32_t p) {
    if (p < (1u << 20)) return mont32_r2(p);
    const float fr = rcp_rn((float)p);
    const uint64_t q0 = f_to_u64(18446744073709551616.0f * fr);
    int64_t rem = (int64_t)(~0ull - q0 * (uint64_t)p);
    for (int pass = 0; pass < 2; pass++) {
        const int32_t q = (int32_t)(s64_to_f(rem) * fr);   // |q| < 2^23
        rem -= (int64_t)q * (int64_t)p;
    }
    if (rem < 0) rem += p;
    if (rem < 0) rem += p;
    if (rem >= (int64_t)p) rem -= p;
    if (rem >= (int64_t)p) rem -= p;
    const uint32_t r = (uint32_t)rem + 1;
    return r == p ? 0u : r;
}

// (r * M + s) mod p for r < p, M < 2^64, s < p, given rt = r R mod p and
// r2 = R^2 mod p: r * M = r * lo + (r * hi) * 2^32 with M = hi 2^32 + lo, each
// part one Montgomery product (no 64-bit division).
CS_HD uint32_t mont32_affine(uint32_t rt, uint64_t M, uint32_t s, uint32_t r2, uint32_t p, uint32_t pinv) {
    uint32_t v = mont32_mul(rt, (uint32_t)M, p, pinv);
    if (M >> 32) {
        uint32_t h = mont32_mul(rt, (uint32_t)(M >> 32), p, pinv);   // r hi mod p
        h = mont32_mul(h, r2, p, pinv);                               // r hi R mod p
        v = v + h >= p ? v + h - p : v + h;
    }
    return v + s >= p ? v + s - p : v + s;
}

// R^e mod p given R mod p and R^2 mod p.  Under mont32_mul the residues
// Y_j = R^(j+1) mod p form a monoid with Y_a * Y_b = Y_(a+b) and identity Y_0 = R,
// so R^e = Y_1^(e-1) by square-and-multiply.  e >= 1.
CS_HD uint32_t mont32_rpow(uint32_t e, uint32_t r1, uint32_t r2, uint32_t p, uint32_t pinv) {
    uint32_t acc = r1, base = r2;
    uint32_t k = e - 1;
    while (k) {
        if (k & 1) acc = mont32_mul(acc, base, p, pinv);
        base = mont32_mul(base, base, p, pinv);
        k >>= 1;
    }
    return acc;
}

// ---------------------------------------------------------------- R = 2^64
CS_HD uint64_t mont64_neg_inv(uint64_t p) {
    uint64_t x = p;
    x *= 2u - p * x;
    x *= 2u - p * x;
    x *= 2u - p * x;
    x *= 2u - p * x;
    x *= 2u - p * x;
    return 0ull - x;
}

// a * b * 2^-64 mod p, fully reduced.  Requires odd p < 2^62, a < p, b < 2^64.
CS_HD uint64_t mont64_mul(uint64_t a, uint64_t b, uint64_t p, uint64_t pinv) {
    uint64_t lo = a * b;
    uint64_t hi = mulhi64(a, b);
    uint64_t m = lo * pinv;
    // lo + low64(m * p) == 0 (mod 2^64): the carry out of that sum is (lo != 0)
    uint64_t r = hi + mulhi64(m, p) + (lo != 0);
    return r >= p ? r - p : r;
}

CS_HD uint64_t mont64_r1(uint64_t p) { return (0ull - p) % p; }
// R^2 mod p = R * 2^64 mod p by 64 modular doublings of R mod p (p < 2^63).
CS_HD uint64_t mont64_r2(uint64_t p) {
    uint64_t r = mont64_r1(p);
    for (int i = 0; i < 64; i++) {
        r <<= 1;
        if (r >= p) r -= p;
    }
    return r;
}

// x mod p for x < 2^61 and odd p with a quotient x / p below 2^20, given
// fp = rcp_rn(u64_to_f(p)): u64_to_f(x) and u64_to_f(p) are each within a
// relative 2^-22 of x and p, the reciprocal and the product each add at most
// 2^-24, so the float quotient is within a relative 2.5 2^-22 of x / p, i.e.
// within 0.63 of it, and its truncation is floor(x / p) or off by one either
// way: one correction each way makes the remainder exact.
CS_HD uint64_t mod_q20(uint64_t x, uint64_t p, float fp) {
    const uint32_t q = (uint32_t)(u64_to_f(x) * fp);
    int64_t r = (int64_t)(x - (uint64_t)q * p);
    if (r < 0) r += (int64_t)p;
    else if (r >= (int64_t)p) r -= (int64_t)p;
    return (uint64_t)r;
}

// R^2 mod p (R = 2^64) for odd 2^20 <= p < 2^40 without a 64-bit division:
// 2^40 mod p (a quotient below 2^20), then x <- x 2^20 mod p four times
// (x 2^20 < 2^60, quotients below 2^20) up to 2^120, and x 2^8 mod p.  Other p
// take the 64 modular doublings of mont64_r2.
CS_HD uint64_t mont64_r2_fast(uint64_t p, float fp) {
    if (p < (1ull << 20) || p >= (1ull << 40)) return mont64_r2(p);
    uint64_t x = mod_q20(1ull << 40, p, fp);
    for (int k = 0; k < 4; k++) x = mod_q20(x << 20, p, fp);
    return mod_q20(x << 8, p, fp);
}

// R^e mod p from R^2 mod p alone (e >= 1), in the Montgomery monoid
// Y_j = R^(j+1) mod p: R^e = Y_(e-1) = Y_1^(e-1), taken as Y_1 * Y_1^(e-2) by
// square-and-multiply without a squaring after the last bit.
CS_HD uint64_t mont64_rpow2(uint32_t e, uint64_t r2, uint64_t p, uint64_t pinv) {
    if (e <= 1) return mont64_mul(r2, 1, p, pinv);   // R mod p
    uint64_t acc = r2, base = r2;
    uint32_t k = e - 2;
    while (k) {
        if (k & 1) acc = mont64_mul(acc, base, p, pinv);
        k >>= 1;
        if (k) base = mont64_mul(base, base, p, pinv);
    }
    return acc;
}

CS_HD uint64_t mont64_rpow(uint32_t e, uint64_t r1, uint64_t r2, uint64_t p, uint64_t pinv) {
    uint64_t acc = r1, base = r2;
    uint32_t k = e - 1;
    while (k) {
        if (k & 1) acc = mont64_mul(acc, base, p, pinv);
        base = mont64_mul(base, base, p, pinv);
        k >>= 1;
    }
    return acc;
}

// --------------------------------------------------------------- division
// Quotients of the solver's operands: 32-bit hardware-friendly division when
// both operands fit in 32 bits, 64-bit otherwise.
CS_HD uint32_t udiv(uint32_t a, uint32_t b) { return a / b; }
CS_HD uint64_t udiv(uint64_t a, uint64_t b) {
    if (((a | b) >> 32) == 0) return (uint32_t)a / (uint32_t)b;
    return a / b;
}

// ----------------------------------------------------------- G(p, K, L, R)
//
// Smallest m >= 0 with L <= m*K mod p <= L + w (Eq. modfunc), for 0 < K < p,
// gcd(K, p) = 1, 0 <= L and L + w < p.  Returns m and y = m*K mod p.
//
// Section 3.3 gives G as a recursion over five cases:
//   a: L = 0                      -> 0
//   C: ceil(L/K) <= floor(R/K)    -> ceil(L/K)
//   D: 2K >= p                    -> G(p, p-K, p-R, p-L)
//   E: otherwise                  -> ceil((L + p*G(K, -p mod K, L mod K, R mod K)) / K)
// (case B, K >= p, is the caller's reduction K mod p).  Case E needs the inner
// answer before it can finish, so a direct transcription keeps a stack.  This
// version runs the same chain of sub-problems forwards and keeps, for the
// current sub-problem (p_k, K_k), the two lattice vectors (U, p_k) and (u, K_k)
// of {(m, y) : y = m*K (mod p)} whose value parts are p_k and K_k, plus an
// affine map y_0 = A + s*y_k from the current window back to the original one
// (s = +-1; case D flips it, case E shifts it by floor(L/K)*K).  When case C
// ends the chain with y_k = c*K_k, the answer is the lattice point
// (B + s*c*u, A + s*c*K_k), where B is the m part accumulated alongside A.
// The window width w = R - L is the same in every sub-problem.
//
// For p < 2^30 all of A, B, U, u stay within (-2^31, 2^31) (|A| < 1.5p,
// |B| < p/2, |u| < 0.62p, |U| < 0.24p), so 32-bit registers suffice.  The
// number of passes is at most about 2*log2(p/(w+1)) + 2; max_iter bounds it.
template <class UT, class ST>
CS_HD bool g_solve(UT p, UT K, UT L, UT w, UT &m_out, UT &y_out, uint32_t &iters, uint32_t max_iter) {
    if (L == 0) {
        m_out = 0;
        y_out = 0;
        return true;
    }
    ST A = 0, B = 0, U = 0, u = 1, s = 1;
    for (uint32_t it = 0; it < max_iter; it++) {
        iters++;
        UT c = udiv((UT)(L + K - 1), K);              // ceil(L/K)
        UT ck = c * K;
        if (ck <= L + w) {                             // case C
            y_out = (UT)(A + s * (ST)ck);
            m_out = (UT)(B + s * (ST)c * u);
            return true;
        }
        if (2 * K >= p) {                              // case D
            A += s * (ST)p;
            B += s * U;
            s = -s;
            u = U - u;
            K = p - K;
            L = p - (L + w);
            continue;
        }
        UT f = c - 1;                                  // case E: floor(L/K), K does not divide L
        A += s * (ST)(f * K);
        B += s * (ST)f * u;
        UT q = udiv((UT)(p + K - 1), K);               // ceil(p/K)
        ST nu = (ST)q * u - U;
        U = u;
        u = nu;
        UT np = K;
        K = q * K - p;                                 // (-p) mod K
        p = np;
        L = L - f * np;                                // L mod K
    }
    return false;
}

// Approximate float reciprocal (one MUFU op; relative error at most 2^-23) for
// quotient estimates that are corrected afterwards.
CS_HD float rcp_approx(float x) {
#if defined(__CUDA_ARCH__)
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
#else
    return 1.0f / x;
#endif
}

// floor(a / b) and a mod b for a < 2^31, 1 <= b, when the quotient is below
// 2^21 + 2, given rb = a reciprocal of b within a relative 2^-23: the float
// estimate a * rb is then within 1/2 of a / b, its truncation within 1 of the
// quotient, and one correction either way makes it exact (the remainder, in
// [-b, 2b), fits 32 signed bits as b < 2^30).  Replaces a full division in the
// Euclid steps, whose partial quotients are small.
CS_HD uint32_t udiv_q21(uint32_t a, uint32_t b, float rb, uint32_t &rem) {
    uint32_t q = (uint32_t)((float)a * rb);
    int32_t r = (int32_t)(a - q * b);
    if (r < 0) {
        q--;
        r += (int32_t)b;
    } else if (r >= (int32_t)b) {
        q++;
        r -= (int32_t)b;
    }
    rem = (uint32_t)r;
    return q;
}

// The same for 64-bit operands, a < 2^62, 1 <= b, a quotient below 2^21 + 2 and
// rb = a reciprocal of u64_to_f(b) within a relative 2^-23: u64_to_f is within a
// relative 2^-23 of its argument (each 32-bit half rounded once, and the sum),
// so u64_to_f(a) * rb is within about 3.5 2^-23 relative, less than 0.875
// absolute, of a / b, and its truncation is the quotient or off by one either
// way (the remainder, in [-b, 2b), fits 64 signed bits).  Replaces the 64-bit
// division of the Euclid steps for primes above 2^32 when p < 2SL 2^21.
CS_HD uint64_t udiv_q21_64(uint64_t a, uint64_t b, float rb, uint64_t &rem) {
    uint64_t q = (uint32_t)(u64_to_f(a) * rb);
    int64_t r = (int64_t)(a - q * b);
    if (r < 0) {
        q--;
        r += (int64_t)b;
    } else if (r >= (int64_t)b) {
        q++;
        r -= (int64_t)b;
    }
    rem = (uint64_t)r;
    return q;
}

// The two steps of the three-gap walk from one run of Euclid's algorithm.
//
// For 0 < r < p with gcd(r, p) = 1 and 1 <= w < p: a = the smallest m > 0 with
// r m mod p in [p - w, p - 1] (da = p - r a mod p) and b = the smallest with
// r m mod p in [1, w] (ub = r b mod p), the same answers as the solver G of
// Section 3.3 gives for those two windows.  Euclid's algorithm on x_0 = p,
// x_1 = r with m_0 = 0, m_1 = 1, x_(k+1) = x_(k-1) - c_k x_k,
// m_(k+1) = m_(k-1) + c_k m_k keeps r m_k = (-1)^(k+1) x_k (mod p), so odd k
// give residues +x_k and even k residues -x_k.  The first m of a given sign
// whose residue is at most w is a convergent or intermediate fraction
// (best approximation): with K the first index where x_K <= w, the sign of K
// is reached at m_(K-2) + t m_(K-1), t = ceil((x_(K-2) - w) / x_(K-1)) (at m_1
// when K = 1), and the other sign at m_(K-1) + t' m_K,
// t' = ceil((x_(K-1) - w) / x_K).  One division per step, against the solver's
// window bookkeeping.  Returns false after max_iter steps (not reached: the
// x_k fall at least as fast as Fibonacci numbers).
template <class UT>
CS_HD bool tg_steps(UT p, UT r, UT w, UT &a, UT &da, UT &b, UT &ub, uint32_t &iters, uint32_t max_iter) {
    UT x_pp = 0, m_pp = 0, x_prev = p, m_prev = 0, x = r, m = 1;
    uint32_t k = 1;
    // 32-bit, p < 2^30 and w >= 512: every partial quotient below x_prev / x <
    // 2^30 / 512 = 2^21, so the float estimate with one correction is exact;
    // 64-bit with p < w 2^21: every partial quotient below p / w < 2^21 likewise
    const bool small_q = sizeof(UT) == 4 && w >= 512 && p < (UT)(1u << 30);
    const bool small_q64 = sizeof(UT) == 8 && (uint64_t)p < ((uint64_t)w << 21);
    while (x > w) {
        if (k > max_iter) return false;
        UT c, xn;
        if (small_q) {
            uint32_t rem;
            c = (UT)udiv_q21((uint32_t)x_prev, (uint32_t)x, rcp_approx((float)x), rem);
            xn = (UT)rem;
        } else if (small_q64) {
            uint64_t rem;
            c = (UT)udiv_q21_64((uint64_t)x_prev, (uint64_t)x, rcp_approx(u64_to_f((uint64_t)x)), rem);
            xn = (UT)rem;
        } else {
            c = udiv(x_prev, x);
            xn = x_prev - c * x;
        }
        const UT mn = m_prev + c * m;
        x_pp = x_prev; m_pp = m_prev;
        x_prev = x; m_prev = m;
        x = xn; m = mn;
        k++;
    }
    iters += k;
    UT ms, xs;                                   // first m with the sign of x_K
    if (k == 1) {
        ms = 1;
        xs = r;
    } else {
        // quotient below x_pp / x_prev + 1 (x_prev > w)
        UT t;
        if (small_q) {
            uint32_t rem;
            t = (UT)udiv_q21((uint32_t)(x_pp - w + x_prev - 1), (uint32_t)x_prev, rcp_approx((float)x_prev), rem);
        } else if (small_q64) {
            uint64_t rem;
            t = (UT)udiv_q21_64((uint64_t)(x_pp - w + x_prev - 1), (uint64_t)x_prev,
                                rcp_approx(u64_to_f((uint64_t)x_prev)), rem);
        } else {
            t = udiv((UT)(x_pp - w + x_prev - 1), x_prev);
        }
        ms = m_pp + t * m_prev;
        xs = x_pp - t * x_prev;
    }
    const UT t2 = udiv((UT)(x_prev - w + x - 1), x);   // first m with the other sign
    const UT mo = m_prev + t2 * m, xo = x_prev - t2 * x;
    if (k & 1) {
        b = ms; ub = xs; a = mo; da = xo;
    } else {
        a = ms; da = xs; b = mo; ub = xo;
    }
    return true;
}

// floor(n / p) for n < 2^62, p < 2^31 and a quotient below 2^32, given
// fr = rcp_rn(p): a float estimate of the quotient (off by less than 2^11),
// its exact remainder in 64-bit arithmetic, one refinement (off by at most
// one) and two corrections each way.
CS_HD uint64_t udiv64_est(uint64_t n, uint32_t p, float fr, int64_t &rem_out) {
    uint64_t q = f_to_u64(u64_to_f(n) * fr);
    int64_t rem = (int64_t)(n - q * p);
    const int32_t q1 = (int32_t)(s64_to_f(rem) * fr);      // |q1| < 2^12
    rem -= (int64_t)q1 * (int64_t)p;
    q += (uint64_t)(int64_t)q1;
    if (rem < 0) { rem += p; q--; }
    if (rem < 0) { rem += p; q--; }
    if (rem >= (int64_t)p) { rem -= p; q++; }
    if (rem >= (int64_t)p) { rem -= p; q++; }
    rem_out = rem;
    return q;
}

// First hit of a walk from the three-gap basis, without a solve.
//
// For 0 < r < p and 1 <= w < p let a > 0 be the smallest m with r m mod p in
// [p - w, p - 1] (r a = -da) and b the smallest with r m mod p in [1, w]
// (r b = ub).  Then a ub + b da = p, so e1 = (a, -da) and e2 = (b, ub) are a
// basis of the lattice {(t, y) : y = r t (mod p)}, and the points of
// (0, v0) + lattice in the strip 0 <= y <= w are (i a + j b, v0 - i da + j ub)
// for the (i, j) with 0 <= v0 - i da + j ub <= w.  Ordered by t they form one
// chain whose steps are e1, e2 or e1 + e2, so i and j never decrease along it.
// With da <= ub the chain runs through blocks of fixed j (i from
// ceil((Y_j - w)/da) to floor(Y_j/da), Y_j = v0 + j ub); the first block whose
// last point has t >= 0 is j = -floor(v0 a / p) or the next one (a da / p < 1),
// and the answer is its first point with t >= 0.  With ub < da the roles of
// (i, a, da) and (j, b, ub) swap, the first block being i = ceil((v0 - w) b / p)
// or the next; the second case is the first one for the reflected strip
// y' = w - y and is computed as such.  Returns the smallest t >= 0 with
// (v0 + r t) mod p <= w, for w < v0 < p < 2^30 and w <= 2^21 (2SL with
// SL <= 2^20; smaller v0 is a hit at t = 0), and in y_out that residue.
CS_HD uint32_t first_hit32(uint32_t p, float fr, uint32_t w, uint32_t a, uint32_t da, uint32_t b,
                           uint32_t ub, uint32_t v0, uint32_t &y_out) {
    // ub < da is the case da <= ub for the reflected strip y' = w - y (start
    // w - v0, steps e2 down by ub and e1 up by da): swap the roles and reflect,
    // so that one branch-free path serves both
    const bool sw = da > ub;
    const uint32_t A = sw ? b : a, DA = sw ? ub : da, B = sw ? a : b, UB = sw ? da : ub;
    const int64_t V0 = sw ? (int64_t)w - (int64_t)v0 : (int64_t)v0;      // |V0| < 2^30
    // floor(x / d) and ceil(x / d) for |x| < 2^31, 0 < d < 2^31
    auto fdiv = [](int64_t x, uint32_t d) -> int64_t {
        const uint32_t ax = (uint32_t)(x < 0 ? -x : x), q = ax / d;
        return x >= 0 ? (int64_t)q : -(int64_t)q - (ax != q * d);
    };
    // first block: J = -floor(V0 A / p) = ceil(-V0 A / p)
    int64_t rem;
    const uint64_t aq = udiv64_est((uint64_t)(V0 < 0 ? -V0 : V0) * A, p, fr, rem);
    int64_t j = V0 >= 0 ? -(int64_t)aq : (int64_t)aq + (rem != 0);
    int64_t Y = V0 + j * (int64_t)UB;                                    // |Y| < 2^31
    // the block's last point must reach t >= 0, else the next block
    if (fdiv(Y, DA) * A + j * (int64_t)B < 0) {
        j++;
        Y += UB;
    }
    int64_t i = -fdiv((int64_t)w - Y, DA);                               // ceil((Y - w) / DA)
    const int64_t t_lo = i * A + j * (int64_t)B;
    if (t_lo < 0) {
        // steps of A to the first point with t >= 0: ceil(-t_lo / A), a quotient
        // below w / DA + 2 <= 2^21 + 2, so one float estimate is off by less
        // than 2 and two corrections each way make it exact
        const int64_t n = -t_lo;                                         // < 2^52
        int64_t q = (int64_t)(uint32_t)(u64_to_f((uint64_t)n) * rcp_rn((float)A));
        int64_t rem = n - q * (int64_t)A;
        if (rem < 0) { rem += A; q--; }
        if (rem < 0) { rem += A; q--; }
        if (rem >= (int64_t)A) { rem -= A; q++; }
        if (rem >= (int64_t)A) { rem -= A; q++; }
        i += q + (rem != 0);
    }
    const uint32_t y = (uint32_t)(Y - i * (int64_t)DA);
    y_out = sw ? w - y : y;
    return (uint32_t)(i * A + j * (int64_t)B);
}

// floor(n / d) for |n / d| < 2^42, 0 < d < 2^41 (n, d as below), given
// fr = rcp_rn(d): a float estimate of the quotient (off by less than 2^19),
// the exact remainder (128-bit, then below 2^61 in magnitude), two refinements
// and two corrections each way.
CS_HD float s128_to_f(__int128 n) {
    const unsigned __int128 m = (unsigned __int128)(n < 0 ? -n : n);
    const float f = u64_to_f((uint64_t)(m >> 64)) * 18446744073709551616.0f + u64_to_f((uint64_t)m);
    return n < 0 ? -f : f;
}
CS_HD int64_t f_to_s64(float x) {   // |x| < 2^63, truncated toward zero
    const uint64_t m = f_to_u64(x < 0 ? -x : x);
    return x < 0 ? -(int64_t)m : (int64_t)m;
}
CS_HD int64_t floor_div_est(__int128 n, uint64_t d, float fr) {
    int64_t q = f_to_s64(s128_to_f(n) * fr);
    int64_t rem = (int64_t)(n - (__int128)q * (__int128)d);
    for (int pass = 0; pass < 2; pass++) {
        const int64_t q1 = f_to_s64(s64_to_f(rem) * fr);
        q += q1;
        rem -= q1 * (int64_t)d;
    }
    if (rem < 0) { rem += d; q--; }
    if (rem < 0) { rem += d; q--; }
    if (rem >= (int64_t)d) { rem -= d; q++; }
    if (rem >= (int64_t)d) { rem -= d; q++; }
    return q;
}

// first_hit32 for 64-bit primes: p < 2^40, w <= 2^21 (SL <= 2^20).  Bounds:
// |V0| < 2^40 and A < 2^40, so V0 A < 2^80 (128-bit) with quotient J below
// 2^40; |Y| < 2^41 (quotients by DA below 2^41); products i A, j B below 2^81
// (128-bit); the block's last point is at most (w / DA + 1) A < 2^61 past its
// first, so the steps to t >= 0 fit in 64 bits.
CS_HD uint64_t first_hit64(uint64_t p, uint64_t w, uint64_t a, uint64_t da, uint64_t b, uint64_t ub,
                           uint64_t v0, uint64_t &y_out) {
    const bool sw = da > ub;
    const uint64_t A = sw ? b : a, DA = sw ? ub : da, B = sw ? a : b, UB = sw ? da : ub;
    const int64_t V0 = sw ? (int64_t)w - (int64_t)v0 : (int64_t)v0;
    const float fp = rcp_rn((float)p), fda = rcp_rn((float)DA);
    // first block: J = -floor(V0 A / p)
    int64_t j = -floor_div_est((__int128)V0 * (__int128)A, p, fp);
    int64_t Y = V0 + j * (int64_t)UB;
    if ((__int128)floor_div_est(Y, DA, fda) * A + (__int128)j * B < 0) {
        j++;
        Y += (int64_t)UB;
    }
    int64_t i = -floor_div_est((int64_t)w - Y, DA, fda);                 // ceil((Y - w) / DA)
    const __int128 t_lo = (__int128)i * A + (__int128)j * B;
    if (t_lo < 0) i += -floor_div_est(t_lo, A, rcp_rn((float)A));     // ceil(-t_lo / A) steps
    const uint64_t y = (uint64_t)(Y - i * (int64_t)DA);
    y_out = sw ? w - y : y;
    return (uint64_t)((__int128)i * A + (__int128)j * B);
}

// ------------------------------------------------- 64-bit primes, narrow steps
// For primes 2^30 <= p < 2^40 and windows 1024 <= w <= 2^21 the walk's item
// preparation runs mostly in 32-bit arithmetic:
//  * tg_steps_w: the same two steps as tg_steps, from the same run of Euclid's
//    algorithm, but the remainders drop below 2^31 after a few steps, and from
//    there each step is a 32-bit division by a corrected float estimate (partial
//    quotients below 2^31 / w <= 2^21).  Along the run m_(k+1) x_k + m_k x_(k+1)
//    = p, so every m_(k+1) taken while x_k > w is below p / w < 2^30; only the
//    two final multipliers can be larger (up to about p when the last remainder
//    is tiny), and they are returned in 64 bits.  da and ub are at most w.
//  * first_hit_w: first_hit32's block construction for such p when both steps
//    are below 2^31; the products V0 A are formed modulo 2^64 around a float
//    estimate of their quotient by p (the exact remainder is small), and every
//    other quantity fits 64 signed bits (|Y| < B DA + UB < 2^52, block indices
//    below 2^32 + 2^21, multipliers i A + j B below 2^63).
CS_HD bool tg_steps_w(uint64_t p, uint64_t r, uint32_t w, uint64_t &a, uint32_t &da, uint64_t &b, uint32_t &ub,
                      uint32_t &iters, uint32_t max_iter) {
    uint64_t x_pp = 0, x_prev = p, x = r;
    uint32_t m_pp = 0, m_prev = 0, m = 1;
    uint32_t k = 1;
    const bool small_q64 = p < ((uint64_t)w << 21);
    // 64-bit remainders while the dividend is 2^31 or more
    while (x > w && x_prev >= (1ull << 31)) {
        if (k > max_iter) return false;
        uint64_t c, xn;
        if (small_q64) {
            c = udiv_q21_64(x_prev, x, rcp_approx(u64_to_f(x)), xn);
        } else {
            c = x_prev / x;
            xn = x_prev - c * x;
        }
        const uint32_t mn = m_prev + (uint32_t)c * m;
        x_pp = x_prev; m_pp = m_prev;
        x_prev = x; m_prev = m;
        x = xn; m = mn;
        k++;
    }
    // 32-bit remainders: dividend below 2^31, quotients below 2^21
    if (x > w) {
        uint32_t xp = (uint32_t)x_prev, xc = (uint32_t)x;
        while (xc > w) {
            if (k > max_iter) return false;
            uint32_t rem;
            const uint32_t c = udiv_q21(xp, xc, rcp_approx((float)xc), rem);
            const uint32_t mn = m_prev + c * m;
            x_pp = xp; m_pp = m_prev;
            xp = xc; m_prev = m;
            xc = rem; m = mn;
            k++;
        }
        x_prev = xp;
        x = xc;
    }
    iters += k;
    uint64_t ms;                                     // first m with the sign of x_K
    uint32_t xs;
    if (k == 1) {
        ms = 1;
        xs = (uint32_t)r;
    } else {
        // t = ceil((x_pp - w) / x_prev), a quotient below x_pp / x_prev + 1
        uint64_t t;
        if (x_pp < (1ull << 30)) {
            uint32_t rem;
            t = udiv_q21((uint32_t)(x_pp - w + x_prev - 1), (uint32_t)x_prev, rcp_approx((float)(uint32_t)x_prev), rem);
        } else if (small_q64) {
            uint64_t rem;
            t = udiv_q21_64(x_pp - w + x_prev - 1, x_prev, rcp_approx(u64_to_f(x_prev)), rem);
        } else {
            t = (x_pp - w + x_prev - 1) / x_prev;
        }
        ms = m_pp + t * m_prev;
        xs = (uint32_t)(x_pp - t * x_prev);
    }
    // the other sign: t2 = ceil((x_prev - w) / x), unbounded when x is small
    const uint64_t num = x_prev - w + x - 1;
    const uint64_t t2 = (num >> 32) == 0 ? (uint64_t)((uint32_t)num / (uint32_t)x) : num / x;
    const uint64_t mo = m_prev + t2 * m;
    const uint32_t xo = (uint32_t)(x_prev - t2 * x);
    if (k & 1) {
        b = ms; ub = xs; a = mo; da = xo;
    } else {
        a = ms; da = xs; b = mo; ub = xo;
    }
    return true;
}

// floor(x / d) for |x| < 2^62, 1 <= d < 2^31 and |x / d| < 2^40, given
// fd = rcp_rn((float)d): the first float estimate is within a relative 2^-21,
// i.e. 2^19 + 1, of the quotient, so the remainder of its truncation is below
// 2^50 d in magnitude and exact; the second estimate, on that remainder, is
// within 1.25, and one correction each way makes the quotient exact.
CS_HD int64_t floor_div_s64(int64_t x, uint32_t d, float fd) {
    int64_t q = f_to_s64(s64_to_f(x) * fd);
    int64_t r = x - q * (int64_t)d;
    const int64_t q1 = f_to_s64(s64_to_f(r) * fd);
    q += q1;
    r -= q1 * (int64_t)d;
    if (r < 0) { r += d; q--; }
    if (r < 0) { r += d; q--; }
    if (r >= (int64_t)d) { r -= d; q++; }
    if (r >= (int64_t)d) { r -= d; q++; }
    return q;
}

// first_hit32 for 2^30 <= p < 2^40, 1024 <= w <= 2^21 and steps a, b below
// 2^31 (da, ub <= w), given fp = rcp_rn(u64_to_f(p)); w < v0 < p.
CS_HD uint64_t first_hit_w(uint64_t p, float fp, uint32_t w, uint32_t a, uint32_t da, uint32_t b, uint32_t ub,
                           uint64_t v0, uint32_t &y_out) {
    const bool sw = da > ub;
    const uint32_t A = sw ? b : a, DA = sw ? ub : da, B = sw ? a : b, UB = sw ? da : ub;
    const int64_t V0 = sw ? (int64_t)w - (int64_t)v0 : (int64_t)v0;     // |V0| < 2^40
    // aq = floor(|V0| A / p) < A < 2^31: a float estimate within 1536 of it
    // (relative 1.5 2^-21), the remainder of |V0| A taken modulo 2^64 (exact:
    // it is below 1537 p < 2^51 in magnitude), one refinement within one, and
    // one correction each way
    const uint64_t av = (uint64_t)(V0 < 0 ? -V0 : V0);
    uint32_t aq = (uint32_t)(u64_to_f(av) * (float)A * fp);
    int64_t rem = (int64_t)(av * (uint64_t)A - (uint64_t)aq * p);
    const int32_t q1 = (int32_t)(s64_to_f(rem) * fp);
    aq += (uint32_t)q1;
    rem -= (int64_t)q1 * (int64_t)p;
    if (rem < 0) { rem += (int64_t)p; aq--; }
    if (rem < 0) { rem += (int64_t)p; aq--; }
    if (rem >= (int64_t)p) { rem -= (int64_t)p; aq++; }
    int64_t j = V0 >= 0 ? -(int64_t)aq : (int64_t)aq + (rem != 0);
    int64_t Y = V0 + j * (int64_t)UB;
    const float fda = rcp_rn((float)DA);
    if (floor_div_s64(Y, DA, fda) * (int64_t)A + j * (int64_t)B < 0) {
        j++;
        Y += UB;
    }
    int64_t i = -floor_div_s64((int64_t)w - Y, DA, fda);                // ceil((Y - w) / DA)
    const int64_t t_lo = i * (int64_t)A + j * (int64_t)B;
    if (t_lo < 0) {
        // ceil(-t_lo / A) steps of A: a quotient below w / DA + 2 <= 2^21 + 2
        const int64_t n = -t_lo;
        int64_t q = (int64_t)(uint32_t)(u64_to_f((uint64_t)n) * rcp_rn((float)A));
        int64_t r = n - q * (int64_t)A;
        if (r < 0) { r += A; q--; }
        if (r < 0) { r += A; q--; }
        if (r >= (int64_t)A) { r -= A; q++; }
        if (r >= (int64_t)A) { r -= A; q++; }
        i += q + (r != 0);
    }
    const uint32_t y = (uint32_t)(Y - i * (int64_t)DA);
    y_out = sw ? w - y : y;
    return (uint64_t)(i * (int64_t)A + j * (int64_t)B);
}

// ------------------------------------------------------------- checksum
CS_HD uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
static constexpr uint64_t kHashStep = 0x9E3779B97F4A7C15ull;

}  // namespace cs
