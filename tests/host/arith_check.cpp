// Host build of the kernels' integer arithmetic (cs_arith.cuh) for CPU tests:
// reads "p K L R" lines, prints "m y" from g_solve (32- or 64-bit).  Mode "r"
// checks the prime generator's division-free R^2 mod p and (r M + s) mod p;
// mode "f" the walk's
// first hit from the three-gap basis; mode "s" the walk's two steps from
// Euclid's algorithm; mode "l" the generator's lazily reduced Montgomery
// product; mode "u" the float-estimate division of 64-bit numerators; mode "F"
// the first hit for 64-bit primes; mode "e" (and "E", 64-bit) the Euclid steps'
// small-quotient division; mode "k" K's factor words; mode "R" the 64-bit
// residue kernel's division-free R^2 mod p, M mod p and R^e mod p; mode "W"
// the narrow-step Euclid run and first hit for 64-bit primes; mode "X" the
// status of a sieve's device error flags.
#include <cstdio>
#include <cstdint>
#include "../../paper_2012_03771_gb300/csrc/cs_arith.cuh"
#include "../../paper_2012_03771_gb300/csrc/cs_words.h"
#include "../../paper_2012_03771_gb300/csrc/cs_errors.h"

int main(int argc, char **argv) {
    const bool narrow = argc > 1 && argv[1][0] == 'n';
    if (argc > 1 && argv[1][0] == 'r') {
        // "p M r s" -> R^2 mod p (division-free) and (r M + s) mod p via mont32_affine
        unsigned long long p, M, r, s;
        while (scanf("%llu %llu %llu %llu", &p, &M, &r, &s) == 4) {
            const uint32_t p32 = (uint32_t)p, pinv = cs::mont32_neg_inv(p32);
            const uint32_t r2 = cs::mont32_r2_fast(p32);
            const uint32_t rt = cs::mont32_mul((uint32_t)r, r2, p32, pinv);
            printf("%u %u\n", r2, cs::mont32_affine(rt, M, (uint32_t)s, r2, p32, pinv));
        }
        return 0;
    }
    if (argc > 1 && argv[1][0] == 'X') {
        // "flags" -> the status cs_sync reports for a sieve's device error word, and its message
        unsigned long long f;
        while (scanf("%llu", &f) == 1) {
            const char *msg = nullptr;
            const int st = cs::status_of_device_errors(f, &msg);
            printf("%d %s\n", st, msg);
        }
        return 0;
    }
    if (argc > 1 && argv[1][0] == 'R') {
        // "p M" -> R^2 mod p (R = 2^64) without a division, M mod p by one float
        // quotient (M / p < 2^20), then R^e mod p for e = 1 .. 40 from R^2 alone
        unsigned long long p, M;
        while (scanf("%llu %llu", &p, &M) == 2) {
            const float fp = cs::rcp_rn(cs::u64_to_f(p));
            const uint64_t pinv = cs::mont64_neg_inv(p);
            const uint64_t r2 = cs::mont64_r2_fast(p, fp);
            printf("%llu %llu", (unsigned long long)r2, (unsigned long long)cs::mod_q20(M, p, fp));
            for (uint32_t e = 1; e <= 40; e++)
                printf(" %llu", (unsigned long long)cs::mont64_rpow2(e, r2, p, pinv));
            printf("\n");
        }
        return 0;
    }
    if (argc > 1 && argv[1][0] == 'W') {
        // "p r w v0" -> the narrow-step Euclid run and first hit for 64-bit primes,
        // beside the general 64-bit ones: ok a da b ub | ok a da b ub | t y | t y
        // (the first hits only when both steps are below 2^31, else "- -")
        unsigned long long p, r, w, v0;
        while (scanf("%llu %llu %llu %llu", &p, &r, &w, &v0) == 4) {
            uint64_t a, b, a2, da2, b2, ub2;
            uint32_t da, ub, it = 0, it2 = 0;
            const bool ok = cs::tg_steps_w(p, r, (uint32_t)w, a, da, b, ub, it, 400);
            const bool ok2 = cs::tg_steps<uint64_t>(p, r, w, a2, da2, b2, ub2, it2, 400);
            printf("%d %llu %u %llu %u %d %llu %llu %llu %llu", ok, (unsigned long long)a, da,
                   (unsigned long long)b, ub, ok2, (unsigned long long)a2, (unsigned long long)da2,
                   (unsigned long long)b2, (unsigned long long)ub2);
            if (ok && a < (1ull << 31) && b < (1ull << 31)) {
                uint32_t y;
                uint64_t y2;
                const uint64_t t = cs::first_hit_w(p, cs::rcp_rn(cs::u64_to_f(p)), (uint32_t)w, (uint32_t)a, da,
                                                   (uint32_t)b, ub, v0, y);
                const uint64_t t2 = cs::first_hit64(p, w, a2, da2, b2, ub2, v0, y2);
                printf(" %llu %u %llu %llu\n", (unsigned long long)t, y, (unsigned long long)t2,
                       (unsigned long long)y2);
            } else {
                printf(" - - - -\n");
            }
        }
        return 0;
    }
    if (argc > 1 && argv[1][0] == 'F') {
        // "p r w v0" -> first hit from the three-gap basis, 64-bit (p < 2^40)
        unsigned long long p, r, w, v0;
        while (scanf("%llu %llu %llu %llu", &p, &r, &w, &v0) == 4) {
            uint64_t a, da, b, ub;
            uint32_t it = 0;
            bool ok = cs::tg_steps<uint64_t>(p, r, w, a, da, b, ub, it, 400);
            uint64_t y = 0;
            const uint64_t t = cs::first_hit64(p, w, a, da, b, ub, v0, y);
            printf("%d %llu %llu\n", ok, (unsigned long long)t, (unsigned long long)y);
        }
        return 0;
    }
    if (argc > 1 && argv[1][0] == 'e') {
        // "a b" -> floor(a / b) and a mod b from udiv_q21, with the reciprocal
        // exact and off by a relative -2^-23 and +2^-23 (the device's approximate one)
        unsigned long long a, b;
        while (scanf("%llu %llu", &a, &b) == 2) {
            const float rb = 1.0f / (float)b;
            const float lo = rb * (1.0f - 1.1920929e-07f), hi = rb * (1.0f + 1.1920929e-07f);
            uint32_t r0, r1, r2;
            const uint32_t q0 = cs::udiv_q21((uint32_t)a, (uint32_t)b, rb, r0);
            const uint32_t q1 = cs::udiv_q21((uint32_t)a, (uint32_t)b, lo, r1);
            const uint32_t q2 = cs::udiv_q21((uint32_t)a, (uint32_t)b, hi, r2);
            printf("%u %u %u %u %u %u\n", q0, r0, q1, r1, q2, r2);
        }
        return 0;
    }
    if (argc > 1 && argv[1][0] == 'k') {
        // "n q_1 ... q_n" -> the words below 2^31, then the words below 2^64, one line each
        unsigned n;
        while (scanf("%u", &n) == 1) {
            std::vector<uint32_t> q(n), w32;
            std::vector<uint64_t> w64;
            for (unsigned i = 0; i < n; i++) scanf("%u", &q[i]);
            cs::pack_k_words(q, w32, w64);
            for (uint32_t w : w32) printf("%u ", w);
            printf("\n");
            for (uint64_t w : w64) printf("%llu ", (unsigned long long)w);
            printf("\n");
        }
        return 0;
    }
    if (argc > 1 && argv[1][0] == 'E') {
        // "a b" -> floor(a / b) and a mod b from udiv_q21_64, with the reciprocal
        // of u64_to_f(b) exact and off by a relative -2^-23 and +2^-23
        unsigned long long a, b;
        while (scanf("%llu %llu", &a, &b) == 2) {
            const float rb = 1.0f / cs::u64_to_f(b);
            const float lo = rb * (1.0f - 1.1920929e-07f), hi = rb * (1.0f + 1.1920929e-07f);
            uint64_t r0, r1, r2;
            const uint64_t q0 = cs::udiv_q21_64(a, b, rb, r0);
            const uint64_t q1 = cs::udiv_q21_64(a, b, lo, r1);
            const uint64_t q2 = cs::udiv_q21_64(a, b, hi, r2);
            printf("%llu %llu %llu %llu %llu %llu\n", (unsigned long long)q0, (unsigned long long)r0,
                   (unsigned long long)q1, (unsigned long long)r1, (unsigned long long)q2, (unsigned long long)r2);
        }
        return 0;
    }
    if (argc > 1 && argv[1][0] == 'u') {
        // "n p" -> floor(n / p) and n mod p from the float-estimate division
        unsigned long long n, p;
        while (scanf("%llu %llu", &n, &p) == 2) {
            int64_t rem = 0;
            const uint64_t q = cs::udiv64_est(n, (uint32_t)p, cs::rcp_rn((float)p), rem);
            printf("%llu %lld\n", (unsigned long long)q, (long long)rem);
        }
        return 0;
    }
    if (argc > 1 && argv[1][0] == 'l') {
        // "p a b" -> a b 2^-32 mod p reduced below 2p (a < 2p, b < 2^31)
        unsigned long long p, a, b;
        while (scanf("%llu %llu %llu", &p, &a, &b) == 3)
            printf("%u\n", cs::mont32_mul_lazy((uint32_t)a, (uint32_t)b, (uint32_t)p, cs::mont32_neg_inv((uint32_t)p)));
        return 0;
    }
    if (argc > 1 && argv[1][0] == 's') {
        // "p r w" -> a da b ub from Euclid's algorithm, 32-bit (p < 2^31) and 64-bit
        unsigned long long p, r, w;
        while (scanf("%llu %llu %llu", &p, &r, &w) == 3) {
            uint32_t it = 0;
            unsigned long long a64, da64, b64, ub64;
            uint64_t A, DA, B, UB;
            bool ok64 = cs::tg_steps<uint64_t>(p, r, w, A, DA, B, UB, it, 200);
            a64 = A; da64 = DA; b64 = B; ub64 = UB;
            uint32_t a = 0, da = 0, b = 0, ub = 0;
            bool ok32 = p < (1ull << 31) && cs::tg_steps<uint32_t>((uint32_t)p, (uint32_t)r, (uint32_t)w, a, da, b, ub, it, 200);
            printf("%d %llu %llu %llu %llu %d %u %u %u %u\n", ok64, a64, da64, b64, ub64, ok32, a, da, b, ub);
        }
        return 0;
    }
    if (argc > 1 && argv[1][0] == 'f') {
        // "p r w v0" -> first t >= 0 with (v0 + r t) mod p <= w from the three-gap basis
        unsigned long long p, r, w, v0;
        while (scanf("%llu %llu %llu %llu", &p, &r, &w, &v0) == 4) {
            uint32_t a, da, b, ub, it = 0;
            bool ok = cs::tg_steps<uint32_t>((uint32_t)p, (uint32_t)r, (uint32_t)w, a, da, b, ub, it, 200);
            uint32_t y = 0;
            const uint32_t t = cs::first_hit32((uint32_t)p, cs::rcp_rn((float)p), (uint32_t)w, a, da, b, ub,
                                               (uint32_t)v0, y);
            printf("%d %u %u\n", ok, t, y);
        }
        return 0;
    }
    unsigned long long p, K, L, R;
    while (scanf("%llu %llu %llu %llu", &p, &K, &L, &R) == 4) {
        uint32_t it = 0;
        if (narrow) {
            uint32_t m = 0, y = 0;
            bool ok = cs::g_solve<uint32_t, int32_t>((uint32_t)p, (uint32_t)(K % p), (uint32_t)L,
                                                     (uint32_t)(R - L), m, y, it, 200);
            printf("%d %u %u\n", ok, m, y);
        } else {
            uint64_t m = 0, y = 0;
            bool ok = cs::g_solve<uint64_t, int64_t>(p, K % p, L, R - L, m, y, it, 300);
            printf("%d %llu %llu\n", ok, (unsigned long long)m, (unsigned long long)y);
        }
    }
    return 0;
}
