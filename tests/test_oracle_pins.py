"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: the expected values are printed
in the paper (tests/golden/*, each with its section), come from a closed form,
from brute force with Python integers, or from an independent library routine.
"""
import math
import random

import numpy as np
import pytest

import oracle.oracle as O
from paper_2012_03771_gb300 import workloads
from tests.conftest import read_golden


def _K(P, d):
    return math.prod(q for q in O._simple_primes(P) if d % q)


def _fermat(n):
    return pow(2, n - 1, n) == 1


# ------------------------------------------------------------------ G

def _G_closed_form(p, K, L, R):
    """min over target values y in [L, R] of y * K^-1 mod p: the smallest m with
    m*K mod p = y, minimised over the window (valid because gcd(K, p) = 1)."""
    inv = pow(K, -1, p)
    return min((y * inv) % p for y in range(L, R + 1))


def test_G_exhaustive_small_primes():
    """Eq. modsol against trying every m, for every K, L <= R below small primes."""
    for p in (3, 5, 7, 11, 13, 17, 19, 23, 29, 31):
        for K in range(1, p):
            for L in range(0, p):
                for R in range(L, p):
                    assert O.G(p, K, L, R) == O.G_brute(p, K, L, R), (p, K, L, R)


def test_G_random_large_against_closed_form():
    """Random 20- to 40-bit primes, narrow windows: result is in the window and
    equals the minimum over the window's values of y*K^-1 mod p."""
    rng = random.Random(12)
    big_primes = [1000003, 999999937, 2**31 - 1, 1099511627689, 68719476731, 4294967291]
    for _ in range(400):
        p = rng.choice(big_primes)
        K = rng.randrange(1, p)
        w = rng.randrange(0, 300)
        L = rng.randrange(0, p - w)
        R = L + w
        m = O.G(p, K, L, R)
        assert L <= (m * K) % p <= R
        assert m == _G_closed_form(p, K, L, R)


def test_G_reduces_K_at_least_p():
    """Case B: K >= p behaves as K mod p."""
    assert O.G(101, 101 + 7, 30, 35) == O.G(101, 7, 30, 35) == O.G_brute(101, 7, 30, 35)


def test_large_prime_walk_equals_traditional_hits():
    """Section 3.2: repeated solves of Eq. modeq enumerate exactly the (m, x)
    that the traditional per-m computation finds, for p > 2*SL."""
    rng = random.Random(5)
    P, d, SL = 37, 6, 40
    K = _K(P, d)
    for p in (83, 97, 211, 1009, 7919, 104729):
        r = K % p
        M_start, M_inc = rng.randrange(1, 10**6), 3000
        hits, solves = O.large_prime_walk(p, r, M_start, M_inc, SL)
        expect = []
        for m in range(M_start, M_start + M_inc):
            n = (m * K) % p
            for x in range(-SL, SL + 1):
                if (n + x) % p == 0:
                    expect.append((m, x))
        assert hits == expect
        # one solve per hit-run plus the final one that leaves the range
        assert len(hits) <= solves + len(hits) <= 2 * len(hits) + 1


# ------------------------------------------------------ structure, K mod p

def test_k_mod_p_against_python_bignum():
    rng = random.Random(3)
    for P, d in ((503, 210), (953, 210), (1019, 2310), (37, 30), (7, 210), (1, 1)):
        K = _K(P, d)
        ps = [p for p in O._simple_primes(20000) if p > P][:200]
        ps += [999999937, 1099511627689, 4294967291, 68719476731]
        ps += [rng.randrange(2, 2**40) | 1 for _ in range(50)]
        assert [K % p for p in ps] == list(O.k_mod_p(P, d, ps))


def test_columns_and_rows_definitions():
    P, d, SL = 37, 30, 200
    K = _K(P, d)
    xs = [x for x in range(-SL, SL + 1) if x and math.gcd(abs(x), K) == 1]
    assert list(O.columns(P, d, SL)) == xs
    assert list(O.columns(1, 1, 5)) == list(range(-5, 6))          # K = 1 keeps x = 0
    assert list(O.rows(30, 100, 50)) == [m for m in range(100, 150) if math.gcd(m, 30) == 1]
    # the configured workloads: widths used by the layout
    assert len(O.columns(503, 210, 7000)) == 4700
    assert len(O.columns(953, 210, 20000)) == 13102
    assert len(O.rows(210, 1, 1000)) == 228


def test_validation_rejects():
    assert O.validate(503, 210, 1, 10, 100, 10**6) == 0
    assert O.validate(503, 4, 1, 10, 100, 10**6) == O.EINVAL          # not squarefree
    assert O.validate(7, 11, 1, 10, 100, 10**6) == O.EINVAL           # 11 does not divide 7#
    assert O.validate(503, 210, 0, 10, 100, 10**6) == O.EINVAL        # m = 0
    assert O.validate(1, 1, 5, 10, 4, 100) == O.EINVAL                # N + x = 1 reachable
    assert O.validate(1, 1, 6, 10, 4, 100) == 0                       # N + x >= 2
    assert O.validate(503, 210, 1, 10, 100, 2**40 + 1) == O.EINVAL    # L too large
    assert O.validate(503, 210, 1, 10, 2**20 + 1, 10**6) == O.EINVAL  # SL too large
    assert O.validate(503, 0, 1, 10, 100, 10**6) == O.EINVAL


# ---------------------------------------------------- brute force (tiny)

def test_sieve_matches_bignum_trial_division():
    """Every stored (m, x) of tiny parameter sets, with Python integers and no
    cached residues: bits, row order, column order and F."""
    n_valid = 0
    for prm in workloads.tiny_cases(120):
        args = prm.as_tuple()
        if O.validate(*args):
            continue
        n_valid += 1
        for wheel in (True, False):
            ms, xs, grid, F = O.brute_force_bits(*args, wheel=wheel)
            m, bits, Fr = O.full_sieve(*args, wheel=wheel)
            assert list(m) == ms
            assert list(O.columns(prm.P, prm.d, prm.SL)) == xs
            expect = O.pack_rows(grid, len(xs))
            assert bits.shape == expect.shape
            assert np.array_equal(bits, expect), prm
            assert int(Fr.sum()) == F, prm
    assert n_valid > 60


def test_prime_survives_when_it_is_a_sieving_prime():
    """N + x = p is not cleared by p itself (p is prime); K = 1001 = 7*11*13."""
    P, d, M_start, SL, L = 13, 30, 1, 300, 2000
    m, bits, F = O.full_sieve(P, d, M_start, 1, SL, L)
    xs = O.columns(P, d, SL)
    row = O.unpack_row(bits[0], len(xs))
    for j, x in enumerate(xs):
        n = 1001 + int(x)
        is_p = n > 1 and all(n % q for q in range(2, int(n**0.5) + 1))
        assert row[j] == is_p, (x, n)


# ------------------------------------------ K = d = 1: survivors are primes

def test_degenerate_K1_survivors_are_primes_and_first_gaps():
    """K = d = 1, one interval [2, 400000] with L >= sqrt(400000): the survivors
    are exactly the primes, which gives the first-occurrence gaps of Section 1."""
    sympy = pytest.importorskip("sympy")
    SL = 199_999
    m, bits, F = O.full_sieve(1, 1, SL + 2, 1, SL, 1000)
    xs = O.columns(1, 1, SL)
    row = O.unpack_row(bits[0], len(xs))
    survivors = [SL + 2 + int(x) for x, b in zip(xs, row) if b]
    assert survivors == list(sympy.primerange(2, 2 * SL + 3))
    gaps = {}
    for a, b in zip(survivors, survivors[1:]):
        gaps.setdefault(b - a, a)
    for gap, first in read_golden("first_gaps.txt"):
        assert gaps[int(gap)] == int(first)


def test_degenerate_K1_many_rows():
    sympy = pytest.importorskip("sympy")
    M_start, M_inc, SL = 1000, 40, 500
    m, bits, F = O.full_sieve(1, 1, M_start, M_inc, SL, 100)     # 100 > sqrt(1540)
    xs = O.columns(1, 1, SL)
    for i, mm in enumerate(m):
        row = O.unpack_row(bits[i], len(xs))
        got = [int(mm) + int(x) for x, b in zip(xs, row) if b]
        assert got == list(sympy.primerange(int(mm) - SL, int(mm) + SL + 1))


# -------------------------------------- Section 3.2 printed hit fractions

def test_hit_fractions_printed_in_section_3_2():
    """X = 100000, N = 503#/210: primes dividing a number of [N - X, N + X]."""
    P, d, SL = 503, 210, 100_000
    small = len(O._simple_primes(P))   # p <= P always divide some N + x (p <= S)
    for lo, hi, hitting, total in read_golden("hit_fractions_503.txt"):
        lo, hi, hitting, total = int(lo), int(hi), int(hitting), int(total)
        count, _, _ = O.prime_stats(lo, hi)
        _, _, n_hit = O.sieve(P, d, SL, hi, [1], p_lo=lo, wheel=False)
        if lo < P:
            n_hit += small                 # the sieve itself only runs p > P
        assert count == total
        assert n_hit == hitting


# ---------------------------------------------- Section 4.1 Mertens table

def test_mertens_table():
    for L, n_primes, theo, exp in read_golden("mertens_table.txt"):
        L, n_primes, theo = int(L), int(n_primes), float(theo)
        decimals = len(exp.split(".")[1])
        count, log_prod, _ = O.prime_stats(0, L)
        assert count == n_primes
        assert abs(math.exp(log_prod) - float(exp)) <= 0.5 * 10**-decimals + 1e-12
        assert abs(1 / (math.log(L) * math.exp(0.5772156649015329)) - theo) <= 0.5e-6


def test_survivor_density_tracks_mertens_product():
    """Without the wheel, survivors over stored cells ~ prod_{P<p<=L}(1-1/p)
    (Eq. sieveeffic restricted to the sieving primes), and F / cells ~ sum 1/p."""
    prm = workloads.PLAIN_503
    m, bits, F = O.full_sieve(*prm.as_tuple(), wheel=False)
    W = len(O.columns(prm.P, prm.d, prm.SL))
    cells = len(m) * W
    surv = int(O.row_counts(bits).sum())
    _, log_prod, inv_sum = O.prime_stats(prm.P, prm.L)
    expect = math.exp(log_prod)
    sigma = math.sqrt(cells * expect * (1 - expect))
    assert abs(surv - cells * expect) < 6 * sigma
    assert abs(int(F.sum()) / cells - inv_sum) < 0.01 * inv_sum


def test_wheel_alone_is_gcd_with_d():
    """With no sieving primes (L = P) a cell survives iff gcd(N + x, d) = 1."""
    P, d, M_start, M_inc, SL = 37, 210, 1, 40, 150
    K = _K(P, d)
    m, bits, F = O.full_sieve(P, d, M_start, M_inc, SL, P)
    xs = O.columns(P, d, SL)
    assert int(F.sum()) == 0
    for i, mm in enumerate(m):
        row = O.unpack_row(bits[i], len(xs))
        expect = [int(math.gcd(int(mm) * K + int(x), d) == 1) for x in xs]
        assert list(row) == expect


def test_cleared_cells_have_a_sieving_factor():
    """Every cleared cell of some rows of the small search has a divisor in
    (P, L] (checked with Python big integers); every survivor has none."""
    prm = workloads.PLAIN_503
    K = _K(prm.P, prm.d)
    m_all = O.rows(prm.d, prm.M_start, prm.M_inc)
    pick = [int(m_all[i]) for i in (0, 77, 227)]
    bits, F, _ = O.sieve(prm.P, prm.d, prm.SL, prm.L, pick, wheel=False)
    xs = O.columns(prm.P, prm.d, prm.SL)
    sp = O.primes(prm.P, prm.L).astype(np.int64)
    kmod = np.array([K % int(p) for p in sp], dtype=np.int64)
    SL = prm.SL
    stored = np.zeros(2 * SL + 1, dtype=bool)
    stored[xs + SL] = True
    small = sp[sp <= 2 * SL]
    for i, mm in enumerate(pick):
        row = O.unpack_row(bits[i], len(xs))
        nmod = (kmod * (mm % sp)) % sp                    # N mod p, numpy int64 (p < 2^24)
        for x, alive in zip(xs[::23], row[::23]):
            has = bool(np.any((nmod + int(x)) % sp == 0))
            assert has == (not alive)
        # F of the row: stored x = -N (mod p) in [-SL, SL], counted per prime
        t = (-nmod) % sp                                  # smallest x >= 0 with p | N + x
        big = sp > 2 * SL
        fr = int(np.count_nonzero(big & (t <= SL) & stored[np.minimum(t, SL) + SL]))
        lo = t - sp
        fr += int(np.count_nonzero(big & (lo >= -SL) & stored[np.maximum(lo, -SL) + SL]))
        for p, tt in zip(small, t[: small.size]):
            start = int(tt) - int(p) * ((int(tt) + SL) // int(p))
            fr += int(np.count_nonzero(stored[start + SL::int(p)]))
        assert fr == int(F[i])


# ------------------------------------------------- Section 1.1 record rows

@pytest.mark.parametrize("which", [0, 1])
def test_record_gap_rows(which):
    """The published gaps: the lower prime survives, the upper one too when it
    is inside the interval, and no survivor strictly inside the gap passes a
    base-2 Fermat test (the gap has no primes)."""
    P, d, m, x_lo, gap = (int(v) for v in read_golden("record_gaps.txt")[which])
    SL, L = (20_000, 10**9) if which == 0 else (25_000, 10**8)
    assert math.gcd(m, d) == 1
    bits, F, _ = O.sieve(P, d, SL, L, [m])
    xs = O.columns(P, d, SL)
    row = O.unpack_row(bits[0], len(xs))
    alive = {int(x) for x, b in zip(xs, row) if b}
    N = m * _K(P, d)
    assert x_lo in alive and _fermat(N + x_lo)
    x_hi = x_lo + gap
    if x_hi <= SL:
        assert x_hi in alive and _fermat(N + x_hi)
    inside = [x for x in alive if x_lo < x < min(x_hi, SL + 1)]
    assert inside and not any(_fermat(N + x) for x in inside)


# ----------------------------------------------------------------- hash

def test_hash_properties():
    rng = np.random.default_rng(0)
    bits = rng.integers(0, 2**63, size=(7, 5), dtype=np.uint64)
    h = O.bitset_hash(bits)
    # additive over row blocks with the global row offset
    assert h == (O.bitset_hash(bits[:3]) + O.bitset_hash(bits[3:], row0=3)) % 2**64
    # any single bit flip changes it; moving a word changes it
    for _ in range(50):
        b2 = bits.copy()
        i, w, k = rng.integers(7), rng.integers(5), rng.integers(64)
        b2[i, w] ^= np.uint64(1 << int(k))
        assert O.bitset_hash(b2) != h
    b3 = bits.copy()
    b3[[0, 1]] = b3[[1, 0]]
    assert O.bitset_hash(b3) != h
    assert list(O.row_counts(bits)) == [sum(bin(int(v)).count("1") for v in r) for r in bits]


def test_compact_layout_is_the_wheel_survivor_subset():
    """Compact rows hold exactly the literal columns with gcd(N + x, d) = 1, in
    order; their popcount equals the literal row's (the wheel cleared the rest)."""
    P, d, M_start, M_inc, SL, L = 37, 210, 1000, 60, 300, 4000
    K = _K(P, d)
    m, bits, F = O.full_sieve(P, d, M_start, M_inc, SL, L)
    comp, W_max, cols = O.compact_layout(P, d, SL, m, bits)
    assert list(O.row_counts(comp)) == list(O.row_counts(bits))
    xs = O.columns(P, d, SL)
    for i, mm in enumerate(m):
        expect = [int(x) for x in xs if math.gcd(int(mm) * K + int(x), d) == 1]
        assert [int(x) for x in cols[i]] == expect
        row = O.unpack_row(comp[i], len(expect))
        lit = dict(zip((int(x) for x in xs), O.unpack_row(bits[i], len(xs))))
        assert list(row) == [lit[x] for x in expect]
    assert W_max == max(sum(1 for x in xs if math.gcd(rho * K + int(x), d) == 1)
                        for rho in range(d) if math.gcd(rho, d) == 1)
