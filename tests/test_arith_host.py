"""The kernels' solver arithmetic (cs_arith.cuh), compiled for the host with
g++, against the paper's recursion G of Section 3.3 in the oracle."""
import math
import os
import random
import subprocess

import pytest

import oracle.oracle as O
from tests.conftest import ROOT

SRC = os.path.join(ROOT, "tests", "host", "arith_check.cpp")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("arith") / "arith_check")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-o", out, SRC])
    return out


@pytest.mark.parametrize("narrow", [True, False])
def test_g_solve_matches_paper_recursion(exe, narrow):
    rng = random.Random(7 + narrow)
    pool = [7, 101, 7919, 1000003, 999999937, (1 << 30) - 35] if narrow else \
           [7, 1000003, 4294967291, 68719476731, 1099511627689]
    cases = []
    for _ in range(3000):
        p = rng.choice(pool)
        K = rng.randrange(1, p)
        w = min(rng.choice([0, 1, 5, 300, 40000, rng.randrange(0, p)]), p - 1)
        L = rng.randrange(0, p - w)
        cases.append((p, K, L, L + w))
    inp = "".join(f"{p} {K} {L} {R}\n" for p, K, L, R in cases)
    out = subprocess.run([exe, "n" if narrow else "w"], input=inp, capture_output=True, text=True,
                         check=True).stdout.split("\n")
    for (p, K, L, R), line in zip(cases, out):
        ok, m, y = (int(v) for v in line.split())
        g = O.G(p, K, L, R)
        assert ok and (m, y) == (g, g * K % p), (p, K, L, R)


def test_narrow_steps_and_first_hit_64(exe):
    """For 2^30 <= p < 2^40 and 1024 <= 2SL <= 2^21: the Euclid run with 32-bit
    steps below 2^31 gives the same two steps as the general 64-bit run, and the
    first hit from them (64-bit products modulo 2^64 around float quotients)
    equals the general first hit and the paper's G of the window, on random
    residues and on the edge cases r = 1, r = p - 1, residues next to the window
    and tiny last remainders."""
    rng = random.Random(41)
    ps = [(1 << 30) + 3, (1 << 31) - 1, (1 << 32) + 15, 99999999977, 100000000003, (1 << 37) - 25,
          (1 << 40) - 87]
    cases = []
    for _ in range(20000):
        p = rng.choice(ps) if rng.random() < 0.2 else rng.randrange(1 << 30, 1 << 40) | 1
        w = rng.choice([1024, 1025, 4000, 40000, 50000, 2 * rng.randrange(512, 1 << 20), 1 << 21])
        w = min(w, p - 2)
        kind = rng.random()
        if kind < 0.05:
            r = rng.choice([1, 2, p - 1, p - 2, w, w + 1, p - w])
        elif kind < 0.1:
            # r just above a multiple of p / k, so that some remainder is tiny
            k = rng.randrange(1, 1000)
            r = (p * rng.randrange(1, k + 1)) // k + rng.randrange(-3, 4)
        else:
            r = rng.randrange(1, p)
        r = min(max(r, 1), p - 1)
        if math.gcd(r, p) != 1:
            continue
        v0 = rng.choice([w + 1, p - 1, rng.randrange(w + 1, p)])
        cases.append((p, r, w, v0))
    inp = "".join(f"{p} {r} {w} {v0}\n" for p, r, w, v0 in cases)
    out = subprocess.run([exe, "W"], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    n_fast = 0
    for (p, r, w, v0), line in zip(cases, out):
        f = line.split()
        assert f[0] == "1" and f[5] == "1", (p, r, w)
        assert [int(x) for x in f[1:5]] == [int(x) for x in f[6:10]], (p, r, w)
        if f[10] != "-":
            n_fast += 1
            t, y, t2, y2 = (int(x) for x in f[10:14])
            g = O.G(p, r, p - v0, p - v0 + w)
            assert (t, y) == (t2, y2) == (g, (v0 + r * g) % p), (p, r, w, v0)
    assert n_fast > 0.9 * len(cases)


def test_device_error_flags_map_to_one_status(exe):
    """The error word a sieve's kernels leave behind (bounded waits and
    capacity checks set flags instead of trapping) becomes one status in
    cs_sync: a prime-buffer overflow first (the result lacks primes), then a
    solver that ran out of passes, then a staging copy that timed out."""
    cases = {0: (0, ""), 1: (-7, "prime buffer overflow"), 2: (-3, "modular solver"),
             4: (-4, "staging copy"), 3: (-7, "prime buffer"), 6: (-3, "modular solver"),
             5: (-7, "prime buffer"), 8: (-3, "unknown")}
    out = subprocess.run([exe, "X"], input="".join(f"{f}\n" for f in cases), capture_output=True, text=True,
                         check=True).stdout.split("\n")
    for (f, (st, msg)), line in zip(cases.items(), out):
        code, _, text = line.partition(" ")
        assert int(code) == st and msg in text, (f, line)


def test_division_free_montgomery_constants_64(exe):
    """R^2 mod p for R = 2^64 from float quotient estimates (odd p in
    [2^20, 2^40); the 64 doublings below), M mod p from one float quotient
    (M / p < 2^20), and R^e mod p for e = 1..40 from R^2 alone, against exact
    integers."""
    rng = random.Random(31)
    ps = [(1 << 20) + 1, (1 << 20) + 7, (1 << 30) - 35, (1 << 30) + 3, (1 << 32) - 5, (1 << 32) + 15,
          (1 << 40) - 87, (1 << 40) - 1, 99999999977, 100000000003, 3, 1000003]
    ps += [rng.randrange(1 << 20, 1 << 40) | 1 for _ in range(20000)]
    ps += [rng.randrange(1 << 39, 1 << 40) | 1 for _ in range(2000)]
    cases = []
    for p in ps:
        hi = min(p * (1 << 20) - 1, (1 << 61) - 1)
        M = rng.choice([0, 1, p - 1, p, p + 1, rng.randrange(0, p), rng.randrange(0, hi + 1), hi])
        cases.append((p, M))
    inp = "".join(f"{p} {M}\n" for p, M in cases)
    out = subprocess.run([exe, "R"], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for (p, M), line in zip(cases, out):
        v = [int(t) for t in line.split()]
        assert v[0] == pow(2, 128, p), p
        if p >= 1 << 20:
            assert v[1] == M % p, (p, M)
        assert v[2:] == [pow(2, 64 * e, p) for e in range(1, 41)], p


def test_division_free_montgomery_constants(exe):
    """R^2 mod p (R = 2^32) from float-reciprocal quotient estimates, and
    (r M + s) mod p from two Montgomery products, against exact integers, for
    odd p across [3, 2^31) (the estimate is used from 2^20 up), M up to 2^40."""
    rng = random.Random(13)
    ps = [3, 5, (1 << 20) - 3, (1 << 20) + 7, (1 << 20) + 1, (1 << 30) - 35, (1 << 31) - 1, (1 << 31) - 19]
    ps += [rng.randrange(1 << 20, 1 << 31) | 1 for _ in range(20000)]
    ps += [rng.randrange(3, 1 << 20) | 1 for _ in range(2000)]
    cases = []
    for p in ps:
        M = rng.choice([0, 1, rng.randrange(1, 1 << 32), rng.randrange(1 << 32, 1 << 40), (1 << 40) - 1])
        cases.append((p, M, rng.randrange(0, p), rng.randrange(0, p)))
    inp = "".join(f"{p} {M} {r} {s}\n" for p, M, r, s in cases)
    out = subprocess.run([exe, "r"], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for (p, M, r, s), line in zip(cases, out):
        r2, v = (int(t) for t in line.split())
        assert r2 == pow(2, 64, p), p
        assert v == (r * M + s) % p, (p, M, r, s)


def test_first_hit_from_three_gap_basis(exe):
    """The walk's first hit without a solve (chain of strip points in the basis
    of the two step vectors) equals the paper's G for the window [p - v0, p - v0 + w],
    including w = 1 and w = 2^21 (the largest 2SL), v0 = w + 1 and v0 = p - 1,
    steps of one residue, and primes up to 2^30."""
    rng = random.Random(17)
    pool = [5, 7, 101, 7919, 104729, 1000003, 999999937, (1 << 30) - 35]
    cases = []
    for _ in range(20000):
        p = rng.choice(pool)
        r = rng.randrange(1, p)
        w = min(rng.choice([1, 2, 3, 17, 300, 40000, 50001, 1 << 21, rng.randrange(1, 1 << 21)]), p - 2)
        v0 = rng.choice([w + 1, p - 1, rng.randrange(w + 1, p)])
        cases.append((p, r, w, v0))
    # a step of 1 in the residue (r = 1 or r = p - 1): blocks of up to w + 1 points
    for p in ((1 << 30) - 35, 999999937):
        for r in (1, p - 1, 2, p - 2):
            for w in (1 << 21, 40000):
                cases += [(p, r, w, w + 1), (p, r, w, p - 1), (p, r, w, p // 2)]
    inp = "".join(f"{p} {r} {w} {v0}\n" for p, r, w, v0 in cases)
    out = subprocess.run([exe, "f"], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for (p, r, w, v0), line in zip(cases, out):
        ok, t, y = (int(x) for x in line.split())
        assert ok and t == O.G(p, r, p - v0, p - v0 + w), (p, r, w, v0)
        assert y == (v0 + r * t) % p, (p, r, w, v0)


def test_three_gap_steps_from_euclid(exe):
    """The walk's two steps from one run of Euclid's algorithm (32- and 64-bit)
    equal the paper's G for the windows [p - w, p - 1] and [1, w]."""
    rng = random.Random(19)
    # 64-bit primes below 2SL 2^21 take the float-estimate division (104857599947
    # is just below 50000 2^21: partial quotients up to 2^21)
    pool = [3, 5, 101, 7919, 1000003, 999999937, (1 << 30) - 35, 4294967291, 1099511627689,
            1073741827, 2999999929, 17179869209, 99999999977, 104857599947, 83886079997]
    cases = []
    for _ in range(20000):
        p = rng.choice(pool)
        r = rng.randrange(1, p)
        w = min(rng.choice([1, 2, 3, 17, 300, 40000, 50000, 50001, rng.randrange(1, p)]), p - 2)
        if w < 1:
            continue
        cases.append((p, r, w))
    inp = "".join(f"{p} {r} {w}\n" for p, r, w in cases)
    out = subprocess.run([exe, "s"], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for (p, r, w), line in zip(cases, out):
        ok64, a, da, b, ub, ok32, a2, da2, b2, ub2 = (int(x) for x in line.split())
        ga, gb = O.G(p, r, p - w, p - 1), O.G(p, r, 1, w)
        want = (ga, p - ga * r % p, gb, gb * r % p)
        assert ok64 and (a, da, b, ub) == want, (p, r, w)
        if p < (1 << 31):
            assert ok32 and (a2, da2, b2, ub2) == want, (p, r, w)


def test_lazy_montgomery_product(exe):
    """a b 2^-32 mod p kept below 2p for a < 2p, b < 2^31, odd p < 2^31 (the
    generator's K mod p chain over factor words below 2^31)."""
    rng = random.Random(23)
    cases = []
    for _ in range(20000):
        p = rng.choice([3, 1009, 999999937, (1 << 31) - 1, rng.randrange(3, 1 << 31) | 1])
        a = rng.choice([0, 2 * p - 1, rng.randrange(0, 2 * p)])
        b = rng.choice([0, (1 << 31) - 1, rng.randrange(0, 1 << 31)])
        cases.append((p, a, b))
    inp = "".join(f"{p} {a} {b}\n" for p, a, b in cases)
    out = subprocess.run([exe, "l"], input=inp, capture_output=True, text=True, check=True).stdout.split()
    for (p, a, b), v in zip(cases, out):
        v = int(v)
        assert v < 2 * p and (v - a * b * pow(2, -32, p)) % p == 0, (p, a, b)


def test_float_estimate_division(exe):
    """floor(n / p) and n mod p for n < 2^62, p < 2^31 and quotients below 2^32,
    from a float reciprocal estimate with exact 64-bit correction."""
    rng = random.Random(29)
    cases = []
    for _ in range(30000):
        p = rng.choice([1, 2, 3, 7, (1 << 31) - 1, rng.randrange(1, 1 << 31), rng.randrange(1, 1 << 16)])
        qmax = min((1 << 32) - 1, ((1 << 62) - 1) // p)
        q = rng.choice([0, 1, qmax, rng.randrange(0, qmax + 1)])
        n = q * p + rng.randrange(0, p)
        if n < (1 << 62):
            cases.append((n, p))
    inp = "".join(f"{n} {p}\n" for n, p in cases)
    out = subprocess.run([exe, "u"], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for (n, p), line in zip(cases, out):
        q, r = (int(x) for x in line.split())
        assert (q, r) == (n // p, n % p), (n, p)


def test_first_hit_64bit(exe):
    """The first hit from the three-gap basis for primes up to 2^40 (the 64-bit
    walk) equals the paper's G for the window [p - v0, p - v0 + w]."""
    rng = random.Random(31)
    pool = [7, 1000003, 999999937, (1 << 30) + 3, 4294967291, 68719476731, 99999999977, 1099511627689]
    cases = []
    for _ in range(20000):
        p = rng.choice(pool)
        r = rng.randrange(1, p)
        w = min(rng.choice([1, 2, 17, 40000, 50000, 1 << 21]), p - 2)
        v0 = rng.choice([w + 1, p - 1, rng.randrange(w + 1, p)])
        cases.append((p, r, w, v0))
    inp = "".join(f"{p} {r} {w} {v0}\n" for p, r, w, v0 in cases)
    out = subprocess.run([exe, "F"], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for (p, r, w, v0), line in zip(cases, out):
        ok, t, y = (int(x) for x in line.split())
        assert ok and t == O.G(p, r, p - v0, p - v0 + w), (p, r, w, v0)
        assert y == (v0 + r * t) % p, (p, r, w, v0)


def test_small_quotient_division(exe):
    """floor(a / b) for a < 2^31 and quotients up to 2^21 + 2 from a float estimate and one
    correction, with the reciprocal exact and perturbed by the relative 2^-23 that the
    device's approximate reciprocal may be off (the Euclid steps' division)."""
    rng = random.Random(37)
    cases = []
    for _ in range(60000):
        b = rng.choice([1, 2, 3, 512, 513, rng.randrange(1, 1 << 10), rng.randrange(1, 1 << 20),
                        rng.randrange(1, 1 << 30)])
        qmax = min((1 << 21) + 2, ((1 << 31) - 1) // b)
        q = rng.choice([0, 1, qmax, qmax - 1, rng.randrange(0, qmax + 1)])
        a = min(q * b + rng.choice([0, b - 1, rng.randrange(0, b)]), (1 << 31) - 1)
        cases.append((a, b))
    inp = "".join(f"{a} {b}\n" for a, b in cases)
    out = subprocess.run([exe, "e"], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for (a, b), line in zip(cases, out):
        v = [int(x) for x in line.split()]
        for k in range(3):
            assert (v[2 * k], v[2 * k + 1]) == (a // b, a % b), (a, b, k)


def test_small_quotient_division_64(exe):
    """floor(a / b) for 64-bit a (up to 2^41) and quotients up to 2^21 + 2 from a float
    estimate through 32-bit halves and one correction, with the reciprocal exact and
    perturbed by a relative 2^-23 (the Euclid steps' division for primes above 2^32)."""
    rng = random.Random(41)
    cases = []
    for _ in range(60000):
        b = rng.choice([1, 2, 3, 50000, 50001, rng.randrange(1, 1 << 16), rng.randrange(1 << 20, 1 << 32),
                        rng.randrange(1 << 32, 1 << 40), (1 << 32) - 1, 1 << 32, (1 << 32) + 1])
        qmax = min((1 << 21) + 2, ((1 << 41) - 1) // b)
        q = rng.choice([0, 1, qmax, qmax - 1, rng.randrange(0, qmax + 1)])
        a = min(q * b + rng.choice([0, b - 1, rng.randrange(0, b)]), (1 << 41) - 1)
        cases.append((a, b))
    inp = "".join(f"{a} {b}\n" for a, b in cases)
    out = subprocess.run([exe, "E"], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for (a, b), line in zip(cases, out):
        v = [int(x) for x in line.split()]
        for k in range(3):
            assert (v[2 * k], v[2 * k + 1]) == (a // b, a % b), (a, b, k)


def test_k_factor_words(exe):
    """K = P#/d packed into words below 2^31 (the 32-bit generator's lazily reduced
    Montgomery product) and below 2^64: each list multiplies to K exactly, every word is
    in range and a product of distinct primes of K, and first fit decreasing needs no
    more words than packing in order (45 instead of 48 for 953#/210)."""
    cases = [(503, 210), (953, 210), (1019, 210), (101, 2310), (37, 30), (7, 210), (953, 1)]
    inp, qks = "", []
    for P, d in cases:
        qK = [q for q in O.primes(1, P) if d % q]
        qks.append([int(q) for q in qK])
        inp += f"{len(qK)} " + " ".join(str(int(q)) for q in qK) + "\n"
    out = subprocess.run([exe, "k"], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    for k, ((P, d), qK) in enumerate(zip(cases, qks)):
        K = 1
        for q in qK:
            K *= q
        w32 = [int(x) for x in out[2 * k].split()]
        w64 = [int(x) for x in out[2 * k + 1].split()]
        for words, limit in ((w32, 1 << 31), (w64, 1 << 64)):
            prod = 1
            for w in words:
                assert 1 < w < limit, (P, d, w)
                prod *= w
            assert prod == K, (P, d)
        # words in order, as packed before: a new word when the next factor does not fit
        seq, acc = 0, 1
        for q in qK:
            if acc * q >= 1 << 31:
                seq, acc = seq + 1, 1
            acc *= q
        seq += acc > 1
        assert len(w32) <= seq, (P, d)
        if (P, d) == (953, 210):
            assert (len(w32), seq) == (45, 48)
