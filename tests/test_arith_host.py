"""The kernels' solver arithmetic (cs_arith.cuh), compiled for the host with
g++, against the paper's recursion G of Section 3.3 in the oracle."""
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
def test_g_solve_and_multi_match_paper_recursion(exe, narrow):
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
        vals = [int(v) for v in line.split()]
        ok, m, y, ok2, m2, y2 = vals[:6]
        g = O.G(p, K, L, R)
        assert ok and ok2
        assert (m, y) == (g, g * K % p), (p, K, L, R)
        assert (m2, y2) == (g, g * K % p), (p, K, L, R)
        if narrow:
            ok4, m4, y4 = vals[6:]
            assert ok4 and (m4, y4) == (g, g * K % p), (p, K, L, R)


def test_shared_reciprocal_quotients(exe):
    """floor(a / d) through one precomputed reciprocal of d, for every size of
    a and d that the 32-bit solver meets (a < 2^31 + 2^30, d < 2^30), with the
    edges where the estimate is one short: a = k d - 1, k d, k d + d - 1."""
    rng = random.Random(11)
    cases = []
    for _ in range(20000):
        d = rng.choice([1, 2, 3, 7, rng.randrange(1, 1 << 16), rng.randrange(1, 1 << 30), (1 << 30) - 35])
        k = rng.randrange(0, (3 << 30) // d + 1)
        for a in (k * d - 1, k * d, k * d + d - 1, rng.randrange(0, 3 << 30)):
            if 0 <= a < (3 << 30):
                cases.append((a, d))
    cases += [(0xffffffff, 1), (0xffffffff, 0xffffffff), (0xfffffffe, 0xffffffff), (0x80000000, 3)]
    inp = "".join(f"{a} {d}\n" for a, d in cases)
    out = subprocess.run([exe, "q"], input=inp, capture_output=True, text=True, check=True).stdout.split()
    assert len(out) == len(cases)
    for (a, d), q in zip(cases, out):
        assert int(q) == a // d, (a, d)
