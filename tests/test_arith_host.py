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
        ok, m, y, ok2, m2, y2 = (int(v) for v in line.split())
        g = O.G(p, K, L, R)
        assert ok and ok2
        assert (m, y) == (g, g * K % p), (p, K, L, R)
        assert (m2, y2) == (g, g * K % p), (p, K, L, R)
