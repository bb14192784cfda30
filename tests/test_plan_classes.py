"""The plan's m-class tiers for the three-gap walk (csrc/cs_classes.h), compiled
for the host: which classes of m each large-prime chunk walks.  A class left
out would lose every hit on its rows, so the first property is coverage."""
import math
import os
import shutil
import subprocess

import pytest

from tests.conftest import ROOT

SRC = os.path.join(ROOT, "tests", "host", "plan_check.cpp")


def _cuda_include():
    cands = [os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"]
    nvcc = shutil.which("nvcc")
    if nvcc:
        cands.append(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))))
    for c in cands:
        if c and os.path.exists(os.path.join(c, "include", "cuda_runtime.h")):
            return os.path.join(c, "include")
    return None


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    inc = _cuda_include()
    if inc is None:
        pytest.skip("CUDA headers not found (cuda_runtime.h)")
    out = str(tmp_path_factory.mktemp("plan") / "plan_check")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-I", inc, "-o", out, SRC])
    return out


def _tiers(exe, rows):
    """rows: (three_gap, d, M_start, M_inc, S, m_classes, min_hits, item_hits, lo)."""
    inp = "".join(" ".join(str(int(v)) for v in r) + "\n" for r in rows)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout.split("\n")
    res = []
    for line in out[:len(rows)]:
        v = [int(x) for x in line.split()]
        Q, n, items = v[:3]
        res.append((Q, n, items, v[3:3 + n]))
    return res


def _chunk_lows(T, L, width=1 << 27):
    """Low ends of the plan's geometric large-prime chunks of (T, L]."""
    lows, lo = [], T
    while lo < L:
        hi = min(L, lo + max(lo, 1), lo + width)
        if lo < (1 << 30) - 1 and hi >= 1 << 30:
            hi = (1 << 30) - 1
        lows.append(lo)
        lo = hi
    return lows


def test_walked_classes_cover_every_row(exe):
    """For every tier and knob the walked residues of m - M_start mod Q include every m
    coprime to d, are distinct, lie below Q, and Q divides d; class items walk exactly
    the phi(Q) classes coprime to Q."""
    rows = []
    for d in (1, 15, 6, 30, 70, 210, 2310, 2 * 3 * 5 * 7 * 97):
        for M_start in (1, 1000, 1003, 10**8, 10**8 + 209, 164_000_000 + 11):
            for m_classes in (0, 1, 2, 3):
                for lo in (600, 10**4, 10**5, 10**6, 10**7, 10**9):
                    rows.append((1, d, M_start, 10**5, 40_001, m_classes, 0, 0, lo))
    got = _tiers(exe, rows)
    for r, (Q, n, items, res) in zip(rows, got):
        _, d, M_start, _, _, m_classes, _, _, lo = r
        assert d % Q == 0 and n == len(set(res)) and all(0 <= x < Q for x in res), r
        walked = set(res)
        for m in range(M_start, M_start + 2 * Q + 7):
            if math.gcd(m, d) == 1:
                assert (m - M_start) % Q in walked, (r, m)
        if items:
            assert items == n == sum(1 for c in range(Q) if math.gcd(c, Q) == 1), r
        if m_classes == 1:
            assert (Q, n) == (1, 1), r
        if m_classes == 3:
            assert Q == next((q for q in (210, 30, 6, 2) if d % q == 0), 1), r


def test_finer_classes_for_primes_with_more_hits(exe):
    """Along the chunks of (T, L] the walked fraction of m never falls as the primes grow
    (fewer hits per prime: fewer classes are worth their set-up), and every chunk walks
    only m with no factor of 2 (or 2, 3) in common with d once 2 | d (6 | d)."""
    for d, M_start in ((210, 10**8), (2310, 164_000_000), (30, 1001), (6, 7), (70, 12345)):
        lows = _chunk_lows(120_003, 10**11)
        got = _tiers(exe, [(1, d, M_start, 10**5, 40_001, 0, 0, 0, lo) for lo in lows])
        frac = [n / Q for Q, n, _, _ in got]
        assert all(a <= b + 1e-12 for a, b in zip(frac, frac[1:])), (d, frac)
        assert max(frac) <= 0.5 and (d % 6 or min(frac) < 0.34), (d, frac)


def test_search_953_tiers_match_the_measured_plan(exe):
    """search_953 at the autotuned T = 3 S = 120,003: 17 chunks, the first five walk class
    items (mod 210, then 30), the next five m = 1, 5 (mod 6), the last seven the odd m,
    as cs_info reported on the GPU ("5 chunks" of class items, "5 of 17" mod 6)."""
    lows = _chunk_lows(120_003, 10**9)
    assert len(lows) == 17
    got = _tiers(exe, [(1, 210, 10**8, 10**5, 40_001, 0, 0, 0, lo) for lo in lows])
    kinds = [(Q, items > 0) for Q, _, items, _ in got]
    assert sum(i for _, i in kinds) == 5 and kinds[0] == (210, True)
    assert sum(1 for Q, i in kinds if Q == 6 and not i) == 5
    assert sum(1 for Q, i in kinds if Q == 2) == 7
    # the paper's one-solve-per-hit walk and SL = 0 take every m
    assert _tiers(exe, [(0, 210, 10**8, 10**5, 40_001, 0, 0, 0, 120_003)])[0][:2] == (1, 1)
