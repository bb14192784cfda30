"""The hit-bucket layout (csrc/cs_buckets.h), compiled for the host: when the
walk's stored hits go through per-band records, how many rows a band holds,
how many records a region holds, and after which chunks the records are
cleared.  Checked on the large search's shape (the values the GPU runs use),
on the search_953 shape (direct clears unless forced) and by properties over
random shapes."""
import math
import os
import random
import shutil
import subprocess

import pytest

from tests.conftest import ROOT

SRC = os.path.join(ROOT, "tests", "host", "bucket_check.cpp")
L2_GB300 = 132644864            # cudaDevAttrL2CacheSize of a GB300 (126.5 MiB)
CTAS = 152 * 3                  # the walk's grid: three CTAs per SM


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not found")
    out = str(tmp_path_factory.mktemp("buckets") / "bucket_check")
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-o", out, SRC])
    return out


def _chunks(T, L, width=1 << 27):
    """The plan's large-prime chunks of (T, L]: doubling up to 2^27 wide, with a
    boundary at 2^30 - 1 (the 32-bit chunks end there)."""
    out, lo = [], T
    while lo < L:
        hi = min(L, lo + max(lo, 1), lo + width)
        if lo < (1 << 30) - 1 and hi >= 1 << 30:
            hi = (1 << 30) - 1
        out.append((lo, hi))
        lo = hi
    return out


def _layout(exe, rows):
    """rows: (hit_buckets, band_rows_log, bucket_records, three_gap, M_c, wpr, W, l2, ctas, chunks)."""
    lines = []
    for r in rows:
        *head, chunks = r
        lines.append(" ".join(str(int(v)) for v in head) + f" {len(chunks)} " +
                     " ".join(f"{lo} {hi}" for lo, hi in chunks))
    out = subprocess.run([exe], input="\n".join(lines) + "\n", capture_output=True, text=True,
                         check=True).stdout.split("\n")
    res = []
    for line in out[:len(rows)]:
        v = [int(x) for x in line.split()]
        res.append({"on": v[0], "band_log": v[1], "n_bands": v[2], "n_regions": v[3], "cap": v[4],
                    "bad": v[5], "after": v[6:]})
    return res


def _expected(lo, hi, M_c, W):
    lo, hi = max(lo, 3.0), max(hi, lo, 3.0)
    return M_c * W * math.log(math.log(hi) / math.log(lo))


def test_large_search_layout(exe):
    """large_1019 (2,285,714 rows of 261 words, 4.77 GB): buckets on by default,
    bands of 8192 rows (17 MB, the largest within a fifth of L2), 280 bands, 456
    regions each of 16,820 records (8 GiB in all), 20 apply groups, as measured
    on the GPU (the plan's info reports the same)."""
    chunks = _chunks(100002, 10**11)
    assert len(chunks) == 756
    b, = _layout(exe, [(0, 0, 0, 1, 2285714, 261, 16682, L2_GB300, CTAS, chunks)])
    assert b["on"] and not b["bad"]
    assert b["band_log"] == 13 and b["n_bands"] == 280 and b["n_regions"] == 456 and b["cap"] == 16820
    assert (1 << 13) * 261 * 8 <= L2_GB300 // 5 < (1 << 14) * 261 * 8
    assert b["cap"] * b["n_bands"] * b["n_regions"] * 4 <= (8 << 30) + 3 * 4 * b["n_bands"] * b["n_regions"]
    assert len(b["after"]) == 756 and sum(b["after"]) == 20 and b["after"][-1] == 1


def test_small_bitset_clears_directly_unless_forced(exe):
    """search_953's 37.5 MB bitset stays in L2: direct clears by default; forced,
    bands within a fifth of L2 and within the bitset."""
    chunks = _chunks(120003, 10**9)
    rows = [(0, 0, 0, 1, 22858, 205, 13102, L2_GB300, CTAS, chunks),
            (1, 0, 0, 1, 22858, 205, 13102, L2_GB300, CTAS, chunks),
            (2, 0, 0, 1, 22858, 205, 13102, L2_GB300, CTAS, chunks),
            (2, 0, 0, 0, 22858, 205, 13102, L2_GB300, CTAS, chunks),   # the paper's walk never buckets
            (2, 0, 0, 1, 22858, 205, 13102, L2_GB300, CTAS, [])]       # no large primes
    auto, off, forced, paper, none = _layout(exe, rows)
    assert not auto["on"] and not off["on"] and not paper["on"] and not none["on"]
    assert forced["on"] and forced["band_log"] == 13 and forced["n_bands"] == 3
    assert sum(forced["after"]) >= 1 and forced["after"][-1] == 1


def test_explicit_band_rows_log_is_checked(exe):
    """An explicit band height whose records would exceed 32 bits, or that gives
    more than 4096 bands, is reported (the plan then fails with CS_EINVAL)."""
    chunks = _chunks(100002, 10**9)
    rows = [(2, 20, 0, 1, 10**6, 100000, 6400000, L2_GB300, CTAS, chunks),   # 64 wpr 2^20 > 2^32
            (2, 1, 0, 1, 10**6, 10, 640, L2_GB300, CTAS, chunks),            # 500,000 bands
            (2, 8, 0, 1, 10**6, 10, 640, L2_GB300, CTAS, chunks)]            # 3907 bands: fine
    big, many, ok = _layout(exe, rows)
    assert big["bad"] and not big["on"]
    assert many["bad"] and not many["on"]
    assert ok["on"] and not ok["bad"] and ok["n_bands"] == -(-10**6 // 256)


def test_layout_properties_on_random_shapes(exe):
    rng = random.Random(29)
    rows = []
    for _ in range(300):
        M_c = rng.choice([1, 7, 1000, 22858, 228571, 2285714, 10**7]) + rng.randint(0, 999)
        W = rng.randint(1, 60000)
        wpr = -(-W // 64)
        l2 = rng.choice([50 << 20, L2_GB300, 256 << 20])
        recs = rng.choice([0, 0, 1, 16, 1000, 5000])
        T = rng.choice([1000, 100002, 10**6])
        L = rng.choice([10**7, 10**9, 10**11])
        rows.append((2, 0, recs, 1, M_c, wpr, W, l2, CTAS, _chunks(T, L) if L > T else []))
    for r, b in zip(rows, _layout(exe, rows)):
        _, _, recs, _, M_c, wpr, W, l2, ctas, chunks = r
        if not chunks:
            assert not b["on"]
            continue
        bl = b["band_log"]
        fits = (64 * wpr) << bl <= 1 << 32
        assert b["on"] == fits, r[:9]
        if not b["on"]:
            continue
        assert b["n_bands"] == -(-M_c // (1 << bl)) and b["n_bands"] <= 4096
        assert b["n_regions"] == ctas
        assert b["cap"] % 4 == 0 and 4 <= b["cap"] <= 1 << 24
        if recs:
            assert b["cap"] == min(max(-(-recs // 4) * 4, 4), 1 << 24)
        # the largest band within a fifth of L2 and the bitset, unless that
        # would give more than 4096 bands
        first = 0
        while (2 << first) * wpr * 8 <= l2 // 5 and (2 << first) <= M_c:
            first += 1
        if -(-M_c // (1 << first)) <= 4096:
            assert bl == first
        else:
            assert bl > first and -(-M_c // (1 << (bl - 1))) > 4096
        # apply groups: greedy, each group within 60% of the regions unless it
        # is a single chunk, and the last chunk ends a group
        room = 0.6 * b["cap"] * b["n_regions"] * b["n_bands"]
        after = b["after"]
        assert len(after) == len(chunks) and after[-1] == 1
        start = 0
        for c, a in enumerate(after):
            if not a:
                continue
            group = sum(_expected(lo, hi, M_c, W) for lo, hi in chunks[start:c + 1])
            assert c == start or group <= room * (1 + 1e-9)
            if c + 1 < len(chunks):
                nxt = _expected(*chunks[c + 1], M_c, W)
                assert group + nxt > room * (1 - 1e-9) or group == 0
            start = c + 1
