"""bench.py's host logic on the CPU: the reference arm's JSON line, the
roofline of the walk from stored ncu counters, and the clock samples that
decide whether a timed run is kept."""
import importlib.util
import json
import os
import subprocess
import sys
from types import SimpleNamespace

import pytest

from tests.conftest import ROOT


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_reference_arm_prints_one_contract_line():
    """`--impl reference` times the oracle on host cores and prints one JSON line with the
    keys the contract names (plain_503 and a few rows keep it to seconds)."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--config",
                          "plain_503", "--steps", "1", "--warmup", "0", "--ref-rows", "4"],
                         capture_output=True, text=True, check=True, timeout=600, cwd=ROOT).stdout
    lines = [l for l in out.strip().split("\n") if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["unit"] == "factors/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["steps"] == 1 and line["warmup"] == 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["cpu_baseline"]["cores"] >= 1 and "sample" in line["cpu_baseline"]
    assert line["e2e"] == {"value": line["value"], "unit": "factors/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("plain_503") and line["config"]["L"] == 10**7


def _info(**kw):
    base = dict(threshold=120003, tile_rows=16, n_large_chunks=17, bitset_bytes=37487120, M_c=22858,
                hit_buckets=0, n_bands=0, apply_launches=0, bucket_bytes=0, prep_chunks=0)
    base.update(kw)
    return SimpleNamespace(**base)


def test_roofline_uses_counters_only_for_the_same_sources_and_setup(bench, monkeypatch):
    """The walk's two bounds: issue (stored thread instructions per launch over the
    launch's timed duration, against the best measured issue rate; the counters
    apply only to the same sources, threshold, tile height and chunking) and
    scattered clears (live stored hits against the measured clear rate).  The
    bound that needs more time binds."""
    ctr = {"csrc_sha": bench.csrc_sha(), "threshold": 120003, "tile_rows": 16, "launches": 17,
           "thread_inst": 8.77e10, "dram_bytes": 1.24e9}
    monkeypatch.setitem(bench.WALK_COUNTERS, "search_953", ctr)
    walk = bench.KC_NAMES.index("large_walk")
    kern_ms = [0.0] * len(bench.KC_NAMES)
    kern_n = [0] * len(bench.KC_NAMES)
    kern_ms[walk], kern_n[walk] = 10 * 5.9, 10 * ctr["launches"]      # 10 sieves
    stats = {"hits_all": 7.47e8, "levels": 4.5e8, "F_large": 1.71e8}
    peaks = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}
    issue = {"add_logic": 20.5, "imad": 19.0, "imad_logic": 38.25}
    args = (None, peaks, "measured", issue, "search_953")
    # issue binds (fast clears, as for a bitset in L2)
    r = bench.roofline(walk, kern_ms, kern_n, stats, _info(), *args, clears_peak=2e11)
    assert r["bound"] == "alu" and r["unit"] == "Tinst/s" and r["peak"] == 38.25
    per_launch_s = 5.9e-3 / ctr["launches"]
    want = ctr["thread_inst"] / ctr["launches"] / per_launch_s / 1e12
    assert abs(r["achieved"] - want) < 1e-9 * want and abs(r["frac"] - want / 38.25) < 1e-12
    assert abs(r["traffic"] - ctr["dram_bytes"] / ctr["launches"]) < 1.0
    assert r["bounds"]["clears"]["min_ms_per_launch"] < r["bounds"]["issue"]["min_ms_per_launch"]
    # clears bind (slow scattered clears, as for a bitset far larger than L2)
    r = bench.roofline(walk, kern_ms, kern_n, stats, _info(), *args, clears_peak=2e10)
    want_c = stats["F_large"] / ctr["launches"] / per_launch_s / 1e9
    assert r["bound"] == "hbm" and r["unit"] == "Gclears/s" and r["peak"] == 20.0
    assert abs(r["achieved"] - want_c) < 1e-9 * want_c and abs(r["frac"] - want_c / 20.0) < 1e-12
    # another threshold, tile height, chunking or source digest: no issue bound
    for other in (_info(threshold=80002), _info(tile_rows=8), _info(n_large_chunks=24)):
        r = bench.roofline(walk, kern_ms, kern_n, stats, other, *args)
        assert r["achieved"] is None and r["frac"] is None and "note" in r
    monkeypatch.setitem(bench.WALK_COUNTERS, "search_953", dict(ctr, csrc_sha="0" * 16))
    r = bench.roofline(walk, kern_ms, kern_n, stats, _info(), *args)
    assert r["achieved"] is None
    # hit buckets: the walk's memory side is the records it writes (4 bytes each,
    # against the HBM copy rate), and the apply kernel gets its own entry
    monkeypatch.setitem(bench.WALK_COUNTERS, "search_953", ctr)
    apply = bench.KC_NAMES.index("hit_apply")
    kb_ms, kb_n = list(kern_ms), list(kern_n)
    kb_ms[apply], kb_n[apply] = 10 * 1.5, 10 * 2
    sb = dict(stats, bucket_records=1.7e8)
    r = bench.roofline(walk, kb_ms, kb_n, sb, _info(hit_buckets=1, n_bands=3, apply_launches=2), *args,
                       clears_peak=2e10, band_peak=1.5e11)
    assert r["bounds"]["clears"] is None and r["bounds"]["records"]["unit"] == "GB/s"
    assert r["bound"] == "alu" and r["unit"] == "Tinst/s"           # 0.68 GB of records per sieve: issue binds
    want_a = 1.7e8 / 1.5e-3
    assert abs(r["apply"]["achieved"] - want_a / 1e9) < 1e-6 * want_a / 1e9
    assert abs(r["apply"]["frac"] - want_a / 1.5e11) < 1e-12 and r["apply"]["unit"] == "Gclears/s"
    # the walker preparation's own entry: its stored instructions per sieve over
    # its timed share, when the stored launch count matches the plan's
    prep = bench.KC_NAMES.index("walk_prep")
    kp_ms, kp_n = list(kern_ms), list(kern_n)
    kp_ms[prep], kp_n[prep] = 10 * 1.7, 10 * 7
    monkeypatch.setitem(bench.WALK_COUNTERS, "search_953", dict(ctr, prep_launches=7, prep_thread_inst=2.56e10))
    r = bench.roofline(walk, kp_ms, kp_n, stats, _info(prep_chunks=7), *args, clears_peak=2e11)
    want_p = 2.56e10 / 1.7e-3 / 1e12
    assert abs(r["prep"]["achieved"] - want_p) < 1e-9 * want_p and abs(r["prep"]["frac"] - want_p / 38.25) < 1e-12
    r = bench.roofline(walk, kp_ms, kp_n, stats, _info(prep_chunks=6), *args, clears_peak=2e11)
    assert "prep" not in r                                          # other chunking: no entry
    monkeypatch.setitem(bench.WALK_COUNTERS, "search_953", ctr)
    # no measured peaks: no fraction (never a derived stand-in)
    monkeypatch.setitem(bench.WALK_COUNTERS, "search_953", ctr)
    r = bench.roofline(walk, kern_ms, kern_n, stats, _info(), None, peaks, "measured", {"error": "x"}, "search_953")
    assert r["peak"] is None and r["frac"] is None


def test_oracle_sample_ranges(bench):
    """The bounded oracle sample: all of (P, L] for small L, else (P, 2^24] plus
    evenly spaced 2^26-wide windows ending at L, disjoint and inside (P, L]."""
    from paper_2012_03771_gb300 import workloads
    assert bench.sample_ranges(workloads.PLAIN_503, 4) == [(503, 10**7)]
    rng = bench.sample_ranges(workloads.LARGE_1019, 4)
    assert rng[0] == (1019, 1 << 24) and len(rng) == 5 and rng[-1][1] == 10**11
    for (a, b), (c, e) in zip(rng, rng[1:]):
        assert b <= c and e - c == 1 << 26
    assert bench.sample_ranges(workloads.LARGE_1019, 0) == [(1019, 10**11)]


def test_clock_samples_median_and_reasons(bench, tmp_path):
    """The nvidia-smi samples of the timed region: median SM clock of this GPU's lines and
    every throttle reason seen active (a run with a slowdown reason is rejected)."""
    path = tmp_path / "clocks.csv"
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "1, 1200, 2070, 500.0, 0x0, Active, Not Active, Not Active, Not Active",   # another GPU
            "0, 2055, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2070, 2070, 1380.0, 0x4, Not Active, Not Active, Not Active, Active",
            "garbage line"]
    path.write_text("\n".join(rows) + "\n")
    c = bench.Clocks(str(path))
    c.proc = SimpleNamespace(terminate=lambda: None, wait=lambda timeout=None: 0, kill=lambda: None)
    c.f = open(os.devnull, "w")
    got = c.stop(device_index=0)
    assert got == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_speedup_curve_interval_count():
    """The speed-up curve's intervals hold exactly M_c values of m coprime to d."""
    import math
    from paper_2012_03771_gb300.speedup_curve import m_inc_for
    for d, M_start in ((210, 1), (210, 10**8), (2310, 7), (1, 5)):
        for m_c in (1, 10, 1000):
            M_inc = m_inc_for(M_start, d, m_c)
            assert sum(math.gcd(m, d) == 1 for m in range(M_start, M_start + M_inc)) == m_c
            assert math.gcd(M_start + M_inc - 1, d) == 1          # the smallest such M_inc
