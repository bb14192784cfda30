"""Benchmark of the Combined Sieve hot path on one or more GPUs.

One step = one full sieve (cs_sieve) of the large single search
K = 1019#/210, m in [1.64e8, 1.74e8) coprime to 210 (2.29M intervals),
X = 25000, primes up to L = 1e11 generated on the device (64-bit arithmetic
above 2^30), 4.77 GB bitset: prime generation, K mod p, small-prime tile
sieve, large-prime walk, counts and checksum.  Metric: enumerated factors per
second (F / time), with F and the bitset checksum checked against the same
values on every step.  --config search_953 selects the smaller paper-shaped
search (K = 953#/210, 22,858 intervals, L = 1e9).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cuda|reference] [--config NAME]

Under torchrun each rank sieves its own m-range (independent problems, no
data-path collective; weak scaling); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import tempfile
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2012_03771_gb300 import workloads  # noqa: E402

def metric_of(params) -> str:
    return f"enumerated factors/s at L={params.L:.0e} (bit-exact bitset + per-m counts)"


METRIC = "enumerated factors/s at L=1e9 (bit-exact bitset + per-m counts)"
UNIT = "factors/s"
KC_NAMES = ["gen_small", "tile_sieve", "gen_large", "large_walk", "final", "hit_apply", "walk_prep"]
# autotuner results for this GPU, one line per (P, d, SL, ceil(log2 L))
TUNE_FILE = os.path.join(ROOT, "paper_2012_03771_gb300", "tune_gb300.txt")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return rank, ws


def _params_for_rank(base: workloads.SieveParams, rank: int) -> workloads.SieveParams:
    return base.with_(M_start=base.M_start + rank * base.M_inc)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, path):
        self.path, self.proc = path, None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, device_index=0):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9 or parts[0] != str(device_index):
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# bounded oracle sample: every prime up to SMALL_ALL (they carry most of the
# enumerated factors: sum 1/p), and WINDOWS windows of WINDOW numbers evenly
# spaced over the rest of (P, L] (they carry most of the per-prime cost)
SAMPLE_SMALL_ALL = 1 << 24
SAMPLE_WINDOW = 1 << 26


def sample_ranges(params: workloads.SieveParams, windows: int):
    """Prime ranges (lo, hi] of the bounded sample: all of (P, L] when that is at
    most 2^24 + windows * 2^26 numbers, else (P, 2^24] and `windows` evenly spaced
    windows of 2^26 numbers above 2^24."""
    P, L = params.P, params.L
    if L - P <= SAMPLE_SMALL_ALL + windows * SAMPLE_WINDOW or windows <= 0:
        return [(P, L)]
    out = [(P, SAMPLE_SMALL_ALL)]
    span = L - SAMPLE_SMALL_ALL
    for k in range(windows):
        hi = SAMPLE_SMALL_ALL + (k + 1) * span // windows
        out.append((hi - SAMPLE_WINDOW, hi))
    return out


def sample_text(params, n_rows, n_all, windows):
    rng = sample_ranges(params, windows)
    pr = ("all primes <= L" if len(rng) == 1 else
          f"primes in ({params.P}, 2^24] and in {len(rng) - 1} windows of 2^26 numbers evenly spaced up to L")
    return f"{n_rows} of {n_all} coprime m (evenly spaced) x {pr}"


def oracle_sample(params: workloads.SieveParams, n_rows: int, windows: int = 4):
    """The CPU oracle (as it stands) on a bounded sample of the workload: n_rows
    evenly spaced coprime m, and the primes of sample_ranges.  Returns
    (factors, seconds, cores, rows, coprime m in the search)."""
    import oracle.oracle as O
    rows = O.rows(params.d, params.M_start, params.M_inc)
    idx = [int(i * (len(rows) - 1) / max(n_rows - 1, 1)) for i in range(n_rows)]
    pick = [int(rows[i]) for i in sorted(set(idx))]
    cores = os.cpu_count() or 1
    F = 0
    t0 = time.perf_counter()
    for lo, hi in sample_ranges(params, windows):
        _, Fr, _ = O.sieve(params.P, params.d, params.SL, hi, pick, p_lo=lo, threads=cores)
        F += int(Fr.sum())
    dt = time.perf_counter() - t0
    return F, dt, cores, len(pick), len(rows)


def run_reference(args, params):
    rank, ws = _dist()
    if rank != 0:
        return
    import oracle.oracle as O
    O.build()
    n_rows = args.ref_rows
    for _ in range(args.warmup):
        oracle_sample(params, n_rows, args.ref_windows)
    Fs, ts = 0, 0.0
    cores, nr, n_all = 1, n_rows, 0
    for _ in range(args.steps):
        F, dt, cores, nr, n_all = oracle_sample(params, n_rows, args.ref_windows)
        Fs += F
        ts += dt
    value = Fs / ts
    sample = sample_text(params, nr, n_all, args.ref_windows) + " per step"
    line = {"impl": "reference", "metric": metric_of(params), "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * ts / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
            "data": "synthetic", "config": _config(params, args.config),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(params, name="large_1019"):
    """The workload, identical for both arms (implementation details go elsewhere)."""
    return {"workload": f"{name}: K={params.P}#/{params.d}, m in [{params.M_start}, {params.M_start + params.M_inc}) "
                        f"coprime to {params.d}, X={params.SL}, primes {params.P} < p <= {params.L}",
            "P": params.P, "d": params.d, "M_start": params.M_start, "M_inc": params.M_inc, "SL": params.SL,
            "L": params.L, "parallelism": "replicas (independent m-ranges per rank)",
            "l2": "flushed between steps (256 MB device write)"}


def _shape(info, tuned):
    return {"M_c": int(info.M_c), "W": int(info.W), "bitset_bytes": int(info.bitset_bytes),
            "threshold": int(info.threshold), "large_mode": int(info.large_mode), "tile_rows": int(info.tile_rows),
            "layout": "compact" if info.layout else "x coprime to K", "autotuned": tuned is not None,
            "m_classes_walked": f"{int(info.m_walked)} of m mod {int(info.m_mod)}",
            "chunks_class_walk": f"{int(info.split_chunks)} of {int(info.n_large_chunks)}",
            "class_items": (f"{int(info.item_chunks)} chunks, finest {int(info.item_classes)} classes of "
                            f"m mod {int(info.item_mod)}" if info.item_chunks else "none"),
            "hit_buckets": ({"bands": int(info.n_bands), "bucket_bytes": int(info.bucket_bytes),
                             "apply_launches": int(info.apply_launches)} if info.hit_buckets else None),
            "prepared_walker_chunks": int(info.prep_chunks)}


def run_cuda(args, params):
    import numpy as np
    import torch
    import paper_2012_03771_gb300 as cs
    from paper_2012_03771_gb300 import build

    rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    cs.load()
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    tuning = dict(profile=True)
    tuned = None
    if not args.threshold and not args.mode and not args.no_autotune:
        # the autotuner's choice for this parameter set, from the committed
        # tuning file (timed on the device and appended there if missing)
        tuned = cs.cs_autotune(*params.as_tuple(), cache_path=TUNE_FILE)
        tuning.update(tuned)
    if args.mode:
        tuning["large_mode"] = args.mode
    if args.threshold:
        tuning["threshold"] = args.threshold
    if args.layout:
        tuning["layout"] = args.layout
    plan = cs.Plan(*params.as_tuple(), **tuning)
    info = plan.info

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            plan.sieve(stream)
        plan.sync()
        F_ref, h_ref = cs.cs_counts(plan.h)
        stats = plan.stats()

        # raw clock samples: CS_CLOCKS_DIR if set (kept for inspection), else a temp file
        clk_dir = os.environ.get("CS_CLOCKS_DIR")
        clocks = Clocks(os.path.join(clk_dir, f"clocks_bench_r{rank}.csv") if clk_dir and os.path.isdir(clk_dir)
                        else os.path.join(tempfile.gettempdir(), f"clocks_{os.getpid()}.csv"))
        clocks.start()
        barrier()
        torch.cuda.synchronize()
        step_ms, kern_ms, kern_n = [], [0.0] * len(KC_NAMES), [0] * len(KC_NAMES)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            flush.fill_(k & 0xff)                       # evict the previous step from L2
            ev[k][0].record(stream)
            plan.sieve(stream)
            ev[k][1].record(stream)
            stream.synchronize()
            ms, n = plan.kernel_times()
            kern_ms = [a + b for a, b in zip(kern_ms, ms)]
            kern_n = [a + b for a, b in zip(kern_n, n)]
            F, h = cs.cs_counts(plan.h)
            if (F, h) != (F_ref, h_ref):
                raise SystemExit(f"step {k}: F/hash changed ({F}, {h:#x}) != ({F_ref}, {h_ref:#x})")
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop(local)
        step_ms = [a.elapsed_time(b) for a, b in ev]

    total_ms = sum(step_ms)
    if ws > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        f = torch.tensor([float(F_ref)], dtype=torch.float64, device="cuda")
        dist.all_reduce(f, op=dist.ReduceOp.SUM)
        F_all = float(f.item())
    else:
        F_all = float(F_ref)
    value = F_all * args.steps / (total_ms / 1e3)
    intervals_s = int(info.M_c) * ws * args.steps / (total_ms / 1e3)

    # ---- end to end through the C ABI with host buffers --------------------
    d2h = int(info.bitset_bytes) + 4 * int(info.M_c) + 16
    host_bits = torch.empty(max(int(info.bitset_bytes) // 8, 1), dtype=torch.int64).pin_memory()
    host_cnt = torch.empty(max(int(info.M_c), 1), dtype=torch.int32).pin_memory()
    e2e_steps = max(1, min(args.steps, 5))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2d = 0
    split = {"plan_ms": 0.0, "sieve_ms": 0.0, "fetch_ms": 0.0, "destroy_ms": 0.0}
    for _ in range(e2e_steps):
        ta = time.perf_counter()
        p2 = cs.Plan(*params.as_tuple(), **{k: v for k, v in tuning.items() if k != "profile"})
        h2d = int(p2.info.h2d_bytes)
        tb = time.perf_counter()
        p2.sieve(stream).sync()
        tb2 = time.perf_counter()
        cs.cs_fetch_bitset(p2.h, host_bits.numpy().view(np.uint64))
        cs.cs_counts(p2.h, host_cnt.numpy().view(np.uint32))
        tc = time.perf_counter()
        p2.close()
        td = time.perf_counter()
        split["plan_ms"] += (tb - ta) * 1e3 / e2e_steps
        split["sieve_ms"] += (tb2 - tb) * 1e3 / e2e_steps
        split["fetch_ms"] += (tc - tb2) * 1e3 / e2e_steps
        split["destroy_ms"] += (td - tc) * 1e3 / e2e_steps
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e_value = F_all / e2e_s if ws == 1 else F_all / e2e_s

    # ---- roofline of the dominant kernel ------------------------------------
    peaks, peak_src = _peaks()
    issue = issue_rates(torch, cs, stream)
    plan.close()                                    # room for the scattered-clear probe
    clears_peak = clear_rate(torch, cs, stream, int(info.bitset_bytes) // 4)
    # the apply kernel clears two bands at a time at most: its peak is the
    # clear rate over a region of two bands' words
    band_peak = (clear_rate(torch, cs, stream, 2 * int(info.bitset_bytes) // max(int(info.n_bands), 1) // 4)
                 if info.hit_buckets else None)
    dom = max(range(len(KC_NAMES)), key=lambda i: kern_ms[i])
    roof = roofline(dom, kern_ms, kern_n, stats, info, params, peaks, peak_src, issue, args.config, clears_peak,
                    band_peak)

    # ---- CPU oracle on a bounded sample -------------------------------------
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu:
        try:
            import oracle.oracle as O
            O.build()
            Fs, dt, cores, nr, n_all = oracle_sample(params, args.ref_rows, args.ref_windows)
            cpu = {"value": Fs / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": sample_text(params, nr, n_all, args.ref_windows) + f" (the reference arm's step); {dt:.1f} s"}
        except Exception as e:  # the oracle is a reported baseline only
            cpu = {"value": None, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                   "sample": f"failed: {e}"}

    if rank == 0:
        line = {
            "metric": metric_of(params), "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32" if info.narrow else "u64",
            "data": "synthetic (parameters of the paper-shaped search; primes generated on device)",
            "config": _config(params, args.config),
            "plan": _shape(info, tuned),
            "intervals_per_s": intervals_s,
            # walk work per second: windows solved (two steps and the first hits per
            # work item in the three-gap walk) and Euclid / solver passes
            "solves_per_s": stats["solves"] * ws / (total_ms / args.steps / 1e3),
            "levels_per_s": stats["levels"] * ws / (total_ms / args.steps / 1e3),
            "F_per_step": int(F_ref), "hash": f"{h_ref:#018x}",
            "stats": stats,
            "kernel_ms_per_step": {n: kern_ms[i] / args.steps for i, n in enumerate(KC_NAMES)},
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "includes": "cs_plan (host tables, H2D, allocation) + cs_sieve + bitset/counts D2H + cs_destroy",
                    "per_step_split": split},
            "gpu_launches": int(info.launches_per_sieve) * args.steps,
        }
        print(json.dumps(line), flush=True)
    plan.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def csrc_sha() -> str:
    """Digest of the sources that make up the large-prime walk kernel, to tell
    whether stored ncu counters still apply to the built code."""
    import hashlib
    h = hashlib.sha256()
    for name in ("cs_large.cu", "cs_arith.cuh", "cs_internal.h", "cs_walker.cuh"):
        f = os.path.join(ROOT, "paper_2012_03771_gb300", "csrc", name)
        h.update(name.encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


# ncu counters of the large-prime walk, summed over the walk's launches of one
# sieve (the first, the bench's warm-up sieve) of each workload, taken with
#   ncu --metrics smsp__thread_inst_executed.sum,gpu__time_duration.sum --clock-control none
#       -k regex:"k_large_tg|k_tg_prep" -c 1424 --csv python bench.py --steps 1 --warmup 1 --no-cpu
#   ncu --metrics gpu__time_duration.sum,smsp__thread_inst_executed.sum,dram__bytes_read.sum,
#       dram__bytes_write.sum --clock-control none -k regex:"k_large_tg|k_tg_prep" -c 24 --csv
#       python bench.py --config search_953 --steps 1 --warmup 1 --no-cpu
# (756 and 17 walk launches, 668 and 7 preparation launches per sieve)
# The work is deterministic (same inputs, same code), so these are per-sieve
# constants for the walk sources whose digest is recorded (csrc_sha) and the
# same threshold, tile height and chunking; otherwise they are not used.
WALK_COUNTERS = {
    # one GB300, walk sources with hit buckets, class-item rows from the steps and
    # prepared walkers for the one-walker chunks (large_1019 buckets its hits,
    # search_953 clears directly); prep_*: the walker-preparation kernel of the
    # same run; large_1019's DRAM bytes were not captured at full size (several
    # passes on a 13 GB working set)
    "large_1019": {"csrc_sha": "c62acc85a540bf78", "threshold": 100002, "tile_rows": 8, "launches": 756,
                   "thread_inst": 8482416284364.0, "dram_bytes": None,
                   "prep_launches": 668, "prep_thread_inst": 3688559218341.0},
    "search_953": {"csrc_sha": "c62acc85a540bf78", "threshold": 120003, "tile_rows": 16, "launches": 17,
                   "thread_inst": 59499229837.0, "dram_bytes": 1798157568.0,
                   "prep_launches": 7, "prep_thread_inst": 25639266207.0},
}


def issue_rates(torch, cs, stream):
    """The measured integer issue rate: thread-level operations per second of the
    cs_issue_rate micro-benchmark (one full-occupancy wave of independent integer
    chains), best of three launches, for each of its three instruction mixes."""
    try:
        n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        sink = torch.zeros(n_sm * 2048, dtype=torch.int32, device="cuda")
        out = {}
        for mix, name in ((0, "add_logic"), (1, "imad"), (2, "imad_logic")):
            best = 0.0
            for _ in range(3):
                ops, ms = cs.cs_issue_rate(mix, 2000, sink.data_ptr(), sink.numel(), stream)
                best = max(best, ops / (ms / 1e3))
            out[name] = best / 1e12
        return out
    except Exception as e:   # reported as missing, never replaced by a derived figure
        return {"error": str(e)}


def clear_rate(torch, cs, stream, words):
    """The measured rate of scattered bit clears (cs_atomic_rate: one-bit 32-bit
    atomic ANDs at random words) over a region of `words` 32-bit words, the
    bitset's size: best of three launches, in clears per second."""
    try:
        buf = torch.full((max(int(words), 1),), -1, dtype=torch.int32, device="cuda")
        best = 0.0
        for _ in range(3):
            n, ms = cs.cs_atomic_rate(buf.data_ptr(), buf.numel(), 256, stream)
            best = max(best, n / (ms / 1e3))
        del buf
        return best
    except Exception:   # reported as missing, never replaced by a derived figure
        return None


def roofline(dom, kern_ms, kern_n, stats, info, params, peaks, peak_src, issue, config, clears_peak=None,
             band_peak=None):
    """Roofline of the dominant kernel class over its average CUDA-event launch
    duration (timed on the launching stream).  The large-prime walk has two
    bounds: the integer issue rate (thread instructions per sieve, from stored
    ncu counters, against cs_issue_rate) and its memory side.  With direct
    clears that is the scattered bit clears (its stored hits, F_large, counted
    live, against cs_atomic_rate over a region of the bitset's size); with hit
    buckets it is the 4-byte records it writes (against the measured HBM copy
    rate), and the apply kernel that clears them gets its own entry (records
    counted live, against cs_atomic_rate over a region of two bands).  The
    bound that needs more time binds; achieved, peak and frac are given in its
    units, the other bound beside it."""
    name = KC_NAMES[dom]
    n_launch = max(kern_n[dom], 1)
    per_launch_s = kern_ms[dom] / n_launch / 1e3
    if name == "final":
        bytes_ = int(info.bitset_bytes) + 4 * int(info.M_c)
        achieved = bytes_ / per_launch_s / 1e9
        peak = float(peaks["hbm_gbs"])
        return {"kernel": "k_final", "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "peak_source": f"hbm_gbs, {peak_src}"}
    # integer kernels: thread-level instructions against the measured integer
    # issue rate (the best mix of the micro-benchmark, timed in this run)
    rates = {k: v for k, v in issue.items() if isinstance(v, float)}
    peak = max(rates.values()) if rates else None
    out = {"kernel": "k_large_tg" if name == "large_walk" else name, "bound": "alu", "achieved": None,
           "peak": peak, "unit": "Tinst/s", "frac": None, "traffic": None,
           "peak_source": "measured in this run: cs_issue_rate integer micro-benchmark, best of its mixes "
                          "(burst, one wave at full occupancy)",
           "issue_rates_Tops": issue}
    if name != "large_walk":
        out["note"] = "no stored instruction counts for this kernel"
        return out
    n_chunks = max(int(info.n_large_chunks), 1)
    ctr = WALK_COUNTERS.get(config)
    # the counters hold for the same sources, threshold, tile height and chunking
    # (one walk launch per large-prime chunk)
    same_setup = ctr is not None and (ctr.get("threshold"), ctr.get("tile_rows"), ctr.get("launches")) == (
        int(info.threshold), int(info.tile_rows), int(info.n_large_chunks))
    issue_b = None
    if ctr and ctr["csrc_sha"] == csrc_sha() and same_setup and peak:
        inst_launch = ctr["thread_inst"] / ctr["launches"]
        achieved = inst_launch / per_launch_s / 1e12
        issue_b = {"achieved": achieved, "peak": peak, "unit": "Tinst/s", "frac": achieved / peak,
                   "min_ms_per_launch": inst_launch / (peak * 1e12) * 1e3, "thread_inst_per_launch": inst_launch}
        if ctr.get("dram_bytes") is not None:
            out["traffic"] = ctr["dram_bytes"] / ctr["launches"]
    clears_b = records_b = None
    if info.hit_buckets:
        rec_launch = stats["bucket_records"] / n_chunks       # records written by one walk launch
        hbm = float(peaks["hbm_gbs"]) * 1e9
        records_b = {"achieved": rec_launch * 4 / per_launch_s / 1e9, "peak": hbm / 1e9, "unit": "GB/s",
                     "frac": rec_launch * 4 / per_launch_s / hbm, "min_ms_per_launch": rec_launch * 4 / hbm * 1e3,
                     "records_per_launch": rec_launch}
        ia = KC_NAMES.index("hit_apply")
        if kern_n[ia] and band_peak:
            apply_s = kern_ms[ia] / 1e3 / max(n_launch / n_chunks, 1)     # apply seconds per sieve
            ach = stats["bucket_records"] / apply_s
            out["apply"] = {"kernel": "k_apply_buckets", "achieved": ach / 1e9, "peak": band_peak / 1e9,
                            "unit": "Gclears/s", "frac": ach / band_peak,
                            "launches_per_sieve": int(info.apply_launches), "ms_per_sieve": apply_s * 1e3,
                            "peak_source": "measured in this run: cs_atomic_rate over a region of two bands' "
                                           "words (best of three launches)"}
    elif clears_peak:
        clears_launch = stats["F_large"] / n_chunks           # stored hits: one bit clear each
        achieved = clears_launch / per_launch_s / 1e9
        clears_b = {"achieved": achieved, "peak": clears_peak / 1e9, "unit": "Gclears/s",
                    "frac": achieved / (clears_peak / 1e9), "min_ms_per_launch": clears_launch / clears_peak * 1e3,
                    "clears_per_launch": clears_launch}
    out["bounds"] = {"issue": issue_b, "clears": clears_b, "records": records_b}
    # the walker preparation of the one-walker chunks (its own kernel, k_tg_prep)
    ip = KC_NAMES.index("walk_prep")
    if kern_n[ip] and issue_b and ctr.get("prep_thread_inst") and ctr.get("prep_launches") == int(info.prep_chunks):
        prep_s = kern_ms[ip] / 1e3 / max(n_launch / n_chunks, 1)       # prep seconds per sieve
        ach = ctr["prep_thread_inst"] / prep_s / 1e12
        out["prep"] = {"kernel": "k_tg_prep", "achieved": ach, "peak": peak, "unit": "Tinst/s",
                       "frac": ach / peak, "ms_per_sieve": prep_s * 1e3, "launches_per_sieve": int(info.prep_chunks)}
    out["launches_timed"] = n_launch
    walk_s = kern_ms[dom] / 1e3 / max(n_launch / n_chunks, 1)   # walk seconds per sieve
    out["per_unit_rates"] = {"visited_hits_per_s": stats["hits_all"] / walk_s, "levels_per_s": stats["levels"] / walk_s,
                             "clears_per_s": stats["F_large"] / walk_s}
    binding = None
    mem_b = clears_b or records_b
    if issue_b and mem_b:
        binding = "memory" if mem_b["min_ms_per_launch"] >= issue_b["min_ms_per_launch"] else "issue"
    elif mem_b:
        binding = "memory"
    elif issue_b:
        binding = "issue"
    if binding == "memory" and records_b:
        binding = "records"
    elif binding == "memory":
        binding = "clears"
    if binding == "issue":
        out.update(achieved=issue_b["achieved"], frac=issue_b["frac"])
    elif binding == "clears":
        out.update(bound="hbm", achieved=clears_b["achieved"], peak=clears_b["peak"], unit="Gclears/s",
                   frac=clears_b["frac"],
                   peak_source="measured in this run: cs_atomic_rate, one-bit 32-bit atomic ANDs at random "
                               "words of a region the size of the bitset (best of three launches)")
    elif binding == "records":
        out.update(bound="hbm", achieved=records_b["achieved"], peak=records_b["peak"], unit="GB/s",
                   frac=records_b["frac"], peak_source=f"hbm_gbs, {peak_src}")
    if not issue_b:
        out["note"] = "ncu instruction counts not recorded for these sources and this threshold / tile height"
    return out




# ------------------------------------------------------------ batched / served

def _flush(torch, buf, k):
    buf.fill_(k & 0xff)


def run_batched(args):
    """64 seeded instances of uneven size (the batched workload), four ways, each
    step timed on one stream with CUDA events:
      plain          one instance after another, each generating its own primes;
      plain_cached   one instance after another, large primes from the shared
                     residue caches (filled once per step, as in the batch);
      batch          the batch graph (worker streams, cache fills inside it)
                     with one walk launch per prime chunk (the default batch);
      graph_jobs     the batch graph with the walks of all instances as jobs of
                     a few persistent launches (CS_BATCH_JOBS=1).
    The headline ratio is batch against plain_cached: the caches on both arms."""
    import numpy as np
    import torch
    import paper_2012_03771_gb300 as cs
    from paper_2012_03771_gb300 import build
    build.build()
    cs.load()
    torch.cuda.set_device(0)
    mix = workloads.batched_instances(64)
    plans = [cs.Plan(*p.as_tuple()) for p in mix]
    s = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # reference results: every instance alone
    ref = []
    for p in plans:
        p.sieve(s).sync()
        counts, F, h = p.counts()
        ref.append((F, h, counts.copy()))
    F_total = sum(r[0] for r in ref)

    def same(ps):
        out = True
        for p, r in zip(ps, ref):
            counts, F, h = p.counts()
            out = out and (F, h) == r[:2] and np.array_equal(counts, r[2])
        return out

    def time_steps(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for k in range(args.steps):
            _flush(torch, flush, k)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            b.record(s)
            s.synchronize()
            ms.append(a.elapsed_time(b))
        return statistics.median(ms)

    def plain():
        for p in plans:
            p.sieve(s)

    arms = {"plain": time_steps(plain)}
    ok = same(plans)
    lim = {}
    for prm in mix:
        lim[(prm.P, prm.d)] = max(lim.get((prm.P, prm.d), 0), prm.L)
    caches = {k: cs.Cache(k[0], k[1], L) for k, L in lim.items()}
    cplans = [cs.Plan(*prm.as_tuple(), cache=caches[(prm.P, prm.d)]) for prm in mix]

    def plain_cached():
        for c in caches.values():
            c.fill(s)
        for p in cplans:
            p.sieve(s)

    arms["plain_cached"] = time_steps(plain_cached)
    ok = ok and same(cplans)
    os.environ["CS_BATCH_JOBS"] = "1"
    b_jobs = cs.Batch(cplans, n_streams=args.batch_streams)
    del os.environ["CS_BATCH_JOBS"]
    arms["graph_jobs"] = time_steps(lambda: b_jobs.run(s))
    b_jobs.sync()
    ok = ok and same(cplans)
    launches_jobs = b_jobs.launches
    b_jobs.close()
    batch = cs.Batch(cplans, n_streams=args.batch_streams)
    arms["batch"] = time_steps(lambda: batch.run(s))
    batch.sync()
    ok = ok and same(cplans)
    cache_bytes = sum(c.info()[1] for c in caches.values())
    line = {"metric": "enumerated factors/s, 64-instance batch (bit-exact)", "unit": UNIT,
            "value": F_total / (arms["batch"] / 1e3), "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": arms["batch"],
            "arms_ms_per_step": arms,
            "arms_value": {k: F_total / (v / 1e3) for k, v in arms.items()},
            "speedup_vs_plain_cached": arms["plain_cached"] / arms["batch"],
            "speedup_vs_plain": arms["plain"] / arms["batch"],
            "residue_caches": {"count": len(caches), "device_bytes": cache_bytes},
            "n_streams": batch.n_streams, "gpu_launches_per_step": batch.launches,
            "gpu_launches_per_step_jobs": launches_jobs, "F_per_step": F_total,
            "results_equal_alone": ok,
            "config": {"workload": "batched_64: P in {503,701,953,1019}, d in {210,2310}, M_inc log-U[1e3,1e6], "
                                   "SL U[5000,25000], L log-U[1e8,1e10], M_start log-U[1e6,1e8], seed 201203771",
                       "l2": "flushed between steps (256 MB device write)"}}
    print(json.dumps(line), flush=True)
    batch.close()
    for p in plans + cplans:
        p.close()
    for c in caches.values():
        c.close()


def run_served(args):
    """Seeded Poisson stream of requests from the batched distribution (seed + 1),
    continuous batching by the request server against one-at-a-time service."""
    import torch
    import paper_2012_03771_gb300 as cs
    from paper_2012_03771_gb300 import build
    build.build()
    cs.load()
    torch.cuda.set_device(0)
    n_req = args.requests
    reqs = workloads.batched_instances(n_req, seed=workloads.BATCH_SEED + 1)
    s = torch.cuda.Stream()
    # service time of each request alone (one stream, one after another)
    alone_ms, ref = [], []
    for prm in reqs:
        p = cs.Plan(*prm.as_tuple())
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        p.sieve(s)
        b.record(s)
        s.synchronize()
        alone_ms.append(a.elapsed_time(b))
        ref.append(cs.cs_counts(p.h))
        p.close()
    mean_ms = statistics.mean(alone_ms)
    rate = args.load / (mean_ms / 1e3)                  # requests/s at `load` of one-at-a-time capacity
    arrivals = workloads.poisson_arrivals(n_req, rate)
    free, total = torch.cuda.mem_get_info()
    budget = int(args.budget_frac * free)
    srv = cs.Server(budget_bytes=budget, max_slots=args.slots)
    lat, queue, pending, results = [0.0] * n_req, list(range(n_req)), {}, {}
    t0 = time.perf_counter()
    while queue or pending:
        now = time.perf_counter() - t0
        while queue and arrivals[queue[0]] <= now:
            i = queue[0]
            t = srv.submit(*reqs[i].as_tuple())
            if t is None:
                break
            pending[t] = i
            queue.pop(0)
        for t in list(pending):
            if srv.poll(t):
                i = pending.pop(t)
                lat[i] = time.perf_counter() - t0 - arrivals[i]
                bp = srv.plan(t)
                try:
                    cs.cs_sync(bp.h)
                    results[i] = cs.cs_counts(bp.h)
                except cs.CSError as e:
                    results[i] = ("error", str(e))
                srv.release(t)
        time.sleep(0.0002)
    makespan = time.perf_counter() - t0
    srv.close()
    # one-at-a-time service of the same arrivals (FIFO, measured service times)
    fifo_lat, end = [], 0.0
    for i in range(n_req):
        start = max(arrivals[i], end)
        end = start + alone_ms[i] / 1e3
        fifo_lat.append(end - arrivals[i])
    F_total = sum(f for f, _ in ref)
    pct = lambda v, q: sorted(v)[min(len(v) - 1, int(q * len(v)))]
    bad = [i for i in range(n_req) if results[i] != ref[i]]
    for i in bad[:8]:
        print(json.dumps({"mismatch": i, "params": reqs[i].as_tuple(), "got": str(results[i]),
                          "alone": list(ref[i])}), file=sys.stderr, flush=True)
    line = {"metric": "served sieve requests: latency and enumerated factors/s (bit-exact)", "unit": UNIT,
            "value": F_total / makespan, "requests": n_req, "arrival_rate_per_s": rate,
            "p50_ms": 1e3 * pct(lat, 0.5), "p99_ms": 1e3 * pct(lat, 0.99),
            "one_at_a_time": {"p50_ms": 1e3 * pct(fifo_lat, 0.5), "p99_ms": 1e3 * pct(fifo_lat, 0.99),
                              "value": F_total / max(end, 1e-9)},
            "slots": args.slots, "budget_bytes": budget,
            "results_equal_alone": all(results[i] == ref[i] for i in range(n_req)),
            "config": {"workload": f"served: {n_req} requests from the batched distribution (seed 201203772), "
                                   f"Poisson arrivals at {args.load:.2f} x the one-at-a-time capacity",
                       "budget": f"{args.budget_frac:.2f} of free device memory"}}
    print(json.dumps(line), flush=True)


def run_fig1(args):
    """The speed-up curve of combined sieving against sieving the intervals one
    at a time (the shape of Figure 1: K = 1511#/210, X = 18,000, L = 1e11), on
    the GPU (median of --fig1-repeats sieves per point), beside the CPU oracle's
    time for one interval: the oracle as it stands on this host's cores, timed
    on a bounded sample of the primes (those up to 2^24 and four windows of
    2^26 numbers) and scaled to all primes of (P, L] by the prime count."""
    import torch
    import paper_2012_03771_gb300 as cs
    from paper_2012_03771_gb300 import build, speedup_curve as sc
    build.build()
    cs.load()
    torch.cuda.set_device(0)
    res = sc.curve(repeats=args.fig1_repeats)
    f = sc.FIG1
    one = workloads.SieveParams(P=f["P"], d=f["d"], M_start=f["M_start"], M_inc=1, SL=f["SL"], L=f["L"])
    with cs.Plan(*one.as_tuple()) as p:
        p.sieve().sync()
        st = p.stats()
    n_all = st["n_small_primes"] + st["n_large_primes"]          # primes in (P, L], counted on the GPU
    oracle = None
    if not args.no_cpu:
        import oracle.oracle as O
        O.build()
        n_sample = sum(O.prime_stats(lo, hi)[0] for lo, hi in sample_ranges(one, args.ref_windows))
        F, dt, cores, _, _ = oracle_sample(one, 1, args.ref_windows)
        per_interval = dt * n_all / max(n_sample, 1)
        oracle = {"seconds_per_interval": per_interval, "sample_seconds": dt, "cores": cores,
                  "sample": f"1 interval (m = 1) x {sample_text(one, 1, 1, args.ref_windows).split(' x ')[1]}; "
                            f"{n_sample} of {n_all} primes, time scaled by the prime count"}
        for pt in res["points"]:
            pt["speedup_vs_oracle"] = pt["M_c"] * per_interval / pt["seconds"]
    line = {"metric": "speed-up of the combined sieve over one interval at a time (Figure 1 shape)",
            "config": {"workload": "fig1_1511: K=1511#/210, X=18000, primes 1511 < p <= 1e11, m from 1"},
            "curve": res, "oracle_one_interval": oracle}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--config", default="large_1019",
                    choices=sorted(workloads.NAMED) + ["batched_64", "served", "fig1_1511"])
    ap.add_argument("--fig1-repeats", type=int, default=5)
    ap.add_argument("--requests", type=int, default=256)
    ap.add_argument("--load", type=float, default=0.8)
    ap.add_argument("--slots", type=int, default=2)
    ap.add_argument("--batch-streams", type=int, default=0)
    ap.add_argument("--budget-frac", type=float, default=0.5)
    ap.add_argument("--mode", type=int, default=0)
    ap.add_argument("--threshold", type=int, default=0)
    ap.add_argument("--ref-rows", type=int, default=256, help="oracle sample: evenly spaced coprime m")
    ap.add_argument("--ref-windows", type=int, default=4, help="oracle sample: prime windows above 2^24")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--layout", type=int, default=0, help="1 = compact rows (no wheel offsets stored)")
    args = ap.parse_args()
    rank, ws = _dist()
    if args.config == "batched_64":
        return run_batched(args)
    if args.config == "served":
        return run_served(args)
    if args.config == "fig1_1511":
        return run_fig1(args)
    params = _params_for_rank(workloads.NAMED[args.config], rank)
    if args.impl == "reference":
        run_reference(args, params)
    else:
        run_cuda(args, params)


if __name__ == "__main__":
    main()
