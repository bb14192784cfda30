"""Speed-up of the combined sieve over sieving its intervals one at a time, as
the number of intervals grows: the shape of the paper's Figure 1 (Section 2,
K = 1511#/7#, X = 18,000, sieving limit 1e11).

For each M_c (intervals m coprime to d, counted from M_start) one plan sieves
all of them at once; the same plan type with M_c = 1 is the one-at-a-time
baseline, so the speed-up is M_c * t(1) / t(M_c).  Times are the wall time of
cs_sieve + cs_sync, `repeats` sieves per point after one untimed sieve; the
speed-up uses the medians, and the spread (fastest, slowest) is reported.
bench.py --config fig1_1511 adds the CPU oracle's time per interval beside it.

  python -m paper_2012_03771_gb300.speedup_curve [--repeats 5] [--out curve.json]
"""
from __future__ import annotations

import argparse
import json
import math
import statistics
import time

from . import Plan


def m_inc_for(M_start: int, d: int, m_c: int) -> int:
    """Smallest M_inc whose interval [M_start, M_start + M_inc) holds m_c values coprime to d."""
    n, m = 0, M_start
    while n < m_c:
        n += math.gcd(m, d) == 1
        m += 1
    return m - M_start


FIG1 = dict(P=1511, d=210, SL=18000, L=10**11, M_start=1)
M_CS = (1, 10, 100, 1000, 10000, 100000)


def curve(P=1511, d=210, SL=18000, L=10**11, M_start=1, m_cs=M_CS, repeats=5):
    points = []
    warm = True
    for m_c in m_cs:
        M_inc = m_inc_for(M_start, d, m_c)
        with Plan(P, d, M_start, M_inc, SL, L) as plan:
            if warm:
                plan.sieve().sync()
                warm = False
            ts = []
            for _ in range(max(repeats, 1)):
                t0 = time.perf_counter()
                plan.sieve().sync()
                ts.append(time.perf_counter() - t0)
            _, F, h = plan.counts()
            points.append({"M_c": int(plan.M_c), "M_inc": M_inc, "seconds": statistics.median(ts),
                           "seconds_min": min(ts), "seconds_max": max(ts), "repeats": len(ts), "F": int(F),
                           "hash": hex(h)})
    base = next(p["seconds"] for p in points if p["M_c"] == 1)
    for p in points:
        p["seconds_per_interval"] = p["seconds"] / p["M_c"]
        p["speedup"] = p["M_c"] * base / p["seconds"]
    return {"K": f"{P}#/{d}", "X": SL, "L": L, "M_start": M_start, "points": points}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--repeats", type=int, default=5)
    args = ap.parse_args()
    res = curve(repeats=args.repeats)
    line = json.dumps(res)
    print(line, flush=True)
    if args.out:
        with open(args.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
