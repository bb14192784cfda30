"""Writes the stored expected values of the whole-workload parity tests.

Every value in the files this script writes comes from the CPU oracle
(``oracle/``: the traditional sieve of Section 2.1 with the cached K mod p of
Section 3.1).  Nothing here imports the CUDA package: the seeded parameter
draws are read from ``paper_2012_03771_gb300/workloads.py`` by file path (that
module holds parameter tuples only, none of the method's arithmetic).

  python tests/golden/make_config_goldens.py [--only NAME ...] [--threads N]

NAME is one of:
  search_953   K = 953#/210, m in [1e8, 1e8 + 1e5) coprime to 210, X = 20000,
               primes up to 1e9: every row (22,858), i.e. per-row survivor
               counts, per-row enumerated factors, per-row checksums, and the
               totals F and checksum.  About 35 minutes on 8 cores.
  large_1019   K = 1019#/210, m in [1.64e8, 1.74e8), X = 25000, primes up to
               1e11: 256 evenly spaced rows plus the row of the 36,702 record
               gap (Section 1.1).  About 35 minutes on 8 cores.
  batched_64   the 64-instance mix (seed 201203771): 4 evenly spaced rows of
               every instance.
  served_256   the 256-request served stream (seed 201203772): 4 evenly
               spaced rows of every request.
  fig1_1511    the speed-up curve's 10-interval point (Figure 1's shape: K =
               1511#/210, X = 18,000, primes up to 1e11, m = 1 .. 41): every
               row.  About 6 minutes on 8 cores.

Per-row checksum: the oracle's bitset checksum of the row alone, taken at the
row's position in the whole bitset (``oracle.bitset_hash(row, row0=i)``); the
checksum of a whole bitset is the sum of its rows' (mod 2^64).

Output: ``tests/golden/<NAME>.npz`` (numpy, compressed).
"""
from __future__ import annotations

import argparse
import importlib.util
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle.oracle as O  # noqa: E402


def _workloads():
    """The seeded input generator module, loaded by path (no package import)."""
    path = os.path.join(ROOT, "paper_2012_03771_gb300", "workloads.py")
    spec = importlib.util.spec_from_file_location("cs_seeded_workloads", path)
    mod = importlib.util.module_from_spec(spec)
    sys.modules[spec.name] = mod
    spec.loader.exec_module(mod)
    return mod


WL = _workloads()
U64 = np.uint64


def _row_hashes(bits: np.ndarray, idx) -> np.ndarray:
    return np.array([O.bitset_hash(bits[k:k + 1], row0=int(i)) for k, i in enumerate(idx)], dtype=U64)


def _even_rows(n_rows: int, k: int):
    """k evenly spaced row indices of [0, n_rows), first and last included."""
    if n_rows <= 0:
        return []
    return sorted({int(round(j * (n_rows - 1) / max(k - 1, 1))) for j in range(k)})


def search_953(threads: int):
    prm = WL.SEARCH_953
    m, bits, F = O.full_sieve(*prm.as_tuple(), threads=threads)
    counts = O.row_counts(bits)
    rh = _row_hashes(bits, range(len(m)))
    total = O.bitset_hash(bits)
    assert int(rh.sum(dtype=U64)) == total           # the checksum is additive over rows
    return dict(params=np.array(prm.as_tuple(), dtype=np.int64), m_first=U64(m[0]), m_last=U64(m[-1]),
                M_c=np.int64(len(m)), W=np.int64(len(O.columns(prm.P, prm.d, prm.SL))),
                counts=counts.astype(np.uint32), F_rows=F.astype(np.uint32), row_hash=rh,
                F=U64(int(F.sum())), hash=U64(total))


def large_1019(threads: int, n_sample: int = 256):
    prm = WL.LARGE_1019
    rows = O.rows(prm.d, prm.M_start, prm.M_inc)
    i_rec = int(np.searchsorted(rows, WL.RECORD_1019[0]))
    assert rows[i_rec] == WL.RECORD_1019[0]
    idx = sorted(set(_even_rows(len(rows), n_sample)) | {i_rec})
    m = rows[idx]
    bits, F, _ = O.sieve(prm.P, prm.d, prm.SL, prm.L, m, threads=threads)
    return dict(params=np.array(prm.as_tuple(), dtype=np.int64), M_c=np.int64(len(rows)),
                row_idx=np.array(idx, dtype=np.int64), m=m.astype(U64), i_record=np.int64(i_rec),
                counts=O.row_counts(bits).astype(np.uint32), F_rows=F.astype(np.uint32),
                row_hash=_row_hashes(bits, idx))


def _instances(mix, threads: int, per: int = 4):
    params, M_c, inst, idx_all, m_all, cnt, Fr, rh = [], [], [], [], [], [], [], []
    for k, prm in enumerate(mix):
        rows = O.rows(prm.d, prm.M_start, prm.M_inc)
        idx = _even_rows(len(rows), per)
        params.append(prm.as_tuple())
        M_c.append(len(rows))
        if not idx:
            continue
        m = rows[idx]
        bits, F, _ = O.sieve(prm.P, prm.d, prm.SL, prm.L, m, threads=threads)
        inst += [k] * len(idx)
        idx_all += idx
        m_all += [int(v) for v in m]
        cnt += [int(c) for c in O.row_counts(bits)]
        Fr += [int(f) for f in F]
        rh += [int(h) for h in _row_hashes(bits, idx)]
        print(f"  instance {k}: {prm.as_tuple()} rows {idx}", flush=True)
    return dict(params=np.array(params, dtype=np.int64), M_c=np.array(M_c, dtype=np.int64),
                inst=np.array(inst, dtype=np.int64), row_idx=np.array(idx_all, dtype=np.int64),
                m=np.array(m_all, dtype=U64), counts=np.array(cnt, dtype=np.uint32),
                F_rows=np.array(Fr, dtype=np.uint32), row_hash=np.array(rh, dtype=U64))


def fig1_1511(threads: int):
    P, d, SL, L = 1511, 210, 18000, 10**11
    rows = O.rows(d, 1, 41)                           # the first 10 m coprime to 210
    assert len(rows) == 10
    bits, F, _ = O.sieve(P, d, SL, L, rows, threads=threads)
    return dict(params=np.array((P, d, 1, 41, SL, L), dtype=np.int64), m=rows.astype(U64),
                counts=O.row_counts(bits).astype(np.uint32), F_rows=F.astype(np.uint32),
                row_hash=_row_hashes(bits, range(len(rows))), F=U64(int(F.sum())), hash=U64(O.bitset_hash(bits)))


def batched_64(threads: int):
    return _instances(WL.batched_instances(64, seed=WL.BATCH_SEED), threads)


def served_256(threads: int):
    return _instances(WL.batched_instances(256, seed=WL.BATCH_SEED + 1), threads)


JOBS = {"search_953": search_953, "large_1019": large_1019, "batched_64": batched_64, "served_256": served_256,
        "fig1_1511": fig1_1511}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--only", nargs="*", default=list(JOBS), choices=list(JOBS))
    ap.add_argument("--threads", type=int, default=0, help="oracle threads (0 = all cores)")
    args = ap.parse_args()
    O.build()
    for name in args.only:
        t0 = time.time()
        print(f"{name} ...", flush=True)
        out = JOBS[name](args.threads)
        out["generator"] = np.array(f"tests/golden/make_config_goldens.py --only {name}")
        path = os.path.join(HERE, f"{name}.npz")
        np.savez_compressed(path, **out)
        print(f"{name}: wrote {path} in {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
