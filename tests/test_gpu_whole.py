"""Whole-workload parity on the GPU against stored oracle values.

The expected values in tests/golden/<name>.npz were written by
tests/golden/make_config_goldens.py, which calls only the CPU oracle (the
traditional sieve of Section 2.1 with the cached K mod p of Section 3.1).  The
CUDA path runs the full workloads through the C ABI, exactly as bench.py does,
and is compared element by element (integers: tolerance 0):

* search_953 (K = 953#/210, 22,858 rows, L = 1e9): every row's survivor count
  and checksum, the total F and the bitset checksum;
* large_1019 (K = 1019#/210, 2.29M rows, L = 1e11, 64-bit path): 257 sampled
  rows (256 evenly spaced and the row of the 36,702 record gap);
* the 64-instance batched mix (seed 201203771) in one batch with shared
  residue caches: four rows of every instance against the oracle, and every
  instance's counts, F and checksum equal to the instance alone;
* the 256-request served stream (seed 201203772) through the request server
  (continuous batching, admission by memory): four rows of every request
  against the oracle, and every request equal to its result alone;
* the speed-up curve's 10-interval point (the shape of Figure 1: K = 1511#/210,
  X = 18,000, primes up to 1e11): every row, F and the checksum.

A row's checksum is the oracle's bitset checksum of that row alone at its
position in the bitset (the checksum of a whole bitset is the sum of its rows').
"""
import os
import time

import numpy as np
import pytest

import oracle.oracle as O
import paper_2012_03771_gb300 as cs
from paper_2012_03771_gb300 import workloads
from tests.conftest import ROOT

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_03771_gb300 import build
    build.build()
    cs.load()
    torch.cuda.set_device(0)


def _golden(name):
    path = os.path.join(GOLDEN, f"{name}.npz")
    assert os.path.exists(path), f"{path} missing: run tests/golden/make_config_goldens.py --only {name}"
    return np.load(path)


def _row_hash(plan, i):
    return O.bitset_hash(plan.fetch_rows(int(i), 1), row0=int(i))


def _check_rows(plan, counts, idx, want_m, want_counts, want_hash, label):
    rows = plan.rows()
    for k, i in enumerate(idx):
        assert int(rows[i]) == int(want_m[k]), (label, i)
        assert int(counts[i]) == int(want_counts[k]), (label, i)
        assert _row_hash(plan, i) == int(want_hash[k]), (label, i)


def test_search_953_every_row_matches_oracle():
    g = _golden("search_953")
    prm = workloads.SEARCH_953
    assert tuple(int(v) for v in g["params"]) == prm.as_tuple()
    with cs.Plan(*prm.as_tuple()) as p:
        p.sieve(torch.cuda.current_stream()).sync()
        counts, F, h = p.counts()
        assert p.M_c == int(g["M_c"]) and p.W == int(g["W"])
        rows = p.rows()
        assert int(rows[0]) == int(g["m_first"]) and int(rows[-1]) == int(g["m_last"])
        assert F == int(g["F"]) and h == int(g["hash"])
        assert np.array_equal(counts, g["counts"])
        bits = p.bitset()
    got = np.array([O.bitset_hash(bits[i:i + 1], row0=i) for i in range(len(bits))], dtype=np.uint64)
    bad = np.nonzero(got != g["row_hash"])[0]
    assert bad.size == 0, f"{bad.size} rows differ, first {bad[:8]}"


def test_large_1019_sampled_rows_match_oracle():
    g = _golden("large_1019")
    prm = workloads.LARGE_1019
    assert tuple(int(v) for v in g["params"]) == prm.as_tuple()
    idx = [int(i) for i in g["row_idx"]]
    assert len(idx) >= 257 and int(g["i_record"]) in idx
    with cs.Plan(*prm.as_tuple()) as p:
        p.sieve(torch.cuda.current_stream()).sync()
        assert p.M_c == int(g["M_c"])
        counts, F, h = p.counts()
        _check_rows(p, counts, idx, g["m"], g["counts"], g["row_hash"], "large_1019")


def _alone(prm):
    with cs.Plan(*prm.as_tuple()) as p:
        p.sieve(torch.cuda.current_stream()).sync()
        counts, F, h = p.counts()
        return counts.copy(), F, h


def _check_instances(g, mix, results, plans_or_rows):
    """Oracle rows of every instance: (instance k, row index, m, count, checksum)."""
    for k in range(len(mix)):
        sel = np.nonzero(g["inst"] == k)[0]
        if not sel.size:
            continue
        counts = results[k][0]
        fetch = plans_or_rows[k]
        for s in sel:
            i = int(g["row_idx"][s])
            m_i, bits_i = fetch(i)
            assert m_i == int(g["m"][s]), (k, i)
            assert int(counts[i]) == int(g["counts"][s]), (k, i)
            assert O.bitset_hash(bits_i, row0=i) == int(g["row_hash"][s]), (k, i)


def test_batched_64_mix_matches_alone_and_oracle():
    g = _golden("batched_64")
    mix = workloads.batched_instances(64, seed=workloads.BATCH_SEED)
    assert [tuple(int(v) for v in r) for r in g["params"]] == [prm.as_tuple() for prm in mix]
    ref = [_alone(prm) for prm in mix]
    lim = {}
    for prm in mix:
        lim[(prm.P, prm.d)] = max(lim.get((prm.P, prm.d), 0), prm.L)
    caches = {k: cs.Cache(k[0], k[1], L) for k, L in lim.items()}
    plans = [cs.Plan(*prm.as_tuple(), cache=caches[(prm.P, prm.d)]) for prm in mix]
    batch = cs.Batch(plans)
    try:
        s = torch.cuda.Stream()
        for _ in range(2):                                   # capture once, replay
            batch.run(s).sync()
            res = [p.counts() for p in plans]
            for k, ((c2, F2, h2), (c1, F1, h1)) in enumerate(zip(res, ref)):
                assert (F2, h2) == (F1, h1), k
                assert np.array_equal(c2, c1), k
        rows = [p.rows() for p in plans]
        fetch = [(lambda i, p=p, r=r: (int(r[i]), p.fetch_rows(i, 1))) for p, r in zip(plans, rows)]
        _check_instances(g, mix, res, fetch)
    finally:
        batch.close()
        for p in plans:
            p.close()
        for c in caches.values():
            c.close()


def test_served_256_stream_matches_alone_and_oracle():
    g = _golden("served_256")
    reqs = workloads.batched_instances(256, seed=workloads.BATCH_SEED + 1)
    assert [tuple(int(v) for v in r) for r in g["params"]] == [prm.as_tuple() for prm in reqs]
    ref = [_alone(prm) for prm in reqs]
    free, _ = torch.cuda.mem_get_info()
    srv = cs.Server(budget_bytes=int(0.5 * free), max_slots=2)
    results, fetched = {}, {}
    want = {}
    for s in range(len(g["inst"])):
        want.setdefault(int(g["inst"][s]), []).append(int(g["row_idx"][s]))
    pending, queue = {}, list(range(len(reqs)))
    t0 = time.time()
    try:
        while queue or pending:
            while queue:
                t = srv.submit(*reqs[queue[0]].as_tuple())
                if t is None:
                    break                                    # no slot or memory: later
                pending[t] = queue.pop(0)
            for t in list(pending):
                if srv.poll(t):
                    k = pending.pop(t)
                    plan = srv.plan(t)
                    plan.sync()
                    counts, F, h = plan.counts()
                    results[k] = (counts.copy(), F, h)
                    rows = plan.rows()
                    fetched[k] = {i: (int(rows[i]), plan.fetch_rows(i, 1)) for i in want.get(k, [])}
                    srv.release(t)
            assert time.time() - t0 < 900, "requests did not finish"
            time.sleep(0.0005)
        assert srv.usage() == (0, 0, 0)
    finally:
        srv.close()
    for k, (c1, F1, h1) in enumerate(ref):
        c2, F2, h2 = results[k]
        assert (F2, h2) == (F1, h1), k
        assert np.array_equal(c2, c1), k
    _check_instances(g, reqs, results, [lambda i, k=k: fetched[k][i] for k in range(len(reqs))])


def test_fig1_point_matches_oracle():
    from paper_2012_03771_gb300.speedup_curve import m_inc_for
    g = _golden("fig1_1511")
    P, d, M_start, M_inc, SL, L = (int(v) for v in g["params"])
    assert M_inc == m_inc_for(M_start, d, 10)
    with cs.Plan(P, d, M_start, M_inc, SL, L) as p:
        p.sieve(torch.cuda.current_stream()).sync()
        counts, F, h = p.counts()
        assert F == int(g["F"]) and h == int(g["hash"])
        _check_rows(p, counts, range(10), g["m"], g["counts"], g["row_hash"], "fig1_1511")
