"""Batched (CUDA graph over worker streams) and served (continuous batching)
execution: every instance's result is the same alone, in a batch and in the
served mix, exactly (integers; tolerance 0)."""
import time

import numpy as np
import pytest

import oracle.oracle as O
import paper_2012_03771_gb300 as cs
from paper_2012_03771_gb300 import workloads

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_03771_gb300 import build
    build.build()
    cs.load()
    torch.cuda.set_device(0)


def _small_mix(n, seed):
    """The batched distribution, shrunk so that the test runs in seconds."""
    out = []
    for prm in workloads.batched_instances(n, seed=seed):
        out.append(prm.with_(M_inc=max(50, prm.M_inc // 200), SL=prm.SL // 5,
                             L=min(prm.L, 3 * 10**8) if prm.L < 2**30 else 2**30 + 10**7))
    return out


def _alone(prm):
    with cs.Plan(*prm.as_tuple()) as p:
        p.sieve(torch.cuda.current_stream()).sync()
        counts, F, h = p.counts()
        return counts.copy(), F, h


def test_batch_equals_alone_and_replays():
    mix = _small_mix(12, seed=5)
    ref = [_alone(prm) for prm in mix]
    plans = [cs.Plan(*prm.as_tuple()) for prm in mix]
    batch = cs.Batch(plans, n_streams=4)
    assert batch.n_streams == 4
    assert batch.launches == sum(int(p.info.launches_per_sieve) for p in plans)
    s = torch.cuda.Stream()
    for _ in range(2):                                   # capture once, replay twice
        batch.run(s).sync()
        for p, (counts, F, h) in zip(plans, ref):
            c2, F2, h2 = p.counts()
            assert (F2, h2) == (F, h)
            assert np.array_equal(c2, counts)
    batch.close()
    for p in plans:
        p.close()


def test_batch_rejects_duplicates_and_profiled_plans():
    prm = _small_mix(1, seed=6)[0]
    with cs.Plan(*prm.as_tuple()) as p, cs.Plan(*prm.as_tuple(), profile=True) as q:
        with pytest.raises(cs.CSError):
            cs.Batch([p, p])
        with pytest.raises(cs.CSError):
            cs.Batch([q])


def test_batched_sample_rows_against_oracle():
    """Two instances of the batch, two rows each, against the CPU oracle."""
    mix = _small_mix(4, seed=7)
    plans = [cs.Plan(*prm.as_tuple()) for prm in mix]
    b = cs.Batch(plans, n_streams=2)
    b.run().sync()
    for prm, p in zip(mix[:2], plans[:2]):
        rows = p.rows()
        bits = p.bitset()
        pick = [0, len(rows) - 1]
        ref, _, _ = O.sieve(prm.P, prm.d, prm.SL, prm.L, [int(rows[i]) for i in pick])
        for k, i in enumerate(pick):
            assert np.array_equal(bits[i], ref[k])
    b.close()
    for p in plans:
        p.close()


def _drain(server, pending, results, t_limit=120.0):
    t0 = time.time()
    while pending and time.time() - t0 < t_limit:
        for t in list(pending):
            if server.poll(t):
                plan = server.plan(t)
                counts, F, h = plan.counts()
                results[pending.pop(t)] = (counts.copy(), F, h)
                server.release(t)
        time.sleep(0.001)
    assert not pending, "requests did not finish"


def test_server_results_equal_alone():
    """Requests that arrive while others run are admitted as slots free up."""
    mix = _small_mix(10, seed=8)
    ref = [_alone(prm) for prm in mix]
    srv = cs.Server(budget_bytes=4 << 30, max_slots=3)
    pending, results, queue = {}, {}, list(enumerate(mix))
    t0 = time.time()
    while queue or pending:
        if queue:
            i, prm = queue[0]
            t = srv.submit(*prm.as_tuple())
            if t is not None:
                pending[t] = i
                queue.pop(0)
        for t in list(pending):
            if srv.poll(t):
                plan = srv.plan(t)
                plan.sync()                                  # device status of the request
                counts, F, h = plan.counts()
                results[pending.pop(t)] = (counts.copy(), F, h)
                srv.release(t)
        assert time.time() - t0 < 300
    for i, (counts, F, h) in enumerate(ref):
        c2, F2, h2 = results[i]
        assert (F2, h2) == (F, h), i
        assert np.array_equal(c2, counts)
    assert srv.usage() == (0, 0, 0)
    srv.close()


def test_server_admission_by_memory_and_slots():
    prm = _small_mix(1, seed=9)[0]
    probe = cs.Server(budget_bytes=1 << 40, max_slots=1)     # device bytes of one request
    t0 = probe.submit(*prm.as_tuple())
    need = probe.usage()[0]
    while not probe.poll(t0):
        time.sleep(0.001)
    probe.close()
    assert need > 0
    srv = cs.Server(budget_bytes=need + need // 2, max_slots=4)
    t1 = srv.submit(*prm.as_tuple())
    assert t1 is not None
    assert srv.submit(*prm.as_tuple()) is None          # over budget: refused, nothing kept
    while not srv.poll(t1):
        time.sleep(0.001)
    assert srv.usage()[2] == 1                          # result still resident
    assert srv.submit(*prm.as_tuple()) is None          # still over budget while resident
    srv.release(t1)
    t2 = srv.submit(*prm.as_tuple())
    assert t2 is not None
    while not srv.poll(t2):
        time.sleep(0.001)
    srv.release(t2)
    one = cs.Server(budget_bytes=1 << 40, max_slots=1)
    a = one.submit(*prm.as_tuple())
    b = one.submit(*prm.as_tuple())                     # the only slot is busy (or just done)
    assert a is not None
    if b is None:
        while not one.poll(a):
            time.sleep(0.001)
        assert one.submit(*prm.as_tuple()) is not None
    one.close()
    srv.close()


# ------------------------------------------------------------- residue cache

def test_cached_plans_equal_plain_plans():
    """Large primes from the shared (p, K mod p) cache give the same bits."""
    cases = [workloads.PLAIN_503,
             workloads.SieveParams(P=503, d=2310, M_start=10**6, M_inc=3000, SL=3000, L=3 * 10**9),
             workloads.SieveParams(P=503, d=210, M_start=7, M_inc=400, SL=2000, L=2 * 10**6)]
    for prm in cases:
        ref = _alone(prm)
        cache = cs.Cache(prm.P, prm.d, 4 * 10**9)
        cache.fill(torch.cuda.current_stream())
        for mode in (1, 2):
            with cs.Plan(*prm.as_tuple(), cache=cache, large_mode=mode) as p:
                p.sieve(torch.cuda.current_stream()).sync()
                counts, F, h = p.counts()
                assert (F, h) == ref[1:], (prm, mode)
                assert np.array_equal(counts, ref[0])
        n_chunks, nbytes, n_primes = cache.info(count=True)
        cache.close()


def test_cache_holds_every_prime():
    cache = cs.Cache(953, 210, 2 * 10**8)
    cache.fill()
    _, _, n = cache.info(count=True)
    count, _, _ = O.prime_stats(0, _cache_limit(2 * 10**8))
    assert n == count
    cache.close()


def _cache_limit(L):
    """Upper end of the cache grid that covers L: (0, 2^16], then doubling
    chunks up to 2^27 wide, then 2^27 wide."""
    hi = 1 << 16
    while hi < L:
        hi += min(hi, 1 << 27)
    return hi


def test_cached_plan_needs_a_filled_cache():
    prm = _small_mix(1, seed=10)[0]
    cache = cs.Cache(prm.P, prm.d, prm.L)
    with cs.Plan(*prm.as_tuple(), cache=cache) as p:
        with pytest.raises(cs.CSError) as e:
            p.sieve()
        assert e.value.code == cs.CS_ESTATE
    with pytest.raises(cs.CSError):
        cs.Plan(prm.P, prm.d, prm.M_start, prm.M_inc, prm.SL, _cache_limit(prm.L) + 1, cache=cache)
    cache.close()


def test_batch_of_cached_plans_equals_alone():
    mix = _small_mix(10, seed=11)
    ref = [_alone(prm) for prm in mix]
    caches = {}
    for prm in mix:
        key = (prm.P, prm.d)
        caches[key] = max(caches.get(key, 0), prm.L)
    caches = {k: cs.Cache(k[0], k[1], L) for k, L in caches.items()}
    plans = [cs.Plan(*prm.as_tuple(), cache=caches[(prm.P, prm.d)]) for prm in mix]
    batch = cs.Batch(plans, n_streams=3)
    for _ in range(2):
        batch.run().sync()
        for p, (counts, F, h) in zip(plans, ref):
            c2, F2, h2 = p.counts()
            assert (F2, h2) == (F, h)
            assert np.array_equal(c2, counts)
    batch.close()
    for p in plans:
        p.close()
    for c in caches.values():
        c.close()


def test_batch_walk_jobs_equal_one_launch_per_chunk(monkeypatch):
    """Cached plans in a batch walk, with CS_BATCH_JOBS=1, as jobs of a few
    persistent launches (one per walk kernel); by default every chunk has its
    own launch.  Both give every instance's alone result, in fewer launches with
    the jobs."""
    mix = _small_mix(12, seed=12) + [workloads.SieveParams(P=503, d=2310, M_start=10**6, M_inc=3000, SL=3000,
                                                           L=3 * 10**9)]
    ref = [_alone(prm) for prm in mix]
    caches = {}
    for prm in mix:
        caches[(prm.P, prm.d)] = max(caches.get((prm.P, prm.d), 0), prm.L)
    caches = {k: cs.Cache(k[0], k[1], L) for k, L in caches.items()}
    plans = [cs.Plan(*prm.as_tuple(), cache=caches[(prm.P, prm.d)]) for prm in mix]
    launches = {}
    for jobs in ("1", "0"):
        monkeypatch.setenv("CS_BATCH_JOBS", jobs)
        batch = cs.Batch(plans, n_streams=2)
        monkeypatch.delenv("CS_BATCH_JOBS")
        launches[jobs] = batch.launches
        for _ in range(2):
            batch.run().sync()
            for p, (counts, F, h) in zip(plans, ref):
                c2, F2, h2 = p.counts()
                assert (F2, h2) == (F, h)
                assert np.array_equal(c2, counts)
        batch.close()
    assert launches["1"] < launches["0"]
    for p in plans:
        p.close()
    for c in caches.values():
        c.close()
