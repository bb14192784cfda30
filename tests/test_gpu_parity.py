"""CUDA path against the CPU oracle, through the C ABI.  Integer work: every
comparison is exact (bitsets, counts, F, checksum, primes, residues, solver)."""
import math
import random

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


def _run(params, **tuning):
    with cs.Plan(*params, **tuning) as plan:
        plan.sieve(torch.cuda.current_stream()).sync()
        bits = plan.bitset()
        counts, F, h = plan.counts()
        return dict(bits=bits, counts=counts, F=F, hash=h, rows=plan.rows(), cols=plan.columns(),
                    stats=plan.stats(), info=plan.info)


def _bits_only(params, **tuning):
    """Bitset, F and counts (also for the compact layout, whose columns vary by row)."""
    with cs.Plan(*params, **tuning) as plan:
        plan.sieve(torch.cuda.current_stream()).sync()
        counts, F, h = plan.counts()
        return dict(bits=plan.bitset(), counts=counts, F=F, hash=h, info=plan.info)


def _check_full(params, got, wheel=True):
    m_ref, bits_ref, F_ref = O.full_sieve(*params, wheel=wheel)
    assert np.array_equal(got["rows"], m_ref)
    assert np.array_equal(got["cols"], O.columns(params[0], params[1], params[4]))
    assert got["bits"].shape == bits_ref.shape
    bad = np.argwhere(got["bits"] != bits_ref)
    assert bad.size == 0, f"{len(bad)} words differ, first {bad[:3].tolist()}"
    assert got["F"] == int(F_ref.sum())
    assert np.array_equal(got["counts"], O.row_counts(bits_ref))
    assert got["hash"] == O.bitset_hash(bits_ref)


# ------------------------------------------------------------- single steps

def test_prime_generator_matches_oracle():
    for lo, hi in ((0, 2), (0, 10**6), (1, 3), (2, 3), (503, 10**7), (10**9 - 10**6, 10**9),
                   (2**31 - 5 * 10**5, 2**31 + 5 * 10**5), (2**40 - 3 * 10**5, 2**40)):
        ref = O.primes(lo, hi)
        cap = ref.size + 64
        buf = torch.zeros(cap, dtype=torch.int64, device="cuda")
        n = cs.cs_primes(lo, hi, buf.data_ptr(), cap, torch.cuda.current_stream())
        got = np.sort(buf[:n].cpu().numpy().astype(np.uint64))
        assert n == ref.size, (lo, hi)
        assert np.array_equal(got, ref), (lo, hi)


def test_prime_generator_overflow_is_reported():
    buf = torch.zeros(10, dtype=torch.int64, device="cuda")
    with pytest.raises(cs.CSError) as e:
        cs.cs_primes(0, 10**4, buf.data_ptr(), 10, torch.cuda.current_stream())
    assert e.value.code == cs.CS_EOVERFLOW


def test_k_mod_p_matches_oracle():
    rng = random.Random(1)
    for P, d in ((503, 210), (953, 210), (1019, 2310), (37, 6), (1, 1), (7, 210)):
        ps = list(O.primes(P, P + 20000)[:300])
        ps += list(O.primes(2**31 - 2000, 2**31 + 2000))
        ps += list(O.primes(2**40 - 5000, 2**40))
        ps += [int(x) for x in O.primes(10**9, 10**9 + 10**5)[::37]]
        p = torch.tensor(np.array(ps, dtype=np.uint64).view(np.int64), device="cuda")
        r = torch.zeros_like(p)
        cs.cs_k_mod_p(P, d, p.data_ptr(), p.numel(), r.data_ptr(), torch.cuda.current_stream())
        got = r.cpu().numpy().view(np.uint64)
        assert np.array_equal(got, O.k_mod_p(P, d, ps)), (P, d)


@pytest.mark.parametrize("narrow", [1, 0])
def test_modsolve_matches_paper_recursion(narrow):
    rng = random.Random(2 + narrow)
    pool = [101, 7919, 1000003, 999999937, (1 << 30) - 35] if narrow else \
           [1000003, 4294967291, 68719476731, 1099511627689, 999999937]
    rows = []
    for _ in range(4000):
        p = rng.choice(pool)
        K = rng.randrange(1, p)
        w = rng.choice([0, 1, 7, 100, 20000, 50000, rng.randrange(0, p // 2)])
        w = min(w, p - 1)
        L = rng.randrange(0, p - w)
        rows.append((p, K, L, L + w))
    arr = np.array(rows, dtype=np.uint64)
    dev = [torch.tensor(arr[:, i].view(np.int64), device="cuda") for i in range(4)]
    m = torch.zeros_like(dev[0])
    cs.cs_modsolve(*(t.data_ptr() for t in dev), m.data_ptr(), len(rows), narrow,
                   torch.cuda.current_stream())
    got = m.cpu().numpy().view(np.uint64)
    for (p, K, L, R), g in zip(rows, got):
        assert int(g) == O.G(p, K, L, R), (p, K, L, R)


# ------------------------------------------------------------- whole sieve

@pytest.mark.parametrize("mode", [1, 2])
def test_tiny_cases_bit_exact(mode):
    n = 0
    for prm in workloads.tiny_cases(150, seed=11):
        args = prm.as_tuple()
        if O.validate(*args):
            assert cs.cs_plan_status(*args) == cs.CS_EINVAL
            continue
        for T in (0, max(2 * prm.SL, 1)):
            got = _run(args, large_mode=mode, threshold=T)
            _check_full(args, got)
        got = _run(args, large_mode=mode, no_wheel=True)
        _check_full(args, got, wheel=False)
        n += 1
    assert n > 80


def _finest_item_mod(d):
    return next((Q for Q in (210, 30, 6, 2) if d % Q == 0), 0)


@pytest.mark.parametrize("m_classes", [1, 2, 3])
def test_m_class_walk_bit_exact(m_classes):
    """The three-gap walk over every m (1), over the m-classes coprime to
    Q = 6 or 2 in every chunk (2), and over class items (one work item per
    class of m mod 210, 30, 6 or 2, the largest that divides d) in every chunk
    (3) give the oracle's bitset; d = 6, 70 (Q = 2), 2310, and odd d (Q = 1),
    with M_start in every residue class mod 6."""
    n = 0
    for prm in workloads.tiny_cases(150, seed=12):
        args = prm.as_tuple()
        if O.validate(*args):
            continue
        got = _run(args, large_mode=2, threshold=max(2 * prm.SL, 1), m_classes=m_classes)
        _check_full(args, got)
        n += 1
    assert n > 80
    for d in (6, 70, 2310, 15):
        for M_start in range(1000, 1006):
            args = (101, d, M_start, 200, 500, 10**6)
            got = _run(args, large_mode=2, threshold=1000, m_classes=m_classes)
            info = got["info"]
            assert info.m_mod == ((6 if d % 6 == 0 else 2 if d % 2 == 0 else 1) if m_classes != 1 else 1)
            if m_classes == 3:
                Q = _finest_item_mod(d)
                assert info.item_mod == Q
                assert info.item_chunks == (info.n_large_chunks if Q else 0)
            else:
                assert info.item_chunks == 0
            _check_full(args, got)


@pytest.mark.parametrize("d", [30, 210, 2310])
def test_class_items_with_segments_bit_exact(d):
    """Class items (m coprime to 30 or 210, one work item per class) whose
    primes are also split into several m-segments: every chunk takes the
    finest class items (class_item_hits = 1) and items of about one hit, with
    M_start in several residue classes mod 210."""
    Q = 210 if d % 210 == 0 else 30
    for M_start in (1000, 1001, 1003, 1049, 1091, 1177):
        args = (101, d, M_start, 600, 300, 200_000)
        # class items in every chunk
        got = _run(args, large_mode=2, threshold=600, m_classes=3, item_hits=1)
        info = got["info"]
        assert info.item_mod == Q and info.item_classes == {30: 8, 210: 48}[Q]
        assert info.item_chunks == info.n_large_chunks > 0
        _check_full(args, got)
        # automatic tiers: class items mod 210 / 30 where a class has a hit per
        # prime, then the mod-6 classes and the odd m
        mixed = _run(args, large_mode=2, threshold=600, class_item_hits=1, item_hits=1)
        assert mixed["info"].item_mod == Q
        assert 0 < mixed["info"].item_chunks < mixed["info"].n_large_chunks
        assert np.array_equal(mixed["bits"], got["bits"]) and mixed["F"] == got["F"]


@pytest.mark.parametrize("band_rows_log, bucket_records", [(1, 0), (3, 16), (2, 1), (0, 0)])
def test_bucketed_hits_bit_exact(band_rows_log, bucket_records):
    """The walk's stored hits written as records to the walking CTA's region for
    their band of rows and cleared band after band give the oracle's bitset:
    with many small bands, with regions so small that most hits clear directly
    (1 or 16 records per region), with automatic bands, in the
    literal and the compact layout, for 32- and 64-bit primes and on the tiny
    brute-force cases."""
    kw = dict(hit_buckets=2, band_rows_log=band_rows_log, bucket_records=bucket_records)
    for prm in (workloads.PLAIN_503.with_(L=3 * 10**6),
                workloads.SieveParams(P=37, d=30, M_start=10**6, M_inc=300, SL=400, L=10**5)):
        args = prm.as_tuple()
        got = _run(args, threshold=max(2 * prm.SL, 1), **kw)
        info = got["info"]
        assert info.hit_buckets == 1 and info.n_bands >= 1 and info.apply_launches >= 1
        if band_rows_log:
            assert info.n_bands == -(-len(got["rows"]) // (1 << band_rows_log))
        assert info.apply_launches <= info.n_large_chunks
        # every stored hit is a record or (its region full) a direct clear
        assert 0 < got["stats"]["bucket_records"] <= got["stats"]["F_large"]
        if bucket_records == 1:
            assert got["stats"]["bucket_records"] < got["stats"]["F_large"]
        _check_full(args, got)
        comp = _bits_only(args, layout=1, **kw)
        lit = _bits_only(args, layout=1, hit_buckets=1)
        assert comp["info"].hit_buckets == 1 and lit["info"].hit_buckets == 0
        assert np.array_equal(comp["bits"], lit["bits"]) and comp["F"] == lit["F"]
    # 64-bit primes (L above 2^30): the whole bitset against direct clears,
    # sampled rows against the oracle
    prm = workloads.SieveParams(P=503, d=2310, M_start=10**6, M_inc=3000, SL=3000, L=3 * 10**9)
    got = _run(prm.as_tuple(), **kw)
    ref = _run(prm.as_tuple(), hit_buckets=1)
    assert got["info"].narrow == 0 and got["info"].hit_buckets == 1 and ref["info"].hit_buckets == 0
    assert ref["stats"]["bucket_records"] == 0
    assert np.array_equal(got["bits"], ref["bits"])
    assert (got["F"], got["hash"]) == (ref["F"], ref["hash"])
    sample = [0, len(got["rows"]) // 2, len(got["rows"]) - 1]
    bits, _, _ = O.sieve(prm.P, prm.d, prm.SL, prm.L, [int(got["rows"][i]) for i in sample])
    for k, i in enumerate(sample):
        assert np.array_equal(got["bits"][i], bits[k])
    n = 0
    for prm in workloads.tiny_cases(150, seed=13):
        args = prm.as_tuple()
        if O.validate(*args):
            continue
        got = _run(args, large_mode=2, threshold=max(2 * prm.SL, 1), **kw)
        _check_full(args, got)
        n += 1
    assert n > 60


def test_prepared_walkers_bit_exact():
    """One-walker chunks whose walkers a preparation kernel computes (first hit
    and steps per prime, then only walked) give the same bitset, F, counts and
    solver statistics as the walk preparing its items itself: 32-bit primes,
    64-bit primes (L above 2^30, with hit buckets too), odd d (every m walked)
    and the tiny brute-force cases against the oracle."""
    cases = [workloads.PLAIN_503.with_(L=3 * 10**6),
             workloads.SieveParams(P=503, d=2310, M_start=10**6, M_inc=3000, SL=3000, L=3 * 10**9),
             workloads.SieveParams(P=97, d=15, M_start=10**5 + 7, M_inc=700, SL=900, L=2 * 10**6)]
    for prm in cases:
        args = prm.as_tuple()
        for extra in ({}, {"hit_buckets": 2}):
            got = _run(args, walk_prep=2, **extra)
            ref = _run(args, walk_prep=1, **extra)
            assert got["info"].prep_chunks > 0 and ref["info"].prep_chunks == 0, prm
            assert np.array_equal(got["bits"], ref["bits"]), prm
            assert (got["F"], got["hash"]) == (ref["F"], ref["hash"])
            assert np.array_equal(got["counts"], ref["counts"])
            for k in ("solves", "levels", "hits_all", "F_large"):
                assert got["stats"][k] == ref["stats"][k], (prm, k)
    _check_full(cases[0].as_tuple(), _run(cases[0].as_tuple(), walk_prep=2))
    n = 0
    for prm in workloads.tiny_cases(150, seed=17):
        args = prm.as_tuple()
        if O.validate(*args):
            continue
        got = _run(args, large_mode=2, threshold=max(2 * prm.SL, 1), walk_prep=2)
        _check_full(args, got)
        n += got["info"].prep_chunks > 0
    assert n > 10


def test_profiled_launches_equal_the_stated_count():
    """The kernels a sieve launches (counted by the plan's own CUDA-event
    brackets, one kernel each for primes below 2^30; a 64-bit chunk's
    generation bracket also holds its residue kernel) are the
    launches_per_sieve the plan states, which bench.py reports as
    gpu_launches."""
    for prm, extra in ((workloads.SEARCH_953, {}), (workloads.PLAIN_503.with_(L=3 * 10**6), {}),
                       (workloads.PLAIN_503.with_(L=3 * 10**6), {"hit_buckets": 2}),
                       (workloads.PLAIN_503.with_(L=3 * 10**6), {"walk_prep": 1})):
        with cs.Plan(*prm.as_tuple(), profile=True, **extra) as plan:
            plan.sieve(torch.cuda.current_stream()).sync()
            ms, n = plan.kernel_times()
            assert sum(n) == int(plan.info.launches_per_sieve), (prm, extra, n)


def test_bucketed_hits_of_the_search_equal_direct_clears():
    """search_953 with its hits bucketed (forced; its 37.5 MB bitset clears
    directly by default) gives the same checksum, F and per-row counts."""
    prm = workloads.SEARCH_953
    a = _run(prm.as_tuple(), hit_buckets=2)
    b = _run(prm.as_tuple())
    assert a["info"].hit_buckets == 1 and b["info"].hit_buckets == 0
    assert 0 < a["stats"]["bucket_records"] <= a["stats"]["F_large"]
    assert (a["F"], a["hash"]) == (b["F"], b["hash"])
    assert np.array_equal(a["counts"], b["counts"])


def test_k1_survivors_are_primes():
    """K = d = 1 and L >= sqrt(N + SL): survivors are the primes (Section 1 gaps)."""
    SL = 199_999
    got = _run((1, 1, SL + 2, 1, SL, 1000))
    xs = got["cols"]
    row = O.unpack_row(got["bits"][0], len(xs))
    survivors = [SL + 2 + int(x) for x, b in zip(xs, row) if b]
    ref = O.primes(1, 2 * SL + 2)
    assert survivors == [int(v) for v in ref]
    gaps = {}
    for a, b in zip(survivors, survivors[1:]):
        gaps.setdefault(b - a, a)
    assert gaps[4] == 7 and gaps[6] == 23 and gaps[96] == 360653


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("T", [14000, 8 * 14001, 100 * 14001, 10**7])
def test_plain_503_bit_exact(mode, T):
    prm = workloads.PLAIN_503
    got = _run(prm.as_tuple(), large_mode=mode, threshold=T)
    _check_full(prm.as_tuple(), got)


@pytest.mark.parametrize("tile_rows", [1, 4, 32])
def test_tile_shapes_do_not_change_output(tile_rows):
    prm = workloads.PLAIN_503.with_(L=3 * 10**6)
    got = _run(prm.as_tuple(), tile_rows=tile_rows, threshold=50_000)
    _check_full(prm.as_tuple(), got)


def test_wide_arithmetic_bit_exact():
    """Sieve limit above 2^30: 64-bit prime entries and solver."""
    prm = workloads.SieveParams(P=503, d=2310, M_start=10**6, M_inc=3000, SL=3000, L=3 * 10**9)
    for mode in (1, 2):
        got = _run(prm.as_tuple(), large_mode=mode)
        assert got["info"].narrow == 0
        sample = [0, 1, 100, len(got["rows"]) // 2, len(got["rows"]) - 1]
        bits, F, _ = O.sieve(prm.P, prm.d, prm.SL, prm.L, [int(got["rows"][i]) for i in sample])
        for k, i in enumerate(sample):
            assert np.array_equal(got["bits"][i], bits[k]), (mode, i)


def test_search_953_sampled_rows_and_invariants():
    """The paper-shaped search at full size: sampled rows against the oracle
    (including the 35,308 record row), and size-independent properties."""
    prm = workloads.SEARCH_953
    got = _run(prm.as_tuple())
    rows = got["rows"]
    m_rec = workloads.RECORD_953[0]
    i_rec = int(np.searchsorted(rows, m_rec))
    assert rows[i_rec] == m_rec
    sample = sorted({0, 1, 2, 777, i_rec, len(rows) // 2, len(rows) - 2, len(rows) - 1})
    bits, F, _ = O.sieve(prm.P, prm.d, prm.SL, prm.L, [int(rows[i]) for i in sample])
    for k, i in enumerate(sample):
        assert np.array_equal(got["bits"][i], bits[k]), i
        assert int(got["counts"][i]) == int(O.row_counts(bits[k:k + 1])[0])
    # the record's lower prime survives
    xs = got["cols"]
    j = int(np.searchsorted(xs, workloads.RECORD_953[1]))
    assert (int(got["bits"][i_rec][j >> 6]) >> (j & 63)) & 1
    # same result with the paper's one-solve-per-hit walk and another threshold
    other = _run(prm.as_tuple(), large_mode=1, threshold=100 * 40001)
    assert other["hash"] == got["hash"] and other["F"] == got["F"]
    assert np.array_equal(other["counts"], got["counts"])
    # Section 3.2: solves ~ M * S * (loglog L - loglog T) + pi(L) - pi(T)
    st = other["stats"]
    T = other["info"].threshold
    n_large, _, inv = O.prime_stats(T, prm.L)
    expect = prm.M_inc * (2 * prm.SL + 1) * inv + n_large
    assert abs(st["solves"] - expect) < 0.01 * expect
    assert st["n_large_primes"] == n_large
    # hits the three-gap walk visits: M S sum 1/p over (T, L] for every m, a third
    # of that when only m = 1, 5 (mod 6) are walked (6 | d)
    T = got["info"].threshold
    _, _, inv = O.prime_stats(T, prm.L)
    all_hits = prm.M_inc * (2 * prm.SL + 1) * inv
    # default: the chunks with the most hits per prime walk class items mod 210
    # (8/35 of the hits) or 30 (4/15), the next ones m = 1, 5 (mod 6), the rest the odd m
    info = got["info"]
    assert (info.item_mod, info.item_classes) in ((30, 8), (210, 48)) and info.item_chunks > 0
    assert all_hits * 8 / 35 * 0.995 < got["stats"]["hits_all"] < all_hits / 2 * 1.005
    for m_classes, frac in ((1, 1.0), (2, 1.0 / 3.0), (3, 8.0 / 35.0)):
        alt = _run(prm.as_tuple(), threshold=T, tile_rows=got["info"].tile_rows, m_classes=m_classes)
        assert alt["hash"] == got["hash"] and alt["F"] == got["F"]
        assert abs(alt["stats"]["hits_all"] - frac * all_hits) < 0.005 * frac * all_hits


def test_autotune_picks_a_valid_tuning_and_caches_it(tmp_path):
    prm = workloads.PLAIN_503.with_(L=10**8)
    path = str(tmp_path / "tune.txt")
    t = cs.cs_autotune(*prm.as_tuple(), cache_path=path)
    assert t["threshold"] >= 2 * prm.SL and t["tile_rows"] in (8, 16, 32) and t["large_mode"] == 2
    assert t["item_hits"] in (0, 32, 64, 256, 512)              # 0: the automatic 128 won
    assert len(open(path).read().split()) == 7                  # one line: key and choice
    assert cs.cs_autotune(*prm.as_tuple(), cache_path=path) == t
    ref = _run(prm.as_tuple())
    got = _run(prm.as_tuple(), **t)
    assert (got["F"], got["hash"]) == (ref["F"], ref["hash"])


def test_environment_overrides_tuning(monkeypatch):
    prm = workloads.PLAIN_503
    monkeypatch.setenv("CS_THRESHOLD", "50000")
    monkeypatch.setenv("CS_TILE_ROWS", "8")
    with cs.Plan(*prm.as_tuple()) as p:
        assert p.info.threshold == 50000 and p.info.tile_rows == 8


def test_wide_interval_uses_several_column_chunks():
    """X = 5e5: one row of raw offsets no longer fits in shared memory, so the
    tile sieve works on column chunks; rows against the oracle."""
    prm = workloads.SieveParams(P=37, d=30, M_start=10**9 + 7, M_inc=12, SL=500_000, L=200_000)
    got = _run(prm.as_tuple())
    assert got["info"].tile_rows == 1
    _check_full(prm.as_tuple(), got)
    got2 = _run(prm.as_tuple(), tile_rows=4)
    assert (got2["F"], got2["hash"]) == (got["F"], got["hash"])


def test_large_divisor_wheel():
    """d with a prime factor above 64 (the wheel's pattern tables grow with q)."""
    prm = workloads.SieveParams(P=101, d=2 * 3 * 5 * 7 * 97, M_start=1000, M_inc=500, SL=3000, L=10**6)
    for no_wheel in (False, True):
        got = _run(prm.as_tuple(), no_wheel=no_wheel)
        _check_full(prm.as_tuple(), got, wheel=not no_wheel)


@pytest.mark.parametrize("mode", [1, 2])
def test_compact_layout_matches_oracle(mode):
    """Layout 1: per-row columns without the wheel's offsets, bit-exact, with the
    same F and per-row counts as the literal layout."""
    for prm in (workloads.PLAIN_503,
                workloads.SieveParams(P=37, d=30, M_start=10**6, M_inc=300, SL=400, L=10**5),
                workloads.SieveParams(P=503, d=2310, M_start=10**6, M_inc=3000, SL=3000, L=3 * 10**9)):
        args = prm.as_tuple()
        lit = _run(args, large_mode=mode)
        with cs.Plan(*args, layout=1, large_mode=mode) as p:
            p.sieve(torch.cuda.current_stream()).sync()
            bits = p.bitset()
            counts, F, h = p.counts()
            m = p.rows()
            pick = list(range(len(m))) if len(m) <= 300 else [0, 1, len(m) // 2, len(m) - 1]
            ref_lit, _, _ = O.sieve(prm.P, prm.d, prm.SL, prm.L, [int(m[i]) for i in pick])
            comp, W_max, cols = O.compact_layout(prm.P, prm.d, prm.SL, [int(m[i]) for i in pick], ref_lit)
            assert p.info.W == W_max and p.info.words_per_row == comp.shape[1]
            for k, i in enumerate(pick):
                assert np.array_equal(bits[i], comp[k]), (prm, i)
                assert np.array_equal(p.row_columns(i), cols[k])
        assert F == lit["F"]
        assert np.array_equal(counts, lit["counts"])


def test_compact_layout_size_of_the_search():
    """search_953 in the compact layout: about 9 MB instead of 37.5 MB."""
    with cs.Plan(*workloads.SEARCH_953.as_tuple(), layout=1) as p:
        assert p.info.bitset_bytes < 9.5e6
