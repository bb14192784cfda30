"""cs_primes_static: the allocation-free prime generator, for callers whose
device memory belongs to a pool of their own or that cannot afford the device
synchronisation of cudaMalloc/cudaFree.  Its output must equal cs_primes's on
the same range, call after call (the static scratch it shares across calls is
reused, and the previous call's contents must not leak into the next).

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes on its own in a fresh process."""
import math

import numpy as np
import pytest

import oracle.oracle as O
import paper_2012_03771_gb300 as cs

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


def _list(fn, lo, hi, cap):
    buf = torch.zeros(cap, dtype=torch.int64, device="cuda")
    n = fn(lo, hi, buf.data_ptr(), cap, torch.cuda.current_stream())
    return n, np.sort(buf[:n].cpu().numpy())


# the last range has isqrt(hi) = 31623 odd, so the base-prime bound isqrt(hi) + 1 is even
RANGES = [(10**9 - 2 * 10**6, 10**9), (2**40 - 4 * 10**5, 2**40), (0, 3 * 10**5),
          (31623**2 + 5 - 10**6, 31623**2 + 5)]


@pytest.mark.parametrize("lo,hi", RANGES)
def test_static_matches_allocating_entry_point_twice(lo, hi):
    cap = 200_000
    n_ref, ref = _list(cs.cs_primes, lo, hi, cap)
    for _ in range(2):   # two calls in a row on the same static scratch
        n, got = _list(cs.cs_primes_static, lo, hi, cap)
        assert n == n_ref
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("lo,hi", RANGES)
def test_static_matches_oracle(lo, hi):
    assert math.isqrt(RANGES[-1][1]) % 2 == 1
    cap = 200_000
    ref = O.primes(lo, hi)
    for _ in range(2):
        n, got = _list(cs.cs_primes_static, lo, hi, cap)
        assert n == ref.size
        assert np.array_equal(got.astype(np.uint64), ref)


def test_static_sequence_of_different_ranges():
    cap = 200_000
    for lo, hi in ((2**40 - 10**5, 2**40), (100, 5000), (2**33, 2**33 + 10**6)):
        n_ref, ref = _list(cs.cs_primes, lo, hi, cap)
        n, got = _list(cs.cs_primes_static, lo, hi, cap)
        assert n == n_ref and np.array_equal(got, ref)


def test_static_rejects_beyond_limit_and_overflow():
    buf = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(cs.CSError) as e:
        cs.cs_primes_static(0, 2**40 + 1, buf.data_ptr(), 16, torch.cuda.current_stream())
    assert e.value.code == cs.CS_EINVAL
    with pytest.raises(cs.CSError) as e:
        cs.cs_primes_static(0, 10**4, buf.data_ptr(), 16, torch.cuda.current_stream())
    assert e.value.code == cs.CS_EOVERFLOW
    assert "cs_primes_static" in cs.cs_last_error()
