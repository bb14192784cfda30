"""Failure handling through the C ABI, with every failure made on the host:
device allocations that fail (injected with CS_FAIL_ALLOC_AT, the n-th
allocation of a plan build fails as if the device were out of memory),
requests released while their sieve still runs (the request server's
cancellation: the result is dropped and its memory returns once the device
work ends), and the library staying usable, with unchanged results, after
each.  No kernel is made to fault, trap or wait forever."""
import time

import numpy as np
import pytest

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


def _alone(prm, **tuning):
    with cs.Plan(*prm.as_tuple(), **tuning) as p:
        p.sieve(torch.cuda.current_stream()).sync()
        counts, F, h = p.counts()
        return counts.copy(), F, h


def _same(a, b):
    return a[1:] == b[1:] and np.array_equal(a[0], b[0])


def test_every_allocation_of_a_plan_build_can_fail_cleanly(monkeypatch):
    """Each device allocation of a plan build, failed in turn, gives CS_ENOMEM
    with its message and no plan; afterwards the same plan builds and sieves
    to the same result, for a plan of 32-bit primes, one of 64-bit primes and
    one whose walk buckets its hits (more allocations)."""
    for prm, tuning in ((workloads.PLAIN_503, {}),
                        (workloads.SieveParams(P=503, d=2310, M_start=10**6, M_inc=3000, SL=3000, L=3 * 10**9),
                         {"item_hits": 32}),
                        (workloads.PLAIN_503, {"hit_buckets": 2})):
        ref = _alone(prm, **tuning)
        tune = cs.make_tuning(**tuning) if tuning else None
        k = 0
        while True:
            k += 1
            monkeypatch.setenv("CS_FAIL_ALLOC_AT", str(k))
            rc = cs.cs_plan_status(*prm.as_tuple(), tune)
            if rc == cs.CS_OK:
                break
            assert rc == cs.CS_ENOMEM, (k, rc)
            assert "CS_FAIL_ALLOC_AT" in cs.cs_last_error()
            assert k < 64
        assert k > 5                                         # several allocations were failed
        monkeypatch.delenv("CS_FAIL_ALLOC_AT")
        assert _same(_alone(prm, **tuning), ref)


def test_server_survives_a_failed_admission_and_a_cancelled_request(monkeypatch):
    """A request whose plan cannot allocate is refused with CS_ENOMEM and leaves
    nothing behind; a request released before it finishes frees its slot and
    memory; the next requests give the same results as alone."""
    small = workloads.PLAIN_503
    big = workloads.SieveParams(P=953, d=210, M_start=10**8, M_inc=20_000, SL=20_000, L=10**9)
    ref = _alone(small)
    srv = cs.Server(budget_bytes=8 << 30, max_slots=2)
    try:
        monkeypatch.setenv("CS_FAIL_ALLOC_AT", "3")
        with pytest.raises(cs.CSError) as e:
            srv.submit(*small.as_tuple())
        assert e.value.code == cs.CS_ENOMEM
        monkeypatch.delenv("CS_FAIL_ALLOC_AT")
        assert srv.usage() == (0, 0, 0)
        # cancel: release right after submission, while the sieve is on the device
        t = srv.submit(*big.as_tuple())
        assert t is not None and srv.usage()[2] == 1
        srv.release(t)
        assert srv.usage() == (0, 0, 0)
        with pytest.raises(cs.CSError) as e:
            srv.poll(t)                                      # the ticket is gone
        assert e.value.code == cs.CS_EINVAL
        for _ in range(2):
            t = srv.submit(*small.as_tuple())
            t0 = time.time()
            while not srv.poll(t):
                assert time.time() - t0 < 120
                time.sleep(0.001)
            plan = srv.plan(t)
            plan.sync()
            assert _same(plan.counts(), ref)
            srv.release(t)
        assert srv.usage() == (0, 0, 0)
    finally:
        srv.close()


def test_parameter_errors_leave_the_library_usable():
    """Rejected parameter sets (CS_EINVAL before any device work) and a fetch
    before cs_sieve (CS_ESTATE) do not disturb a following plan."""
    ref = _alone(workloads.PLAIN_503)
    for bad in ((503, 4, 1, 1000, 7000, 10**7),            # d not squarefree
                (503, 210, 0, 1000, 7000, 10**7),          # M_start = 0
                (503, 210, 1, 1000, 7000, 2**40 + 1),      # L above 2^40
                (503, 210, 1, 2**31, 7000, 10**7)):        # M_inc too large
        assert cs.cs_plan_status(*bad) == cs.CS_EINVAL
    with cs.Plan(*workloads.PLAIN_503.as_tuple()) as p:
        with pytest.raises(cs.CSError) as e:
            p.counts()
        assert e.value.code == cs.CS_ESTATE
    with pytest.raises(cs.CSError) as e:
        cs.Plan(*workloads.PLAIN_503.as_tuple(), m_classes=4)
    assert e.value.code == cs.CS_EINVAL
    assert _same(_alone(workloads.PLAIN_503), ref)
