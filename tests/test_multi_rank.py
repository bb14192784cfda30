"""The multi-GPU form of bench.py on the CPU: two gloo ranks, each sieving its
own m-range (replicas, weak scaling), with the max-over-ranks time and the sum
of F reduced the way bench.py does.  The oracle stands in for the GPU."""
import os

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    import oracle.oracle as O
    from paper_2012_03771_gb300 import workloads
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, ws = bench._dist()
    base = workloads.SieveParams(P=37, d=30, M_start=10**6, M_inc=40, SL=200, L=5000)
    prm = bench._params_for_rank(base, r)
    m, bits, F = O.full_sieve(*prm.as_tuple())
    t = torch.tensor([float(1 + r)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    f = torch.tensor([float(F.sum())], dtype=torch.float64)
    dist.all_reduce(f, op=dist.ReduceOp.SUM)
    out[rank] = (prm.M_start, prm.M_inc, int(F.sum()), float(t.item()), float(f.item()), [int(v) for v in m])
    dist.destroy_process_group()


def test_two_ranks_shard_the_m_range():
    world = 2
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    (s0, n0, F0, t0, f0, m0), (s1, n1, F1, t1, f1, m1) = res[0], res[1]
    assert s1 == s0 + n0 and n1 == n0                       # contiguous, disjoint m-ranges
    assert not set(m0) & set(m1)
    assert t0 == t1 == 2.0                                   # max over ranks
    assert f0 == f1 == F0 + F1                               # whole-job F
    import oracle.oracle as O
    m, bits, F = O.full_sieve(37, 30, 10**6, 80, 200, 5000)  # one job over both ranges
    assert int(F.sum()) == F0 + F1 and list(m) == m0 + m1
