"""Host logic of a replicated multi-rank bench run on CPU (gloo, two ranks):
the job time is the slowest rank's and the throughput counts every rank's
units.  No GPU is involved."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(10.0 + 5.0 * rank)      # rank 1 is the slow one
    out[rank] = (t, bench.job_rate(1000, world, 4, t))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_two_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, rate = res[r]
        assert t == 15.0                                  # every rank sees the max
        assert rate == pytest.approx(2 * 1000 * 4 / 15e-3 / 1e6)


def test_single_rank_is_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(1e6, 1, 2, 1000.0) == pytest.approx(2.0)
