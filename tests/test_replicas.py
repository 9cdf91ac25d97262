"""The multi-GPU form of the benchmark is N independent replicas (the path
needs no exchange between GPUs): each rank grids its own copy, the job takes
as long as its slowest rank, and the whole-job rate sums the ranks' work.
This checks that bookkeeping with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 10.0 + 5.0 * rank          # rank 1 is the slowest
    rate, ms = bench.job_rate(1_000_000, ms_local, dist, "cpu")
    out[rank] = (rate, ms)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_replica_rate_uses_slowest_rank_and_sums_work():
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        rate, ms = res[rank]
        assert ms == 15.0
        assert rate == pytest.approx(2 * 1_000_000 / 0.015)


def test_single_process_rate():
    import bench
    rate, ms = bench.job_rate(500, 2.0)
    assert ms == 2.0 and rate == pytest.approx(250_000.0)
