"""The N > 1 host path of bench.py on CPU: two `gloo` ranks (one process
each) time different totals; both receive the slowest rank's total, and the
whole-job throughput counts every rank's frames over that time.  The path
has no data collective (replicas only): this reduction of the timed total is
its only cross-rank step."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, totals, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        worst = bench.max_over_ranks(totals[rank], dist)
        out[rank] = (worst, bench.job_throughput(world, 10, worst))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_total():
    world = 2
    totals = [123.5, 987.25]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), totals, out), nprocs=world, join=True)
        res = dict(out)
    assert set(res) == {0, 1}
    for r in range(world):
        worst, value = res[r]
        assert worst == max(totals)
        assert value == pytest.approx(world * 10 / (max(totals) / 1e3))


def test_job_throughput_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_throughput(1, 100, 500.0) == pytest.approx(200.0)
