"""The multi-rank host logic of bench.py on CPU: two gloo ranks (127.0.0.1), each with
its own local time; the job time is the slowest rank's and the job rate counts the
units of both ranks (weak scaling of independent replicas, no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, rate = bench.job_rate(10.0 + 5.0 * rank, 1e9, world, dist, "cpu")
    out[rank] = (ms, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_over_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, rate = res[r]
        assert ms == 15.0                           # the slower rank's time, on every rank
        assert abs(rate - 2 * 1e9 / 15e-3 / 1e9) < 1e-9


def test_job_rate_single_rank():
    import bench
    ms, rate = bench.job_rate(20.0, 4e9, 1)
    assert ms == 20.0 and abs(rate - 200.0) < 1e-12
