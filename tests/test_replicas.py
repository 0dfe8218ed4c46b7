"""The multi-GPU form is replicas only: each rank steps its own copy of the
problem and the job time is the slowest rank's.  Checked with two gloo
processes on the CPU (no GPU, no collective on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 1000.0 + 250.0 * rank                   # rank 1 is the slow replica
    worst = bench.max_over_ranks(ms, "cpu")
    out[rank] = (worst, bench.job_value(world, 8, worst))
    dist.barrier()
    dist.destroy_process_group()


def test_job_time_is_the_slowest_replica():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        worst, value = res[r]
        assert worst == 1250.0
        assert value == pytest.approx(2 * 8 / 1.25)


def test_single_process_is_its_own_max():
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.job_value(1, 4, 2000.0) == 2.0
