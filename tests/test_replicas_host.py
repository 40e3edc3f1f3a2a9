"""The multi-GPU path is replicas only: every rank runs the same workload,
the ranks' timings meet in one all-reduce MAX and the value counts every
rank's units.  Two gloo ranks on the CPU check that host logic."""
import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, local_ms, units, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = bench.replica_throughput(local_ms[rank], units, world, "cpu")
    finally:
        dist.destroy_process_group()


def test_replica_throughput_two_gloo_ranks():
    world, units = 2, 3.0e12
    local_ms = [10.0, 14.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), local_ms, units, out), nprocs=world,
                 join=True)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 14.0                                   # the slowest rank's time
        assert value == pytest.approx(world * units / 0.014 / 1e12)


def test_replica_throughput_one_rank():
    ms, value = bench.replica_throughput(5.0, 1.0e12, 1)
    assert ms == 5.0 and value == pytest.approx(1.0e12 / 0.005 / 1e12)
