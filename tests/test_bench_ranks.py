"""The multi-GPU form of the benchmark runs replicas: each rank solves its own
copy and only the timing is combined (the slowest rank's time, the bytes of
all ranks).  That combination runs here on two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, u = bench.aggregate(torch, dist, seconds=1.0 + rank, units=10.0 * (rank + 1), device="cpu")
        out[rank] = (t, u)
    finally:
        dist.destroy_process_group()


def test_replica_timing_takes_the_slowest_rank_and_sums_the_work():
    import torch.multiprocessing as mp
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1] == (2.0, 30.0)


def test_single_rank_is_unchanged():
    import bench
    assert bench.aggregate(torch, None, 1.5, 7.0, "cpu") == (1.5, 7.0)
