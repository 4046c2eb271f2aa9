"""Replica timing and sharding across ranks: two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2510_03557_gb300 import replicas


def test_shard_is_a_partition():
    for count in (0, 1, 7, 64, 2000):
        for world in (1, 2, 3, 8):
            blocks = [replicas.shard(count, r, world) for r in range(world)]
            flat = [u for b in blocks for u in b]
            assert flat == list(range(count))
            sizes = [len(b) for b in blocks]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard(4, 2, 2)


def test_single_process_needs_no_group():
    assert replicas.max_over_ranks(3.5) == 3.5
    assert replicas.job_throughput(1000, 2.0) == (500000.0, 2.0)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        units = len(replicas.shard(10, rank, world)) * 1000  # particles of this rank's boxes
        ms = 10.0 * (rank + 1)                                # the slower rank sets the time
        dist.barrier()
        value, t = replicas.job_throughput(units, ms, dist)
        out[rank] = (value, t, replicas.max_over_ranks(-rank, dist))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_all_units():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        value, t, mx = res[rank]
        assert t == 20.0                      # max over ranks
        assert value == 10 * 1000 / 0.020     # all ranks' units over the slowest time
        assert mx == 0.0
