"""Replica bookkeeping for runs on several GPUs of one node.

The short-range solver shards by whole boxes or jobs: every rank owns its
own particles, trees and pair lists, and no collective touches the data
path.  Only the timing needs the ranks together: a barrier on both sides of
the timed region and the maximum of the ranks' times, so that the job's
throughput is the units of all ranks over the slowest rank's time (weak
scaling).  These helpers hold that logic; they work with any process group
backend (NCCL on GPUs, gloo on CPUs)."""
from __future__ import annotations


def shard(count: int, rank: int, world: int) -> range:
    """The contiguous block of `count` units (boxes, requests) that `rank` of
    `world` processes; the blocks are disjoint, cover every unit and differ in
    size by at most one."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    base, extra = divmod(count, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over the ranks of the default process group (the
    value itself without one)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    """The sum of `value` over the ranks (units processed by the whole job)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(units: float, ms: float, dist=None, device=None) -> tuple[float, float]:
    """(units of all ranks per second over the slowest rank's time, that time
    in ms)."""
    t_max = max_over_ranks(ms, dist, device)
    total = sum_over_ranks(units, dist, device)
    return total / (t_max / 1e3), t_max
