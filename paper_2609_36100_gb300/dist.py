"""Multi-process helpers for running independent work on several GPUs.

A single simulation does not shard without an all-to-all per 3D FFT, so
several ranks run independent replicas; an ensemble shards by member with no
collective on the data path.  The only collectives are the timing barrier and
the max-over-ranks reduction of elapsed times (any torch.distributed backend:
gloo on CPU tensors, nccl on CUDA tensors)."""
from __future__ import annotations


def shard(n_items: int, rank: int, world: int):
    """Round-robin share of items 0..n_items-1 for `rank` of `world`."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world")
    return list(range(rank, n_items, world))


def max_over_ranks(value: float, device=None) -> float:
    """Max of a scalar over all ranks (the value itself without a process
    group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
