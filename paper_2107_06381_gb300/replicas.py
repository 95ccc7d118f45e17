"""Replicas across GPUs: the all-at-once solve needs no exchange between
independent instances, so N GPUs each take a disjoint share of the instances
(weak scaling) and only the timing is reduced (max over ranks).

These helpers are pure host logic over torch.distributed; the tests run them
with the gloo backend on CPU ranks.
"""
from __future__ import annotations


def shard(items, rank: int, world: int):
    """Round-robin share of `items` for `rank` of `world` (every item exactly once)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    return [it for i, it in enumerate(items) if i % world == rank]


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank float over the default process group (the slowest
    rank's time is the job's time); identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
