"""Multi-GPU form: independent replicas (one process per GPU), no data-path collective.

Frames, views and served requests are independent, so N GPUs render disjoint shares of
the work; the only cross-rank operations are for measurement (a barrier and the maximum
of the per-rank times). The screen-space split of one frame over several GPUs (each
rasterising its own tiles after a full setup and binning, then one gather of the tiles)
lives in partition.py.
"""
from __future__ import annotations


def shard(items, rank: int, world: int):
    """Round-robin share of items for this rank (every item lands on exactly one rank)."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    return [x for i, x in enumerate(items) if i % world == rank]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over all ranks (the job's wall time is set by the slowest)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist=None, device=None) -> float:
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
