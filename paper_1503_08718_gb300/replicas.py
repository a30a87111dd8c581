"""Host logic for running independent solves on several GPUs, one process per
GPU: the path partitions into independent problems (cells, directions,
lateral types), so ranks share no data and exchange only timings and
results.  Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations


def partition(n_items: int, rank: int, world: int) -> list[int]:
    """Round-robin share of items 0..n_items-1 for `rank` of `world`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world size")
    return list(range(rank, n_items, world))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over all ranks (the slowest rank's time)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_results(local: dict[int, float], n_items: int, device=None) -> list[float]:
    """Collects per-item results computed on different ranks into one list
    (items no rank computed stay NaN)."""
    import math

    import torch
    import torch.distributed as dist

    vals = torch.full((n_items,), math.nan, dtype=torch.float64, device=device)
    for i, v in local.items():
        vals[i] = v
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        # every item is owned by exactly one rank: replace NaN by 0 and sum
        mask = torch.isnan(vals)
        vals = torch.where(mask, torch.zeros_like(vals), vals)
        own = (~mask).to(torch.float64)
        dist.all_reduce(vals)
        dist.all_reduce(own)
        vals = torch.where(own > 0, vals, torch.full_like(vals, math.nan))
    return [float(v) for v in vals.cpu()]
