"""Term sharding across ranks and rank aggregation of benchmark timings.

A decomposition of chi_total terms splits into contiguous global term ranges,
one per rank (lrs_init_terms' alpha0 / chi / chi_total); every estimator of the
path then ends in one sum over terms, so partial results of the ranks add up.
These helpers hold only that arithmetic and the torch.distributed calls.
"""
from __future__ import annotations


def shard_range(chi_total: int, rank: int, world: int) -> tuple[int, int]:
    """(alpha0, chi) of `rank`: contiguous, covering [0, chi_total) exactly."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, rem = divmod(chi_total, world)
    alpha0 = rank * base + min(rank, rem)
    return alpha0, base + (1 if rank < rem else 0)


def allreduce_sum(t):
    """Sum a tensor over ranks in place (no-op without an initialised group)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def max_over_ranks(value: float, device=None) -> float:
    """Largest value over ranks (the job's step time is its slowest rank's)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
