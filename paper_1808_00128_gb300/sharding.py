"""Term sharding across ranks and rank aggregation of benchmark timings.

A decomposition of chi_total terms splits into contiguous global term ranges,
one per rank (lrs_init_terms' alpha0 / chi / chi_total); every estimator of the
path then ends in one sum over terms, so partial results of the ranks add up.
These helpers hold only that arithmetic, the torch.distributed calls and the order of
the calls of a term-sharded Metropolis chain (the decisions are the library's).
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


def _sum_parts(parts, allreduce):
    tot = parts[0].clone()
    for p in parts[1:]:
        tot += p
    if allreduce is not None:
        allreduce(tot)
    return tot


def chains_init_sharded(shards, x, allreduce=None):
    """Start chains at the strings x on every term shard of this process: each shard's
    partial <x|psi> is summed over the shards (and, through `allreduce`, over the other
    ranks' shards), and every shard takes P(x) = |<x|psi>|^2 from that sum."""
    amp = _sum_parts([s.amplitude(x) for s in shards], allreduce)
    for s in shards:
        s.chains_init(x)
        s.chains_set_amplitude(amp)
    return amp


def metropolis_sharded(shards, steps, seed, step0=0, trace=None, allreduce=None):
    """`steps` single-flip Metropolis steps (Sec. 4.2) on a term-sharded decomposition:
    per step every shard forms its partial amplitudes of the proposals, they are summed
    (the one exchange of the step: 2 C values per shard, all-reduced over ranks), and
    every shard applies the same accept decision from the same draws.  trace[t] (may be
    None) receives the chains' strings after step t."""
    for t in range(steps):
        step = step0 + t
        amp = _sum_parts([s.metropolis_propose(seed, step) for s in shards], allreduce)
        for i, s in enumerate(shards):
            s.metropolis_accept(amp, seed, step, trace=trace[t] if (trace is not None and i == 0) else None)


def amplitude_sharded(shards, x, allreduce=None):
    """<x|psi> over a term-sharded decomposition: the shards' amplitudes added (and
    all-reduced over ranks)."""
    return _sum_parts([s.amplitude(x) for s in shards], allreduce)


def norm_estimate_sharded(shards, L, seed, allreduce=None):
    """eta_l = 2^n |<phi_{A_l}|psi>|^2 over a term-sharded decomposition: the shards'
    overlaps summed (and all-reduced over ranks) before the library squares them."""
    ov = _sum_parts([s.norm_overlaps(L, seed) for s in shards], allreduce)
    return shards[0].norm_eta_from_overlaps(ov)
