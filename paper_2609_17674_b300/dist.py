"""Multi-GPU bookkeeping (one process per GPU, no data-path collective).

Independent problems (the batched bands) are sharded across ranks: each rank owns a
contiguous block of them and runs its own context with problem_base set to the block's
first index, so every problem draws the same random numbers as in a single context over
the whole set and the union of the ranks' results is the single-GPU result.  Only the
measurement is reduced: the elapsed time as the maximum over ranks and the evaluation
counts as their sum.
"""
from __future__ import annotations

import dataclasses


def shard(n_units: int, world: int, rank: int):
    """Contiguous block of unit indices for rank (sizes differ by at most one)."""
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def shard_problems(wl, world: int, rank: int):
    """(workload of the problems rank owns, their indices in wl).  The shard keeps the
    problems' global indices as its Philox keys (problem_base)."""
    idx = shard(len(wl.problems), world, rank)
    if not idx:
        return None, idx
    sub = dataclasses.replace(wl, problems=[wl.problems[b] for b in idx],
                              problem_base=wl.problem_base + idx[0],
                              name=f"{wl.name}[{idx[0]}:{idx[-1] + 1}]")
    return sub, idx


def rank_seed(seed: int, rank: int) -> int:
    """Data and Philox seed of a rank's independent problem."""
    return seed + 1000 * rank


def reduce_measurement(ms: float, cs: float, group=None, device=None):
    """(max elapsed ms over ranks, total component*samples over ranks)."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return ms, cs
    t = torch.tensor([ms, -cs], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    s = torch.tensor([cs], dtype=torch.float64, device=device)
    dist.all_reduce(s, op=dist.ReduceOp.SUM, group=group)
    return float(t[0].item()), float(s[0].item())
