"""Multi-GPU: the two ways the path shards (one process per GPU).

Independent problems (the batched bands) are sharded across ranks with no data-path
collective: each rank owns a contiguous block of them and runs its own context with
problem_base set to the block's first index, so every problem draws the same random
numbers as in a single context over the whole set and the union of the ranks' results is
the single-GPU result.  Only the measurement is reduced: the elapsed time as the maximum
over ranks and the evaluation counts as their sum.

The particles of one problem can be sharded too (Sec. 6: moves are independent per
particle; reweighting, the ESS and resampling are the global steps).  Each rank's context
holds a block of particles (particles_global, particle_base) and a stage needs one
all-gather of the new-sample log-likelihoods, identical tempering and systematic ancestors
on every rank (computed by the library from the whole population), one exchange of the
particles the ancestors name, and two all-reduces of small sums (metric and step size).
The helpers below are the host side of that exchange; the arithmetic stays in the library.
"""
from __future__ import annotations

import dataclasses

import numpy as np


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


# ---------------------------------------------------------------------------
# Particles of one problem sharded across ranks
# ---------------------------------------------------------------------------
def particle_shards(P_global: int, world: int):
    """[(particle_base, count)] per rank: contiguous blocks (sizes differ by at most one)."""
    out = []
    for r in range(world):
        idx = shard(P_global, world, r)
        out.append((idx[0] if idx else 0, len(idx)))
    return out


def exchange_plan(anc, shards, rank):
    """Who sends which rows to whom after resampling, identical on every rank.

    anc: [n_problems][P_global] global ancestors.  A rank's local rows are ordered
    (problem, particle).  Returns (send, recv_counts, take):
      send[d]        local rows of `rank` that rank d needs, in the order d needs them;
      recv_counts[s] rows `rank` receives from rank s;
      take           for each of `rank`'s new local rows (its order), the position of the
                     row in the concatenation of what it received (sources in rank order).
    """
    anc = np.asarray(anc).reshape(len(anc), -1)
    n_prob = anc.shape[0]
    bases = np.array([b for b, _ in shards], dtype=np.int64)
    counts = np.array([c for _, c in shards], dtype=np.int64)

    def sources(d):   # (owner rank, owner's local row) of the rows rank d needs, in order
        b, c = shards[d]
        a = anc[:, b:b + c].astype(np.int64)                       # [n_prob][c]
        own = np.searchsorted(bases + counts, a, side="right")     # owner of each ancestor
        loc = np.arange(n_prob, dtype=np.int64)[:, None] * counts[own] + (a - bases[own])
        return own.ravel(), loc.ravel()

    send = []
    for d in range(len(shards)):
        own, loc = sources(d)
        send.append(loc[own == rank])
    own, _ = sources(rank)
    recv_counts = np.bincount(own, minlength=len(shards))
    offsets = np.concatenate([[0], np.cumsum(recv_counts)[:-1]])
    take = np.empty(own.shape[0], dtype=np.int64)
    seen = np.zeros(len(shards), dtype=np.int64)
    for q, s_ in enumerate(own):       # rows from source s_ arrive in the order rank needs them
        take[q] = offsets[s_] + seen[s_]
        seen[s_] += 1
    return send, recv_counts, take


def _comm_device(x, group=None):
    """Device of the tensors the group's collectives take: CUDA for NCCL, the host for gloo."""
    import torch
    import torch.distributed as dist

    return x.device if dist.get_backend(group) == "nccl" else torch.device("cpu")


def exchange_rows(rows, anc, shards, rank, group=None):
    """New local rows after resampling: rows [local_rows][W], exchanged with one
    all_to_all_single (returned on the device of `rows`)."""
    import torch
    import torch.distributed as dist

    send, recv_counts, take = exchange_plan(anc, shards, rank)
    cdev = _comm_device(rows, group)
    send_idx = torch.as_tensor(np.concatenate(send), dtype=torch.long, device=rows.device)
    payload = rows.index_select(0, send_idx).contiguous().to(cdev)
    out_rows = int(np.sum(recv_counts))
    recv = torch.empty((out_rows,) + tuple(rows.shape[1:]), dtype=rows.dtype, device=cdev)
    dist.all_to_all_single(recv, payload, output_split_sizes=[int(x) for x in recv_counts],
                           input_split_sizes=[len(x) for x in send], group=group)
    recv = recv.to(rows.device)
    return recv.index_select(0, torch.as_tensor(take, dtype=torch.long, device=rows.device))


def all_gather_particles(x, shards, group=None):
    """x [n_problems][count of this rank] -> [n_problems][P_global] in global particle order
    (every rank's block in rank order), on the device of x."""
    import torch
    import torch.distributed as dist

    cdev = _comm_device(x, group)
    width = max(c for _, c in shards)          # blocks differ by at most one: pad, then trim
    padded = torch.zeros((x.shape[0], width) + tuple(x.shape[2:]), dtype=x.dtype, device=cdev)
    padded[:, :x.shape[1]] = x.to(cdev)
    parts = [torch.empty_like(padded) for _ in shards]
    dist.all_gather(parts, padded, group=group)
    return torch.cat([part[:, :c] for part, (_, c) in zip(parts, shards)], dim=1).to(x.device)


def all_reduce_sum(x, group=None):
    """In-place sum over ranks of a small tensor (through the host for gloo)."""
    import torch.distributed as dist

    cdev = _comm_device(x, group)
    y = x.to(cdev)
    dist.all_reduce(y, group=group)
    x.copy_(y)


def sharded_stage(ctx, stage, shards, rank, group=None):
    """One SMC stage of a population whose particles are sharded across the ranks of
    `group` (each rank calls it with its own context; see include/tsmc.h for the order of
    the library calls).  Returns (beta, log Z, ESS) per problem."""
    import torch

    n_prob = ctx.cfg.n_problems
    P_loc = ctx.cfg.particles
    dev = ctx.ws.device
    beta0, _, _ = ctx.temper_state()
    z, K, lo, ln = ctx.get_population()
    ell = all_gather_particles(ln.view(n_prob, P_loc), shards, group)
    P_glob = ell.shape[1]
    anc = torch.empty(n_prob * P_glob, dtype=torch.int32, device=dev)
    ctx.temper_resample_global(stage, ell.contiguous(), anc)
    ctx.sync()
    anc_h = anc.cpu().numpy().reshape(n_prob, P_glob)
    anc_h[beta0 >= 1.0] = np.arange(P_glob)   # finished problems are not resampled
    kd = z.shape[1] * z.shape[2]
    rows = torch.cat([z.view(-1, kd), K.double()[:, None], lo[:, None], ln[:, None]], dim=1)
    new = exchange_rows(rows, anc_h, shards, rank, group)
    ctx.load_population(new[:, :kd].contiguous().view_as(z), new[:, kd].round().int().contiguous(),
                        new[:, kd + 1].contiguous(), new[:, kd + 2].contiguous())
    sums = torch.zeros(n_prob * 5, dtype=torch.float64, device=dev)
    ctx.metric_sums(sums)
    ctx.sync()
    all_reduce_sum(sums, group)
    ctx.metric_apply(sums)
    stats = torch.zeros(n_prob * 2, dtype=torch.float64, device=dev)
    ctx.mutation_rounds(stage, stats)
    ctx.sync()
    all_reduce_sum(stats, group)
    ctx.eps_update_apply(stats)
    return ctx.temper_state()
