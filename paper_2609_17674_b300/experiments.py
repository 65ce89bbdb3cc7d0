"""Segment experiment of the paper's pulse example (Sec. 5.1, prior-start against
posterior-start): data arrive in segments, each 20 s longer than the last.

- prior-start: every segment is analysed from the prior (bridge Eq. prior_bridge);
- posterior-start: the first segment from the prior, every later one from the previous
  segment's particles after assimilating the new samples (bridge Eq. reuse_bridge).

Reported per segment: SMC stages to reach beta = 1, log Z (increments summed along the
posterior-start chain), the posterior over K and the wall time.
"""
from __future__ import annotations

import time

import numpy as np

from . import capi, sampler
from .synth import Workload


def _k_hist(ctx, kmax):
    K = ctx.get_population()[1].cpu().numpy()
    return np.bincount(K, minlength=kmax + 1)[: kmax + 1] / K.shape[0]


def segment_bounds(wl: Workload, seg_seconds: float = 20.0):
    pr = wl.problems[0]
    per = int(round(seg_seconds / pr.dt))
    return [min(per * (i + 1), pr.n) for i in range((pr.n + per - 1) // per)]


def segment_experiment(wl: Workload, seg_seconds: float = 20.0, precision: int = capi.MIXED,
                       max_stages: int = 400, stream=None):
    import torch

    pr = wl.problems[0]
    bounds = segment_bounds(wl, seg_seconds)

    def run(ctx, **kw):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = sampler.run_smc(ctx, max_stages=max_stages, **kw)
        torch.cuda.synchronize()
        return out, time.perf_counter() - t0

    posterior = []
    ctx = sampler.open_context(wl, precision, n_use=bounds[0], n_capacity=[pr.n], stream=stream)
    logz = 0.0
    for i, nb in enumerate(bounds):
        if i == 0:
            out, wall = run(ctx)
        else:
            ctx.assimilate(0, pr.d[bounds[i - 1]:nb])
            out, wall = run(ctx, stage0=1000 * i, init_prior=False)
        logz += float(out["logz"][-1][0])
        posterior.append(dict(seconds=nb * pr.dt, stages=out["n_stages"], logz=logz,
                              reached=bool(out["beta"][-1][0] >= 1.0),
                              k_hist=_k_hist(ctx, wl.kmax).tolist(), wall_s=wall))
    ctx.close()
    prior = []
    for nb in bounds:
        ctx = sampler.open_context(wl, precision, n_use=nb, n_capacity=[pr.n], stream=stream)
        out, wall = run(ctx)
        prior.append(dict(seconds=nb * pr.dt, stages=out["n_stages"],
                          logz=float(out["logz"][-1][0]),
                          reached=bool(out["beta"][-1][0] >= 1.0),
                          k_hist=_k_hist(ctx, wl.kmax).tolist(), wall_s=wall))
        ctx.close()
    return dict(workload=wl.name, segments_s=[nb * pr.dt for nb in bounds], prior=prior,
                posterior=posterior)
