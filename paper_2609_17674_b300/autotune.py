"""Launch-shape autotuner for the particle-block kernels.

The tunables are the threads per particle block and the samples each thread keeps
in registers per segment (tsmc_config.threads / samples_per_thread).  For a
workload the tuner times, on the device, the batched logL+gradient evaluation and
one NUTS transition of a frozen prior population for each candidate and keeps the
fastest; results are cached per (model, precision, N_max, K_max, P_total).
"""
from __future__ import annotations

import json
import os

from . import capi, sampler, synth

CANDIDATES = ((128, 32), (96, 32), (64, 32), (256, 32), (128, 16))
_cache: dict = {}


def _key(wl, precision):
    return (wl.model, precision, max(p.n for p in wl.problems), wl.kmax,
            wl.P * len(wl.problems))


def tune(wl, precision=capi.MIXED, candidates=CANDIDATES, nuts=True, seed=11, cache_file=None):
    """Returns {'threads', 'samples_per_thread', 'ms': {(T, R): ms}} for the workload."""
    import torch

    key = _key(wl, precision)
    if cache_file and os.path.exists(cache_file):
        for rec in json.load(open(cache_file)):
            if tuple(rec["key"]) == key:
                _cache[key] = rec["best"]
    if key in _cache:
        return _cache[key]
    z, K = synth.prior_population(wl, seed)
    zd = torch.as_tensor(z, device="cuda")
    Kd = torch.as_tensor(K, device="cuda")
    nb = len(wl.problems)
    beta = torch.full((nb,), 0.5, dtype=torch.float64, device="cuda")
    times = {}
    for T, R in candidates:
        if precision == capi.FP64 and R != 32:
            continue
        ctx = sampler.open_context(wl, precision, threads=T, samples_per_thread=R)
        ctx.set_population(zd, Kd, beta=[1e-3] * nb)
        ctx.update_metric()
        ctx.profile(True, events=64)
        ctx.profile_read(reset=True)
        ctx.eval(zd, Kd, beta, grad=True)
        ms = ctx.profile_read(reset=True)["eval"][1]
        if nuts:
            ctx.nuts_move(0, 0)
            ms += ctx.profile_read(reset=True)["nuts"][1]
        times[(T, R)] = ms
        ctx.close()
    (T, R) = min(times, key=times.get)
    best = {"threads": T, "samples_per_thread": R,
            "ms": {f"{t}x{r}": v for (t, r), v in times.items()}}
    _cache[key] = best
    if cache_file:
        recs = json.load(open(cache_file)) if os.path.exists(cache_file) else []
        recs = [r for r in recs if tuple(r["key"]) != key] + [{"key": list(key), "best": best}]
        json.dump(recs, open(cache_file, "w"), indent=1)
    return best


def open_tuned_context(wl, precision=capi.MIXED, **kw):
    """open_context with the tuned launch shape for this workload."""
    best = tune(wl, precision)
    return sampler.open_context(wl, precision, threads=best["threads"],
                                samples_per_thread=best["samples_per_thread"], **kw)
