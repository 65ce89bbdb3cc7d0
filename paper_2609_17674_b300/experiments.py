"""Experiments on the sampler.

Segment experiment of the paper's pulse example (Sec. 5.1, prior-start against
posterior-start): data arrive in segments, each 20 s longer than the last.

- prior-start: every segment is analysed from the prior (bridge Eq. prior_bridge);
- posterior-start: the first segment from the prior, every later one from the previous
  segment's particles after assimilating the new samples (bridge Eq. reuse_bridge).

Reported per segment: SMC stages to reach beta = 1, log Z (increments summed along the
posterior-start chain), the posterior over K and the wall time.

Also: the population birth proposal against prior births; the throughput of the batched
logL + gradient evaluation per precision (``python -m paper_2609_17674_b300.experiments eval
--precision fp64``); NUTS transitions of one workload after a few stages (``... nuts
--workload gb --particles 512``, the small case of the kernel profiles); and the posterior
start over 2^17, 2^18 and 2^19 samples at P = 16384 (``... assimilation``).  Each prints one
JSON line.
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
            if not posterior[-1]["reached"]:
                raise RuntimeError(f"segment {i - 1} stopped at beta < 1 after {max_stages} "
                                   "stages: its particles are not a posterior to start from")
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


def birth_proposal_comparison(wl: Workload, mid_stages: int = 12, rounds: int = 5,
                              precision: int = capi.MIXED, max_stages: int = 400, stream=None):
    """Births from the prior against births from the population mixture
    (tsmc_build_birth_proposal): full prior-start runs with each, and the birth acceptance
    of both on one population taken after mid_stages stages of the prior-proposal run."""
    import copy

    import torch

    runs = {}
    for bp in (0, 1):
        w = copy.copy(wl)
        w.birth_proposal = bp
        ctx = sampler.open_context(w, precision, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = sampler.run_smc(ctx, max_stages=max_stages)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        kh = _k_hist(ctx, w.kmax)
        runs[bp] = dict(stages=out["n_stages"], wall_s=wall, logz=float(out["logz"][-1][0]),
                        mean_k=float(np.dot(kh, np.arange(w.kmax + 1))),
                        reached=bool(out["beta"][-1][0] >= 1.0))
        ctx.close()
    # birth acceptance on a common mid-run population
    w0 = copy.copy(wl)
    w0.birth_proposal = 0
    ctx = sampler.open_context(w0, precision, stream=stream)
    sampler.run_smc(ctx, max_stages=mid_stages)
    z, K, _, _ = ctx.get_population()
    z, K = z.clone(), K.clone()
    torch.cuda.synchronize()   # the clones run on torch's stream, the contexts on theirs
    beta = ctx.temper_state()[0]
    ctx.close()
    acc, outs, m_built = {}, {}, 0
    for bp in (0, 1):
        w = copy.copy(wl)
        w.birth_proposal = bp
        c = sampler.open_context(w, precision, stream=stream)
        zr, Kr = z.clone(), K.clone()
        torch.cuda.synchronize()
        c.set_population(zr, Kr, beta=beta)
        c.build_birth_proposal(mid_stages)
        if bp:
            m_built = c.get_birth_proposal(0)[0]
        outd = torch.zeros(K.shape[0], dtype=torch.int32, device=z.device)
        born, proposed, allo = 0, 0, []
        for r in range(rounds):
            zr, Kr = z.clone(), K.clone()
            torch.cuda.synchronize()
            c.set_population(zr, Kr, beta=beta)
            c.rj_move(mid_stages, r, outd)
            c.sync()                   # the move runs on the context's stream
            o = outd.cpu().numpy()
            allo.append(o.copy())
            born += int(np.sum(o == 1))
            proposed += int(np.sum((o == 1) | (o == -1)))
        acc[bp] = born / max(proposed, 1)
        outs[bp] = np.concatenate(allo)
        c.close()
    return dict(workload=wl.name, prior_births=runs[0], population_births=runs[1],
                mid_stage=mid_stages, mid_beta=float(beta[0]), proposal_centres=m_built,
                outcomes_differing=int(np.sum(outs[0] != outs[1])),
                birth_acceptance_prior=acc[0], birth_acceptance_population=acc[1])


def eval_throughput(wl: Workload, precision: int, reps: int = 3, seed: int = 1,
                    beta: float = 0.5, pulse_window: int = 1) -> dict:
    """Batched logL + gradient over a prior population of the workload (K_p N counted per
    particle): one warm-up launch, then the best of reps launches timed with CUDA events on
    the context's stream."""
    import torch

    from . import synth

    z, K = synth.prior_population(wl, seed)
    nb = len(wl.problems)
    stream = torch.cuda.Stream()
    zd = torch.as_tensor(z, device="cuda")
    Kd = torch.as_tensor(K, device="cuda")
    bt = torch.full((nb,), beta, dtype=torch.float64, device="cuda")
    ctx = sampler.open_context(wl, precision, stream=stream, pulse_window=pulse_window)
    ctx.set_population(zd, Kd, beta=[beta] * nb)
    g = torch.empty_like(zd)
    with torch.cuda.stream(stream):
        ctx.eval(zd, Kd, bt, grad=True, g=g)
        best = float("inf")
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(stream)
            ctx.eval(zd, Kd, bt, grad=True, g=g)
            e1.record(stream)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
    ctx.close()
    cs = float(K.astype(np.int64).sum()) * wl.problems[0].n
    return dict(workload=wl.name, precision="fp64" if precision == capi.FP64 else "mixed",
                ms_per_launch=best, cs_per_s=cs / (best * 1e-3))


def nuts_launch_timing(wl: Workload, precision: int = capi.MIXED, warm_stages: int = 3,
                       launches: int = 3) -> dict:
    """A prior start of the workload, warm_stages SMC stages, then `launches` NUTS transitions
    of the population, each timed with CUDA events on the context's stream; returns the
    fastest with the component*samples it evaluated (nominal and computed)."""
    import torch

    stream = torch.cuda.Stream()
    ctx = sampler.open_context(wl, precision, stream=stream)
    ctx.init_population()
    for st in range(warm_stages):
        ctx.run_stage(st, use_graph=False, read=False)
    torch.cuda.synchronize()
    best = None
    for r in range(launches):
        ctx.counters(reset=True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.nuts_move(warm_stages, r)
        e1.record(stream)
        torch.cuda.synchronize()
        (_, cs, _, cc), _ = ctx.counters(reset=True)
        ms = e0.elapsed_time(e1)
        if best is None or ms < best[0]:
            best = (ms, cs, cc)
    ctx.close()
    ms, cs, cc = best
    return dict(workload=wl.name, precision="fp64" if precision == capi.FP64 else "mixed",
                ms=ms, cs_nominal=cs, cs_computed=cc, nominal_cs_per_s=cs / (ms * 1e-3),
                computed_cs_per_s=cc / (ms * 1e-3))


def assimilation_experiment(P: int = 16384, sizes=(1 << 17, 1 << 18, 1 << 19),
                            precision: int = capi.MIXED, max_stages: int = 400,
                            prior_start: bool = True, posterior_start: bool = True) -> dict:
    """Posterior start on the assimilation workload (K_true = 14 pulses on t_n = n / 2^19):
    a prior start on the first sizes[0] samples, then for every later size the new samples are
    assimilated (Eq. reuse_bridge) and the run continues from the previous posterior; with
    prior_start, also a prior start on each size.  Per segment: SMC stages, wall time,
    component*sample evaluations per second (device counters), log Z and mean K."""
    import torch

    from . import synth

    wl = synth.assimilation_pulse_k14(P=P, n_full=sizes[-1])
    pr = wl.problems[0]

    def run(ctx, **kw):
        ctx.counters(reset=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = sampler.run_smc(ctx, max_stages=max_stages, **kw)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        (ce, cn, _, _), _ = ctx.counters(reset=True)
        return out, wall, (ce + cn) / wall

    def summary(ctx, n, out, wall, rate, logz):
        K = ctx.get_population()[1].cpu().numpy()
        return dict(samples=n, stages=out["n_stages"], wall_s=round(wall, 3), cs_per_s=rate,
                    logz=logz, reached=bool(out["beta"][-1][0] >= 1.0), mean_k=float(K.mean()))

    res = dict(workload=wl.name, P=P, sizes=list(sizes), posterior=[], prior=[])
    ctx = sampler.open_context(wl, precision, n_use=sizes[0], n_capacity=[pr.n])
    logz = 0.0
    for i, n in enumerate(sizes if posterior_start else []):
        if i == 0:
            out, wall, rate = run(ctx)
        else:
            if not res["posterior"][-1]["reached"]:
                raise RuntimeError("segment stopped at beta < 1: no posterior to start from")
            ctx.assimilate(0, pr.d[sizes[i - 1]:n])
            out, wall, rate = run(ctx, stage0=1000 * i, init_prior=False)
        logz += float(out["logz"][-1][0])
        res["posterior"].append(summary(ctx, n, out, wall, rate, logz))
    ctx.close()
    if prior_start:
        for n in sizes[1:]:
            ctx = sampler.open_context(wl, precision, n_use=n, n_capacity=[pr.n])
            out, wall, rate = run(ctx)
            res["prior"].append(summary(ctx, n, out, wall, rate, float(out["logz"][-1][0])))
            ctx.close()
    return res


def _main(argv=None):
    import argparse
    import json

    from . import synth

    ap = argparse.ArgumentParser(prog="python -m paper_2609_17674_b300.experiments")
    sub = ap.add_subparsers(dest="cmd", required=True)
    ev = sub.add_parser("eval", help="batched logL + gradient throughput (pulse workload)")
    ev.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ev.add_argument("--particles", type=int, default=8192)
    ev.add_argument("--samples", type=int, default=16384)
    ev.add_argument("--reps", type=int, default=3)
    nu = sub.add_parser("nuts", help="NUTS transitions after a few SMC stages (one workload)")
    nu.add_argument("--workload", choices=["pulse", "gb", "gb_ae"], default="pulse")
    nu.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    nu.add_argument("--particles", type=int, default=1024)
    nu.add_argument("--warm-stages", type=int, default=3)
    nu.add_argument("--launches", type=int, default=3)
    asm = sub.add_parser("assimilation", help="posterior start over 2^17, 2^18, 2^19 samples")
    asm.add_argument("--particles", type=int, default=16384)
    asm.add_argument("--max-stages", type=int, default=400)
    asm.add_argument("--no-prior-start", action="store_true")
    asm.add_argument("--no-posterior-start", action="store_true")
    a = ap.parse_args(argv)
    prec = capi.FP64 if getattr(a, "precision", "mixed") == "fp64" else capi.MIXED
    if a.cmd == "eval":
        wl = synth.pulse_k20(P=a.particles, n=a.samples)
        print(json.dumps(eval_throughput(wl, prec, reps=a.reps)))
    elif a.cmd == "nuts":
        wl = {"pulse": lambda: synth.pulse_k20(P=a.particles),
              "gb": lambda: synth.gb_band_k10(P=a.particles),
              "gb_ae": lambda: synth.ae_workload(f"gb_ae_n262144x2_k10_p{a.particles}", 1 << 18,
                                                 10, 30, a.particles, 1007)}[a.workload]()
        print(json.dumps(nuts_launch_timing(wl, prec, a.warm_stages, a.launches)))
    else:
        print(json.dumps(assimilation_experiment(a.particles, max_stages=a.max_stages,
                                                 prior_start=not a.no_prior_start,
                                                 posterior_start=not a.no_posterior_start)))


if __name__ == "__main__":
    _main()
