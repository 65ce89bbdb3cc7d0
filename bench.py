"""Benchmark: SMC stages of the transdimensional sampler on one B300 per rank.

A step is one whole stage of the hot path (ESS bisection, reweight, systematic
resampling, metric, then n_mut rounds of reversible-jump birth/death + NUTS)
on the Gaussian-pulse workload at scale: N = 16384 samples, K_true = 20,
K_max = 40, P = 8192 particles, mixed precision (FP32 templates and residuals,
FP64 sums, anchors and log-weights).  The metric is component*sample logL+grad
evaluations per second, counted on the device by the kernels themselves (the
batched metric evaluation plus every NUTS leaf and initial point).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs its own independent problem (weak scaling, no
data-path collective), and the extras split the 64 batched bands across the ranks
(each rank a contiguous block, no exchange); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "component*sample logL+grad evals/s"
UNIT = "cs-evals/s"
OPS_PER_CS = {0: 9.0, 1: 14.0}   # algorithmic FP32 lane-ops per component*sample (fwd+adj)
FP32_LANES_PER_SM = 128
# DRAM bytes (read + write) per particle of one NUTS launch, from an ncu capture of the
# same kernel on a 1024-particle launch of this workload
# (profiles/k_nuts_mixed_pulse_n16384_p1024.md); traffic scales with the particle count (z
# rows in and out; the samples stay in L2).  None when the kernel has changed since the
# capture.
NUTS_DRAM_BYTES_PER_PARTICLE = 579.0
NUTS_TRAFFIC_NOTE = ("ncu dram__bytes_read+write of a 1024-particle launch, scaled per "
                     "particle (profiles/k_nuts_mixed_pulse_n16384_p1024.md)")


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--particles", type=int, default=8192)
    ap.add_argument("--samples", type=int, default=16384)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--clock-ms", type=int, default=500,
                    help="nvidia-smi sampling interval (200 ms polling slows kernels on this part)")
    ap.add_argument("--clock-fields", default="full", choices=["full", "reasons", "clocks"])
    return ap.parse_args()


def workload(rank: int, P: int, n: int):
    from paper_2609_17674_b300 import dist as tdist, synth

    return synth.pulse_k20(seed=tdist.rank_seed(1002, rank), P=P, n=n)


# ---------------------------------------------------------------------------
# CPU side: the oracle timed on a bounded sample (reference arm, cpu_baseline)
# ---------------------------------------------------------------------------
def _oracle_worker(args):
    """One oracle stage sample: metric on the slice, one RJ + NUTS round (oracle as is)."""
    wl_seed, P, n, idx, stage, rnd = args
    import oracle
    from paper_2609_17674_b300 import synth

    wl = synth.pulse_k20(seed=wl_seed, P=P, n=n)
    o = oracle.Oracle(wl)
    z, K = synth.prior_population(wl, 7)
    z, K = z[idx].copy(), K[idx].copy()
    t0 = time.perf_counter()
    r = o.logl_grad(z, K, 1e-4, want_scale=False)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    minv = o.metric(z, K, 1e-4)
    o.rj_move(stage, rnd, 1e-4, z, K, lo, ln)
    Kn = K.copy()
    acc, nl, fl = o.nuts_move(stage, rnd, 1e-4, o.eps_initial(), minv, z, K, lo, ln)
    dt = time.perf_counter() - t0
    cs = float(np.sum(K.astype(np.float64) * n)) * 2  # gradient eval + metric eval of the slice
    cs += float(np.sum(Kn.astype(np.float64) * n * np.where(nl > 0, nl + 1, 0)))
    return cs, dt


def oracle_sample(wl_seed, P, n, cores, per_core, step):
    import multiprocessing as mp

    rng = np.random.default_rng(step)
    idx = rng.choice(P, cores * per_core, replace=False)
    jobs = [(wl_seed, P, n, idx[c * per_core:(c + 1) * per_core], step, 0) for c in range(cores)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map(_oracle_worker, jobs)
    wall = time.perf_counter() - t0
    cs = sum(r[0] for r in res)
    busy = max(r[1] for r in res)
    return cs, wall, busy


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = len(os.sched_getaffinity(0))
    per_core = 1
    wl = workload(0, a.particles, a.samples)
    for s in range(a.warmup):
        oracle_sample(wl.seed, a.particles, a.samples, cores, per_core, 1000 + s)
    tot_cs, tot_wall = 0.0, 0.0
    for s in range(a.steps):
        cs, wall, busy = oracle_sample(wl.seed, a.particles, a.samples, cores, per_core, s)
        tot_cs += cs
        tot_wall += busy
    v = tot_cs / tot_wall
    sample = (f"oracle (single-threaded FP64 C) per core: {per_core} particle(s) of the same "
              f"workload, logL+grad + metric + one RJ move + one NUTS transition per step, "
              f"{cores} processes")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": a.gpus,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": 1e3 * tot_wall / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "N": a.samples, "P": a.particles, "kmax": 40,
                   "K_true": 20, "precision": "fp64 oracle"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------------
# GPU side
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 200, fields: str = "full"):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = {"full": self.FIELDS,
             "reasons": self.FIELDS.replace("power.draw,", ""),
             "clocks": "index,clocks.sm,clocks.max.sm"}[fields]
        self.cols = q.split(",")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms",
                                       str(interval_ms), "-i", str(gpu_index)],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def wait_first(self, timeout_s: float = 10.0):
        """Returns once nvidia-smi has written its first sample (its start-up, which
        initialises NVML on the device, stays outside the timed region)."""
        t0 = time.perf_counter()
        while self.p is not None and time.perf_counter() - t0 < timeout_s:
            if os.path.getsize(self.f.name) > 0 or self.p.poll() is not None:
                return
            time.sleep(0.02)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        self.f.seek(0)
        ix = {c: i for i, c in enumerate(self.cols)}
        rows = [[v.strip() for v in r.split(",")] for r in self.f.read().strip().splitlines()]
        rows = [r for r in rows if len(r) == len(self.cols)]
        os.unlink(self.f.name)

        def num(r, c):
            v = r[ix[c]]
            return float(v) if v.replace(".", "").isdigit() else None

        sm = [x for x in (num(r, "clocks.sm") for r in rows) if x is not None]
        mx = [x for x in (num(r, "clocks.max.sm") for r in rows) if x is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n in names
                          if "clocks_event_reasons." + n in ix
                          and "Active" in r[ix["clocks_event_reasons." + n]]
                          and "Not" not in r[ix["clocks_event_reasons." + n]]})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def _events_ms(stream, fn):
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def measure_extras(stream):
    """Secondary measurements: mixed vs FP64 logL+grad throughput, SMC wall time at equal
    error against the oracle reference, the 64-band batched workload, the paper's segment
    experiment on its pulse example and the population birth proposal on it."""
    import json as _json

    import torch

    from paper_2609_17674_b300 import autotune, capi, sampler, synth

    out = {}
    # (1) batched logL+grad kernel, pulse N=16384, K_max=40, P=8192, prior population
    wl = synth.pulse_k20()
    z, K = synth.prior_population(wl, 1)
    zd, Kd = torch.as_tensor(z, device="cuda"), torch.as_tensor(K, device="cuda")
    beta = torch.tensor([0.5], dtype=torch.float64, device="cuda")
    cs = float(K.sum()) * wl.problems[0].n
    thr = {}
    for name, prec, win in (("mixed", capi.MIXED, 1), ("mixed_no_window", capi.MIXED, 0),
                            ("fp64", capi.FP64, 0)):
        ctx = sampler.open_context(wl, prec, stream=stream, pulse_window=win)
        ctx.set_population(zd, Kd, beta=[0.5])
        g = torch.empty_like(zd)
        with torch.cuda.stream(stream):
            ctx.eval(zd, Kd, beta, grad=True, g=g)
        ms = min(_events_ms(stream, lambda: ctx.eval(zd, Kd, beta, grad=True, g=g))
                 for _ in range(2 if prec == capi.FP64 else 5))
        thr[name] = cs / (ms * 1e-3)
        ctx.close()
    out["logl_grad_kernel"] = {"workload": wl.name + " (prior population)", "unit": UNIT,
                               **thr, "mixed_over_fp64": thr["mixed"] / thr["fp64"],
                               "mixed_no_window_over_fp64": thr["mixed_no_window"] / thr["fp64"]}
    # (2) full SMC, N=1024 pulses, FP64 vs mixed, against the 20-run oracle reference
    gold = os.path.join(ROOT, "tests", "golden", "smc_pulse_n1024_oracle.json")
    if os.path.exists(gold):
        runs = _json.load(open(gold))["runs"]
        gh = np.array([r["hist"] for r in runs])
        gz = np.array([r["logz"] for r in runs])
        res = {}
        for name, prec in (("fp64", capi.FP64), ("mixed", capi.MIXED)):
            hs, zs, ts = [], [], []
            for seed in range(4):
                w1 = synth.pulse_n1024_k3()
                w1.seed = seed
                ctx = sampler.open_context(w1, prec, stream=stream)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                o = sampler.run_smc(ctx, max_stages=400)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
                _, Kp, _, _ = ctx.get_population()
                hs.append(np.bincount(Kp.cpu().numpy(), minlength=w1.kmax + 1) / w1.P)
                zs.append(o["logz"][-1][0])
                ctx.close()
            hs, zs = np.array(hs), np.array(zs)
            se_h = np.sqrt(hs.var(0, ddof=1) / len(hs) + gh.var(0, ddof=1) / len(gh))
            se_z = math.sqrt(zs.var(ddof=1) / len(zs) + gz.var(ddof=1) / len(gz))
            res[name] = {"wall_s_per_run": float(np.median(ts)), "logz": float(zs.mean()),
                         "within_3se": bool(np.all(np.abs(hs.mean(0) - gh.mean(0))
                                                   <= np.maximum(3 * se_h, 1.0 / w1.P))
                                            and abs(zs.mean() - gz.mean()) <= 3 * se_z)}
        res["oracle_logz"] = float(gz.mean())
        res["fp64_over_mixed_wall"] = res["fp64"]["wall_s_per_run"] / res["mixed"]["wall_s_per_run"]
        out["smc_equal_error_pulse_n1024_p512"] = res
    # (2a) single-channel Galactic-binary band at full size: N = 2^18 at dt = 15 s,
    # K_true = 10, K_max = 30, P = 4096: logL+grad (mixed and FP64), one NUTS transition
    # and one whole SMC stage from the prior start (mixed)
    wg = synth.gb_band_k10()
    zg, Kg = synth.prior_population(wg, 3)
    zdg, Kdg = torch.as_tensor(zg, device="cuda"), torch.as_tensor(Kg, device="cuda")
    csg = float(Kg.astype(np.float64).sum()) * wg.problems[0].n
    bg = torch.tensor([0.5], dtype=torch.float64, device="cuda")
    gbr = {"workload": wg.name, "unit": UNIT}
    for name, prec in (("mixed", capi.MIXED), ("fp64", capi.FP64)):
        ctx = sampler.open_context(wg, prec, stream=stream)
        ctx.set_population(zdg, Kdg, beta=[1e-3])
        gg = torch.empty_like(zdg)
        ctx.eval(zdg, Kdg, bg, grad=True, g=gg)
        msg = min(_events_ms(stream, lambda: ctx.eval(zdg, Kdg, bg, grad=True, g=gg))
                  for _ in range(3 if prec == capi.MIXED else 1))
        gbr[f"logl_grad_kernel_{name}"] = csg / (msg * 1e-3)
        if prec == capi.MIXED:
            ctx.update_metric()
            ctx.counters(reset=True)
            msn = _events_ms(stream, lambda: ctx.nuts_move(0, 0))
            (_, cng, _, _), _ = ctx.counters(reset=True)
            gbr["nuts_transition_mixed"] = cng / (msn * 1e-3)
            gbr["nuts_ms_mixed"] = msn
            ctx.init_population()
            ctx.counters(reset=True)
            mss = _events_ms(stream, lambda: ctx.run_stage(0, use_graph=True, read=False))
            (ce, cn, _, _), _ = ctx.counters(reset=True)
            gbr["stage_ms_mixed"] = mss
            gbr["stage_mixed"] = (ce + cn) / (mss * 1e-3)
        ctx.close()
    gbr["mixed_over_fp64_logl_grad"] = (gbr["logl_grad_kernel_mixed"]
                                        / gbr["logl_grad_kernel_fp64"])
    out["gb_band_n262144_k10_p4096"] = gbr
    # (2b) two channels A and E (eq. gw_likelihood, flat PSD, simplified response):
    # 2^18 samples per channel, K_max = 30, P = 4096, logL + gradient and one NUTS round;
    # the value counts K_p x 2^19 component*samples (both channels)
    wa = synth.ae_workload("gb_ae_n262144x2_k10_p4096", 1 << 18, 10, 30, 4096, 1007)
    za, Ka = synth.prior_population(wa, 3)
    zda, Kda = torch.as_tensor(za, device="cuda"), torch.as_tensor(Ka, device="cuda")
    ctx = sampler.open_context(wa, capi.MIXED, stream=stream)
    ctx.set_population(zda, Kda, beta=[1e-3])
    ba = torch.tensor([0.5], dtype=torch.float64, device="cuda")
    ga = torch.empty_like(zda)
    csa = float(Ka.sum()) * wa.problems[0].n
    msa = min(_events_ms(stream, lambda: ctx.eval(zda, Kda, ba, grad=True, g=ga)) for _ in range(3))
    ctx.update_metric()
    ctx.counters(reset=True)
    msn = _events_ms(stream, lambda: ctx.nuts_move(0, 0))
    (_, cna, _, _), _ = ctx.counters(reset=True)
    out["two_channel_band"] = {"workload": wa.name, "unit": UNIT,
                               "logl_grad_kernel": csa / (msa * 1e-3),
                               "nuts_transition": cna / (msn * 1e-3), "nuts_ms": msn}
    ctx.close()
    # (3) 64 independent GB bands (N_b 2^14..2^18, P=2048 each) in one launch
    w5 = synth.gb_bands()
    nb = len(w5.problems)
    best = autotune.tune(w5, capi.MIXED, nuts=False)
    ctx = sampler.open_context(w5, capi.MIXED, stream=stream, threads=best["threads"],
                               samples_per_thread=best["samples_per_thread"])
    z5, K5 = band_population(w5, range(nb))
    zd5, Kd5 = torch.as_tensor(z5, device="cuda"), torch.as_tensor(K5, device="cuda")
    ctx.set_population(zd5, Kd5, beta=[1e-3] * nb)
    b5 = torch.full((nb,), 0.5, dtype=torch.float64, device="cuda")
    g5 = torch.empty_like(zd5)
    cs5 = float(sum(K5[b * w5.P:(b + 1) * w5.P].sum() * w5.problems[b].n for b in range(nb)))
    ms5 = min(_events_ms(stream, lambda: ctx.eval(zd5, Kd5, b5, grad=True, g=g5)) for _ in range(3))
    ctx.update_metric()
    ctx.counters(reset=True)
    msn = _events_ms(stream, lambda: ctx.nuts_move(0, 0))
    (_, cn, _, _), _ = ctx.counters(reset=True)
    out["gb_bands_64x2048"] = {"unit": UNIT, "launch_shape": best,
                               "logl_grad_kernel": cs5 / (ms5 * 1e-3),
                               "nuts_transition": cn / (msn * 1e-3), "nuts_ms": msn}
    ctx.close()
    # (4) the paper's pulse example (Sec. 5.1): 10 noise-free pulses in 200 s, P=6000,
    # alpha=0.9, mixture moves 0.6/0.2/0.2, K in [1, 10]; 20 s segments, prior-start on
    # each against posterior-start from the previous segment
    from paper_2609_17674_b300 import experiments

    wp = synth.paper_pulse_workload(P=6000)
    r = experiments.segment_experiment(wp, seg_seconds=20.0, precision=capi.MIXED, stream=stream)
    ks = np.arange(wp.kmax + 1)
    out["paper_pulse_segments"] = {
        "workload": wp.name, "segments_s": r["segments_s"],
        "stages_prior_start": [x["stages"] for x in r["prior"]],
        "stages_posterior_start": [x["stages"] for x in r["posterior"]],
        "wall_s_prior_start": [round(x["wall_s"], 3) for x in r["prior"]],
        "wall_s_posterior_start": [round(x["wall_s"], 3) for x in r["posterior"]],
        "logz_prior_start": [round(x["logz"], 2) for x in r["prior"]],
        "logz_posterior_start": [round(x["logz"], 2) for x in r["posterior"]],
        "mean_k_prior_start": [round(float(np.dot(x["k_hist"], ks)), 3) for x in r["prior"]],
        "mean_k_posterior_start": [round(float(np.dot(x["k_hist"], ks)), 3)
                                   for x in r["posterior"]],
        "k_mode_all_data": [int(np.argmax(r["prior"][-1]["k_hist"])),
                            int(np.argmax(r["posterior"][-1]["k_hist"]))]}
    # (5) births from the prior against births from the population mixture (Sec. 6
    # suggestion): full runs of the same example, and birth acceptance on one mid-run
    # population under both proposals
    cmp = experiments.birth_proposal_comparison(wp, mid_stages=40, precision=capi.MIXED,
                                                stream=stream)
    out["birth_proposal_paper_pulses"] = cmp
    return out


def _snapshot(ctx):
    """Device copies of the population and the per-problem state a stage starts from."""
    z, K, _, _ = ctx.get_population()
    beta, logz, _ = ctx.temper_state()
    eps, minv = ctx.get_kernel_params()
    return dict(z=z.clone(), K=K.clone(), beta=beta, logz=logz, eps=eps, minv=minv)


def _restore(ctx, snap):
    ctx.set_population(snap["z"].clone(), snap["K"].clone(), beta=snap["beta"],
                       logz=snap["logz"])
    ctx.set_kernel_params(snap["eps"], snap["minv"])
    ctx.sync()


def band_population(full, bands):
    """Frozen prior populations of the batched bands (seed 100 + global band index)."""
    from paper_2609_17674_b300 import synth

    zs, Ks = [], []
    for b in bands:
        zb, Kb = synth.prior_population(full, 100 + b, full.P)
        zs.append(zb)
        Ks.append(Kb)
    return np.concatenate(zs), np.concatenate(Ks)


def measure_sharded_bands(stream, world, rank, local, barrier):
    """The 64 batched bands split across the ranks (each rank a contiguous block, its own
    context, no exchange): logL+grad and one NUTS transition per rank, the whole job's
    component*samples over the slowest rank's time (strong scaling: the total is fixed)."""
    import torch

    from paper_2609_17674_b300 import capi, sampler, synth
    from paper_2609_17674_b300 import dist as tdist

    full = synth.gb_bands()
    wl, idx = tdist.shard_problems(full, world, rank)
    dev = torch.device("cuda", local)
    ms_e = ms_n = cs_e = cs_n = 0.0
    if wl is not None:
        z, K = band_population(full, idx)
        zd, Kd = torch.as_tensor(z, device=dev), torch.as_tensor(K, device=dev)
        ctx = sampler.open_context(wl, capi.MIXED, stream=stream)
        ctx.set_population(zd, Kd, beta=[1e-3] * len(idx))
        ctx.update_metric()
        bt = torch.full((len(idx),), 0.5, dtype=torch.float64, device=dev)
        g = torch.empty_like(zd)
        ctx.eval(zd, Kd, bt, grad=True, g=g)
        barrier()
        ms_e = _events_ms(stream, lambda: ctx.eval(zd, Kd, bt, grad=True, g=g))
        cs_e = float(sum(K[i * wl.P:(i + 1) * wl.P].astype(np.float64).sum() * wl.problems[i].n
                         for i in range(len(idx))))
        ctx.counters(reset=True)
        barrier()
        ms_n = _events_ms(stream, lambda: ctx.nuts_move(0, 0))
        (_, c_n, _, _), _ = ctx.counters(reset=True)
        cs_n = float(c_n)
        ctx.close()
    else:
        barrier()
        barrier()
    me, ce = tdist.reduce_measurement(ms_e, cs_e, device=dev)
    mn, cn = tdist.reduce_measurement(ms_n, cs_n, device=dev)
    return {"workload": full.name, "ranks": world, "bands_per_rank": len(idx),
            "unit": UNIT, "logl_grad_kernel": ce / (me * 1e-3),
            "nuts_transition": cn / (mn * 1e-3), "scaling": "strong (64 bands in total)"}


def run_gpu(a):
    import torch

    from paper_2609_17674_b300 import capi, sampler
    from paper_2609_17674_b300 import dist as tdist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    props = torch.cuda.get_device_properties(local)
    wl = workload(rank, a.particles, a.samples)
    stream = torch.cuda.Stream()
    ctx = sampler.open_context(wl, capi.MIXED, stream=stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ctx.init_population()
    ctx.profile(True, events=200 * a.steps)
    stage = 0
    for _ in range(a.warmup):   # the same calls as a timed step (first use loads their kernels)
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
        ctx.run_stage(stage, use_graph=False, read=False)
        stage += 1
    torch.cuda.synchronize()
    stage0 = stage
    snap = _snapshot(ctx)     # the state both legs start from: the same stage window
    ctx.counters(reset=True)
    ctx.profile_read(reset=True)
    clocks = ClockSampler(local, a.clock_ms, a.clock_fields)
    clocks.wait_first()
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(a.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)          # L2 flush between steps (256 MB write)
        # eager launches with an event pair around each kernel (the per-kernel times of the
        # roofline come from this same region); queued: no host sync per stage
        ctx.run_stage(stage, use_graph=False, read=False)
        stage += 1
    ev1.record(stream)
    torch.cuda.synchronize()
    betas = [float(ctx.temper_state()[0][0])]
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    (cs_eval, cs_nuts, cc_eval, cc_nuts), launches = ctx.counters(reset=True)
    prof = ctx.profile_read(reset=True)
    ms_max, cs_total = tdist.reduce_measurement(ms, float(cs_eval + cs_nuts),
                                                device=torch.device("cuda", local))
    _, cc_total = tdist.reduce_measurement(ms, float(cc_eval + cc_nuts),
                                           device=torch.device("cuda", local))
    value = cs_total / (ms_max * 1e-3)
    value_computed = cc_total / (ms_max * 1e-3)

    # roofline of the dominant kernel (NUTS transition), ALU bound (FP32 pipe), on the
    # component*samples it computed (the support window skips the rest)
    n_nuts, ms_nuts = prof["nuts"]
    per_launch_ms = ms_nuts / max(n_nuts, 1)
    ops = OPS_PER_CS[wl.model] * cc_nuts
    achieved = ops / max(ms_nuts * 1e-3, 1e-12) / 1e12
    mhz = clk.get("sm_mhz") or 2032.0
    n_sm = props.multi_processor_count
    peak = FP32_LANES_PER_SM * n_sm * mhz * 1e6 / 1e12
    roof = {"kernel": "k_nuts_mixed<PULSE,32>", "bound": "alu", "achieved": achieved,
            "peak": peak, "unit": "Tops/s (FP32 lane-ops, FMA=1)", "frac": achieved / peak,
            "traffic": NUTS_DRAM_BYTES_PER_PARTICLE * a.particles if NUTS_DRAM_BYTES_PER_PARTICLE
            else None,
            "traffic_note": NUTS_TRAFFIC_NOTE,
            "launches": n_nuts, "ms_per_launch": per_launch_ms,
            "share_of_step": ms_nuts / ms,
            "peak_basis": f"128 FP32 lanes x {n_sm} SMs (device properties) x {mhz:.0f} MHz "
                          "(median SM clock sampled during the timed region)",
            "ops_per_cs": OPS_PER_CS[wl.model],
            "work_basis": "component*samples the NUTS launches computed (device counter)",
            "cs_nominal": cs_nuts, "cs_computed": cc_nuts,
            "computed_cs_per_s": cc_nuts / max(ms_nuts * 1e-3, 1e-12),
            "nominal_cs_per_s": cs_nuts / max(ms_nuts * 1e-3, 1e-12),
            "kernels_ms": {k: v[1] for k, v in prof.items()}}

    # end to end through the public API with the population on the host (pinned) between
    # stages, over the same stage window from the same starting state and in the same
    # execution mode (eager, per-kernel events) as the device-timed region
    e2e = None
    if not a.no_e2e:
        _restore(ctx, snap)
        zh = torch.empty(snap["z"].shape, dtype=snap["z"].dtype, pin_memory=True)
        Kh = torch.empty(snap["K"].shape, dtype=snap["K"].dtype, pin_memory=True)
        lnh = torch.empty(snap["K"].shape, dtype=torch.float64, pin_memory=True)
        zh.copy_(snap["z"])
        Kh.copy_(snap["K"])
        zd, Kd = torch.empty_like(snap["z"]), torch.empty_like(snap["K"])
        state = dict(eps=snap["eps"], beta=snap["beta"], logz=snap["logz"])

        def e2e_step(st):
            with torch.cuda.stream(stream):
                zd.copy_(zh, non_blocking=True)
                Kd.copy_(Kh, non_blocking=True)
            ctx.set_population(zd, Kd, beta=state["beta"], logz=state["logz"])
            ctx.set_kernel_params(state["eps"])
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
            b, lz, _ = ctx.run_stage(st, use_graph=False)
            zo, Ko, _, lno = ctx.get_population()
            with torch.cuda.stream(stream):
                zh.copy_(zo, non_blocking=True)
                Kh.copy_(Ko, non_blocking=True)
                lnh.copy_(lno, non_blocking=True)
            state["eps"], _ = ctx.get_kernel_params()
            stream.synchronize()
            state["beta"], state["logz"] = b, lz

        ctx.counters(reset=True)
        ctx.profile_read(reset=True)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for st in range(stage0, stage0 + a.steps):
            e2e_step(st)
        t1 = time.perf_counter()
        barrier()
        (ce, cn, _, _), _ = ctx.counters(reset=True)
        ctx.profile_read(reset=True)
        el, cst = tdist.reduce_measurement((t1 - t0) * 1e3, float(ce + cn),
                                           device=torch.device("cuda", local))
        h2d = zh.numel() * 8 + Kh.numel() * 4 + 8 * 4
        d2h = zh.numel() * 8 + Kh.numel() * 4 + lnh.numel() * 8 + 8 * 5
        e2e = {"value": cst / (el * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "stages": [stage0, stage0 + a.steps],
               "path": "pinned host population -> tsmc_set_population -> tsmc_run_stage "
                       "(eager, per-kernel events, as the device-timed region) -> "
                       "tsmc_get_population -> pinned host; same stages and starting state "
                       "as the device-timed region"}
    ctx.profile(False)

    sharded = None
    if world > 1 and not a.no_extras:
        sharded = measure_sharded_bands(stream, world, rank, local, barrier)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    cpu = None
    if not a.no_cpu:
        cores = len(os.sched_getaffinity(0))
        cs, wall, busy = oracle_sample(wl.seed, a.particles, a.samples, cores, 1, 0)
        cpu = {"value": cs / busy, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{cores} particles of the same workload (one per core, {cores} "
                         "processes): logL+grad, metric, one RJ move and one NUTS transition "
                         f"each; {busy:.1f} s"}
    extras = None if a.no_extras else measure_extras(stream)
    if extras is not None and sharded is not None:
        extras["gb_bands_sharded"] = sharded
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "value_computed": value_computed,
        "value_basis": "value: every K_p*N component*sample of each logL+grad evaluation "
                       "(the metric's definition); value_computed: the component*samples "
                       "the kernels computed (the support window skips terms < 2^-26 A); "
                       "the roofline uses the computed work",
        "config": {"workload": wl.name + " (SMC stage: ESS bisection, resampling, metric, "
                                         "5 x [RJ birth/death + NUTS depth<=6])",
                   "N": a.samples, "P": a.particles, "kmax": 40, "K_true": 20,
                   "precision": "mixed: FP32 templates/residuals, FP64 sums/anchors/log-weights",
                   "l2": "flushed between steps (256 MB write)",
                   "mode": "eager launches, an event pair per kernel (no CUDA graph)",
                   "pulse_window": "on: (component, warp range) pairs with |t - t0| > 6 w "
                                   "(every term < 2^-26 A) skipped",
                   "computed_fraction": (cc_eval + cc_nuts) / max(cs_eval + cs_nuts, 1),
                   "parallelism": f"{world} independent problem(s), one per GPU",
                   "stages": [stage0, stage0 + a.steps],
                   "beta_end": betas[-1]},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
        "clocks": clk, "extras": extras,
    }
    print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)


if __name__ == "__main__":
    main()
