"""Writes smc_sinusoid_wrap_oracle.json: 20 oracle SMC runs on a small sinusoid band with
periodic phases (wrap bit on phi0).

Calls only the oracle (and the shared input generator).  The band: N = 1024 samples at
dt = 15 s, two sources with f in [3.0, 3.6] mHz (about nine frequency bins of 1/T, so the
sources are resolved), SNR ~ U[10, 40], white noise sigma = 1, the first source's phase
placed at 0.05 rad next to 0 = 2 pi (the case the periodic map is for); prior K ~ U{0..5},
P = 256, alpha = 0.5, 5 rounds of RJ + NUTS per stage, Philox seeds 0..19.  Stored per run:
the K histogram, log Z, the stage count, beta and log Z after every stage and, among
particles with K = K_true, the mean sorted frequencies and the mean (cos phi0, sin phi0) of
the frequency-ordered components.
Run:  python tests/golden/make_smc_sinusoid_wrap.py   (about four minutes on 8 cores)
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

PHASE, WRAP = 3, 1 << 3


def workload(seed=0, P=256):
    from paper_2609_17674_b300 import synth

    rng = np.random.default_rng(3101)
    pr = synth.sinusoid_problem(rng, 1024, 2, f_lo=3.0e-3, f_hi=3.6e-3)
    th = pr.truth.copy()
    th[0, PHASE] = 0.05
    t = pr.t_origin + pr.dt * np.arange(pr.n)
    d = np.zeros(pr.n)
    for A, f, fd, p0 in th:
        d += A * np.cos(synth._sin_phase(t, f, fd, p0))
    pr.d = d + pr.sigma * rng.standard_normal(pr.n)
    pr.truth = th
    return synth.Workload(name="gb_wrap_n1024_k2_p256", model=synth.SINUSOID, kmax=5, P=P,
                          problems=[pr], lo=pr.lo, hi=pr.hi, logmask=0b0001, seed=seed,
                          wrapmask=WRAP)


def summaries(wl, z, K):
    kt = wl.problems[0].truth.shape[0]
    hist = np.bincount(K, minlength=wl.kmax + 1) / len(K)
    sel = np.where(K == kt)[0]
    lo, hi = wl.bounds(0)
    out = {"hist": hist.tolist(), "mean_K": float(np.mean(K)), "n_ktrue": int(len(sel))}
    if len(sel):
        f = lo[1] + (hi[1] - lo[1]) / (1.0 + np.exp(-z[sel, :kt, 1]))
        order = np.argsort(f, axis=1)
        u = np.take_along_axis(z[sel, :kt, PHASE], order, 1)
        ph = lo[PHASE] + (hi[PHASE] - lo[PHASE]) * (u - np.floor(u))
        out["f_sorted_mean"] = np.take_along_axis(f, order, 1).mean(0).tolist()
        out["cos_by_f_mean"] = np.cos(ph).mean(0).tolist()
        out["sin_by_f_mean"] = np.sin(ph).mean(0).tolist()
    return out


def run(seed):
    import oracle

    wl = workload(seed)
    res = oracle.Oracle(wl).smc_run(wl.P, max_stages=400)
    s = summaries(wl, res["z"], res["K"])
    s.update(seed=seed, logz=float(res["logz"]), n_stages=int(res["n_stages"]),
             beta_last=float(res["beta"][-1]), beta_hist=[float(b) for b in res["beta"]],
             logz_hist=[float(x) for x in res["logz_hist"]])
    return s


if __name__ == "__main__":
    import oracle

    oracle.build()
    with mp.get_context("spawn").Pool(min(8, os.cpu_count())) as pool:
        runs = pool.map(run, range(20))
    out = {"workload": "gb_wrap_n1024_k2_p256 (data seed 3101, phi0 periodic), Philox seeds 0..19",
           "runs": runs}
    with open(os.path.join(HERE, "smc_sinusoid_wrap_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", len(runs), "runs")
