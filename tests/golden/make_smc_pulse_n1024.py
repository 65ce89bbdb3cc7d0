"""Writes smc_pulse_n1024_oracle.json: 20 oracle SMC runs on the N=1024 pulse workload.

Calls only the oracle (and the shared input generator).  Each run is a prior-start
SMC (P=512, K ~ U{0..10}, alpha=0.5, 5 rounds of RJ + NUTS per stage) with Philox
seed s; the data are the same for every run.  Stored per run: the K histogram of
the final population, log Z, the stage count, beta and log Z after every stage, and
label-invariant summaries (mean K; mean sorted pulse centres and amplitudes for
particles with K = K_true).
Run:  python tests/golden/make_smc_pulse_n1024.py   (about 5 minutes on 8 cores)
"""
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))


def summaries(wl, z, K):
    from paper_2609_17674_b300 import synth

    kt = wl.problems[0].truth.shape[0]
    hist = np.bincount(K, minlength=wl.kmax + 1) / len(K)
    sel = np.where(K == kt)[0]
    lo, hi = wl.bounds(0)
    out = {"hist": hist.tolist(), "mean_K": float(np.mean(K)), "n_ktrue": int(len(sel))}
    if len(sel):
        zz = z[sel, :kt]
        s = 1.0 / (1.0 + np.exp(-zz))
        t0 = lo[1] + (hi[1] - lo[1]) * s[..., 1]
        A = lo[0] + (hi[0] - lo[0]) * s[..., 0]
        order = np.argsort(t0, axis=1)
        out["t0_sorted_mean"] = np.take_along_axis(t0, order, 1).mean(0).tolist()
        out["A_by_t0_mean"] = np.take_along_axis(A, order, 1).mean(0).tolist()
    return out


def run(seed):
    import oracle
    from paper_2609_17674_b300 import synth

    wl = synth.pulse_n1024_k3()
    wl.seed = seed
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
    out = {"workload": "pulse_n1024_k3_p512 (data seed 1001), Philox seeds 0..19",
           "runs": runs}
    with open(os.path.join(HERE, "smc_pulse_n1024_oracle.json"), "w") as f:
        json.dump(out, f, indent=1)
    print("wrote", len(runs), "runs")
