"""The paper's pulse example (Sec. 5.1) end to end on the GPU, at reduced scale.

Noise-free 10-pulse signal in 200 s, K prior U{1..10}, alpha = 0.9, mixture moves
0.6 / 0.2 / 0.2, data arriving in 40 s segments (2000 particles instead of 6000, 40 s
instead of 20 s segments, to keep the test short).  Checked, as the paper reports:
- posterior-start needs fewer SMC stages than prior-start on every later segment, while
  prior-start needs more as the data grow;
- both modes reach the same posterior over K and the same evidence on every segment;
- with all 200 s the posterior over K peaks at the 10 injected pulses.
"""
import numpy as np
import pytest

import oracle
from paper_2609_17674_b300 import capi, experiments, sampler, synth

pytestmark = pytest.mark.gpu


def test_segment_experiment_prior_vs_posterior_start():
    wl = synth.paper_pulse_workload(P=2000)
    r = experiments.segment_experiment(wl, seg_seconds=40.0, precision=capi.MIXED)
    pri, post = r["prior"], r["posterior"]
    assert all(s["reached"] for s in pri + post)
    # stage counts: posterior-start cheaper on every later segment; prior-start grows
    for a, b in zip(pri[1:], post[1:]):
        assert b["stages"] < a["stages"], (a["stages"], b["stages"])
    assert pri[-1]["stages"] > pri[0]["stages"]
    # same K posterior and evidence in both modes
    ks = np.arange(wl.kmax + 1)
    for a, b in zip(pri, post):
        ea, eb = np.dot(a["k_hist"], ks), np.dot(b["k_hist"], ks)
        assert abs(ea - eb) <= 0.35, (a["seconds"], ea, eb)
        assert abs(a["logz"] - b["logz"]) <= 2.0, (a["seconds"], a["logz"], b["logz"])
    # all the data: the 10 injected pulses
    assert int(np.argmax(pri[-1]["k_hist"])) == 10
    assert int(np.argmax(post[-1]["k_hist"])) == 10


def test_paper_workload_first_stages_match_oracle_fp64():
    """Two SMC stages of the paper's settings (K floor 1, alpha 0.9, mixture moves, uniform
    width prior) on the first 20 s, FP64 path against the oracle."""
    wl = synth.paper_pulse_workload(P=128)
    n = 200
    ctx = sampler.open_context(wl, capi.FP64, n_use=n, n_capacity=[wl.problems[0].n])
    ctx.init_population()
    betas = [ctx.run_stage(s, use_graph=False)[0][0] for s in range(2)]
    z, K, _, _ = ctx.get_population()
    res = oracle.Oracle(wl, n=n).smc_run(128, max_stages=2)
    np.testing.assert_allclose(betas, res["beta"][:2], rtol=0, atol=1e-12)
    Kg = K.cpu().numpy()
    assert Kg.min() >= 1 and res["K"].min() >= 1
    assert np.mean(Kg == res["K"]) > 0.95
    same = Kg == res["K"]
    close = np.all(np.isclose(z.cpu().numpy(), res["z"], rtol=1e-8, atol=1e-8), axis=(1, 2))
    assert np.mean(close[same]) > 0.9
