"""Whole SMC runs at the benchmark sizes, checked against the injection.

At N = 16384 (20 pulses) and N = 2^18 (10 sinusoids) the oracle cannot run an SMC, so a run
of the mixed GPU path is held to what the posterior must satisfy (Sec. 5.1, 5.2):

- every problem reaches beta = 1;
- the population reaches the likelihood level of the injection.  For p = D K_true
  parameters the log-likelihood of a posterior draw differs from the injection's by
  (chi2_p - chi2'_p) / 2 (noise fitted minus posterior spread): mean ~0, standard deviation
  ~sqrt(p).  The median of a sample of particles, scored by the oracle, must lie above
  logL(injection) - p / 2;
- the modal K is within one or two of K_true;
- on the sinusoid band (resolved sources), the frequencies of the particles with K = K_true,
  sorted, agree with the injected ones within 3 population standard deviations (plus a tenth
  of a frequency bin 1/T).

The 20 pulses of the N = 16384 workload overlap heavily (widths up to 0.05 of the span, support
+-6 widths), and a run may settle on a configuration of centres that explains the data as
well as the injection does (its likelihood is at or above the injection's) but not at the
injected centres, so there the check is the likelihood level, not the centres.
"""
import numpy as np
import pytest

import oracle
from paper_2609_17674_b300 import capi, sampler, synth
from gpu_helpers import torch

pytestmark = pytest.mark.gpu


def _run(wl, max_stages):
    ctx = sampler.open_context(wl, capi.MIXED)
    out = sampler.run_smc(ctx, max_stages=max_stages)
    z, K, _, _ = ctx.get_population()
    ctx.close()
    return out, z.cpu().numpy(), K.cpu().numpy()


def _likelihood_level(wl, z, K, n_sample=64, seed=0):
    """Oracle log-likelihood (beta = 1) of the injection and of sampled particles."""
    ora = oracle.Oracle(wl)
    truth = wl.problems[0].truth
    zt = np.zeros((1, wl.kmax, wl.D))
    zt[0, : truth.shape[0]] = synth.theta_to_z(wl, 0, truth)
    lt = ora.logl_grad(zt, np.array([truth.shape[0]], np.int32), 1.0, want_scale=False)["ll_new"][0]
    idx = np.random.default_rng(seed).choice(len(K), n_sample, replace=False)
    lp = ora.logl_grad(z[idx], K[idx], 1.0, want_scale=False)["ll_new"]
    return lt, lp


def test_pulse_n16384_k20_full_smc_reaches_the_injection_likelihood():
    torch()
    wl = synth.pulse_k20()                    # N = 16384, K_true = 20, K_max = 40, P = 8192
    out, z, K = _run(wl, max_stages=400)
    assert out["beta"][-1][0] == 1.0
    kt = wl.problems[0].truth.shape[0]
    hist = np.bincount(K, minlength=wl.kmax + 1)
    assert abs(int(np.argmax(hist)) - kt) <= 1, hist
    lt, lp = _likelihood_level(wl, z, K)
    assert np.all(np.isfinite(lp))
    p = wl.D * kt
    assert np.median(lp) >= lt - p / 2, (np.median(lp), lt)


@pytest.mark.parametrize("periodic_phase", [False, True])
def test_gb_band_n262144_k10_full_smc_recovers_the_injection(periodic_phase):
    torch()
    wl = synth.gb_band_k10(P=1024)           # N = 2^18 at 15 s, K_true = 10, K_max = 30
    if periodic_phase:
        wl.wrapmask = 1 << 3                 # phi0 on the circle
    out, z, K = _run(wl, max_stages=400)
    assert out["beta"][-1][0] == 1.0
    pr = wl.problems[0]
    kt = pr.truth.shape[0]
    hist = np.bincount(K, minlength=wl.kmax + 1)
    assert abs(int(np.argmax(hist)) - kt) <= 2, hist
    lt, lp = _likelihood_level(wl, z, K)
    assert np.all(np.isfinite(lp))
    assert np.median(lp) >= lt - wl.D * kt / 2, (np.median(lp), lt)
    # frequencies of the K = K_true particles, sorted (labels are exchangeable)
    sel = np.where(K == kt)[0]
    assert len(sel) >= 0.05 * len(K)
    lo, hi = wl.bounds(0)
    f = lo[1] + (hi[1] - lo[1]) / (1.0 + np.exp(-z[sel, :kt, 1]))
    f = np.sort(f, axis=1)
    T = pr.n * pr.dt
    dev = np.abs(f.mean(0) - np.sort(pr.truth[:, 1]))
    assert np.all(dev <= 3 * f.std(0) + 0.1 / T), (dev, f.std(0))
    if periodic_phase:
        # phases of the same components (labels ordered by frequency), on the circle
        order = np.argsort(lo[1] + (hi[1] - lo[1]) / (1.0 + np.exp(-z[sel, :kt, 1])), axis=1)
        u = np.take_along_axis(z[sel, :kt, 3], order, 1)
        ph = 2 * np.pi * (u - np.floor(u))
        m = np.mean(np.exp(1j * ph), axis=0)
        sd = np.sqrt(-2.0 * np.log(np.abs(m)))
        tr = pr.truth[np.argsort(pr.truth[:, 1]), 3]
        err = np.abs(np.angle(m * np.exp(-1j * tr)))
        assert np.all(err <= 3 * sd + 0.05), (err, sd)


def test_batched_gb_bands_full_smc_reach_their_injections():
    """Eight bands of the batched workload (ragged N_b in [2^14, 2^18], K_true in 1..15),
    512 particles each, in one context: every band reaches beta = 1 and its likelihood
    level.  K is not checked here: a 5 uHz window spans 5e-6 N_b dt frequency bins, about
    one at N_b = 2^14, so the sources of the shorter bands are not resolved and K is not
    identified by their data."""
    torch()
    wl = synth.gb_bands(n_bands=8, P=512)
    ctx = sampler.open_context(wl, capi.MIXED)
    out = sampler.run_smc(ctx, max_stages=400)
    z, K, _, _ = ctx.get_population()
    ctx.close()
    assert np.all(out["beta"][-1] == 1.0)
    z, K = z.cpu().numpy(), K.cpu().numpy()
    P = wl.P
    for b, pr in enumerate(wl.problems):
        zb, Kb = z[b * P:(b + 1) * P], K[b * P:(b + 1) * P]
        kt = pr.truth.shape[0]
        ora = oracle.Oracle(wl, b)
        zt = np.zeros((1, wl.kmax, wl.D))
        zt[0, :kt] = synth.theta_to_z(wl, b, pr.truth)
        lt = ora.logl_grad(zt, np.array([kt], np.int32), 1.0, want_scale=False)["ll_new"][0]
        idx = np.random.default_rng(b).choice(P, 32, replace=False)
        lp = ora.logl_grad(zb[idx], Kb[idx], 1.0, want_scale=False)["ll_new"]
        assert np.all(np.isfinite(lp))
        assert np.median(lp) >= lt - wl.D * kt / 2, (b, np.median(lp), lt)
