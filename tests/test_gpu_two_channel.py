"""Sinusoids in the two noise-orthogonal channels A and E (Sec. 5.2, eq. gw_likelihood with
a flat PSD, computed in the time domain; the oracle's pins tie it to the frequency-domain
inner product) through the C ABI against the oracle: evaluation, Gauss-Newton sums,
reversible jump, NUTS and one SMC stage, a full-size band on a sample of particles, and the
argument checks.  The relative mixed-path comparisons use data with white noise; on the
paper's noise-free data a particle at the injection has a residual near zero, so there the
mixed path is held to an absolute bound scaled by the data energy."""
import numpy as np
import pytest

import oracle
from paper_2609_17674_b300 import capi, sampler, synth
from gpu_helpers import (TOL, assert_eval_parity, context_with_population, data_scale_gscale,
                         dev_tensor, population, torch)

pytestmark = pytest.mark.gpu


def _near_injection(wl, z, K, every=2, jitter=0.01):
    zt = synth.theta_to_z(wl, 0, wl.problems[0].truth)
    for i in range(2, z.shape[0], every):
        k = min(max(K[i], 1), zt.shape[0])
        K[i] = k
        z[i] = 0.0
        z[i, :k] = zt[:k] + jitter * np.random.default_rng(i).standard_normal((k, 4))
    return z, K


@pytest.mark.parametrize("prec", [capi.FP64, capi.MIXED])
@pytest.mark.parametrize("n", [4096, 1056])
def test_eval_parity(prec, n):
    t = torch()
    wl = synth.ae_workload("t", n, 3, 5, 24, 41, noise=True)
    z, K = _near_injection(wl, *population(wl, 5, 24))
    ctx, zd, Kd = context_with_population(wl, prec, z, K, 0.37)
    lo, ln, lp, g, _ = ctx.eval(zd, Kd, dev_tensor([0.37], t.float64), grad=True)
    t.cuda.synchronize()
    ora = oracle.Oracle(wl)
    res = ora.logl_grad(z, K, 0.37)
    assert_eval_parity(ora, res, lo, ln, lp, g, K, TOL[prec], 4)


@pytest.mark.parametrize("jitter", [1e-3, 1e-6])
def test_mixed_eval_noise_free_absolute_bound(jitter):
    """The paper's data are noise-free (Sec. 5.2), so a particle at the injection has a residual
    near zero and no relative bound on its likelihood is meaningful.  With FP32 templates each
    residual carries an error of a few eps32 times the signal, which moves the energy by at
    most ~2 eps32 sqrt(E D) + O(eps32^2 D) <= eps32 (E + D), D = sum d^2 / sigma^2 the data
    energy: the mixed path is held to |dlogL| <= 1e-5 (1/2 D + |logL|) on every particle,
    near the injection and far from it, and its gradient to 1e-5 of the sum of absolute
    terms at the residual plus the same sum at the data scale."""
    t = torch()
    wl = synth.ae_workload("t", 4096, 3, 5, 24, 44, noise=False)
    z, K = population(wl, 6, 24)
    K[2::2] = 3
    z, K = _near_injection(wl, z, K, jitter=jitter)
    ctx, zd, Kd = context_with_population(wl, capi.MIXED, z, K, 0.8)
    lo, ln, lp, g, _ = ctx.eval(zd, Kd, dev_tensor([0.8], t.float64), grad=True)
    t.cuda.synchronize()
    res = oracle.Oracle(wl).logl_grad(z, K, 0.8)
    pr = wl.problems[0]
    half_D = 0.5 * float(np.sum(pr.d ** 2)) / pr.sigma ** 2
    err = np.abs(ln.cpu().numpy() - res["ll_new"])
    assert np.all(err <= 1e-5 * (half_D + np.abs(res["ll_new"]))), (err.max(), half_D)
    hard = [i for i in range(2, 24, 2) if K[i] == 3]          # all three sources, at the truth
    assert len(hard) >= 4 and np.max(np.abs(res["ll_new"][hard])) < 0.1 * half_D
    gerr = np.abs(g.cpu().numpy() - res["grad"])
    gs = res["gscale"] + data_scale_gscale(wl, z, K, 0.8)
    assert np.all(gerr <= 1e-5 * gs + 1e-300), float(np.max(gerr / (gs + 1e-300)))


@pytest.mark.parametrize("prec", [capi.FP64, capi.MIXED])
def test_fisher_parity(prec):
    t = torch()
    wl = synth.ae_workload("t", 4096, 3, 4, 12, 42, noise=True)
    z, K = _near_injection(wl, *population(wl, 9, 12))
    ctx, zd, Kd = context_with_population(wl, prec, z, K, 0.5)
    _, _, _, _, fis = ctx.eval(zd, Kd, dev_tensor([0.5], t.float64), grad=True, fisher=True)
    res = oracle.Oracle(wl).logl_grad(z, K, 0.5, want_fisher=True)
    np.testing.assert_allclose(fis.cpu().numpy(), res["fisher"].sum(1),
                               rtol=1e-10 if prec == capi.FP64 else 1e-4)


def test_rj_move_parity_fp64():
    t = torch()
    wl = synth.ae_workload("t", 2048, 3, 6, 160, 43)
    z, K = _near_injection(wl, *population(wl, 13, 160), every=3, jitter=0.02)
    beta = 0.45
    ora = oracle.Oracle(wl)
    ctx, _, _ = context_with_population(wl, capi.FP64, z, K, beta)
    r = ora.logl_grad(z, K, beta)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    zo, Ko = z.copy(), K.copy()
    out_o = ora.rj_move(4, 2, beta, zo, Ko, lo, ln)
    outd = t.zeros(160, dtype=t.int32, device="cuda")
    ctx.rj_move(4, 2, outd)
    zg, Kg, _, lng = ctx.get_population()
    assert np.array_equal(outd.cpu().numpy(), out_o)
    assert np.array_equal(Kg.cpu().numpy(), Ko)
    np.testing.assert_allclose(zg.cpu().numpy(), zo, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(lng.cpu().numpy(), ln, rtol=1e-10)


def test_nuts_parity_fp64():
    t = torch()
    wl = synth.ae_workload("t", 1024, 2, 3, 48, 44)
    ora = oracle.Oracle(wl)
    rng = np.random.default_rng(0)
    zt = synth.theta_to_z(wl, 0, wl.problems[0].truth)
    K = np.full(48, 2, np.int32)
    z = np.zeros((48, 3, 4))
    z[:, :2] = zt[None] + 0.002 * rng.standard_normal((48, 2, 4))
    beta = 0.3
    minv = ora.metric(z, K, beta)
    eps = 0.05
    ctx, _, _ = context_with_population(wl, capi.FP64, z, K, beta)
    ctx.set_kernel_params([eps], minv[None, :])
    acc = t.zeros(48, dtype=t.float64, device="cuda")
    nl = t.zeros(48, dtype=t.int32, device="cuda")
    fl = t.zeros(48, dtype=t.int32, device="cuda")
    ctx.nuts_move(3, 1, acc, nl, fl)
    zg, _, _, ln_g = ctx.get_population()
    r = ora.logl_grad(z, K, beta)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    zo = z.copy()
    acc_o, nl_o, fl_o = ora.nuts_move(3, 1, beta, eps, minv, zo, K, lo, ln)
    assert np.array_equal(nl.cpu().numpy(), nl_o)
    assert np.array_equal(fl.cpu().numpy(), fl_o)
    np.testing.assert_allclose(zg.cpu().numpy(), zo, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(ln_g.cpu().numpy(), ln, rtol=1e-10)
    assert np.mean(nl_o) > 1


def test_smc_stage_matches_oracle_fp64():
    wl = synth.ae_workload("t", 1024, 2, 4, 128, 45)
    ctx = sampler.open_context(wl, capi.FP64)
    ctx.init_population()
    b, lz, _ = ctx.run_stage(0, use_graph=False)
    z, K, _, _ = ctx.get_population()
    res = oracle.Oracle(wl).smc_run(128, max_stages=1)
    assert b[0] == pytest.approx(res["beta"][0], abs=1e-13)
    assert lz[0] == pytest.approx(res["logz"], rel=1e-11, abs=1e-11)
    Kg = K.cpu().numpy()
    assert np.mean(Kg == res["K"]) > 0.95


def test_full_size_band_sampled():
    """2^18 samples per channel (2^19 in all), K_max = 30, P = 1024; oracle on a sample."""
    t = torch()
    wl = synth.ae_workload("gb_ae", 1 << 18, 10, 30, 1024, 46, noise=True)
    z, K = _near_injection(wl, *population(wl, 1, 1024), every=7, jitter=1e-4)
    ctx, zd, Kd = context_with_population(wl, capi.MIXED, z, K, 0.9)
    lo, ln, lp, g, _ = ctx.eval(zd, Kd, dev_tensor([0.9], t.float64), grad=True)
    t.cuda.synchronize()
    idx = np.array([0, 1, 2, 3, 9, 16])
    res = oracle.Oracle(wl).logl_grad(z[idx], K[idx], 0.9)
    assert_eval_parity(None, res, lo[idx], ln[idx], lp[idx], g[idx], K[idx], TOL[capi.MIXED], 4)


def test_two_channel_arguments_checked():
    wl = synth.ae_workload("t", 1024, 2, 4, 8, 47)
    cfg = sampler.make_config(wl, capi.MIXED)
    for bad in ("model", "response"):
        c2 = sampler.make_config(wl, capi.MIXED)
        if bad == "model":
            c2.model = capi.PULSE
        else:
            c2.response[2] = 0.0
        with pytest.raises(capi.TsmcError):
            capi.Context(c2, [2048])
    ctx = sampler.open_context(wl, capi.MIXED)
    with pytest.raises(capi.TsmcError):      # 2 x 1000: not a multiple of 32 per channel
        ctx.set_problem(0, np.zeros(2000), 0.0, 15.0, 1.0, wl.lo, wl.hi, wl.logmask)
    ctx.init_population()
    with pytest.raises(capi.TsmcError):      # no appended samples for two channels
        ctx.assimilate(0, np.zeros(64))
    assert cfg.channels == 2
