"""Periodic phase coordinates (tsmc_config.wrap_mask) on the GPU against the oracle.

The same parity bars as the logit-mapped parameters: FP64 path to rounding (exact draws,
RJ outcomes, NUTS trees), mixed path to its tolerance, with phase coordinates spread over
several periods so that the fractional part is exercised, and one whole FP64 stage.
"""
import numpy as np
import pytest

import oracle
from paper_2609_17674_b300 import capi, sampler, synth
from gpu_helpers import (assert_eval_parity, context_with_population, dev_tensor, population,
                         torch)

pytestmark = pytest.mark.gpu

PHASE, WRAP = 3, 1 << 3
TOL = {capi.FP64: 1e-12, capi.MIXED: 1e-5}


def _wl(n=5000, P=64, seed=43, kmax=8):
    wl = synth.sinusoid_workload("t", n, 3, kmax, P, seed)
    wl.wrapmask = WRAP
    return wl


def _spread(z, seed):
    """Shift every phase coordinate by a whole number of periods in [-4, 5]."""
    rng = np.random.default_rng(seed)
    z = z.copy()
    z[..., PHASE] += rng.integers(-4, 6, size=z.shape[:-1])
    return z


@pytest.mark.parametrize("prec", [capi.FP64, capi.MIXED])
@pytest.mark.parametrize("n1", [0, 1777])
def test_eval_parity_with_periodic_phase(prec, n1):
    t = torch()
    wl = _wl()
    z, K = population(wl, 5, wl.P)
    zt = synth.theta_to_z(wl, 0, wl.problems[0].truth)
    for i in range(2, wl.P, 2):          # half near the injection (small residuals)
        k = min(K[i], 3)
        K[i] = k
        z[i, :k] = zt[:k] + 0.01 * np.random.default_rng(i).standard_normal((k, 4))
    z = _spread(z, 9)
    z[np.arange(wl.kmax)[None, :] >= K[:, None]] = 0.0
    beta = 0.41
    ctx, zd, Kd = context_with_population(wl, prec, z, K, beta, n1=n1)
    lo, ln, lp, g, _ = ctx.eval(zd, Kd, dev_tensor([beta], t.float64), grad=True)
    t.cuda.synchronize()
    ora = oracle.Oracle(wl, n1=n1)
    res = ora.logl_grad(z, K, beta)
    assert_eval_parity(ora, res, lo, ln, lp, g, K, TOL[prec], wl.D)
    if n1 > 0:
        return
    # the phase coordinates carry no prior gradient: with every sample tempered, at beta = 0
    # their gradient is exactly 0
    _, _, _, g0, _ = ctx.eval(zd, Kd, dev_tensor([0.0], t.float64), grad=True)
    g0 = g0.cpu().numpy()
    for i in range(wl.P):
        assert np.all(g0[i, : K[i], PHASE] == 0.0)


@pytest.mark.parametrize("prec,tol", [(capi.FP64, 1e-10), (capi.MIXED, 1e-4)])
def test_fisher_parity_with_periodic_phase(prec, tol):
    t = torch()
    wl = _wl()
    z, K = population(wl, 6, wl.P)
    z = _spread(z, 4)
    z[np.arange(wl.kmax)[None, :] >= K[:, None]] = 0.0
    beta = 0.7
    ctx, zd, Kd = context_with_population(wl, prec, z, K, beta)
    _, _, _, _, fis = ctx.eval(zd, Kd, dev_tensor([beta], t.float64), grad=True, fisher=True)
    res = oracle.Oracle(wl).logl_grad(z, K, beta, want_fisher=True)
    np.testing.assert_allclose(fis.cpu().numpy(), res["fisher"].sum(1), rtol=tol)


def test_init_population_with_periodic_phase_matches_oracle():
    wl = _wl(P=512)
    ctx = sampler.open_context(wl, capi.FP64)
    ctx.init_population()
    z, K, _, _ = ctx.get_population()
    zo, Ko = oracle.Oracle(wl).init_population(512)
    assert np.array_equal(K.cpu().numpy(), Ko)
    z = z.cpu().numpy()
    # logit coordinates to the last bits of log / log1p; periodic ones are u itself
    np.testing.assert_allclose(z, zo, rtol=1e-15, atol=1e-15)
    assert np.array_equal(z[..., PHASE], zo[..., PHASE])
    ph = np.concatenate([zo[i, : Ko[i], PHASE] for i in range(512)])
    assert np.all((ph > 0) & (ph < 1))


def test_rj_move_with_periodic_phase_matches_oracle_fp64():
    t = torch()
    wl = _wl(P=256)
    z, K = population(wl, 11, wl.P)
    z = _spread(z, 2)
    z[np.arange(wl.kmax)[None, :] >= K[:, None]] = 0.0
    beta = 0.3
    ora = oracle.Oracle(wl)
    ctx, _, _ = context_with_population(wl, capi.FP64, z, K, beta)
    r = ora.logl_grad(z, K, beta)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    zo, Ko = z.copy(), K.copy()
    out_o = ora.rj_move(2, 1, beta, zo, Ko, lo, ln)
    outd = t.zeros(wl.P, dtype=t.int32, device="cuda")
    ctx.rj_move(2, 1, outd)
    zg, Kg, _, lng = ctx.get_population()
    assert np.array_equal(outd.cpu().numpy(), out_o)
    assert np.any(out_o == 1) and np.any(out_o == 2)
    assert np.array_equal(Kg.cpu().numpy(), Ko)
    zg = zg.cpu().numpy()
    np.testing.assert_allclose(zg, zo, rtol=1e-14, atol=1e-14)
    assert np.array_equal(zg[..., PHASE], zo[..., PHASE])
    np.testing.assert_allclose(lng.cpu().numpy(), ln, rtol=1e-10)


@pytest.mark.parametrize("prec", [capi.FP64, capi.MIXED])
def test_nuts_with_periodic_phase(prec):
    """Near the injection, phases started on other periods: FP64 the oracle's trees and end
    points (phases reduced to one period on both sides); mixed the same trees for almost
    every particle."""
    t = torch()
    wl = synth.sinusoid_workload("t", 1024, 2, 4, 96, 47)
    wl.wrapmask = WRAP
    ora = oracle.Oracle(wl)
    beta = 0.35
    rng = np.random.default_rng(5)
    zt = synth.theta_to_z(wl, 0, wl.problems[0].truth)
    K = np.full(96, 2, np.int32)
    z = np.zeros((96, 4, 4))
    z[:, :2] = zt[None] + 0.002 * rng.standard_normal((96, 2, 4))
    z = _spread(z, 8)
    minv = ora.metric(z, K, beta)
    ctx, _, _ = context_with_population(wl, prec, z, K, beta)
    ctx.set_kernel_params([0.5], minv[None, :])
    acc = t.zeros(96, dtype=t.float64, device="cuda")
    nl = t.zeros(96, dtype=t.int32, device="cuda")
    fl = t.zeros(96, dtype=t.int32, device="cuda")
    ctx.nuts_move(3, 2, acc, nl, fl)
    zg, _, _, ln_g = ctx.get_population()
    zg = zg.cpu().numpy()
    r = ora.logl_grad(z, K, beta)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    zo = z.copy()
    _, nl_o, fl_o = ora.nuts_move(3, 2, beta, 0.5, minv, zo, K, lo, ln)
    assert np.all((zg[:, :2, PHASE] >= 0.0) & (zg[:, :2, PHASE] <= 1.0))
    assert len(np.unique(fl_o >> 8)) >= 3
    if prec == capi.MIXED:
        same = (nl.cpu().numpy() == nl_o) & (fl.cpu().numpy() == fl_o)
        assert np.mean(same) >= 0.9, np.mean(same)
        close = np.all(np.isclose(zg, zo, rtol=1e-4, atol=1e-5), axis=(1, 2))
        assert np.mean(close[same]) >= 0.9, np.mean(close[same])
        return
    assert np.array_equal(nl.cpu().numpy(), nl_o)
    assert np.array_equal(fl.cpu().numpy(), fl_o)
    np.testing.assert_allclose(zg, zo, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(ln_g.cpu().numpy(), ln, rtol=1e-10)


def test_smc_stage_with_periodic_phase_matches_oracle_fp64():
    wl = synth.sinusoid_workload("t", 1024, 2, 4, 128, 61)
    wl.wrapmask = WRAP
    wl.n_mut = 2
    ctx = sampler.open_context(wl, capi.FP64)
    ctx.init_population()
    b, lz, _ = ctx.run_stage(0, use_graph=False)
    z, K, _, _ = ctx.get_population()
    res = oracle.Oracle(wl).smc_run(128, max_stages=1)
    assert b[0] == pytest.approx(res["beta"][0], abs=1e-13)
    assert lz[0] == pytest.approx(res["logz"], rel=1e-11, abs=1e-11)
    np.testing.assert_array_equal(K.cpu().numpy(), res["K"])
    np.testing.assert_allclose(z.cpu().numpy(), res["z"], rtol=1e-9, atol=1e-9)


def test_phase_posterior_crosses_the_seam():
    """One source with phi0 next to 0 = 2 pi: on the circle its posterior is one mode
    straddling the seam (which the logit map would cut), so the K = 1 particles' phases lie
    on both sides of it and their circular mean is within three circular standard
    deviations of the injected phase (phi0 is correlated with f, so its marginal is wide)."""
    rng = np.random.default_rng(3)
    wl = synth.sinusoid_workload("t", 4096, 1, 2, 512, 71, noise=False)
    pr = wl.problems[0]
    th = pr.truth.copy()
    th[0, PHASE] = 0.004
    t = pr.t_origin + pr.dt * np.arange(pr.n)
    pr.d = synth._sin_phase(t, th[0, 1], th[0, 2], th[0, 3])
    pr.d = th[0, 0] * np.cos(pr.d) + pr.sigma * 0.3 * rng.standard_normal(pr.n)
    pr.truth = th
    wl.wrapmask = WRAP
    ctx = sampler.open_context(wl, capi.MIXED)
    out = sampler.run_smc(ctx, max_stages=300)
    assert out["beta"][-1][0] == 1.0
    z, K, _, _ = ctx.get_population()
    z, K = z.cpu().numpy(), K.cpu().numpy()
    sel = K == 1
    assert np.mean(sel) > 0.5
    phi = 2 * np.pi * (z[sel, 0, PHASE] - np.floor(z[sel, 0, PHASE]))
    assert np.mean(phi < np.pi) > 0.05 and np.mean(phi > np.pi) > 0.05   # both sides
    m = np.mean(np.exp(1j * phi))
    sd = np.sqrt(-2.0 * np.log(np.abs(m)))              # circular standard deviation
    assert abs(np.angle(m * np.exp(-1j * th[0, PHASE]))) <= 3 * sd, (np.angle(m), sd)


@pytest.mark.parametrize("prec", [capi.FP64, capi.MIXED])
def test_two_channel_eval_parity_with_periodic_phase(prec):
    """Channels A and E add their response phase to phi0; with the periodic map phi0 comes
    from the fraction of z first."""
    t = torch()
    wl = synth.ae_workload("t", 4096, 3, 5, 24, 41, noise=True)
    wl.wrapmask = WRAP
    z, K = population(wl, 5, 24)
    zt = synth.theta_to_z(wl, 0, wl.problems[0].truth)
    for i in range(2, 24, 2):
        k = min(K[i], 3)
        K[i] = k
        z[i, :k] = zt[:k] + 0.01 * np.random.default_rng(i).standard_normal((k, 4))
    z = _spread(z, 6)
    z[np.arange(wl.kmax)[None, :] >= K[:, None]] = 0.0
    ctx, zd, Kd = context_with_population(wl, prec, z, K, 0.37)
    lo, ln, lp, g, _ = ctx.eval(zd, Kd, dev_tensor([0.37], t.float64), grad=True)
    t.cuda.synchronize()
    ora = oracle.Oracle(wl)
    res = ora.logl_grad(z, K, 0.37)
    assert_eval_parity(ora, res, lo, ln, lp, g, K, TOL[prec], wl.D)


def test_rj_move_with_periodic_phase_mixed_agrees():
    t = torch()
    wl = _wl(P=512)
    z, K = population(wl, 12, wl.P)
    z = _spread(z, 3)
    z[np.arange(wl.kmax)[None, :] >= K[:, None]] = 0.0
    beta = 0.3
    ora = oracle.Oracle(wl)
    ctx, _, _ = context_with_population(wl, capi.MIXED, z, K, beta)
    r = ora.logl_grad(z, K, beta)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    zo, Ko = z.copy(), K.copy()
    out_o = ora.rj_move(2, 1, beta, zo, Ko, lo, ln)
    outd = t.zeros(wl.P, dtype=t.int32, device="cuda")
    ctx.rj_move(2, 1, outd)
    assert np.mean(outd.cpu().numpy() == out_o) > 0.99
    zg = ctx.get_population()[0].cpu().numpy()
    same = outd.cpu().numpy() == out_o
    assert np.array_equal(zg[same][..., PHASE], zo[same][..., PHASE])


def test_periodic_parameter_cannot_be_log_uniform():
    wl = _wl(P=8)
    ctx = sampler.open_context(wl, capi.MIXED)
    pr = wl.problems[0]
    with pytest.raises(capi.TsmcError):      # bit 3 both periodic and log-uniform
        ctx.set_problem(0, pr.d, pr.t_origin, pr.dt, pr.sigma, (1.0, 1.0, 1.0, 0.1),
                        (2.0, 2.0, 2.0, 2 * np.pi), wl.logmask | WRAP)
    ctx.set_problem(0, pr.d, pr.t_origin, pr.dt, pr.sigma, pr.lo, pr.hi, wl.logmask)
