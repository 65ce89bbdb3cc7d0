"""CUDA path vs the oracle, through the C ABI, on the same seeded inputs.

Sizes span several segments of samples per block and a ragged tail; K ranges
over 0..kmax.  FP64 path: relative 1e-12; mixed path: relative 1e-5 (gradients
relative to the sum of absolute terms, i.e. the condition of the sum).
"""
import math

import numpy as np
import pytest

import oracle
from paper_2609_17674_b300 import capi, sampler, synth
from gpu_helpers import (TOL, assert_eval_parity, context_with_population, data_scale_gscale,
                         dev_tensor, population, torch)

pytestmark = pytest.mark.gpu


def test_philox_matches_oracle():
    wl = synth.pulse_n1024_k3()
    ctx = sampler.open_context(wl, capi.FP64)
    rng = np.random.default_rng(3)
    ctr = rng.integers(0, 2**63, size=(64, 4), dtype=np.uint64)
    out = ctx.philox(ctr.ravel(), 12345, 678)
    for i in range(64):
        assert (out[4 * i: 4 * i + 4] == oracle.philox(ctr[i], [12345, 678])).all()


CASES = [
    # model, N, kmax, n1, P
    ("pulse", 3000, 6, 0, 48),
    ("pulse", 5000, 5, 1700, 40),
    ("pulse", 100, 4, 0, 16),
    ("sinusoid", 9000, 5, 0, 24),
    ("sinusoid", 6000, 4, 2500, 16),
    # ragged tails at every alignment: odd N and n1 inside a thread's samples, one sample
    # past a full segment, N below one warp range, a single sample
    ("pulse", 1001, 7, 333, 24),
    ("pulse", 4097, 40, 0, 16),
    ("pulse", 37, 3, 0, 8),
    ("pulse", 1, 2, 0, 4),
    ("sinusoid", 777, 3, 101, 8),
]


def _wl(model, n, kmax, P, seed=41):
    if model == "pulse":
        return synth.pulse_workload("t", n, 3, kmax, P, seed)
    return synth.sinusoid_workload("t", n, 3, kmax, P, seed)


@pytest.mark.parametrize("prec", [capi.FP64, capi.MIXED])
@pytest.mark.parametrize("model,n,kmax,n1,P", CASES)
def test_eval_parity(prec, model, n, kmax, n1, P):
    t = torch()
    wl = _wl(model, n, kmax, P)
    z, K = population(wl, 5, P)
    if model == "sinusoid":
        # half the particles near the injection (small residuals: the hard case)
        zt = synth.theta_to_z(wl, 0, wl.problems[0].truth)
        for i in range(2, P, 2):
            k = min(K[i], zt.shape[0])
            K[i] = k
            z[i, :k] = zt[:k] + 0.01 * np.random.default_rng(i).standard_normal((k, 4))
    beta = 0.37
    ctx, zd, Kd = context_with_population(wl, prec, z, K, beta, n_use=n, n1=n1)
    bt = dev_tensor([beta], t.float64)
    lo, ln, lp, g, _ = ctx.eval(zd, Kd, bt, grad=True)
    t.cuda.synchronize()
    ora = oracle.Oracle(wl, n=n, n1=n1)
    res = ora.logl_grad(z, K, beta)
    assert_eval_parity(ora, res, lo, ln, lp, g, K, TOL[prec], wl.D)


@pytest.mark.parametrize("prec", [capi.FP64, capi.MIXED])
@pytest.mark.parametrize("model", ["pulse", "sinusoid"])
def test_eval_parity_at_the_component_limit(prec, model):
    """K_max = 64, the library's limit (components 32..63 live in the second ballot word and
    the second slot of every lane), with K from 0 to 64 and a ragged tail."""
    t = torch()
    wl = _wl(model, 5000, 64, 12, seed=43)
    z, K = population(wl, 9, 12)
    K[2:] = [64, 63, 33, 32, 31, 1, 48, 64, 17, 40]
    ctx, zd, Kd = context_with_population(wl, prec, z, K, 0.6)
    lo, ln, lp, g, _ = ctx.eval(zd, Kd, dev_tensor([0.6], t.float64), grad=True)
    t.cuda.synchronize()
    res = oracle.Oracle(wl).logl_grad(z, K, 0.6)
    assert_eval_parity(None, res, lo, ln, lp, g, K, TOL[prec], wl.D)


@pytest.mark.parametrize("prec", [capi.FP64, capi.MIXED])
def test_eval_parity_at_the_sample_limit(prec):
    """N = 2^24 samples, the largest capacity the library accepts (sample indices stay exact
    in FP32 and 32-bit arithmetic), on a few particles against the oracle."""
    t = torch()
    n = 1 << 24
    wl = synth.pulse_workload("t", n, 3, 4, 4, 44)
    z, K = population(wl, 10, 4)
    K[2:] = [3, 4]
    ctx, zd, Kd = context_with_population(wl, prec, z, K, 0.7)
    lo, ln, lp, g, _ = ctx.eval(zd, Kd, dev_tensor([0.7], t.float64), grad=True)
    t.cuda.synchronize()
    res = oracle.Oracle(wl).logl_grad(z, K, 0.7)
    assert_eval_parity(None, res, lo, ln, lp, g, K, TOL[prec], 3)
    with pytest.raises(capi.TsmcError):   # one sample more than the limit is refused
        capi.Context(sampler.make_config(wl, prec), [n + 1])


@pytest.mark.parametrize("prec", [capi.FP64, capi.MIXED])
def test_linamp_eval_and_fisher(prec):
    t = torch()
    wl = synth.linamp_workload(n=2100, k=3, P=8)
    rng = np.random.default_rng(2)
    z = rng.normal(1.0, 1.0, (8, 3, 1))
    K = np.full(8, 3, np.int32)
    ctx, zd, Kd = context_with_population(wl, prec, z, K, 0.8)
    bt = dev_tensor([0.8], t.float64)
    lo, ln, lp, g, fis = ctx.eval(zd, Kd, bt, grad=True, fisher=True)
    res = oracle.Oracle(wl).logl_grad(z, K, 0.8, want_fisher=True)
    assert_eval_parity(None, res, lo, ln, lp, g, K, TOL[prec], 1)
    np.testing.assert_allclose(fis.cpu().numpy()[:, 0], res["fisher"].sum(1)[:, 0],
                               rtol=1e-10 if prec == capi.FP64 else 1e-4)


@pytest.mark.parametrize("prec", [capi.FP64, capi.MIXED])
def test_linamp_nuts_parity(prec):
    """Linear-amplitude model (fixed centres and widths, Gaussian amplitude prior): one NUTS
    transition against the oracle; FP64: the same trees (leaf counts, depths) and end
    points; mixed: the same trees for almost every particle."""
    t = torch()
    wl = synth.linamp_workload(n=512, k=3, P=64, seed=33)
    ora = oracle.Oracle(wl)
    rng = np.random.default_rng(4)
    z = rng.normal(1.0, 1.0, (64, 3, 1))
    K = np.full(64, 3, np.int32)
    beta, eps = 0.5, 0.02
    minv = ora.metric(z, K, beta)
    ctx, _, _ = context_with_population(wl, prec, z, K, beta)
    ctx.set_kernel_params([eps], minv[None, :])
    acc = t.zeros(64, dtype=t.float64, device="cuda")
    nl = t.zeros(64, dtype=t.int32, device="cuda")
    fl = t.zeros(64, dtype=t.int32, device="cuda")
    ctx.nuts_move(2, 0, acc, nl, fl)
    zg = ctx.get_population()[0].cpu().numpy()
    r = ora.logl_grad(z, K, beta)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    zo = z.copy()
    acc_o, nl_o, fl_o = ora.nuts_move(2, 0, beta, eps, minv, zo, K, lo, ln)
    assert len(np.unique(fl_o >> 8)) >= 4
    if prec == capi.FP64:
        assert np.array_equal(nl.cpu().numpy(), nl_o)
        assert np.array_equal(fl.cpu().numpy(), fl_o)
        np.testing.assert_allclose(zg, zo, rtol=1e-9, atol=1e-9)
    else:
        same = (nl.cpu().numpy() == nl_o) & (fl.cpu().numpy() == fl_o)
        assert np.mean(same) >= 0.9, np.mean(same)
        close = np.all(np.isclose(zg, zo, rtol=1e-4, atol=1e-5), axis=(1, 2))
        assert np.mean(close[same]) >= 0.9, np.mean(close[same])


@pytest.mark.parametrize("prec", [capi.FP64, capi.MIXED])
@pytest.mark.parametrize("model", ["pulse", "sinusoid"])
def test_fisher_parity(prec, model):
    t = torch()
    wl = _wl(model, 4000, 4, 12)
    z, K = population(wl, 9, 12)
    ctx, zd, Kd = context_with_population(wl, prec, z, K, 0.5)
    bt = dev_tensor([0.5], t.float64)
    _, _, _, _, fis = ctx.eval(zd, Kd, bt, grad=True, fisher=True)
    res = oracle.Oracle(wl).logl_grad(z, K, 0.5, want_fisher=True)
    np.testing.assert_allclose(fis.cpu().numpy(), res["fisher"].sum(1),
                               rtol=1e-10 if prec == capi.FP64 else 1e-4)


@pytest.mark.parametrize("kmin", [0, 1])
def test_init_population_matches_oracle(kmin):
    wl = synth.pulse_n1024_k3()
    wl.P = 300
    wl.kmin = kmin
    ctx = sampler.open_context(wl, capi.FP64)
    ctx.init_population()
    z, K, lo, ln = ctx.get_population()
    zo, Ko = oracle.Oracle(wl).init_population(300)
    assert np.array_equal(K.cpu().numpy(), Ko)
    np.testing.assert_allclose(z.cpu().numpy(), zo, rtol=1e-15, atol=1e-15)
    res = oracle.Oracle(wl).logl_grad(zo, Ko, 0.0)
    np.testing.assert_allclose(ln.cpu().numpy(), res["ll_new"], rtol=1e-12)


@pytest.mark.parametrize("n1,kmin", [(0, 0), (700, 0), (0, 2)])
def test_rj_move_parity_fp64(n1, kmin):
    t = torch()
    wl = synth.pulse_workload("t", 1500, 3, 6, 200, 77)
    wl.kmin = kmin
    z, K = population(wl, 13, 200, include_edges=kmin == 0)
    if kmin:
        K[:40] = kmin          # deaths proposed at the floor are rejected
        z[:40, kmin:] = 0.0
    ora = oracle.Oracle(wl, n=1500, n1=n1)
    beta = 0.45
    ctx, zd, Kd = context_with_population(wl, capi.FP64, z, K, beta, n_use=1500, n1=n1)
    r = ora.logl_grad(z, K, beta)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    zo, Ko = z.copy(), K.copy()
    out_o = ora.rj_move(4, 2, beta, zo, Ko, lo, ln)
    # the GPU move reads beta from the context (set_population set it)
    outd = t.zeros(200, dtype=t.int32, device="cuda")
    ctx.rj_move(4, 2, outd)
    zg, Kg, log_, lng = ctx.get_population()
    assert np.array_equal(outd.cpu().numpy(), out_o)
    assert np.array_equal(Kg.cpu().numpy(), Ko)
    np.testing.assert_allclose(zg.cpu().numpy(), zo, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(lng.cpu().numpy(), ln, rtol=1e-10)
    np.testing.assert_allclose(log_.cpu().numpy(), lo, rtol=1e-10, atol=1e-9)
    assert set(np.unique(out_o)) >= {1, 2, -1} or len(np.unique(out_o)) >= 3
    assert Kg.cpu().numpy().min() >= kmin
    if kmin:
        assert np.any(out_o == -2)


def test_rj_move_mixed_agrees():
    t = torch()
    wl = synth.pulse_k20(P=512, n=16384)
    z, K = population(wl, 21, 512)
    ora = oracle.Oracle(wl)
    ctx, zd, Kd = context_with_population(wl, capi.MIXED, z, K, 0.01)
    r = ora.logl_grad(z, K, 0.01, want_scale=False)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    zo, Ko = z.copy(), K.copy()
    out_o = ora.rj_move(1, 0, 0.01, zo, Ko, lo, ln)
    outd = t.zeros(512, dtype=t.int32, device="cuda")
    ctx.rj_move(1, 0, outd)
    zg, Kg, _, lng = ctx.get_population()
    agree = np.mean(outd.cpu().numpy() == out_o)
    assert agree > 0.99
    same = outd.cpu().numpy() == out_o
    np.testing.assert_allclose(lng.cpu().numpy()[same], ln[same], rtol=1e-5)


def test_nuts_parity_fp64():
    t = torch()
    wl = synth.pulse_workload("t", 512, 3, 4, 64, 88)
    ora = oracle.Oracle(wl)
    rng = np.random.default_rng(0)
    K = rng.integers(1, 5, 64).astype(np.int32)
    zt = synth.theta_to_z(wl, 0, wl.problems[0].truth)
    z = np.zeros((64, 4, 3))
    for i in range(64):
        k = min(K[i], 3)
        K[i] = k
        z[i, :k] = zt[:k] + 0.05 * rng.standard_normal((k, 3))
    beta = 0.6
    minv = ora.metric(z, K, beta)
    eps = 0.2
    ctx, zd, Kd = context_with_population(wl, capi.FP64, z, K, beta)
    ctx.set_kernel_params([eps], minv[None, :])
    acc = t.zeros(64, dtype=t.float64, device="cuda")
    nl = t.zeros(64, dtype=t.int32, device="cuda")
    fl = t.zeros(64, dtype=t.int32, device="cuda")
    ctx.nuts_move(3, 1, acc, nl, fl)
    zg, Kg, lo_g, ln_g = ctx.get_population()
    r = ora.logl_grad(z, K, beta)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    zo = z.copy()
    acc_o, nl_o, fl_o = ora.nuts_move(3, 1, beta, eps, minv, zo, K, lo, ln)
    assert np.array_equal(nl.cpu().numpy(), nl_o)
    assert np.array_equal(fl.cpu().numpy(), fl_o)
    np.testing.assert_allclose(zg.cpu().numpy(), zo, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(acc.cpu().numpy(), acc_o, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(ln_g.cpu().numpy(), ln, rtol=1e-10)
    assert np.mean(nl_o) > 3  # the trees were non-trivial


def test_sinusoid_rj_parity_fp64():
    """Single-channel sinusoids (FP64 path): a birth/death move with the oracle's outcomes,
    K, z and carried likelihoods."""
    t = torch()
    wl = synth.sinusoid_workload("t", 1024, 2, 4, 96, 47)
    ora = oracle.Oracle(wl)
    z, K = population(wl, 14, 96)
    beta = 0.35
    ctx, _, _ = context_with_population(wl, capi.FP64, z, K, beta)
    r = ora.logl_grad(z, K, beta)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    zo, Ko = z.copy(), K.copy()
    out_o = ora.rj_move(6, 1, beta, zo, Ko, lo, ln)
    outd = t.zeros(96, dtype=t.int32, device="cuda")
    ctx.rj_move(6, 1, outd)
    zg, Kg, _, lng = ctx.get_population()
    assert np.array_equal(outd.cpu().numpy(), out_o)
    assert np.array_equal(Kg.cpu().numpy(), Ko)
    np.testing.assert_allclose(zg.cpu().numpy(), zo, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(lng.cpu().numpy(), ln, rtol=1e-10)
    assert len(np.unique(out_o)) >= 3


@pytest.mark.parametrize("prec,eps", [(capi.FP64, 0.5), (capi.FP64, 1.0), (capi.MIXED, 0.5)])
def test_sinusoid_nuts_parity(prec, eps):
    """Single-channel sinusoids near the injection: one NUTS transition against the oracle.
    FP64: the same leaf counts, depth and divergence flags, end points and acceptance
    statistics (eps 0.5: U-turns at depths 2-6; eps 1.0: divergences as well); mixed: the
    same trees for almost every particle and the same end points where they agree."""
    t = torch()
    wl = synth.sinusoid_workload("t", 1024, 2, 4, 96, 47)
    ora = oracle.Oracle(wl)
    beta = 0.35
    rng = np.random.default_rng(5)
    zt = synth.theta_to_z(wl, 0, wl.problems[0].truth)
    K = np.full(96, 2, np.int32)
    z = np.zeros((96, 4, 4))
    z[:, :2] = zt[None] + 0.002 * rng.standard_normal((96, 2, 4))
    minv = ora.metric(z, K, beta)
    ctx, _, _ = context_with_population(wl, prec, z, K, beta)
    ctx.set_kernel_params([eps], minv[None, :])
    acc = t.zeros(96, dtype=t.float64, device="cuda")
    nl = t.zeros(96, dtype=t.int32, device="cuda")
    fl = t.zeros(96, dtype=t.int32, device="cuda")
    ctx.nuts_move(3, 2, acc, nl, fl)
    zg, _, _, ln_g = ctx.get_population()
    r = ora.logl_grad(z, K, beta)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    zo = z.copy()
    acc_o, nl_o, fl_o = ora.nuts_move(3, 2, beta, eps, minv, zo, K, lo, ln)
    assert len(np.unique(fl_o >> 8)) >= 3
    if eps == 1.0:
        assert np.any(fl_o & 1)
    if prec == capi.MIXED:
        same = (nl.cpu().numpy() == nl_o) & (fl.cpu().numpy() == fl_o)
        assert np.mean(same) >= 0.9, np.mean(same)
        close = np.all(np.isclose(zg.cpu().numpy(), zo, rtol=1e-4, atol=1e-5), axis=(1, 2))
        assert np.mean(close[same]) >= 0.9, np.mean(close[same])
        return
    assert np.array_equal(nl.cpu().numpy(), nl_o)
    assert np.array_equal(fl.cpu().numpy(), fl_o)
    np.testing.assert_allclose(zg.cpu().numpy(), zo, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(acc.cpu().numpy(), acc_o, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(ln_g.cpu().numpy(), ln, rtol=1e-10)


def test_nuts_mixed_moves_and_stays_finite():
    t = torch()
    wl = synth.pulse_k20(P=256, n=16384)
    z, K = population(wl, 2, 256)
    ctx, zd, Kd = context_with_population(wl, capi.MIXED, z, K, 0.001)
    ctx.update_metric()
    acc = t.zeros(256, dtype=t.float64, device="cuda")
    nl = t.zeros(256, dtype=t.int32, device="cuda")
    ctx.nuts_move(0, 0, acc, nl, None)
    zg, Kg, _, ln = ctx.get_population()
    assert np.all(np.isfinite(zg.cpu().numpy()))
    assert np.all(np.isfinite(ln.cpu().numpy()))
    moved = nl.cpu().numpy() > 0
    assert np.all(moved == (K > 0))
    # carried likelihoods belong to the returned points (mixed path, same kernel)
    _, ln2, _, _, _ = ctx.eval(zg, Kg, dev_tensor([0.001], t.float64))
    np.testing.assert_allclose(ln.cpu().numpy(), ln2.cpu().numpy(), rtol=1e-12)


def test_nuts_mixed_agrees_with_oracle():
    """Mixed path (FP32 templates and tree control, same Philox streams) against the FP64
    oracle: the same trees for almost every particle, and the same end points to FP32
    accuracy where the trees agree."""
    t = torch()
    wl = synth.pulse_workload("t", 512, 3, 4, 64, 88)
    ora = oracle.Oracle(wl)
    rng = np.random.default_rng(0)
    K = rng.integers(1, 5, 64).astype(np.int32)
    zt = synth.theta_to_z(wl, 0, wl.problems[0].truth)
    z = np.zeros((64, 4, 3))
    for i in range(64):
        k = min(K[i], 3)
        K[i] = k
        z[i, :k] = zt[:k] + 0.05 * rng.standard_normal((k, 3))
    beta = 0.6
    minv = ora.metric(z, K, beta)
    eps = 0.2
    ctx, zd, Kd = context_with_population(wl, capi.MIXED, z, K, beta)
    ctx.set_kernel_params([eps], minv[None, :])
    acc = t.zeros(64, dtype=t.float64, device="cuda")
    nl = t.zeros(64, dtype=t.int32, device="cuda")
    fl = t.zeros(64, dtype=t.int32, device="cuda")
    ctx.nuts_move(3, 1, acc, nl, fl)
    zg = ctx.get_population()[0].cpu().numpy()
    r = ora.logl_grad(z, K, beta)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    zo = z.copy()
    acc_o, nl_o, fl_o = ora.nuts_move(3, 1, beta, eps, minv, zo, K, lo, ln)
    same = (nl.cpu().numpy() == nl_o) & (fl.cpu().numpy() == fl_o)
    assert np.mean(same) >= 0.9, np.mean(same)
    close = np.all(np.isclose(zg, zo, rtol=1e-4, atol=1e-5), axis=(1, 2))
    assert np.mean(close[same]) >= 0.9, np.mean(close[same])
    np.testing.assert_allclose(acc.cpu().numpy()[same], acc_o[same], rtol=1e-3, atol=1e-6)


@pytest.mark.parametrize("model", ["pulse", "sinusoid"])
@pytest.mark.parametrize("prec", [capi.FP64, capi.MIXED])
def test_extreme_coordinates_stay_finite(prec, model):
    """z = +-1e308 puts theta on a prior bound with log prior -1e308 (FP64; the oracle's
    value) or -inf (mixed: |z| is beyond the FP32 range).  The likelihood and gradient stay
    those of the bound, a mixed-path NUTS transition from such a point diverges at its first
    leaf and leaves it in place, the extreme coordinates are never moved, and no NaN reaches
    the population through a whole SMC stage."""
    t = torch()
    if model == "pulse":
        wl = synth.pulse_workload("t", 1024, 3, 10, 64, 91)
    else:
        wl = synth.sinusoid_workload("t", 4096, 3, 6, 64, 93)
    z, K = population(wl, 7, 64, include_edges=False)
    K[:4] = np.maximum(K[:4], 1)
    ext = [(0, 0, 1, 1e308), (1, 0, 2, -1e308), (2, 0, 0, 1e308), (3, 0, wl.D - 1, -1e308)]
    for i, k, d, v in ext:
        z[i, k, d] = v
    beta = 0.3
    ctx, zd, Kd = context_with_population(wl, prec, z, K, beta)
    bt = dev_tensor([beta], t.float64)
    lo, ln, lp, g, _ = ctx.eval(zd, Kd, bt, grad=True)
    lo, ln, lp, g = (x.cpu().numpy() for x in (lo, ln, lp, g))
    res = oracle.Oracle(wl).logl_grad(z, K, beta)
    tol = TOL[prec]
    np.testing.assert_allclose(ln, res["ll_new"], rtol=tol)
    assert np.all(np.isfinite(g))
    for i, k, d, v in ext:
        assert g[i, k, d] == pytest.approx(-np.sign(v), rel=1e-6)
    if prec == capi.FP64:
        np.testing.assert_allclose(lp, res["logp"], rtol=tol)
    else:
        assert np.all(lp[:4] == -np.inf)
        np.testing.assert_allclose(lp[4:], res["logp"][4:], rtol=tol)
    eps = [0.05]
    ctx.set_kernel_params(eps, np.ones((1, wl.D)))
    acc = t.zeros(64, dtype=t.float64, device="cuda")
    nl = t.zeros(64, dtype=t.int32, device="cuda")
    fl = t.zeros(64, dtype=t.int32, device="cuda")
    ctx.nuts_move(2, 0, acc, nl, fl)
    zg, Kg, lo_g, ln_g = (x.cpu().numpy() for x in ctx.get_population())
    assert not np.any(np.isnan(zg)) and np.all(np.isfinite(ln_g)) and np.all(np.isfinite(lo_g))
    assert np.all(np.isfinite(acc.cpu().numpy()))
    for i, k, d, v in ext:
        assert zg[i, k, d] == v
    if prec == capi.MIXED:
        assert np.all(fl.cpu().numpy()[:4] & 1)
        np.testing.assert_array_equal(zg[:4], z[:4])
        assert np.all(acc.cpu().numpy()[:4] == 0.0)
    assert np.mean(nl.cpu().numpy()[4:] > 0) > 0.5     # the other particles moved
    ctx.rj_move(2, 1)
    ctx.update_metric()
    _, minv = ctx.get_kernel_params()
    assert np.all(np.isfinite(minv)) and np.all(minv > 0)
    ctx.run_stage(3, use_graph=False)
    zg, Kg, lo_g, ln_g = (x.cpu().numpy() for x in ctx.get_population())
    assert not np.any(np.isnan(zg))
    assert np.all(np.isfinite(ln_g)) and np.all(np.isfinite(lo_g))
    b, lz, ess = ctx.temper_state()
    assert np.all(np.isfinite(b)) and np.all(np.isfinite(lz)) and np.all(np.isfinite(ess))


@pytest.mark.parametrize("prec", [capi.FP64, capi.MIXED])
def test_nan_particle_has_zero_density(prec):
    """A particle with a NaN coordinate has a NaN likelihood (zero density): its NUTS
    transition diverges at the first leaf, it does not enter the population metric (which
    equals the metric with that particle's K set to 0), it gets zero weight at the next
    reweighting, and after one SMC stage no NaN is left in the population."""
    t = torch()
    wl = synth.pulse_workload("t", 1024, 3, 10, 64, 92)
    z, K = population(wl, 8, 64, include_edges=False)
    K[5] = max(K[5], 1)
    z[5, 0, 1] = np.nan
    beta = 0.2
    ctx, zd, Kd = context_with_population(wl, prec, z, K, beta)
    lo, ln, lp, g, _ = ctx.eval(zd, Kd, dev_tensor([beta], t.float64), grad=True)
    ln, lp = ln.cpu().numpy(), lp.cpu().numpy()
    assert np.isnan(ln[5]) and np.isnan(lp[5])
    others = np.arange(64) != 5
    res = oracle.Oracle(wl).logl_grad(z[others], K[others], beta)
    np.testing.assert_allclose(ln[others], res["ll_new"], rtol=TOL[prec])
    ctx.update_metric()
    _, minv = ctx.get_kernel_params()
    K0 = K.copy()
    K0[5] = 0
    ctx0, _, _ = context_with_population(wl, prec, z, K0, beta)
    ctx0.update_metric()
    _, minv0 = ctx0.get_kernel_params()
    assert np.all(np.isfinite(minv))
    np.testing.assert_array_equal(minv, minv0)
    acc = t.zeros(64, dtype=t.float64, device="cuda")
    nl = t.zeros(64, dtype=t.int32, device="cuda")
    fl = t.zeros(64, dtype=t.int32, device="cuda")
    ctx.nuts_move(2, 0, acc, nl, fl)
    assert fl.cpu().numpy()[5] & 1 and acc.cpu().numpy()[5] == 0.0
    zg = ctx.get_population()[0].cpu().numpy()
    assert np.isnan(zg[5, 0, 1]) and not np.any(np.isnan(np.delete(zg, 5, axis=0)))
    b, lz, ess = ctx.run_stage(3, use_graph=False)
    zg, Kg, lo_g, ln_g = (x.cpu().numpy() for x in ctx.get_population())
    anc = ctx.get_ancestors().cpu().numpy()
    assert 5 not in anc
    assert not np.any(np.isnan(zg)) and np.all(np.isfinite(ln_g)) and np.all(np.isfinite(lo_g))
    assert np.all(np.isfinite(b)) and np.all(np.isfinite(lz)) and np.all(np.isfinite(ess))


def test_temper_and_resample_parity():
    wl = synth.pulse_n1024_k3()
    wl.P = 512
    ctx = sampler.open_context(wl, capi.FP64)
    ctx.init_population()
    _, _, _, ln = ctx.get_population()
    ell = ln.cpu().numpy()
    b, lz, e = ctx.temper_reweight_resample(5)
    bo, inco, esso, logw = oracle.temper(ell, wl.alpha, 0.0)
    assert b[0] == pytest.approx(bo, abs=1e-13)
    assert lz[0] == pytest.approx(inco, rel=1e-12, abs=1e-12)
    assert e[0] == pytest.approx(esso, rel=1e-9)
    anc = ctx.get_ancestors().cpu().numpy()
    anc_o = oracle.Oracle(wl).resample(5, logw)
    assert np.array_equal(anc, anc_o)       # exact integer prefix sums: index work is exact
    assert np.all(np.diff(anc) >= 0)


@pytest.mark.parametrize("P", [1, 7, 1000, 3000])
def test_resample_ancestors_exact(P):
    """Systematic ancestors on quantised weights are the same bit for bit on both sides for
    ragged particle counts (one thread chunk, several warps, several chunks per thread)."""
    wl = synth.pulse_workload("t", 700, 3, 6, P, 17)
    for stage in (0, 1):
        ctx = sampler.open_context(wl, capi.FP64)
        ctx.init_population()
        ell = ctx.get_population()[3].cpu().numpy()
        ctx.temper_reweight_resample(stage)
        _, _, _, logw = oracle.temper(ell, wl.alpha, 0.0)
        anc = ctx.get_ancestors().cpu().numpy()
        assert np.array_equal(anc, oracle.Oracle(wl).resample(stage, logw)), stage
        ctx.close()


def test_metric_parity():
    wl = synth.pulse_workload("t", 2048, 3, 5, 64, 5)
    z, K = population(wl, 8, 64)
    ctx, zd, Kd = context_with_population(wl, capi.FP64, z, K, 0.3)
    ctx.update_metric()
    _, m = ctx.get_kernel_params()
    mo = oracle.Oracle(wl).metric(z, K, 0.3)
    np.testing.assert_allclose(m[0], mo, rtol=1e-10)


def test_stage_graph_matches_eager():
    res = []
    for graph in (False, True):
        wl = synth.pulse_n1024_k3()
        wl.P = 256
        ctx = sampler.open_context(wl, capi.FP64)
        ctx.init_population()
        out = [ctx.run_stage(s, use_graph=graph) for s in range(3)]
        z, K, _, ln = ctx.get_population()
        res.append((out, z.cpu().numpy(), K.cpu().numpy()))
    (o1, z1, k1), (o2, z2, k2) = res
    assert np.array_equal(k1, k2)
    np.testing.assert_array_equal(z1, z2)
    for a, b in zip(o1, o2):
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("model,schedule", [("pulse", 0), ("pulse", 1), ("sinusoid", 0)])
def test_fused_mutation_rounds_match_per_round_launches(model, schedule):
    """The mixed path's persistent launch of a stage's rounds (each block pulls particles and
    runs all their rounds) gives bit for bit the results of one launch per move and round:
    the same particles, K, likelihoods and step size after three stages, eager and graph."""
    res = []
    for fused, graph in ((0, False), (1, False), (1, True)):
        wl = (synth.pulse_workload("t", 3000, 3, 8, 200, 61) if model == "pulse"
              else synth.sinusoid_workload("t", 4000, 3, 6, 150, 62))
        if schedule == 1:
            wl.schedule, wl.p_nuts, wl.p_birth, wl.p_death = capi.SCHED_MIXTURE, 0.6, 0.2, 0.2
        wl.n_mut = 3
        ctx = sampler.open_context(wl, capi.MIXED, fused_rounds=fused)
        ctx.init_population()
        out = [ctx.run_stage(s, use_graph=graph) for s in range(3)]
        z, K, lo, ln = (x.cpu().numpy() for x in ctx.get_population())
        eps, minv = ctx.get_kernel_params()
        res.append((out, z, K, lo, ln, eps, minv))
        ctx.close()
    for other in res[1:]:
        for a, b in zip(res[0][1:], other[1:]):
            np.testing.assert_array_equal(a, b)
        for sa, sb in zip(res[0][0], other[0]):
            for x, y in zip(sa, sb):
                np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("seed", [1001, 7, 8])
def test_smc_stage_matches_oracle_fp64(seed):
    """One full stage (temper, resample, metric, RJ + NUTS rounds) on both sides: the same
    ancestors, then every particle's K exactly and its coordinates to 1e-9."""
    wl = synth.pulse_n1024_k3()
    wl.P = 128
    wl.n_mut = 2
    wl.seed = seed
    ctx = sampler.open_context(wl, capi.FP64)
    ctx.init_population()
    ell = ctx.get_population()[3].cpu().numpy()
    b, lz, _ = ctx.run_stage(0, use_graph=False)
    z, K, _, ln = ctx.get_population()
    ora = oracle.Oracle(wl)
    _, _, _, logw = oracle.temper(ell, wl.alpha, 0.0)
    assert np.array_equal(ctx.get_ancestors().cpu().numpy(), ora.resample(0, logw))
    res = ora.smc_run(128, max_stages=1)
    assert b[0] == pytest.approx(res["beta"][0], abs=1e-13)
    assert lz[0] == pytest.approx(res["logz"], rel=1e-11, abs=1e-11)
    np.testing.assert_array_equal(K.cpu().numpy(), res["K"])
    np.testing.assert_allclose(z.cpu().numpy(), res["z"], rtol=1e-9, atol=1e-9)


@pytest.mark.parametrize("prec", [capi.FP64, capi.MIXED])
def test_full_size_pulse_sampled(prec):
    """N=16384, K_max=40, P=8192 in the benchmark launch configuration; logL and gradient
    against the oracle on 64 particles (K = 0, K = K_max and 62 drawn at random)."""
    t = torch()
    wl = synth.pulse_k20()
    z, K = population(wl, 1, wl.P)
    ctx, zd, Kd = context_with_population(wl, prec, z, K, 0.25)
    bt = dev_tensor([0.25], t.float64)
    lo, ln, lp, g, _ = ctx.eval(zd, Kd, bt, grad=True)
    t.cuda.synchronize()
    idx = np.r_[0, 1, np.random.default_rng(0).choice(np.arange(2, wl.P), 62, replace=False)]
    res = oracle.Oracle(wl).logl_grad(z[idx], K[idx], 0.25)
    assert_eval_parity(None, res, lo[idx], ln[idx], lp[idx], g[idx], K[idx], TOL[prec], 3)


def test_mixed_sinusoid_noise_free_absolute_bound():
    """Single-channel band on noise-free data (Sec. 5.2's example has no noise): particles
    at the injection (tiny residual) and from the prior, |dlogL| <= 1e-5 (1/2 D + |logL|)
    with D = sum d^2 / sigma^2 (FP32 templates err by ~eps32 of the signal), and the gradient
    within 1e-5 of its sum of absolute terms at the residual plus that at the data scale."""
    t = torch()
    wl = synth.sinusoid_workload("t", 9000, 3, 5, 16, 52, noise=False)
    clean = wl.problems[0].d
    z, K = population(wl, 3, 16)
    zt = synth.theta_to_z(wl, 0, wl.problems[0].truth)
    for i in range(2, 16, 2):
        K[i] = 3
        z[i] = 0.0
        z[i, :3] = zt + 1e-6 * np.random.default_rng(i).standard_normal((3, 4))
    ctx, zd, Kd = context_with_population(wl, capi.MIXED, z, K, 1.0)
    lo, ln, lp, g, _ = ctx.eval(zd, Kd, dev_tensor([1.0], t.float64), grad=True)
    t.cuda.synchronize()
    res = oracle.Oracle(wl).logl_grad(z, K, 1.0)
    half_D = 0.5 * float(np.sum(clean ** 2)) / wl.problems[0].sigma ** 2
    err = np.abs(ln.cpu().numpy() - res["ll_new"])
    assert np.all(err <= 1e-5 * (half_D + np.abs(res["ll_new"]))), (err.max(), half_D)
    assert np.max(np.abs(res["ll_new"][2::2])) < 0.1 * half_D
    gerr = np.abs(g.cpu().numpy() - res["grad"])
    gs = res["gscale"] + data_scale_gscale(wl, z, K, 1.0)
    assert np.all(gerr <= 1e-5 * gs + 1e-300), float(np.max(gerr / (gs + 1e-300)))


@pytest.mark.parametrize("prec", [capi.MIXED])
def test_full_size_sinusoid_sampled(prec):
    """N=2^18 Galactic-binary band, K_max=30, P=4096; oracle on a sample of particles."""
    t = torch()
    wl = synth.gb_band_k10()
    z, K = population(wl, 1, wl.P)
    zt = synth.theta_to_z(wl, 0, wl.problems[0].truth)
    for i in range(2, 40, 2):
        K[i] = 10
        z[i, :10] = zt + 1e-4 * np.random.default_rng(i).standard_normal((10, 4))
        z[i, 10:] = 0.0
    ctx, zd, Kd = context_with_population(wl, prec, z, K, 0.9)
    bt = dev_tensor([0.9], t.float64)
    lo, ln, lp, g, _ = ctx.eval(zd, Kd, bt, grad=True)
    t.cuda.synchronize()
    idx = np.array([0, 1, 2, 3, 4, 8, 9])
    res = oracle.Oracle(wl).logl_grad(z[idx], K[idx], 0.9)
    assert_eval_parity(None, res, lo[idx], ln[idx], lp[idx], g[idx], K[idx], TOL[prec], 4)


def test_full_size_assimilation_sampled():
    """N=2^19 samples, P=16384, K_max=40: the largest configuration, with the second half
    of the data new (tempered) and the first half assimilated; oracle on a sample."""
    t = torch()
    wl = synth.assimilation_pulse_k14()
    n = wl.problems[0].n
    z, K = population(wl, 4, wl.P)
    ctx, zd, Kd = context_with_population(wl, capi.MIXED, z, K, 0.3, n_use=n, n1=n // 2)
    bt = dev_tensor([0.3], t.float64)
    lo, ln, lp, g, _ = ctx.eval(zd, Kd, bt, grad=True)
    t.cuda.synchronize()
    idx = np.r_[0, 1, np.random.default_rng(3).choice(wl.P, 6, replace=False)]
    res = oracle.Oracle(wl, n=n, n1=n // 2).logl_grad(z[idx], K[idx], 0.3)
    assert_eval_parity(None, res, lo[idx], ln[idx], lp[idx], g[idx], K[idx], TOL[capi.MIXED], 3)


def test_autograd_function_backward():
    t = torch()
    wl = synth.pulse_workload("t", 2048, 3, 4, 8, 3)
    z, K = population(wl, 3, 8)
    ctx, zd, Kd = context_with_population(wl, capi.FP64, z, K, 1.0)
    zr = zd.clone().requires_grad_(True)
    logp = sampler.LoglGrad.apply(ctx, zr, Kd)
    w = t.arange(8, dtype=t.float64, device="cuda")
    (logp * w).sum().backward()
    res = oracle.Oracle(wl).logl_grad(z, K, 1.0)
    np.testing.assert_allclose(zr.grad.cpu().numpy(), res["grad"] * np.arange(8)[:, None, None],
                               rtol=1e-10, atol=1e-10)


def test_bad_arguments_rejected():
    wl = synth.pulse_n1024_k3()
    ctx = sampler.open_context(wl, capi.FP64)
    with pytest.raises(capi.TsmcError):
        ctx.set_problem(0, np.array([1.0, np.nan]), 0.0, 1.0, 0.1, synth.PULSE_LO, synth.PULSE_HI, 4)
    with pytest.raises(capi.TsmcError):
        ctx.set_problem(3, np.ones(8), 0.0, 1.0, 0.1, synth.PULSE_LO, synth.PULSE_HI, 4)
    with pytest.raises(capi.TsmcError):
        ctx.nuts_move(-1, 0)
    t = torch()
    with pytest.raises(capi.TsmcError):
        ctx.set_population(dev_tensor(np.zeros((512, 10, 3))),
                           dev_tensor(np.full(512, 11, np.int32)))


def test_pulse_window_matches_full_evaluation():
    """The support window changes nothing beyond FP32 resolution and skips real work."""
    t = torch()
    wl = synth.pulse_k20(P=256)
    z, K = population(wl, 4, 256)
    out = []
    for win in (0, 1):
        ctx = sampler.open_context(wl, capi.MIXED, pulse_window=win)
        zd, Kd = dev_tensor(z, t.float64), dev_tensor(K, t.int32)
        ctx.set_population(zd, Kd, beta=[0.3])
        ctx.counters(reset=True)
        lo, ln, lp, g, _ = ctx.eval(zd, Kd, dev_tensor([0.3], t.float64), grad=True)
        (nom, _, comp, _), _ = ctx.counters()
        out.append((ln.cpu().numpy(), g.cpu().numpy(), nom, comp))
    (l0, g0, n0, c0), (l1, g1, n1, c1) = out
    assert n0 == n1 == c0 and c1 < 0.7 * n1
    np.testing.assert_allclose(l1, l0, rtol=1e-6)
    res = oracle.Oracle(wl).logl_grad(z[:8], K[:8], 0.3)
    assert np.all(np.abs(g1[:8] - g0[:8]) <= 1e-5 * res["gscale"] + 1e-300)


def test_mixture_schedule_stage_matches_oracle_fp64():
    """The paper's kernel mixture (p_NUTS, p_birth, p_death = 0.6, 0.2, 0.2 per round)."""
    wl = synth.pulse_n1024_k3()
    wl.P = 128
    wl.n_mut = 3
    wl.schedule = synth.SCHED_MIXTURE
    wl.p_nuts, wl.p_birth, wl.p_death = 0.6, 0.2, 0.2
    ctx = sampler.open_context(wl, capi.FP64)
    ctx.init_population()
    b, lz, _ = ctx.run_stage(0, use_graph=False)
    z, K, _, _ = ctx.get_population()
    res = oracle.Oracle(wl).smc_run(128, max_stages=1)
    assert b[0] == pytest.approx(res["beta"][0], abs=1e-13)
    Kg = K.cpu().numpy()
    assert np.mean(Kg == res["K"]) > 0.95
    same = Kg == res["K"]
    close = np.all(np.isclose(z.cpu().numpy(), res["z"], rtol=1e-8, atol=1e-8), axis=(1, 2))
    assert np.mean(close[same]) > 0.9


def test_mixture_schedule_unequal_birth_death_rj_parity_fp64():
    """Mixture schedule with p_birth != p_death (0.35 / 0.15), where the acceptance's
    log(p_death / p_birth) term does not vanish: one birth/death round with the oracle's
    move types, outcomes, K, z and likelihoods."""
    t = torch()
    wl = synth.pulse_workload("t", 1500, 3, 6, 200, 77)
    wl.schedule = synth.SCHED_MIXTURE
    wl.p_nuts, wl.p_birth, wl.p_death = 0.5, 0.35, 0.15
    z, K = population(wl, 15, 200)
    beta = 0.02
    ora = oracle.Oracle(wl)
    ctx, _, _ = context_with_population(wl, capi.FP64, z, K, beta)
    r = ora.logl_grad(z, K, beta)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    zo, Ko = z.copy(), K.copy()
    out_o = ora.rj_move(4, 1, beta, zo, Ko, lo, ln)
    outd = t.zeros(200, dtype=t.int32, device="cuda")
    ctx.rj_move(4, 1, outd)
    zg, Kg, _, lng = ctx.get_population()
    assert np.array_equal(outd.cpu().numpy(), out_o)
    assert np.array_equal(Kg.cpu().numpy(), Ko)
    np.testing.assert_allclose(zg.cpu().numpy(), zo, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(lng.cpu().numpy(), ln, rtol=1e-10)
    assert set(np.unique(out_o)) >= {0, 1, -1, 2}


@pytest.mark.parametrize("prec", [capi.FP64, capi.MIXED])
def test_linear_gaussian_evidence_on_gpu(prec):
    """SMC log Z and posterior mean against the closed form of the linear-Gaussian model."""
    lz, mu = [], []
    for seed in range(8):
        wl = synth.linamp_workload(n=256, k=3, P=1024, seed=31)
        wl.seed = 200 + seed
        ctx = sampler.open_context(wl, prec)
        out = sampler.run_smc(ctx, max_stages=200)
        z, _, _, _ = ctx.get_population()
        lz.append(out["logz"][-1][0])
        mu.append(z.cpu().numpy().reshape(-1, 3).mean(0))
        ctx.close()
    pr = wl.problems[0]
    t = np.arange(pr.n) / pr.n
    G = np.exp(-((t[:, None] - wl.fixed_tw[None, :, 0]) ** 2) / (2 * wl.fixed_tw[None, :, 1] ** 2))
    s2 = pr.sigma ** 2
    S = s2 * np.eye(pr.n) + wl.amp_sd ** 2 * G @ G.T
    res_ = pr.d - G @ np.full(3, wl.amp_mean)
    logz_full = -0.5 * res_ @ np.linalg.solve(S, res_) - 0.5 * np.linalg.slogdet(S)[1] \
        - 0.5 * pr.n * math.log(2 * math.pi)
    logz_exact = logz_full + 0.5 * pr.n * math.log(2 * math.pi * s2)
    prec_m = np.eye(3) / wl.amp_sd ** 2 + G.T @ G / s2
    cov = np.linalg.inv(prec_m)
    mean = cov @ (np.full(3, wl.amp_mean) / wl.amp_sd ** 2 + G.T @ pr.d / s2)
    lz, mu = np.array(lz), np.array(mu)
    se = max(lz.std(ddof=1) / math.sqrt(len(lz)), 0.01)
    assert abs(lz.mean() - logz_exact) < 3 * se + 0.02, (lz.mean(), logz_exact, se)
    sem = np.sqrt(np.diag(cov) / 1024 + mu.var(0, ddof=1) / len(mu))
    assert np.all(np.abs(mu.mean(0) - mean) < 4 * sem)


def test_state_errors_and_constant_ell():
    t = torch()
    wl = synth.pulse_n1024_k3()
    cfg = sampler.make_config(wl, capi.FP64)
    ctx = capi.Context(cfg, [1024])
    with pytest.raises(capi.TsmcError, match="error -6"):     # no data yet
        ctx.init_population()
    with pytest.raises(capi.TsmcError, match="error -6"):     # no population yet
        ctx.nuts_move(0, 0)
    # all particles with K = 0 have the same likelihood: ESS = P at any beta -> beta' = 1
    ctx2 = sampler.open_context(wl, capi.FP64)
    ctx2.set_population(dev_tensor(np.zeros((512, 10, 3))), dev_tensor(np.zeros(512, np.int32)),
                        beta=[0.0])
    b, lz, e = ctx2.temper_reweight_resample(0)
    d = wl.problems[0].d
    assert b[0] == 1.0 and e[0] == pytest.approx(512.0)
    assert lz[0] == pytest.approx(-0.5 * np.sum(d * d) / 0.01, rel=1e-12)
    anc = ctx2.get_ancestors().cpu().numpy()
    assert np.array_equal(anc, np.arange(512))


def test_mixed_temper_matches_oracle():
    """The mixed path's FP32 bisection passes choose the same beta as the FP64 definition
    (to the precision of an FP32 ESS) and the FP64 evidence increment."""
    wl = synth.pulse_k20(P=8192)
    z, K = synth.prior_population(wl, 3)
    t = torch()
    ctx = sampler.open_context(wl, capi.MIXED)
    ctx.set_population(dev_tensor(z, t.float64), dev_tensor(K, t.int32), beta=[0.0])
    _, _, _, ln = ctx.get_population()
    ell = ln.cpu().numpy()
    b, lz, e = ctx.temper_reweight_resample(2)
    bo, inco, esso, _ = oracle.temper(ell, wl.alpha, 0.0)
    assert b[0] == pytest.approx(bo, rel=1e-5)
    assert e[0] == pytest.approx(esso, rel=1e-3)
    assert lz[0] == pytest.approx(inco, rel=1e-4, abs=1e-4)
