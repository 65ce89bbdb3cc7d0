"""Population birth proposal (Sec. 6 suggestion; tsmc_build_birth_proposal) against the
oracle: the proposal built from the same population and stage, reversible-jump moves
that use it, whole SMC stages with it switched on, and the posterior it reaches."""
import importlib.util
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2609_17674_b300 import capi, sampler, synth
from gpu_helpers import context_with_population, population, torch

pytestmark = pytest.mark.gpu


def _wl(P=200, seed=77):
    wl = synth.pulse_workload("t", 1500, 3, 6, P, seed)
    wl.birth_proposal, wl.birth_prior_weight = 1, 0.2
    return wl


def _posterior_like(wl, seed):
    """Population concentrated near the injection (what a late stage looks like)."""
    rng = np.random.default_rng(seed)
    zt = synth.theta_to_z(wl, 0, wl.problems[0].truth)
    K = rng.integers(1, 5, wl.P).astype(np.int32)
    z = np.zeros((wl.P, wl.kmax, 3))
    for i in range(wl.P):
        k = min(K[i], zt.shape[0])
        K[i] = k
        z[i, :k] = zt[:k] + 0.05 * rng.standard_normal((k, 3))
    return z, K


def test_build_matches_oracle():
    wl = _wl()
    z, K = population(wl, 13, wl.P)
    ctx, _, _ = context_with_population(wl, capi.FP64, z, K, 0.3)
    m0, _, _ = ctx.get_birth_proposal(0)
    assert m0 == 0                      # nothing built yet: births come from the prior
    ctx.build_birth_proposal(7)
    m, h, c = ctx.get_birth_proposal(0)
    kde = oracle.Oracle(wl).kde_build(z, K, 7)
    assert m == kde.m == oracle.KDE_M
    assert np.array_equal(c, kde.centres(3))
    np.testing.assert_allclose(h[:3], np.array(kde.h[:3]), rtol=1e-15)


@pytest.mark.parametrize("pop", ["prior", "posterior"])
def test_rj_move_with_proposal_matches_oracle_fp64(pop):
    t = torch()
    wl = _wl()
    z, K = population(wl, 13, wl.P) if pop == "prior" else _posterior_like(wl, 5)
    beta = 0.45
    ora = oracle.Oracle(wl)
    ctx, _, _ = context_with_population(wl, capi.FP64, z, K, beta)
    ctx.build_birth_proposal(4)
    kde = ora.kde_build(z, K, 4)
    r = ora.logl_grad(z, K, beta)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    zo, Ko = z.copy(), K.copy()
    out_o = ora.rj_move(4, 2, beta, zo, Ko, lo, ln, kde=kde)
    outd = t.zeros(wl.P, dtype=t.int32, device="cuda")
    ctx.rj_move(4, 2, outd)
    zg, Kg, _, lng = ctx.get_population()
    assert np.array_equal(outd.cpu().numpy(), out_o)
    assert np.array_equal(Kg.cpu().numpy(), Ko)
    np.testing.assert_allclose(zg.cpu().numpy(), zo, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(lng.cpu().numpy(), ln, rtol=1e-10)
    assert np.sum(out_o == 1) > 0          # accepted births; deaths too from the prior
    assert pop == "posterior" or np.sum(out_o == 2) > 0


def test_smc_stages_with_proposal_match_oracle_fp64():
    wl = synth.pulse_n1024_k3()
    wl.P = 128
    wl.birth_proposal, wl.birth_prior_weight = 1, 0.3
    ctx = sampler.open_context(wl, capi.FP64)
    ctx.init_population()
    betas = [ctx.run_stage(s, use_graph=False)[0][0] for s in range(2)]
    z, K, _, _ = ctx.get_population()
    res = oracle.Oracle(wl).smc_run(128, max_stages=2)
    np.testing.assert_allclose(betas, res["beta"][:2], rtol=0, atol=1e-12)
    Kg = K.cpu().numpy()
    assert np.mean(Kg == res["K"]) > 0.95
    same = Kg == res["K"]
    close = np.all(np.isclose(z.cpu().numpy(), res["z"], rtol=1e-8, atol=1e-8), axis=(1, 2))
    assert np.mean(close[same]) > 0.9


def test_rj_move_with_proposal_mixed_agrees():
    t = torch()
    wl = _wl(P=400)
    z, K = _posterior_like(wl, 9)
    beta = 0.5
    ora = oracle.Oracle(wl)
    ctx, _, _ = context_with_population(wl, capi.MIXED, z, K, beta)
    ctx.build_birth_proposal(4)
    kde = ora.kde_build(z, K, 4)
    r = ora.logl_grad(z, K, beta)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    zo, Ko = z.copy(), K.copy()
    out_o = ora.rj_move(4, 2, beta, zo, Ko, lo, ln, kde=kde)
    outd = t.zeros(wl.P, dtype=t.int32, device="cuda")
    ctx.rj_move(4, 2, outd)
    assert np.mean(outd.cpu().numpy() == out_o) > 0.99


def test_smc_with_population_births_reaches_the_oracle_posterior():
    """Twenty mixed-path runs of the N=1024 pulse workload with births from the population
    mixture against the twenty oracle runs with births from the prior
    (tests/golden/smc_pulse_n1024_oracle.json): the proposal changes the path, not the target,
    so the K histogram, log Z and the parameter summaries agree within 3 standard errors."""
    here = os.path.dirname(__file__)
    gold = json.load(open(os.path.join(here, "golden", "smc_pulse_n1024_oracle.json")))["runs"]
    spec = importlib.util.spec_from_file_location(
        "mk", os.path.join(here, "golden", "make_smc_pulse_n1024.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    runs = []
    for r0 in gold:
        wl = synth.pulse_n1024_k3()
        wl.seed = r0["seed"]
        wl.birth_proposal, wl.birth_prior_weight = 1, 0.2
        ctx = sampler.open_context(wl, capi.MIXED)
        out = sampler.run_smc(ctx, max_stages=400)
        z, K, _, _ = ctx.get_population()
        r = mk.summaries(wl, z.cpu().numpy(), K.cpu().numpy())
        r["logz"] = float(out["logz"][-1][0])
        runs.append(r)
        ctx.close()

    def mean_se(x):
        x = np.asarray(x, dtype=float)
        return x.mean(0), x.std(0, ddof=1) / math.sqrt(len(x))

    hg, sg = mean_se([r["hist"] for r in runs])
    ho, so = mean_se([r["hist"] for r in gold])
    # 3 standard errors, floored at one particle's mass (the histogram's resolution)
    assert np.all(np.abs(hg - ho) <= np.maximum(3 * np.sqrt(sg**2 + so**2), 1.0 / 512)), (hg, ho)
    lg, slg = mean_se([r["logz"] for r in runs])
    lo, slo = mean_se([r["logz"] for r in gold])
    assert abs(lg - lo) <= 3 * math.hypot(slg, slo), (lg, lo)
    for key in ("t0_sorted_mean", "A_by_t0_mean"):
        xg = [r[key] for r in runs if key in r]
        xo = [r[key] for r in gold if key in r]
        mg, seg = mean_se(xg)
        mo, seo = mean_se(xo)
        assert np.all(np.abs(mg - mo) <= 3 * np.sqrt(seg**2 + seo**2) + 1e-4), (key, mg, mo)
