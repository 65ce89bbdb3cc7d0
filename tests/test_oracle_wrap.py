"""Periodic (wrapped) coordinates for phase parameters, pinned on the CPU.

The sinusoid phase phi0 is uniform on [0, 2 pi) (Sec. 5.2), a circle.  With the wrap bit
set, theta = lo + (hi - lo)(z - floor z): the prior density of z is flat on every period
(log 0, no gradient, no curvature) and the posterior can straddle phi0 = 0 = 2 pi, which the
logit map cuts.  Pinned here against what the mathematics fixes: the same theta reached
through the logit map gives the same likelihood; the map is periodic in z; the gradient
matches finite differences across the period boundary; the log prior differs from the
logit map's exactly by the logistic density term; prior draws and birth/death at beta = 0
keep z uniform on one period; NUTS leaves wrapped coordinates reduced to one period.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2609_17674_b300 import synth

PHASE = 3            # sinusoid parameter index of phi0
WRAP = 1 << PHASE


def _wl(wrap=True, n=4096, P=1, seed=31):
    wl = synth.sinusoid_workload("t", n, 3, 4, P, seed)
    if wrap:
        wl.wrapmask = WRAP
    return wl


def _near_truth(wl, phases):
    """One particle at the injection with the given phases (radians) in place of phi0."""
    pr = wl.problems[0]
    th = pr.truth.copy()
    th[:, PHASE] = phases
    z = np.zeros((1, wl.kmax, 4))
    z[0, :3] = synth.theta_to_z(wl, 0, th)
    return z, np.array([3], np.int32), th


def test_wrapped_map_gives_the_logit_maps_likelihood_at_the_same_theta():
    ww, wl = _wl(True), _wl(False)
    zw, K, th = _near_truth(ww, [0.01, 3.1, 6.27])
    zl, _, _ = _near_truth(wl, [0.01, 3.1, 6.27])
    assert np.all((zw[0, :3, PHASE] >= 0) & (zw[0, :3, PHASE] < 1))
    rw = oracle.Oracle(ww).logl_grad(zw, K, 0.6)
    rl = oracle.Oracle(wl).logl_grad(zl, K, 0.6)
    np.testing.assert_allclose(rw["ll_new"], rl["ll_new"], rtol=1e-10)
    # log prior: the wrapped coordinate carries none; the logit one its logistic density
    a = np.abs(zl[0, :3, PHASE])
    logistic_term = np.sum(-a - 2.0 * np.log1p(np.exp(-a)))
    assert rw["logp"][0] - rl["logp"][0] == pytest.approx(-logistic_term, rel=1e-9, abs=1e-9)
    # d logL / d theta agrees; dtheta/dz is the span for the wrapped map
    span = 2 * math.pi
    sl = 1.0 / (1.0 + np.exp(-zl[0, :3, PHASE]))
    dth_l = span * sl * (1 - sl)
    pg_l = 1 - 2 * sl
    dl_dth_l = (rl["grad"][0, :3, PHASE] - pg_l) / dth_l
    dl_dth_w = rw["grad"][0, :3, PHASE] / span
    np.testing.assert_allclose(dl_dth_w, dl_dth_l, rtol=1e-6, atol=1e-9)


def test_wrapped_map_is_periodic():
    ww = _wl(True)
    z, K, _ = _near_truth(ww, [0.4, 2.0, 5.5])
    o = oracle.Oracle(ww)
    r0 = o.logl_grad(z, K, 0.8)
    for shift in (-3.0, 1.0, 7.0):
        zs = z.copy()
        zs[0, :3, PHASE] += shift
        r = o.logl_grad(zs, K, 0.8)
        np.testing.assert_allclose(r["logp"], r0["logp"], rtol=1e-12)
        np.testing.assert_allclose(r["grad"], r0["grad"], rtol=1e-7, atol=1e-9)


def _fd(o, z, K, beta, idx, h):
    def f(zz):
        return o.logl_grad(zz, K, beta, want_scale=False)["logp"][0]

    def cd(hh):
        zp, zm = z.copy(), z.copy()
        zp.flat[idx] += hh
        zm.flat[idx] -= hh
        return (f(zp) - f(zm)) / (2 * hh)

    return (4 * cd(h / 2) - cd(h)) / 3


def test_wrapped_gradient_matches_finite_differences_across_the_period_boundary():
    ww = _wl(True)
    o = oracle.Oracle(ww)
    z, K, _ = _near_truth(ww, [0.3, 1.0, 2.0])
    # phase coordinates just below the end of a period, at a negative period, far out
    z[0, :3, PHASE] = [0.9999995, -0.37, 12.25]
    g = o.logl_grad(z, K, 0.45)["grad"][0]
    for k in range(3):
        for d in range(4):
            q = k * 4 + d
            fd = _fd(o, z, K, 0.45, q, 1e-5)
            assert g.flat[q] == pytest.approx(fd, rel=2e-6, abs=1e-6 * (1 + abs(fd))), (k, d)


def test_wrapped_prior_has_no_gradient_or_curvature():
    ww = _wl(True)
    o = oracle.Oracle(ww)
    z, K, _ = _near_truth(ww, [0.3, 1.0, 2.0])
    # beta = 0: only the prior acts; the phase entries of gradient and metric vanish
    r = o.logl_grad(z, K, 0.0, want_fisher=True)
    assert np.all(r["grad"][0, :3, PHASE] == 0.0)
    assert np.all(r["fisher"][0, :3, PHASE] == 0.0)
    assert np.all(r["grad"][0, :3, :PHASE] != 0.0)


def test_wrapped_initial_draws_are_uniform_on_one_period():
    ww = _wl(True, P=1)
    ww.kmax, ww.seed = 6, 1
    z, K = oracle.Oracle(ww).init_population(6000)
    ph = np.concatenate([z[i, : K[i], PHASE] for i in range(6000)])
    other = np.concatenate([z[i, : K[i], 0] for i in range(6000)])
    assert np.all((ph > 0) & (ph < 1))
    assert stats.kstest(ph, "uniform").pvalue > 1e-3
    assert stats.kstest(other, "logistic").pvalue > 1e-3


def test_birth_death_keeps_the_wrapped_prior_at_beta_zero():
    ww = synth.sinusoid_workload("t", 64, 1, 5, 1, 3)
    ww.wrapmask = WRAP
    o = oracle.Oracle(ww)
    P = 4000
    z = np.zeros((P, 5, 4))
    K = np.zeros(P, np.int32)
    lo, ln = np.zeros(P), np.zeros(P)
    for rnd in range(120):
        o.rj_move(rnd // 16, rnd % 16, 0.0, z, K, lo, ln)
    assert stats.chisquare(np.bincount(K, minlength=6)).pvalue > 1e-3
    ph = np.concatenate([z[i, : K[i], PHASE] for i in range(P)])
    assert stats.kstest(ph, "uniform").pvalue > 1e-3
    fr = np.concatenate([z[i, : K[i], 1] for i in range(P)])
    assert stats.kstest(fr, "logistic").pvalue > 1e-3


def test_nuts_leaves_wrapped_coordinates_on_one_period():
    ww = _wl(True, P=8)
    o = oracle.Oracle(ww)
    z = np.zeros((8, 4, 4))
    K = np.full(8, 3, np.int32)
    for i in range(8):
        z[i] = _near_truth(ww, [0.2 + i, 1.0, 3.0])[0][0]
    z[:, :3, PHASE] += np.arange(8)[:, None] - 4.0          # start on other periods
    r = o.logl_grad(z, K, 0.5)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    zin = z.copy()
    o.nuts_move(0, 0, 0.5, 0.01, np.full(4, 1e-2), z, K, lo, ln)
    ph = z[:, :3, PHASE]
    assert np.all((ph >= 0.0) & (ph <= 1.0))
    # the other coordinates are not reduced; an unmoved particle's phases are only reduced
    assert np.any(z[:, :3, :PHASE] != zin[:, :3, :PHASE])
    same = np.all(z[:, :3, :PHASE] == zin[:, :3, :PHASE], axis=(1, 2))
    red = zin[:, :3, PHASE] - np.floor(zin[:, :3, PHASE])
    assert np.all(ph[same] == red[same])
