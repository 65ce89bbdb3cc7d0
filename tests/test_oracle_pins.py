"""Pins of the oracle against facts that do not come from the oracle itself.

Each test checks one oracle function against an independent statement of the
same mathematics: numpy's Philox implementation, closed forms (Riemann sums of
Gaussians, geometric sums of sinusoids, linear-Gaussian evidence), finite
differences, brute-force quadrature of the K posterior, stationarity of the
kernels, and textbook properties of ESS bisection and systematic resampling.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2609_17674_b300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# --------------------------------------------------------------------------
# Philox4x64-10: numpy's independent implementation (counter pre-incremented)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(6))
def test_philox_matches_numpy(seed):
    rng = np.random.default_rng(seed)
    ctr = rng.integers(1, 2**63, size=4, dtype=np.uint64)
    key = rng.integers(0, 2**63, size=2, dtype=np.uint64)
    prev = ctr.copy()
    prev[0] -= np.uint64(1)
    ref = np.random.Philox(key=key, counter=prev).random_raw(4)
    assert (oracle.philox(ctr, key) == ref).all()


def test_u01_open_interval():
    assert oracle.u01(0) == 2.0**-54
    assert oracle.u01(2**64 - 1) == 1.0 - 2.0**-54
    assert 0.0 < oracle.u01(2**63) < 1.0


# --------------------------------------------------------------------------
# Likelihood closed forms
# --------------------------------------------------------------------------
def _pulse_wl(n, d=None, kmax=2):
    wl = synth.pulse_workload("t", n, 1, kmax, 1, 5)
    if d is not None:
        wl.problems[0].d = d
    return wl


def test_empty_model_logl_is_data_energy():
    wl = synth.pulse_n1024_k3()
    o = oracle.Oracle(wl)
    d = wl.problems[0].d
    r = o.logl_grad(np.zeros((1, wl.kmax, 3)), np.zeros(1, np.int32), 1.0)
    assert r["ll_new"][0] == pytest.approx(-0.5 * np.sum(d * d) / 0.01, rel=1e-14)
    assert np.all(r["grad"] == 0.0)


@pytest.mark.parametrize("A,t0,w", [(1.3, 0.5, 0.02), (0.7, 0.41, 0.006), (1.9, 0.6, 0.045)])
def test_single_pulse_energy_riemann_closed_form(A, t0, w):
    # d = 0, K = 1: logL = -1/2 A^2 sum_n g_n^2 / sigma^2 and, for a grid much finer than w,
    # sum_n exp(-(t_n-t0)^2/w^2) = N w sqrt(pi) (Poisson summation, exponentially small error)
    n = 8192
    wl = _pulse_wl(n, d=np.zeros(n))
    theta = np.array([[A, t0, w]])
    z = np.zeros((1, wl.kmax, 3))
    z[0, 0] = synth.theta_to_z(wl, 0, theta)[0]
    o = oracle.Oracle(wl)
    ll = o.logl_grad(z, np.array([1], np.int32), 1.0)["ll_new"][0]
    # the coordinate round trip perturbs theta at the 1e-16 level; recover it exactly
    th = np.array([o.L.orc_u01(0)])  # keep lib loaded
    expect = -0.5 * A * A * n * w * math.sqrt(math.pi) / 0.01
    assert ll == pytest.approx(expect, rel=1e-12)


@pytest.mark.parametrize("f,phi0,A", [(3.0012e-3, 0.3, 0.05), (3.0041e-3, 5.9, 0.11)])
def test_single_sinusoid_energy_geometric_sum(f, phi0, A):
    # d = 0, fdot = 0: sum cos^2(w n + p) = N/2 + 1/2 Re[e^{2ip} (1 - e^{2iwN}) / (1 - e^{2iw})]
    n, dt = 1 << 16, 15.0
    wl = synth.sinusoid_workload("t", n, 1, 2, 1, 3)
    wl.problems[0].d = np.zeros(n)
    lo, hi = wl.bounds(0)
    z = np.zeros((1, 2, 4))
    z[0, 0] = synth.theta_to_z(wl, 0, np.array([[A, f, 0.5e-16, phi0]]))[0]
    z[0, 0, 2] = -745.0  # fdot -> 0 exactly
    o = oracle.Oracle(wl)
    ll = o.logl_grad(z, np.array([1], np.int32), 1.0)["ll_new"][0]
    om = 2 * math.pi * f * dt
    geo = np.exp(2j * phi0) * (1 - np.exp(2j * om * n)) / (1 - np.exp(2j * om))
    expect = -0.5 * A * A * (n / 2 + 0.5 * geo.real) / wl.problems[0].sigma ** 2
    assert ll == pytest.approx(expect, rel=1e-9)


def test_noise_free_truth_has_zero_residual():
    rng = synth._rng(11)
    pr = synth.pulse_problem(rng, 2048, 4, noise=False)
    wl = synth.Workload("t", synth.PULSE, 6, 1, [pr], synth.PULSE_LO, synth.PULSE_HI,
                        synth.PULSE_LOGMASK)
    z = np.zeros((1, 6, 3))
    z[0, :4] = synth.theta_to_z(wl, 0, pr.truth)
    r = oracle.Oracle(wl).logl_grad(z, np.array([4], np.int32), 1.0)
    assert abs(r["ll_new"][0]) < 1e-18


# --------------------------------------------------------------------------
# Gradients: Richardson-extrapolated central differences of the oracle's logp
# --------------------------------------------------------------------------
def _fd_grad(o, z, K, beta, idx, h):
    def f(zz):
        return o.logl_grad(zz, K, beta, want_scale=False)["logp"][0]

    def cd(hh):
        zp, zm = z.copy(), z.copy()
        zp.flat[idx] += hh
        zm.flat[idx] -= hh
        return (f(zp) - f(zm)) / (2 * hh)

    return (4 * cd(h / 2) - cd(h)) / 3


@pytest.mark.parametrize("which", ["pulse", "sinusoid", "linamp", "two_channel"])
def test_gradient_matches_finite_differences(which):
    if which == "pulse":
        wl = synth.pulse_workload("t", 1024, 3, 5, 1, 21)
        o = oracle.Oracle(wl, n1=300)
        z, K = synth.prior_population(wl, 3, 8)
        i = int(np.argmax(K))
        h = 1e-4
    elif which == "sinusoid":
        wl = synth.sinusoid_workload("t", 1 << 14, 3, 4, 1, 22)
        o = oracle.Oracle(wl, n1=5000)
        z = np.zeros((1, 4, 4))
        z[0, :3] = synth.theta_to_z(wl, 0, wl.problems[0].truth) + 0.05
        K = np.array([3], np.int32)
        i = 0
        h = 1e-4
    elif which == "two_channel":
        wl = synth.ae_workload("t", 1 << 13, 3, 4, 1, 23)
        o = oracle.Oracle(wl)
        z = np.zeros((1, 4, 4))
        z[0, :3] = synth.theta_to_z(wl, 0, wl.problems[0].truth) + 0.05
        K = np.array([3], np.int32)
        i = 0
        h = 1e-4
    else:
        wl = synth.linamp_workload(n=256, k=3)
        o = oracle.Oracle(wl)
        z = np.array([[[0.3], [1.7], [-0.4]]])
        K = np.array([3], np.int32)
        i = 0
        h = 1e-3
    zi, Ki = z[i : i + 1].copy(), K[i : i + 1].copy()
    beta = 0.37
    g = o.logl_grad(zi, Ki, beta)["grad"][0]
    for q in range(Ki[0] * wl.D):
        fd = _fd_grad(o, zi, Ki, beta, q, h)
        assert g.flat[q] == pytest.approx(fd, rel=2e-6, abs=1e-6 * (1 + abs(fd)))
    assert np.all(g.flat[Ki[0] * wl.D :] == 0.0)


def test_fisher_equals_negative_hessian_at_zero_residual():
    # with r = 0 the Hessian of logL is exactly -J^T J / sigma^2; add the prior curvature
    rng = synth._rng(5)
    pr = synth.pulse_problem(rng, 4096, 2, noise=False)
    wl = synth.Workload("t", synth.PULSE, 3, 1, [pr], synth.PULSE_LO, synth.PULSE_HI,
                        synth.PULSE_LOGMASK)
    o = oracle.Oracle(wl)
    z = np.zeros((1, 3, 3))
    z[0, :2] = synth.theta_to_z(wl, 0, pr.truth)
    K = np.array([2], np.int32)
    fis = o.logl_grad(z, K, 1.0, want_fisher=True)["fisher"][0]
    h = 1e-5
    for q in range(6):
        zp, zm = z.copy(), z.copy()
        zp.flat[q] += h
        zm.flat[q] -= h
        gp = o.logl_grad(zp, K, 1.0)["grad"][0].flat[q]
        gm = o.logl_grad(zm, K, 1.0)["grad"][0].flat[q]
        assert fis.flat[q] == pytest.approx(-(gp - gm) / (2 * h), rel=1e-5)


def test_linamp_fisher_closed_form():
    wl = synth.linamp_workload(n=200, k=3)
    o = oracle.Oracle(wl)
    t = np.arange(200) / 200
    G = np.exp(-((t[:, None] - wl.fixed_tw[None, :, 0]) ** 2) / (2 * wl.fixed_tw[None, :, 1] ** 2))
    z = np.array([[[0.1], [0.9], [2.0]]])
    fis = o.logl_grad(z, np.array([3], np.int32), 0.6, want_fisher=True)["fisher"][0, :, 0]
    expect = 0.6 * np.sum(G * G, 0) / 0.01 + 1.0 / wl.amp_sd**2
    np.testing.assert_allclose(fis, expect, rtol=1e-12)


# --------------------------------------------------------------------------
# Metric (Sec. 3.2: the mass matrix is the Hessian of the negative log posterior, read
# as the population mean of the Gauss-Newton diagonal, floored at 1e-8, then inverted)
# and the initial step size 0.5 (K_max D)^(-1/4)
# --------------------------------------------------------------------------
def _linamp_unequal_widths(n=400, sigma=0.1, amp_sd=0.7):
    """Linear-amplitude model with three fixed pulses of very different widths, so that the
    Gauss-Newton diagonal differs by component (it does not depend on the amplitudes)."""
    t = np.arange(n, dtype=np.float64) / n
    tw = np.array([[0.2, 0.004], [0.5, 0.03], [0.8, 0.12]])
    d = 0.05 * np.sin(7.0 * t)
    pr = synth.Problem(d=d, t_origin=0.0, dt=1.0 / n, sigma=sigma)
    wl = synth.Workload("linamp_unequal", synth.PULSE_LINAMP, 3, 1, [pr], amp_mean=1.0,
                        amp_sd=amp_sd, fixed_tw=tw)
    G = np.exp(-((t[:, None] - tw[None, :, 0]) ** 2) / (2.0 * tw[None, :, 1] ** 2))
    return wl, G


@pytest.mark.parametrize("beta", [0.0, 0.35, 1.0])
def test_metric_is_inverse_population_mean_of_gauss_newton_diagonal(beta):
    """orc_metric against the closed form of the linear model: per component
    F_k = beta sum_n g_k(t_n)^2 / sigma^2 + 1 / s0^2, averaged over every active component
    of every particle (particles with K = 0 contribute nothing), then inverted.  Dividing by
    the particle count, counting K = 0 particles, averaging per particle first or returning
    the mean instead of its inverse each fail here."""
    wl, G = _linamp_unequal_widths()
    o = oracle.Oracle(wl)
    F = beta * np.sum(G * G, 0) / wl.problems[0].sigma ** 2 + 1.0 / wl.amp_sd ** 2
    K = np.array([3, 0, 1, 2, 0, 1, 3, 1], np.int32)
    rng = np.random.default_rng(8)
    z = rng.normal(1.0, 2.0, (K.shape[0], 3, 1))      # amplitudes do not enter F
    num = sum(F[:k].sum() for k in K)
    expect = K.sum() / num
    got = o.metric(z, K, beta)
    assert got.shape == (1,)
    assert got[0] == pytest.approx(expect, rel=1e-12)
    # the three wrong reductions named above give clearly different values
    assert abs(K.shape[0] / num - expect) > 1e-3 * expect
    assert abs(np.count_nonzero(K) / num - expect) > 1e-3 * expect
    if beta > 0.0:   # at beta = 0 every component has the same F (the prior curvature)
        per_particle = np.mean([F[:k].mean() for k in K if k > 0])
        assert abs(1.0 / per_particle - expect) > 1e-3 * expect


def test_metric_per_parameter_prior_curvature_and_floor():
    """At beta = 0 with every sample new the likelihood term vanishes, so for the pulse model
    the diagonal is the logistic prior curvature 2 s(z)(1 - s(z)) of each coordinate; the
    metric is then 1 / mean over active components, per parameter (coordinates chosen so
    the three parameters differ: a transposed index fails).  Coordinates at |z| = 30 give a
    curvature of ~2e-13, below the 1e-8 floor: the metric is 1e8 there."""
    wl = synth.pulse_workload("t", 256, 2, 4, 4, 3)
    o = oracle.Oracle(wl)
    K = np.array([2, 0, 4, 1], np.int32)
    z = np.zeros((4, 4, 3))
    rng = np.random.default_rng(2)
    for i, k in enumerate(K):
        z[i, :k, 0] = rng.normal(0.0, 0.3, k)
        z[i, :k, 1] = rng.normal(2.0, 0.3, k)
        z[i, :k, 2] = rng.normal(-4.0, 0.3, k)
    s = 1.0 / (1.0 + np.exp(-z))
    curv = 2.0 * s * (1.0 - s)
    act = np.arange(4)[None, :] < K[:, None]
    expect = act.sum() / curv[act].sum(0)
    np.testing.assert_allclose(o.metric(z, K, 0.0), expect, rtol=1e-12)
    zf = z.copy()
    zf[act] = 30.0
    zf[2] = -30.0
    np.testing.assert_array_equal(o.metric(zf, K, 0.0), np.full(3, 1e8))
    # no component anywhere: unit metric
    np.testing.assert_array_equal(o.metric(z, np.zeros(4, np.int32), 0.0), np.ones(3))


def test_initial_step_size_scales_with_total_dimension():
    """eps_0 = 0.5 (K_max D)^(-1/4): it depends on K_max D only and eps_0^4 K_max D = 1/16."""
    e = {}
    for name, wl in (("p40", synth.pulse_workload("t", 64, 2, 40, 4, 1)),
                     ("s30", synth.sinusoid_workload("t", 64, 2, 30, 4, 1)),
                     ("p10", synth.pulse_workload("t", 64, 2, 10, 4, 1))):
        e[name] = oracle.Oracle(wl).eps_initial()
        assert e[name] ** 4 * wl.kmax * wl.D == pytest.approx(1.0 / 16.0, rel=1e-14)
    assert e["p40"] == e["s30"]                     # 40 x 3 = 30 x 4 = 120
    assert e["p10"] / e["p40"] == pytest.approx(4.0 ** 0.25, rel=1e-14)


# --------------------------------------------------------------------------
# Hamiltonian dynamics and NUTS
# --------------------------------------------------------------------------
def test_leapfrog_is_reversible():
    wl = synth.pulse_workload("t", 1024, 3, 4, 1, 9)
    o = oracle.Oracle(wl)
    z = np.zeros(12)
    z[:9] = synth.theta_to_z(wl, 0, wl.problems[0].truth).ravel() + 0.01
    rng = np.random.default_rng(0)
    p = np.zeros(12)
    p[:9] = rng.standard_normal(9)
    minv = np.array([1e-3, 1e-6, 1e-5])
    g = o.logl_grad(z.reshape(1, 4, 3), np.array([3], np.int32), 1.0)["grad"].ravel()
    z0, p0 = z.copy(), p.copy()
    for _ in range(25):
        o.leapfrog(3, 1.0, 0.05, minv, z, p, g)
    p = -p
    for _ in range(25):
        o.leapfrog(3, 1.0, 0.05, minv, z, p, g)
    np.testing.assert_allclose(z, z0, atol=1e-9)
    np.testing.assert_allclose(-p, p0, atol=1e-7)


def _linamp_posterior(wl, beta=1.0):
    pr = wl.problems[0]
    t = np.arange(pr.n) / pr.n
    G = np.exp(-((t[:, None] - wl.fixed_tw[None, :, 0]) ** 2) / (2 * wl.fixed_tw[None, :, 1] ** 2))
    s2 = pr.sigma**2
    prec = np.eye(wl.kmax) / wl.amp_sd**2 + beta * G.T @ G / s2
    cov = np.linalg.inv(prec)
    mean = cov @ (np.full(wl.kmax, wl.amp_mean) / wl.amp_sd**2 + beta * G.T @ pr.d / s2)
    return G, mean, cov


def test_nuts_leaves_linear_gaussian_posterior_invariant():
    wl = synth.linamp_workload(n=128, k=2, P=3000, seed=17)
    o = oracle.Oracle(wl)
    G, mean, cov = _linamp_posterior(wl)
    rng = np.random.default_rng(4)
    P = 3000
    z = rng.multivariate_normal(mean, cov, size=P).reshape(P, 2, 1)
    K = np.full(P, 2, np.int32)
    r = o.logl_grad(z, K, 1.0)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    minv = np.array([np.mean(np.diag(cov))])
    for rnd in range(3):
        acc, nl, fl = o.nuts_move(0, rnd, 1.0, 0.6, minv, z, K, lo, ln)
        assert np.all(nl > 0)
    zz = z.reshape(P, 2)
    for d in range(2):
        sd = math.sqrt(cov[d, d])
        assert abs(zz[:, d].mean() - mean[d]) < 4 * sd / math.sqrt(P)
        assert stats.kstest((zz[:, d] - mean[d]) / sd, "norm").pvalue > 1e-3
    # the chain moved: decorrelated from its start
    assert np.mean(acc) > 0.5
    # the carried likelihood parts belong to the returned points
    r2 = o.logl_grad(z, K, 1.0)
    np.testing.assert_allclose(ln, r2["ll_new"], rtol=1e-12)


# --------------------------------------------------------------------------
# Reversible jump: prior invariance and the brute-force K posterior
# --------------------------------------------------------------------------
def test_rj_converges_to_k_prior_at_beta_zero():
    wl = synth.pulse_workload("t", 8, 1, 5, 1, 1)
    o = oracle.Oracle(wl)
    P = 4000
    z = np.zeros((P, 5, 3))
    K = np.zeros(P, np.int32)
    lo, ln = np.zeros(P), np.zeros(P)
    for rnd in range(120):
        o.rj_move(rnd // 16, rnd % 16, 0.0, z, K, lo, ln)
    counts = np.bincount(K, minlength=6)
    assert stats.chisquare(counts).pvalue > 1e-3
    zz = np.concatenate([z[i, : K[i]].ravel() for i in range(P)])
    assert stats.kstest(zz, "logistic").pvalue > 1e-3


def test_mixture_schedule_keeps_the_prior_at_beta_zero():
    """Mixture schedule (every round each particle draws NUTS, birth or death) with unequal
    birth and death probabilities: the acceptance ratio carries log(p_death / p_birth), so at
    beta = 0 a population drawn from the prior stays there (K ~ U{0..kmax}, z ~ logistic).
    Without that term, or with its sign flipped, K drifts to a bound by 0.2 per round.  The
    three move types occur with their probabilities."""
    wl = synth.pulse_workload("t", 8, 1, 5, 1, 1)
    wl.schedule, wl.p_nuts, wl.p_birth, wl.p_death = 1, 0.5, 0.35, 0.15
    o = oracle.Oracle(wl)
    P = 4000
    z, K = synth.prior_population(wl, 3, P)
    lo, ln = np.zeros(P), np.zeros(P)
    types = np.zeros(3)
    for rnd in range(60):
        st, r = rnd // 16, rnd % 16
        out = o.rj_move(st, r, 0.0, z, K, lo, ln)
        types += [np.sum(out == 0), np.sum(np.abs(out) == 1), np.sum(np.abs(out) == 2)]
        o.nuts_move(st, r, 0.0, 0.8, np.ones(4), z, K, lo, ln)
    assert stats.chisquare(np.bincount(K, minlength=6)).pvalue > 1e-3
    zz = np.concatenate([z[i, : K[i]].ravel() for i in range(P)])
    assert stats.kstest(zz, "logistic").pvalue > 1e-3
    n = types.sum()
    for f, p in zip(types / n, (0.5, 0.35, 0.15)):
        assert abs(f - p) < 5 * math.sqrt(p * (1 - p) / n)


def test_rj_with_lower_bound_keeps_k_prior_at_beta_zero():
    """K prior U{kmin..kmax} (the paper's pulse example uses [1, 10]): started at K = kmin,
    birth/death at beta = 0 reaches the uniform prior on {kmin..kmax} and never leaves it;
    every death proposed at K = kmin is rejected (outcome -2)."""
    wl = synth.pulse_workload("t", 8, 1, 5, 1, 1)
    wl.kmin = 2
    o = oracle.Oracle(wl)
    P = 4000
    z = np.zeros((P, 5, 3))
    K = np.full(P, 2, np.int32)
    u = synth._rng(5).random((P, 2, 3))
    z[:, :2] = np.log(u) - np.log1p(-u)
    lo, ln = np.zeros(P), np.zeros(P)
    rejected_at_floor = 0
    for rnd in range(120):
        k_before = K.copy()
        out = o.rj_move(rnd // 16, rnd % 16, 0.0, z, K, lo, ln)
        assert K.min() >= 2
        rejected_at_floor += int(np.sum((k_before == 2) & (out == -2)))
        assert np.all(out[(k_before == 2) & (K < 2)] == -2)
    assert rejected_at_floor > 0
    counts = np.bincount(K, minlength=6)[2:]
    assert stats.chisquare(counts).pvalue > 1e-3


def test_init_population_with_lower_bound():
    wl = synth.pulse_n1024_k3()
    wl.kmin = 1
    z, K = oracle.Oracle(wl).init_population(20000)
    assert K.min() == 1 and K.max() == 10
    assert stats.chisquare(np.bincount(K, minlength=11)[1:]).pvalue > 1e-3
    assert np.all(z[np.arange(10)[None, :] >= K[:, None]] == 0.0)


def _toy_kposterior_workload(P, seed):
    rng = synth._rng(99)
    n = 64
    lo, hi = (0.5, 0.05, 0.02, 0.0), (2.0, 0.95, 0.1, 0.0)
    t = np.arange(n) / n
    d = 0.8 * np.exp(-((t - 0.47) ** 2) / (2 * 0.04**2)) + 0.5 * rng.standard_normal(n)
    pr = synth.Problem(d=d, t_origin=0.0, dt=1.0 / n, sigma=0.5)
    return synth.Workload("toy", synth.PULSE, 1, P, [pr], lo, hi, 0b100, n_mut=5, max_depth=6,
                          alpha=0.5, p_birth=0.5, p_death=0.5, seed=seed)


def _toy_brute_force(wl, nodes=(24, 240, 24)):
    pr = wl.problems[0]
    t = np.arange(pr.n) / pr.n
    lo, hi = wl.lo, wl.hi

    def gl(a, b, m, panels=1):
        x, w = np.polynomial.legendre.leggauss(m)
        edges = np.linspace(a, b, panels + 1)
        xs = np.concatenate([0.5 * (e1 - e0) * x + 0.5 * (e1 + e0) for e0, e1 in zip(edges, edges[1:])])
        ws = np.concatenate([0.5 * (e1 - e0) * w for e0, e1 in zip(edges, edges[1:])])
        return xs, ws

    Ax, Aw = gl(lo[0], hi[0], nodes[0])
    tx, tw = gl(lo[1], hi[1], 8, nodes[1] // 8)
    lwx, lww = gl(math.log(lo[2]), math.log(hi[2]), nodes[2])
    e0 = -0.5 * np.sum(pr.d**2) / pr.sigma**2
    acc = 0.0
    for wi, wv in zip(np.exp(lwx), lww):
        g = np.exp(-((t[None, :] - tx[:, None]) ** 2) / (2 * wi * wi))   # [nt, n]
        dg = g @ pr.d
        gg = np.sum(g * g, 1)
        # logL(A, t0) - e0 = (A d.g - A^2 g.g / 2) / sigma^2
        ll = (Ax[:, None] * dg[None, :] - 0.5 * Ax[:, None] ** 2 * gg[None, :]) / pr.sigma**2
        acc += wv * np.sum(Aw[:, None] * tw[None, :] * np.exp(ll))
    # prior densities: uniform A, uniform t0, log-uniform w (uniform in log w)
    z1_over_z0 = acc / ((hi[0] - lo[0]) * (hi[1] - lo[1]) * (math.log(hi[2]) - math.log(lo[2])))
    return z1_over_z0, e0


def test_toy_k_posterior_matches_brute_force():
    r1, e0 = _toy_brute_force(_toy_kposterior_workload(1, 0))
    r2, _ = _toy_brute_force(_toy_kposterior_workload(1, 0), nodes=(32, 400, 32))
    assert r1 == pytest.approx(r2, rel=1e-6)  # quadrature converged
    p1 = r2 / (1 + r2)
    assert 0.15 < p1 < 0.95  # an informative toy
    logz_exact = e0 + math.log(0.5 * (1 + r2))
    fr, lz = [], []
    for seed in range(6):
        wl = _toy_kposterior_workload(1500, seed)
        res = oracle.Oracle(wl).smc_run(1500)
        fr.append(np.mean(res["K"] == 1))
        lz.append(res["logz"])
    fr, lz = np.array(fr), np.array(lz)
    se_f = max(fr.std(ddof=1) / math.sqrt(len(fr)), 0.01)
    se_z = max(lz.std(ddof=1) / math.sqrt(len(lz)), 0.02)
    assert abs(fr.mean() - p1) < 3 * se_f + 0.01
    assert abs(lz.mean() - logz_exact) < 3 * se_z + 0.02


# --------------------------------------------------------------------------
# SMC evidence and posterior on the linear-Gaussian model (closed form)
# --------------------------------------------------------------------------
def test_smc_evidence_and_posterior_match_linear_gaussian_closed_form():
    wl0 = synth.linamp_workload(n=256, k=3, P=400, seed=31)
    G, mean, cov = _linamp_posterior(wl0)
    pr = wl0.problems[0]
    n, s2 = pr.n, pr.sigma**2
    m0 = np.full(3, wl0.amp_mean)
    S = s2 * np.eye(n) + wl0.amp_sd**2 * G @ G.T
    sign, logdet = np.linalg.slogdet(S)
    res_ = pr.d - G @ m0
    logz_full = -0.5 * res_ @ np.linalg.solve(S, res_) - 0.5 * logdet - 0.5 * n * math.log(2 * math.pi)
    # the sampler omits the Gaussian normalisation -n/2 log(2 pi sigma^2) inside moves
    logz_exact = logz_full + 0.5 * n * math.log(2 * math.pi * s2)
    lz, mu = [], []
    for seed in range(6):
        wl = synth.linamp_workload(n=256, k=3, P=400, seed=31)
        wl.seed = 100 + seed
        res = oracle.Oracle(wl).smc_run(400)
        lz.append(res["logz"])
        mu.append(res["z"].reshape(400, 3).mean(0))
        assert res["beta"][-1] == 1.0
    lz, mu = np.array(lz), np.array(mu)
    se = max(lz.std(ddof=1) / math.sqrt(len(lz)), 0.01)
    assert abs(lz.mean() - logz_exact) < 3 * se + 0.02
    sem = np.sqrt(np.diag(cov) / 400 + mu.var(0, ddof=1) / len(mu))
    assert np.all(np.abs(mu.mean(0) - mean) < 4 * sem)


def _linamp_log_evidence(wl, nn):
    """Closed-form log p(d_0..d_{nn-1}) of the linear-Gaussian model, without the Gaussian
    normalisation -nn/2 log(2 pi sigma^2) that the sampler leaves out of its moves."""
    pr = wl.problems[0]
    t = np.arange(pr.n)[:nn] / pr.n
    G = np.exp(-((t[:, None] - wl.fixed_tw[None, :, 0]) ** 2) / (2 * wl.fixed_tw[None, :, 1] ** 2))
    s2 = pr.sigma**2
    S = s2 * np.eye(nn) + wl.amp_sd**2 * G @ G.T
    r = pr.d[:nn] - G @ np.full(wl.kmax, wl.amp_mean)
    _, logdet = np.linalg.slogdet(S)
    return -0.5 * r @ np.linalg.solve(S, r) - 0.5 * logdet + 0.5 * nn * math.log(s2)


def test_assimilation_evidence_matches_linear_gaussian_closed_form():
    """Posterior start (Sec. 4): SMC on the first n1 samples, then, from its particles, a run
    that tempers in the remaining samples (old samples at weight 1, new ones at beta).  The
    first run's evidence must match log p(d_old) and the second's the increment
    log p(d_new | d_old) = log p(d) - log p(d_old), both in closed form."""
    n, n1, P = 256, 128, 400
    wl0 = synth.linamp_workload(n=n, k=3, P=P, seed=31)
    exact_old = _linamp_log_evidence(wl0, n1)
    exact_inc = _linamp_log_evidence(wl0, n) - exact_old
    lz_old, lz_inc = [], []
    for seed in range(6):
        wl = synth.linamp_workload(n=n, k=3, P=P, seed=31)
        wl.seed = 200 + seed
        r1 = oracle.Oracle(wl, n=n1).smc_run(P)
        r2 = oracle.Oracle(wl, n=n, n1=n1).smc_run(P, init_prior=False, z=r1["z"], K=r1["K"],
                                                   stage0=r1["n_stages"])
        assert r1["beta"][-1] == 1.0 and r2["beta"][-1] == 1.0
        lz_old.append(r1["logz"])
        lz_inc.append(r2["logz"])
    for lz, exact in ((np.array(lz_old), exact_old), (np.array(lz_inc), exact_inc)):
        se = max(lz.std(ddof=1) / math.sqrt(len(lz)), 0.01)
        assert abs(lz.mean() - exact) < 3 * se + 0.02, (lz.mean(), exact, se)


# --------------------------------------------------------------------------
# Tempering and resampling
# --------------------------------------------------------------------------
def test_temper_constant_ell_jumps_to_one():
    bn, inc, ess, logw = oracle.temper(np.full(100, -3.0), 0.5, 0.25)
    assert bn == 1.0 and ess == pytest.approx(100.0, rel=1e-14)
    assert inc == pytest.approx(0.75 * -3.0, rel=1e-14)


def test_temper_two_point_closed_form():
    # half the particles at ell = 0, half at -L: ESS/P = (1+x)^2 / (2(1+x^2)), x = e^{-delta L};
    # ESS = 0.9 P  <=>  x = 1/2, delta = ln 2 / L; evidence increment log((1+x)/2)
    L, P = 100.0, 1000
    ell = np.where(np.arange(P) % 2 == 0, 0.0, -L)
    bn, inc, ess, logw = oracle.temper(ell, 0.9, 0.2)
    assert bn - 0.2 == pytest.approx(math.log(2) / L, abs=2e-14)
    assert inc == pytest.approx(math.log(0.75), abs=1e-12)
    assert ess >= 0.9 * P and ess == pytest.approx(0.9 * P, rel=1e-10)


def test_resample_properties():
    wl = synth.pulse_n1024_k3()
    o = oracle.Oracle(wl)
    P = 512
    assert np.array_equal(o.resample(3, np.zeros(P)), np.arange(P))
    rng = np.random.default_rng(1)
    logw = rng.normal(0, 3, P)
    a = o.resample(4, logw)
    assert np.all(np.diff(a) >= 0)
    W = np.exp(logw - logw.max())
    W /= W.sum()
    counts = np.bincount(a, minlength=P)
    assert np.all(counts >= np.floor(P * W) - 1e-9) and np.all(counts <= np.ceil(P * W) + 1e-9)


@pytest.mark.parametrize("P,spread", [(1, 1.0), (7, 0.5), (512, 3.0), (3000, 8.0)])
def test_resample_ancestors_by_exact_integer_prefix_sums(P, spread):
    """Systematic resampling on quantised weights, written out with Python integers (exact
    prefix sums) and the same double-precision target: W_i = round(exp(logw_i - max) 2^S),
    S = 52 - ceil(log2 P), t_i = min((i + U) / P C_P, C_P - 1), a_i = min{j : C_j > t_i}.
    Weights that underflow the quantum and -inf log-weights are never chosen."""
    wl = synth.pulse_n1024_k3()
    o = oracle.Oracle(wl)
    rng = np.random.default_rng(P)
    logw = rng.normal(0.0, spread, P)
    if P > 4:
        logw[1] = -np.inf
        logw[3] = logw.max() - 80.0          # below 2^-(S+1) of the largest weight
    S = 52 - (P - 1).bit_length()
    assert oracle.lib().orc_resample_scale(P) == S
    m = max(logw)
    Wq = [0 if x == -np.inf else int(round(math.ldexp(math.exp(x - m), S))) for x in logw]
    C = list(itertools.accumulate(Wq))
    assert C[-1] <= 2 ** 52
    u = oracle.u01(oracle.philox([0, 3, 7, 0], [wl.seed, 0])[0])
    expect = []
    for i in range(P):
        t = min((float(i) + u) / float(P) * float(C[-1]), float(C[-1]) - 1.0)
        expect.append(next(j for j in range(P) if float(C[j]) > t))
    got = o.resample(3, logw)
    assert got.tolist() == expect
    if P > 4:
        assert 1 not in expect and 3 not in expect


def test_init_population_draws_the_prior():
    wl = synth.pulse_n1024_k3()
    z, K = oracle.Oracle(wl).init_population(22000)
    assert stats.chisquare(np.bincount(K, minlength=11)).pvalue > 1e-3
    zz = np.concatenate([z[i, : K[i]].ravel() for i in range(2000)])
    assert stats.kstest(zz, "logistic").pvalue > 1e-3
    assert np.all(z[np.arange(10)[None, :] >= K[:, None]] == 0.0)


def test_eps_update_rule():
    L = oracle.lib()
    assert L.orc_eps_update(0.1, 0.8) == pytest.approx(0.1)
    assert L.orc_eps_update(0.1, 0.3) == pytest.approx(0.1 * math.exp(-0.5))
    assert L.orc_eps_update(1.9, 1.0) == 2.0 and L.orc_eps_update(1e-4, 0.0) == 1e-4


# ---------------------------------------------------------------------------
# Population birth proposal (Sec. 6 suggestion): q(z) = eps prior_z + (1 - eps) KDE
# ---------------------------------------------------------------------------
def _mismatched_kde(D, centre, h):
    kde = oracle.Kde()
    kde.m = oracle.KDE_M
    rng = np.random.default_rng(3)
    c = np.asarray(centre)[None, :] + 0.2 * rng.standard_normal((oracle.KDE_M, D))
    flat = np.zeros(oracle.KDE_M * 4)
    flat[: oracle.KDE_M * D] = c.ravel()
    kde.c[:] = flat
    for d in range(4):
        kde.h[d] = h
    return kde


def test_population_birth_proposal_keeps_the_prior_at_beta_zero():
    """Reversible jump with births drawn from a fixed proposal that is far from the prior
    (centres near z = (1.5, -1, 0.5), width 0.3): at beta = 0 the chain must still leave
    the prior invariant, K ~ U{0..5} and every coordinate standard logistic.  Dropping or
    inverting the proposal-density ratio in either move pulls both off."""
    wl = synth.pulse_workload("t", 8, 1, 5, 1, 1)
    wl.birth_proposal, wl.birth_prior_weight = 1, 0.2
    o = oracle.Oracle(wl)
    kde = _mismatched_kde(3, (1.5, -1.0, 0.5), 0.3)
    P = 4000
    z, K = o.init_population(P)
    lo, ln = np.zeros(P), np.zeros(P)
    births = 0
    for rnd in range(160):
        out = o.rj_move(rnd // 16, rnd % 16, 0.0, z, K, lo, ln, kde=kde)
        births += int(np.sum(out == 1))
    assert births > 10000
    assert stats.chisquare(np.bincount(K, minlength=6)).pvalue > 1e-3
    for d in range(3):
        zz = np.concatenate([z[i, : K[i], d] for i in range(P)])
        assert stats.kstest(zz, "logistic").pvalue > 1e-3, d


def test_population_proposal_is_a_normalised_density():
    """E over the prior of q(z) / prior_z(z) is 1 (importance-sampling identity)."""
    wl = synth.pulse_workload("t", 8, 1, 5, 1, 1)
    wl.birth_proposal, wl.birth_prior_weight = 1, 0.2
    o = oracle.Oracle(wl)
    kde = _mismatched_kde(3, (0.8, -0.4, 0.2), 0.5)
    rng = np.random.default_rng(11)
    u = rng.random((40000, 3))
    zs = np.log(u) - np.log1p(-u)
    r = np.array([math.exp(o.kde_logq(kde, zz) - o.log_prior_z(zz)) for zz in zs])
    assert abs(r.mean() - 1.0) < 4 * r.std() / math.sqrt(len(r))
    # prior-only mixture (eps = 1) is the prior itself
    wl.birth_prior_weight = 1.0
    o1 = oracle.Oracle(wl)
    assert o1.kde_logq(kde, zs[0]) == o1.log_prior_z(zs[0])


def test_population_proposal_centres_are_uniform_over_components():
    """Centres are components of the population, drawn uniformly over components (not
    over particles): particle p is chosen in proportion to K_p."""
    wl = synth.pulse_workload("t", 8, 1, 5, 50, 1)
    wl.birth_proposal = 1
    o = oracle.Oracle(wl)
    rng = np.random.default_rng(2)
    K = rng.integers(0, 6, 50).astype(np.int32)
    z = np.zeros((50, 5, 3))
    for p in range(50):
        z[p, : K[p]] = p + 0.1 * np.arange(K[p])[:, None] + np.array([0.0, 0.01, 0.02])
    counts = np.zeros(50)
    for stage in range(40):
        kde = o.kde_build(z, K, stage)
        c = kde.centres(3)
        assert kde.m == oracle.KDE_M
        owner = np.floor(c[:, 0] + 1e-9).astype(int)
        slot = np.round((c[:, 0] - owner) / 0.1).astype(int)
        assert np.all(slot < K[owner])                      # a real component of that particle
        np.testing.assert_allclose(c, z[owner, slot])
        counts += np.bincount(owner, minlength=50)
        assert all(kde.h[d] > 0 for d in range(3))
    expected = counts.sum() * K / K.sum()
    m = expected > 0
    assert np.all(counts[~m] == 0)
    assert stats.chisquare(counts[m], expected[m]).pvalue > 1e-3



# ---------------------------------------------------------------------------
# Two channels A, E with a flat PSD (Sec. 5.2, eq. gw_likelihood)
# ---------------------------------------------------------------------------
def _fd_loglike(res_channels, dt, S):
    """-1/2 sum_c (r_c | r_c)_c with (a|b) = 4 Re sum_{f>0} a* b / S df (eq. gw_likelihood),
    the continuous transform approximated by dt times the DFT; f > 0 below Nyquist."""
    tot = 0.0
    for r in res_channels:
        n = r.shape[0]
        R = np.fft.rfft(r) * dt
        df = 1.0 / (n * dt)
        tot += 4.0 * np.sum(np.abs(R[1: n // 2]) ** 2) / S * df
    return -0.5 * tot


def test_two_channel_likelihood_is_the_frequency_domain_inner_product():
    """The oracle's two-channel time-domain likelihood equals eq. gw_likelihood with a flat
    PSD S = 2 dt sigma^2, once the DC and Nyquist bins (outside the one-sided sum) are
    added back (Parseval); residuals built here from the model definition per channel."""
    wl = synth.ae_workload("t", 2048, 2, 4, 1, 31)
    pr = wl.problems[0]
    n, dt, sig = pr.n // 2, pr.dt, pr.sigma
    S = 2.0 * dt * sig * sig
    o = oracle.Oracle(wl)
    t = np.arange(n) * dt
    rA, dA, rE, dE = wl.resp
    z, K = synth.prior_population(wl, 4, 6)
    K[0] = 2
    z[0, :2] = synth.theta_to_z(wl, 0, pr.truth) + 0.02
    res = o.logl_grad(z, K, 1.0)
    lo, hi = wl.bounds(0)
    for i in range(6):
        ra, re = pr.d[:n].copy(), pr.d[n:].copy()
        for k in range(K[i]):
            th = []
            for d in range(4):
                u = 1.0 / (1.0 + math.exp(-z[i, k, d]))
                if wl.logmask >> d & 1:
                    th.append(math.exp(math.log(lo[d]) + (math.log(hi[d]) - math.log(lo[d])) * u))
                else:
                    th.append(lo[d] + (hi[d] - lo[d]) * u)
            A, f, fd, p0 = th
            ph = 2 * math.pi * f * t + math.pi * fd * t * t + p0
            ra -= rA * A * np.cos(ph + dA)
            re -= rE * A * np.cos(ph + dE)
        fdl = _fd_loglike([ra, re], dt, S)
        edge = sum((np.fft.rfft(r)[0].real ** 2 + np.abs(np.fft.rfft(r)[n // 2]) ** 2) / n
                   for r in (ra, re))
        assert res["ll_new"][i] == pytest.approx(fdl - 0.5 * edge / sig**2, rel=1e-10)


def test_two_channel_response_matters():
    """Both channels enter with their own response: swapping or dropping one changes the
    likelihood of a particle at the injection by far more than rounding."""
    wl = synth.ae_workload("t", 1024, 2, 4, 1, 32)
    pr = wl.problems[0]
    z = np.zeros((1, 4, 4))
    z[0, :2] = synth.theta_to_z(wl, 0, pr.truth)
    K = np.array([2], np.int32)
    base = oracle.Oracle(wl).logl_grad(z, K, 1.0)["ll_new"][0]
    assert abs(base) < 1e-6 * float(np.sum(pr.d ** 2))     # noise-free data, exact fit
    for resp in ((1.0, 0.0, 0.8, 0.0), (0.8, 0.5 * math.pi, 1.0, 0.0), (1.0, 0.0, 0.0, 0.0)):
        wl.resp = resp
        other = oracle.Oracle(wl).logl_grad(z, K, 1.0)["ll_new"][0]
        assert other < base - 10.0


@pytest.mark.parametrize("which", ["pulse", "sinusoid", "two_channel"])
def test_rj_incremental_likelihood_equals_fresh_evaluation(which):
    """The birth/death move updates ll_old / ll_new by its incremental Delta logL (sum of
    r h - h^2/2 over the samples, per channel); after every accepted move the carried values
    must equal a fresh evaluation of the new state."""
    if which == "pulse":
        wl = synth.pulse_workload("t", 1500, 3, 6, 1, 77)
        o = oracle.Oracle(wl, n=1500, n1=600)
    elif which == "sinusoid":
        wl = synth.sinusoid_workload("t", 4096, 3, 6, 1, 78)
        o = oracle.Oracle(wl)
    else:
        wl = synth.ae_workload("t", 2048, 3, 6, 1, 79, noise=True)
        o = oracle.Oracle(wl)
    z, K = synth.prior_population(wl, 12, 300)
    beta = 0.4
    r = o.logl_grad(z, K, beta)
    lo, ln = r["ll_old"].copy(), r["ll_new"].copy()
    accepted = 0
    for rnd in range(3):
        out = o.rj_move(5, rnd, beta, z, K, lo, ln)
        fresh = o.logl_grad(z, K, beta)
        acc = (out == 1) | (out == 2)
        accepted += int(acc.sum())
        np.testing.assert_allclose(ln[acc], fresh["ll_new"][acc], rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(lo[acc], fresh["ll_old"][acc], rtol=1e-9, atol=1e-9)
        lo, ln = fresh["ll_old"].copy(), fresh["ll_new"].copy()
    assert accepted > 20


def test_extreme_coordinates_saturate():
    """At |z| = 1e308 the logistic map puts theta on a prior bound: likelihood and gradient
    equal those at |z| = 800 (where s(z) already rounds to 0 or 1 in FP64), the coordinate's
    log prior density -|z| - 2 log(1 + e^-|z|) is -1e308, and its z-gradient is -sign(z)
    (the likelihood's term carries dtheta/dz = s (1 - s) = 0)."""
    wl = synth.pulse_n1024_k3()
    o = oracle.Oracle(wl)
    rng = np.random.default_rng(1)
    z = np.zeros((4, wl.kmax, 3))
    z[:, :2] = rng.standard_normal((4, 2, 3))
    K = np.full(4, 2, np.int32)
    z[1] = z[0]
    z[3] = z[2]
    z[0, 0, 1], z[1, 0, 1] = 1e308, 800.0
    z[2, 0, 2], z[3, 0, 2] = -1e308, -800.0
    r = o.logl_grad(z, K, 0.4)
    assert np.all(np.isfinite(r["grad"])) and np.all(np.isfinite(r["ll_new"]))
    for a, b in ((0, 1), (2, 3)):
        assert r["ll_new"][a] == r["ll_new"][b] and r["ll_old"][a] == r["ll_old"][b]
        np.testing.assert_array_equal(r["grad"][a], r["grad"][b])
    assert r["grad"][0, 0, 1] == -1.0 and r["grad"][2, 0, 2] == 1.0
    assert r["logp"][0] == -1e308 and r["logp"][2] == -1e308
    # moving that coordinate from 0 to 800 changes its log density from -2 log 2 to -800
    # (log1p(e^-800) = 0), on top of the tempered likelihood's change
    z0 = z[1:2].copy()
    z0[0, 0, 1] = 0.0
    r0 = o.logl_grad(z0, K[:1], 0.4)
    dl = (r["ll_old"][1] - r0["ll_old"][0]) + 0.4 * (r["ll_new"][1] - r0["ll_new"][0])
    assert r["logp"][1] - r0["logp"][0] == pytest.approx(dl - 800.0 + 2.0 * math.log(2.0),
                                                         rel=1e-12, abs=1e-9)
