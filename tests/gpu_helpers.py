"""Shared set-up for the GPU parity tests: one workload, the oracle and the CUDA path."""
import numpy as np

import oracle
from paper_2609_17674_b300 import capi, sampler, synth

# tolerances (relative, conditioned on the sum of absolute terms for gradients)
TOL = {capi.FP64: 1e-12, capi.MIXED: 1e-5}


def torch():
    import torch as t

    return t


def dev_tensor(a, dtype=None):
    t = torch()
    return t.as_tensor(np.ascontiguousarray(a), device="cuda", dtype=dtype)


def context_with_population(wl, precision, z, K, beta, n_use=None, n1=0, threads=0, spt=0):
    """CUDA context holding population (z, K) at temperature beta; samples [n1, n_use) new."""
    pr = wl.problems[0]
    n_use = n_use or pr.n
    ctx = sampler.open_context(wl, precision, n_use=n1 if n1 > 0 else n_use,
                               n_capacity=[p.n for p in wl.problems], threads=threads,
                               samples_per_thread=spt)
    t = torch()
    zt = dev_tensor(z, t.float64)
    Kt = dev_tensor(K, t.int32)
    if n1 > 0:
        # assimilation starts from a posterior (beta = 1) of the first n1 samples
        ctx.set_population(zt, Kt, beta=[1.0] * len(wl.problems))
        ctx.assimilate(0, pr.d[n1:n_use])
    ctx.set_population(zt, Kt, beta=[beta] * len(wl.problems))
    return ctx, zt, Kt


def population(wl, seed, P, include_edges=True):
    z, K = synth.prior_population(wl, seed, P)
    if include_edges and P >= 2:
        K[0] = 0
        K[1] = wl.kmax
        rng = np.random.default_rng(seed)
        u = rng.random((wl.kmax, wl.D)).clip(1e-9, 1 - 1e-9)
        z[1] = np.log(u) - np.log1p(-u)
        z[0] = 0.0
    return z, K


def assert_eval_parity(ora, res, ll_old, ll_new, logp, grad, K, tol, D):
    ll_old, ll_new, logp = (x.cpu().numpy() for x in (ll_old, ll_new, logp))
    for name, g, r in (("ll_old", ll_old, res["ll_old"]), ("ll_new", ll_new, res["ll_new"]),
                       ("logp", logp, res["logp"])):
        err = np.abs(g - r)
        bound = tol * (np.abs(r) + 1e-300) + 1e-300
        assert np.all(err <= bound), (name, float(np.max(err / (np.abs(r) + 1e-300))))
    if grad is not None:
        g = grad.cpu().numpy()
        err = np.abs(g - res["grad"])
        bound = tol * res["gscale"] + 1e-300
        worst = float(np.max(err / (res["gscale"] + 1e-300)))
        assert np.all(err <= bound), ("grad", worst)
        # rows beyond K_p are zero
        for i, k in enumerate(K):
            assert np.all(g[i, k:] == 0.0)


def data_scale_gscale(wl, z, K, beta, b=0):
    """Gradient condition at the data scale: the oracle's sum of absolute terms evaluated on
    data 2d, where a particle near the injection has residual ~d (used with noise-free data,
    where the residual itself vanishes at the injection but FP32 template errors do not)."""
    import copy

    w2 = copy.deepcopy(wl)
    w2.problems[b].d = 2.0 * w2.problems[b].d
    return oracle.Oracle(w2, b).logl_grad(z, K, beta)["gscale"]
