"""High-level driver: a transdimensional SMC run on the CUDA library.

The loop follows Sec. 4 of the paper: start from the prior (or from a previous
posterior), then repeat {choose beta by ESS, reweight, resample, mutate} until
beta = 1.  Every step is one call of the C ABI (``capi``); this module only
sequences them and marshals tensors.
"""
from __future__ import annotations

import numpy as np

from . import capi
from .synth import Workload


def make_config(wl: Workload, precision: int = capi.MIXED, threads: int = 0,
                samples_per_thread: int = 0, pulse_window: int = 1,
                fused_rounds: int = 0, particle_shard=None) -> capi.Config:
    """particle_shard = (particle_base, particles_global): the context holds wl.P particles
    of each problem starting at particle_base, of particles_global in all."""
    return capi.Config(model=wl.model, precision=precision, schedule=wl.schedule,
                       n_problems=len(wl.problems), particles=wl.P, kmax=wl.kmax, kmin=wl.kmin,
                       birth_proposal=wl.birth_proposal,
                       birth_prior_weight=wl.birth_prior_weight, channels=wl.channels,
                       response=(capi.C.c_double * 4)(*wl.resp),
                       n_mut=wl.n_mut, max_depth=wl.max_depth, alpha=wl.alpha, p_nuts=wl.p_nuts,
                       p_birth=wl.p_birth, p_death=wl.p_death, amp_mean=wl.amp_mean,
                       amp_sd=wl.amp_sd, seed=wl.seed, threads=threads,
                       samples_per_thread=samples_per_thread,
                       pulse_window=pulse_window if precision == capi.MIXED else 0,
                       problem_base=wl.problem_base, fused_rounds=fused_rounds,
                       particle_base=particle_shard[0] if particle_shard else 0,
                       particles_global=particle_shard[1] if particle_shard else 0,
                       wrap_mask=wl.wrapmask)


def open_context(wl: Workload, precision=capi.MIXED, n_use=None, n_capacity=None, threads=0,
                 samples_per_thread=0, stream=None, pulse_window=1,
                 fused_rounds=0, particle_shard=None) -> capi.Context:
    """Context with every problem's data uploaded (first n_use samples of each)."""
    cfg = make_config(wl, precision, threads, samples_per_thread, pulse_window, fused_rounds,
                      particle_shard)
    nb = len(wl.problems)
    n_use = n_use or [p.n for p in wl.problems]
    if np.isscalar(n_use):
        n_use = [int(n_use)] * nb
    cap = n_capacity or [p.n for p in wl.problems]
    ctx = capi.Context(cfg, cap, stream=stream)
    for b, pr in enumerate(wl.problems):
        lo, hi = wl.bounds(b)
        ctx.set_problem(b, pr.d[: n_use[b]], pr.t_origin, pr.dt, pr.sigma, lo, hi, wl.logmask)
    if wl.model == capi.PULSE_LINAMP:
        ctx.set_fixed_components(wl.fixed_tw)
    return ctx


def run_smc(ctx: capi.Context, max_stages: int = 500, stage0: int = 0, use_graph: bool = True,
            init_prior: bool = True):
    """Prior-start (or continue) SMC until every problem reaches beta = 1."""
    if init_prior:
        ctx.init_population()
    betas, logzs, esss = [], [], []
    for s in range(max_stages):
        b, lz, e = ctx.run_stage(stage0 + s, use_graph)
        betas.append(b)
        logzs.append(lz)
        esss.append(e)
        if np.all(b >= 1.0):
            break
    return dict(n_stages=len(betas), beta=np.array(betas), logz=np.array(logzs),
                ess=np.array(esss))


class LoglGrad:
    """torch.autograd.Function over the adjoint kernel: logp(z) per particle.

    forward(z, K) returns logp [P_total]; backward multiplies the kernel's
    gradient dlogp/dz by the incoming gradient.
    """

    _fn = None

    @classmethod
    def apply(cls, ctx: capi.Context, z, K, beta=None):
        if cls._fn is None:
            import torch

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(fctx, z, K, cctx, beta):
                    _, _, logp, g, _ = cctx.eval(z.detach().contiguous(), K, beta, grad=True)
                    fctx.save_for_backward(g)
                    return logp

                @staticmethod
                def backward(fctx, gout):
                    (g,) = fctx.saved_tensors
                    return gout[:, None, None] * g, None, None, None

            cls._fn = _F
        return cls._fn.apply(z, K, ctx, beta)
