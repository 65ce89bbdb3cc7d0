"""Python access to the oracle (plain single-threaded FP64 C, ``tsmc_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The product path never imports this
package.  The oracle shares no code with the CUDA library; the two meet only
through the seeded inputs of ``paper_2609_17674_b300.synth``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tsmc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "tsmc_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Cfg(C.Structure):
    _fields_ = [
        ("model", C.c_int32), ("D", C.c_int32), ("kmax", C.c_int32), ("kmin", C.c_int32),
        ("birth_proposal", C.c_int32), ("birth_prior_weight", C.c_double),
        ("channels", C.c_int32), ("resp", C.c_double * 4),
        ("n_mut", C.c_int32),
        ("max_depth", C.c_int32), ("schedule", C.c_int32), ("alpha", C.c_double),
        ("p_nuts", C.c_double), ("p_birth", C.c_double), ("p_death", C.c_double),
        ("lo", C.c_double * 4), ("hi", C.c_double * 4), ("logmask", C.c_uint32),
        ("amp_mean", C.c_double), ("amp_sd", C.c_double), ("fixed_tw", C.c_void_p),
        ("seed", C.c_uint64), ("wrapmask", C.c_uint32),
    ]


KDE_M = 256


class Kde(C.Structure):
    """Population birth proposal: centres [m][D] and bandwidths in z coordinates."""
    _fields_ = [("m", C.c_int32), ("h", C.c_double * 4), ("c", C.c_double * (KDE_M * 4))]

    def centres(self, D):
        return np.ctypeslib.as_array(self.c)[: self.m * D].reshape(self.m, D).copy()


class Data(C.Structure):
    _fields_ = [("d", C.c_void_p), ("n", C.c_int64), ("n1", C.c_int64),
                ("t_origin", C.c_double), ("dt", C.c_double), ("sigma", C.c_double)]


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
        sig = {
            "orc_philox": (None, [P, P, P]),
            "orc_u01": (D, [C.c_uint64]),
            "orc_logl_grad_batch": (None, [P, P, P, P, I32, D, P, P, P, P, P, P]),
            "orc_init_population": (None, [P, I32, I32, P, P]),
            "orc_rj_move": (None, [P, P, I32, I32, I32, D, I32, P, P, P, P, P]),
            "orc_rj_move_q": (None, [P, P, I32, I32, I32, D, I32, P, P, P, P, P, P]),
            "orc_kde_build": (None, [P, I32, I32, I32, P, P, P]),
            "orc_kde_logq": (D, [P, P, P]),
            "orc_log_prior_z": (D, [P, P]),
            "orc_nuts_move": (None, [P, P, I32, I32, I32, D, D, P, I32, P, P, P, P, P, P, P]),
            "orc_leapfrog": (None, [P, P, I32, D, D, P, P, P, P, P]),
            "orc_temper": (None, [I32, P, D, D, P, P, P, P]),
            "orc_resample": (None, [P, I32, I32, I32, P, P]),
            "orc_resample_scale": (I32, [I32]),
            "orc_metric": (None, [P, P, P, P, I32, D, P]),
            "orc_eps_update": (D, [D, D]),
            "orc_eps_initial": (D, [P]),
            "orc_smc_run": (I32, [P, P, I32, I32, I32, I32, I32, P, P, P, P, P, P, P, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


class Oracle:
    """One problem of a workload, bound to oracle structs (keeps arrays alive)."""

    def __init__(self, wl, b: int = 0, n: int | None = None, n1: int | None = None):
        self.wl, self.b = wl, b
        pr = wl.problems[b]
        lo, hi = wl.bounds(b)
        self.d = np.ascontiguousarray(pr.d[: (n or pr.n)], dtype=np.float64)
        self.fixed = (np.ascontiguousarray(wl.fixed_tw, dtype=np.float64)
                      if wl.fixed_tw is not None else None)
        self.cfg = Cfg(model=wl.model, D=wl.D, kmax=wl.kmax, kmin=wl.kmin,
                       birth_proposal=wl.birth_proposal,
                       birth_prior_weight=wl.birth_prior_weight, channels=wl.channels,
                       resp=(C.c_double * 4)(*wl.resp), n_mut=wl.n_mut,
                       max_depth=wl.max_depth, schedule=wl.schedule, alpha=wl.alpha,
                       p_nuts=wl.p_nuts, p_birth=wl.p_birth, p_death=wl.p_death,
                       lo=(C.c_double * 4)(*lo), hi=(C.c_double * 4)(*hi), logmask=wl.logmask,
                       amp_mean=wl.amp_mean, amp_sd=wl.amp_sd,
                       fixed_tw=(self.fixed.ctypes.data if self.fixed is not None else None),
                       seed=wl.seed, wrapmask=wl.wrapmask)
        self.data = Data(d=self.d.ctypes.data, n=self.d.shape[0],
                         n1=(pr.n1 if n1 is None else n1), t_origin=pr.t_origin, dt=pr.dt,
                         sigma=pr.sigma)
        self.L = lib()

    @property
    def stride(self):
        return self.wl.kmax * self.wl.D

    def logl_grad(self, z, K, beta, want_scale=True, want_fisher=False):
        z = np.ascontiguousarray(z, dtype=np.float64)
        K = np.ascontiguousarray(K, dtype=np.int32)
        P = K.shape[0]
        out = {k: np.zeros(P) for k in ("ll_old", "ll_new", "logp")}
        out["grad"] = np.zeros((P, self.wl.kmax, self.wl.D))
        out["gscale"] = np.zeros_like(out["grad"]) if want_scale else None
        out["fisher"] = np.zeros_like(out["grad"]) if want_fisher else None
        self.L.orc_logl_grad_batch(C.byref(self.cfg), C.byref(self.data), _p(z), _p(K), P, beta,
                                   _p(out["ll_old"]), _p(out["ll_new"]), _p(out["logp"]),
                                   _p(out["grad"]),
                                   _p(out["gscale"]) if want_scale else None,
                                   _p(out["fisher"]) if want_fisher else None)
        return out

    def init_population(self, P):
        z = np.zeros((P, self.wl.kmax, self.wl.D))
        K = np.zeros(P, dtype=np.int32)
        self.L.orc_init_population(C.byref(self.cfg), self.b, P, _p(z), _p(K))
        return z, K

    def rj_move(self, stage, rnd, beta, z, K, ll_old, ll_new, kde=None):
        P = K.shape[0]
        out = np.zeros(P, dtype=np.int32)
        self.L.orc_rj_move_q(C.byref(self.cfg), C.byref(self.data), self.b, stage, rnd, beta, P,
                             _p(z), _p(K), _p(ll_old), _p(ll_new), _p(out),
                             C.byref(kde) if kde is not None else None)
        return out

    def kde_build(self, z, K, stage):
        kde = Kde()
        z = np.ascontiguousarray(z, dtype=np.float64)
        K = np.ascontiguousarray(K, dtype=np.int32)
        self.L.orc_kde_build(C.byref(self.cfg), self.b, stage, K.shape[0], _p(z), _p(K),
                             C.byref(kde))
        return kde

    def kde_logq(self, kde, z):
        z = np.ascontiguousarray(z, dtype=np.float64)
        return self.L.orc_kde_logq(C.byref(self.cfg), C.byref(kde), _p(z))

    def log_prior_z(self, z):
        z = np.ascontiguousarray(z, dtype=np.float64)
        return self.L.orc_log_prior_z(C.byref(self.cfg), _p(z))

    def nuts_move(self, stage, rnd, beta, eps, minv, z, K, ll_old, ll_new):
        P = K.shape[0]
        acc = np.zeros(P)
        nl = np.zeros(P, dtype=np.int32)
        fl = np.zeros(P, dtype=np.int32)
        minv = np.ascontiguousarray(minv, dtype=np.float64)
        self.L.orc_nuts_move(C.byref(self.cfg), C.byref(self.data), self.b, stage, rnd, beta, eps,
                             _p(minv), P, _p(z), _p(K), _p(ll_old), _p(ll_new), _p(acc), _p(nl),
                             _p(fl))
        return acc, nl, fl

    def leapfrog(self, K, beta, eps, minv, z, p, grad):
        lp = np.zeros(1)
        minv = np.ascontiguousarray(minv, dtype=np.float64)
        self.L.orc_leapfrog(C.byref(self.cfg), C.byref(self.data), K, beta, eps, _p(minv), _p(z),
                            _p(p), _p(grad), _p(lp))
        return lp[0]

    def resample(self, stage, logw):
        logw = np.ascontiguousarray(logw, dtype=np.float64)
        anc = np.zeros(logw.shape[0], dtype=np.int32)
        self.L.orc_resample(C.byref(self.cfg), self.b, stage, logw.shape[0], _p(logw), _p(anc))
        return anc

    def metric(self, z, K, beta):
        minv = np.zeros(4)
        self.L.orc_metric(C.byref(self.cfg), C.byref(self.data), _p(z), _p(K), K.shape[0], beta,
                          _p(minv))
        return minv[: self.wl.D]

    def eps_initial(self):
        return self.L.orc_eps_initial(C.byref(self.cfg))

    def smc_run(self, P, init_prior=True, z=None, K=None, stage0=0, max_stages=500, eps=None):
        if init_prior:
            z = np.zeros((P, self.wl.kmax, self.wl.D))
            K = np.zeros(P, dtype=np.int32)
        z = np.ascontiguousarray(z, dtype=np.float64).copy()
        K = np.ascontiguousarray(K, dtype=np.int32).copy()
        lo, ln, logz = np.zeros(P), np.zeros(P), np.zeros(1)
        bh, zh, eh = np.zeros(max_stages), np.zeros(max_stages), np.zeros(max_stages)
        e = np.array([self.eps_initial() if eps is None else eps])
        ns = self.L.orc_smc_run(C.byref(self.cfg), C.byref(self.data), self.b, P,
                                1 if init_prior else 0, stage0, max_stages, _p(e), _p(z), _p(K),
                                _p(lo), _p(ln), _p(logz), _p(bh), _p(zh), _p(eh))
        return dict(z=z, K=K, ll_old=lo, ll_new=ln, logz=logz[0], n_stages=ns, eps=e[0],
                    beta=bh[:ns], logz_hist=zh[:ns], ess=eh[:ns])


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox(_p(c), _p(k), _p(out))
    return out


def temper(ell, alpha, beta):
    ell = np.ascontiguousarray(ell, dtype=np.float64)
    P = ell.shape[0]
    bn, inc, ess = np.zeros(1), np.zeros(1), np.zeros(1)
    logw = np.zeros(P)
    lib().orc_temper(P, _p(ell), alpha, beta, _p(bn), _p(inc), _p(ess), _p(logw))
    return bn[0], inc[0], ess[0], logw


def u01(x):
    return lib().orc_u01(int(x))
