"""Thin ctypes binding of ``libtsmc.so`` (the C ABI in ``include/tsmc.h``).

Argument marshalling only: every step of the sampler runs in the library's
CUDA kernels.  PyTorch supplies device memory (the workspace and I/O tensors)
and the CUDA stream.  ``lib()`` raises when the shared library is missing;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtsmc.so")
_lib = None

OK, EINVAL, ENOMEM, ECUDA, ENONFINITE, ETIMEOUT, ESTATE = 0, -1, -2, -3, -4, -5, -6
PULSE, SINUSOID, PULSE_LINAMP = 0, 1, 2
FP64, MIXED = 0, 1
SCHED_ROUNDS, SCHED_MIXTURE = 0, 1

# every entry point declared in include/tsmc.h, with its ctypes signature
P, I32, I64, D, U32, U64, SZ = (C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_uint32,
                               C.c_uint64, C.c_size_t)
SIGNATURES = {
    "tsmc_workspace_bytes": (I32, [P, P, P]),
    "tsmc_create": (I32, [P, P, P, SZ, P, P]),
    "tsmc_destroy": (I32, [P]),
    "tsmc_last_error": (C.c_char_p, [P]),
    "tsmc_set_problem": (I32, [P, I32, P, I64, D, D, D, P, P, U32]),
    "tsmc_set_fixed_components": (I32, [P, P]),
    "tsmc_init_population": (I32, [P]),
    "tsmc_set_population": (I32, [P, P, P, P, P]),
    "tsmc_get_population": (I32, [P, P, P, P, P]),
    "tsmc_eval_logl_grad": (I32, [P, P, P, P, P, P, P, P, P]),
    "tsmc_rj_move": (I32, [P, I32, I32, P]),
    "tsmc_nuts_move": (I32, [P, I32, I32, P, P, P]),
    "tsmc_set_kernel_params": (I32, [P, P, P]),
    "tsmc_get_kernel_params": (I32, [P, P, P]),
    "tsmc_build_birth_proposal": (I32, [P, I32]),
    "tsmc_get_birth_proposal": (I32, [P, I32, P, I64]),
    "tsmc_update_metric": (I32, [P]),
    "tsmc_temper_reweight_resample": (I32, [P, I32, P, P, P]),
    "tsmc_get_state": (I32, [P, P, P, P]),
    "tsmc_get_ancestors": (I32, [P, P]),
    "tsmc_run_stage": (I32, [P, I32, I32, P, P, P]),
    "tsmc_assimilate": (I32, [P, I32, P, I64]),
    "tsmc_philox": (I32, [P, P, U64, U64, I64, P]),
    "tsmc_counters": (I32, [P, P, P, I32]),
    "tsmc_profile": (I32, [P, I32]),
    "tsmc_profile_read": (I32, [P, P, P, I32]),
    "tsmc_resample_systematic_static": (I32, [P, I32, I32, U64, I32, P, P]),
    "tsmc_temper_resample_global": (I32, [P, I32, P, P]),
    "tsmc_load_population": (I32, [P, P, P, P, P]),
    "tsmc_metric_sums": (I32, [P, P]),
    "tsmc_metric_apply": (I32, [P, P]),
    "tsmc_mutation_rounds": (I32, [P, I32, P]),
    "tsmc_eps_update_apply": (I32, [P, P]),
    "tsmc_sync": (I32, [P]),
}

KERNEL_CLASSES = ("eval", "rj", "nuts", "temper", "resample", "gather", "metric", "other")


class Config(C.Structure):
    _fields_ = [
        ("model", C.c_int32), ("precision", C.c_int32), ("schedule", C.c_int32),
        ("n_problems", C.c_int32), ("particles", C.c_int32), ("kmax", C.c_int32),
        ("n_mut", C.c_int32), ("max_depth", C.c_int32), ("alpha", C.c_double),
        ("p_nuts", C.c_double), ("p_birth", C.c_double), ("p_death", C.c_double),
        ("amp_mean", C.c_double), ("amp_sd", C.c_double), ("seed", C.c_uint64),
        ("threads", C.c_int32), ("samples_per_thread", C.c_int32),
        ("pulse_window", C.c_int32), ("kmin", C.c_int32),
        ("birth_proposal", C.c_int32), ("birth_prior_weight", C.c_double),
        ("channels", C.c_int32), ("response", C.c_double * 4),
        ("problem_base", C.c_int32), ("fused_rounds", C.c_int32),
        ("particles_global", C.c_int32), ("particle_base", C.c_int32),
        ("wrap_mask", C.c_uint32),
    ]


class TsmcError(RuntimeError):
    pass


def lib():
    """Load libtsmc.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise TsmcError(f"libtsmc.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(t):
    """Device or host pointer of a torch tensor or numpy array (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _check_device_array(name, t, dtype, n):
    """t must be a contiguous CUDA tensor of dtype on the current device with >= n elements
    (the C side cannot check the size of a device buffer)."""
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if t.device.index != torch.cuda.current_device():
        raise ValueError(f"{name} is on {t.device}, not the current device")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} elements, needs {n}")


def resample_systematic_static(logw, n_problems, particles, seed, stage, ancestors, stream):
    """Allocation-free systematic resampling (static device scratch); see include/tsmc.h."""
    import torch

    n = int(n_problems) * int(particles)
    if n_problems >= 1 and particles >= 1:   # sizes themselves are checked by the library
        _check_device_array("logw", logw, torch.float64, n)
        _check_device_array("ancestors", ancestors, torch.int32, n)
    L = lib()
    st = L.tsmc_resample_systematic_static(_ptr(logw), n_problems, particles, seed, stage,
                                           _ptr(ancestors), stream.cuda_stream)
    if st != OK:
        msg = L.tsmc_last_error(None)
        raise TsmcError(f"tsmc error {st}: {msg.decode() if msg else ''}")


class Context:
    """Owns a tsmc context, its workspace tensor and the stream it launches on."""

    def __init__(self, cfg: Config, n_capacity, device="cuda", stream=None):
        import torch

        self.torch = torch
        self.cfg = cfg
        self.L = lib()
        cap = np.ascontiguousarray(n_capacity, dtype=np.int64)
        nbytes = C.c_size_t(0)
        self._check(self.L.tsmc_workspace_bytes(C.byref(cfg), _ptr(cap), C.byref(nbytes)), None)
        self.ws = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=device)
        base = self.ws.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        h = C.c_void_p()
        self._check(self.L.tsmc_create(C.byref(cfg), _ptr(cap), self._ws_ptr, int(nbytes.value),
                                       self.stream.cuda_stream, C.byref(h)), None)
        self.h = h
        self.D = {PULSE: 3, SINUSOID: 4, PULSE_LINAMP: 1}[cfg.model]
        self.P_total = cfg.n_problems * cfg.particles

    def _check(self, st, h="self"):
        if st != OK:
            hh = self.h if h == "self" else None
            msg = self.L.tsmc_last_error(hh)
            raise TsmcError(f"tsmc error {st}: {msg.decode() if msg else ''}")

    def close(self):
        if getattr(self, "h", None):
            self.L.tsmc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- problem data ----
    def set_problem(self, b, d, t_origin, dt, sigma, lo=(0, 0, 0, 0), hi=(1, 1, 1, 1), logmask=0):
        d = np.ascontiguousarray(d, dtype=np.float64)
        lo = np.ascontiguousarray(lo, dtype=np.float64)
        hi = np.ascontiguousarray(hi, dtype=np.float64)
        self._check(self.L.tsmc_set_problem(self.h, b, _ptr(d), d.shape[0], t_origin, dt, sigma,
                                            _ptr(lo), _ptr(hi), logmask))

    def set_fixed_components(self, tw):
        tw = np.ascontiguousarray(tw, dtype=np.float64)
        self._check(self.L.tsmc_set_fixed_components(self.h, _ptr(tw)))

    # ---- population ----
    def init_population(self):
        self._check(self.L.tsmc_init_population(self.h))

    def set_population(self, z, K, beta=None, logz=None):
        b = None if beta is None else np.ascontiguousarray(beta, dtype=np.float64)
        lz = None if logz is None else np.ascontiguousarray(logz, dtype=np.float64)
        self._check(self.L.tsmc_set_population(self.h, _ptr(z), _ptr(K), _ptr(b), _ptr(lz)))

    def get_population(self):
        t = self.torch
        dev = self.ws.device
        z = t.empty((self.P_total, self.cfg.kmax, self.D), dtype=t.float64, device=dev)
        K = t.empty(self.P_total, dtype=t.int32, device=dev)
        lo = t.empty(self.P_total, dtype=t.float64, device=dev)
        ln = t.empty(self.P_total, dtype=t.float64, device=dev)
        self._check(self.L.tsmc_get_population(self.h, _ptr(z), _ptr(K), _ptr(lo), _ptr(ln)))
        self.sync()
        return z, K, lo, ln

    def eval(self, z, K, beta=None, grad=False, fisher=False, ll_old=None, ll_new=None, logp=None,
             g=None, fis=None):
        t = self.torch
        dev = z.device
        n = z.shape[0]
        ll_old = ll_old if ll_old is not None else t.empty(n, dtype=t.float64, device=dev)
        ll_new = ll_new if ll_new is not None else t.empty(n, dtype=t.float64, device=dev)
        logp = logp if logp is not None else t.empty(n, dtype=t.float64, device=dev)
        if grad and g is None:
            g = t.empty_like(z)
        if fisher and fis is None:
            fis = t.empty((n, self.D), dtype=t.float64, device=dev)
        self._check(self.L.tsmc_eval_logl_grad(self.h, _ptr(z), _ptr(K), _ptr(beta), _ptr(ll_old),
                                               _ptr(ll_new), _ptr(logp), _ptr(g) if grad else None,
                                               _ptr(fis) if fisher else None))
        return ll_old, ll_new, logp, g, fis

    def rj_move(self, stage, rnd, outcome=None):
        self._check(self.L.tsmc_rj_move(self.h, stage, rnd, _ptr(outcome)))

    def nuts_move(self, stage, rnd, acc=None, nleaf=None, flags=None):
        self._check(self.L.tsmc_nuts_move(self.h, stage, rnd, _ptr(acc), _ptr(nleaf), _ptr(flags)))

    def set_kernel_params(self, eps=None, minv=None):
        e = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
        m = None if minv is None else np.ascontiguousarray(minv, dtype=np.float64)
        self._check(self.L.tsmc_set_kernel_params(self.h, _ptr(e), _ptr(m)))

    def get_kernel_params(self):
        e = np.zeros(self.cfg.n_problems)
        m = np.zeros((self.cfg.n_problems, self.D))
        self._check(self.L.tsmc_get_kernel_params(self.h, _ptr(e), _ptr(m)))
        return e, m

    def update_metric(self):
        self._check(self.L.tsmc_update_metric(self.h))

    def build_birth_proposal(self, stage):
        self._check(self.L.tsmc_build_birth_proposal(self.h, stage))

    def get_birth_proposal(self, problem=0):
        """(m, h[4], centres [m][D]) of the population birth proposal of one problem."""
        out = np.zeros(5 + 256 * self.D)
        self._check(self.L.tsmc_get_birth_proposal(self.h, problem, _ptr(out), out.size))
        m = int(out[0])
        return m, out[1:5].copy(), out[5:].reshape(256, self.D)[:m].copy()

    def temper_reweight_resample(self, stage):
        b, lz, e = (np.zeros(self.cfg.n_problems) for _ in range(3))
        self._check(self.L.tsmc_temper_reweight_resample(self.h, stage, _ptr(b), _ptr(lz), _ptr(e)))
        return b, lz, e

    def temper_state(self):
        """(beta, log Z, last ESS) per problem."""
        b, lz, e = (np.zeros(self.cfg.n_problems) for _ in range(3))
        self._check(self.L.tsmc_get_state(self.h, _ptr(b), _ptr(lz), _ptr(e)))
        return b, lz, e

    def get_ancestors(self):
        a = self.torch.empty(self.P_total, dtype=self.torch.int32, device=self.ws.device)
        self._check(self.L.tsmc_get_ancestors(self.h, _ptr(a)))
        self.sync()
        return a

    def run_stage(self, stage, use_graph=True, read=True):
        """One stage; read=False queues it without synchronising (returns None)."""
        if not read:
            self._check(self.L.tsmc_run_stage(self.h, stage, 1 if use_graph else 0, None, None,
                                              None))
            return None
        b, lz, e = (np.zeros(self.cfg.n_problems) for _ in range(3))
        self._check(self.L.tsmc_run_stage(self.h, stage, 1 if use_graph else 0, _ptr(b), _ptr(lz),
                                          _ptr(e)))
        return b, lz, e

    def assimilate(self, b, d_new):
        d = np.ascontiguousarray(d_new, dtype=np.float64)
        self._check(self.L.tsmc_assimilate(self.h, b, _ptr(d), d.shape[0]))

    def philox(self, ctr, key0, key1):
        t = self.torch
        c = t.as_tensor(np.ascontiguousarray(ctr, dtype=np.uint64).view(np.int64),
                        device=self.ws.device)
        out = t.empty_like(c)
        self._check(self.L.tsmc_philox(self.h, _ptr(c), key0, key1, c.shape[0] // 4, _ptr(out)))
        self.sync()
        return out.cpu().numpy().view(np.uint64)

    def counters(self, reset=False):
        """((batched cs, NUTS cs, batched cs computed, NUTS cs computed), kernels launched)."""
        cs = np.zeros(4, dtype=np.uint64)
        n = C.c_int64(0)
        self._check(self.L.tsmc_counters(self.h, _ptr(cs), C.byref(n), 1 if reset else 0))
        return tuple(int(x) for x in cs), int(n.value)

    def profile(self, enable=True, events=0):
        """Per-kernel-class event timing; events > 0 pre-creates that many events."""
        self._check(self.L.tsmc_profile(self.h, max(int(events), 1) if enable else 0))

    def profile_read(self, reset=True):
        n = np.zeros(8, dtype=np.int64)
        ms = np.zeros(8)
        self._check(self.L.tsmc_profile_read(self.h, _ptr(n), _ptr(ms), 1 if reset else 0))
        return {k: (int(n[i]), float(ms[i])) for i, k in enumerate(KERNEL_CLASSES)}

    # ---- a population sharded across processes (see include/tsmc.h) ----
    def temper_resample_global(self, stage, ell, anc):
        self._check(self.L.tsmc_temper_resample_global(self.h, stage, _ptr(ell), _ptr(anc)))

    def load_population(self, z, K, ll_old, ll_new):
        self._check(self.L.tsmc_load_population(self.h, _ptr(z), _ptr(K), _ptr(ll_old),
                                                _ptr(ll_new)))

    def metric_sums(self, sums):
        self._check(self.L.tsmc_metric_sums(self.h, _ptr(sums)))

    def metric_apply(self, sums):
        self._check(self.L.tsmc_metric_apply(self.h, _ptr(sums)))

    def mutation_rounds(self, stage, stats):
        self._check(self.L.tsmc_mutation_rounds(self.h, stage, _ptr(stats)))

    def eps_update_apply(self, stats):
        self._check(self.L.tsmc_eps_update_apply(self.h, _ptr(stats)))

    def sync(self):
        self._check(self.L.tsmc_sync(self.h))
