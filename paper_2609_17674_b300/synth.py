"""Seeded synthetic workloads: injected data sets and frozen particle populations.

This module is the only thing the CUDA path and the oracle share.  It holds
no step of the sampler: it draws injection parameters, simulates the observed
data d_n = sum_k h(t_n; theta_k) + sigma * noise, and builds frozen particle
populations for benchmarks.  Both sides receive its arrays as plain inputs.

The workloads stand in for the paper's two applications (Sec. 5.1: a sequence
of Gaussian pulses; Sec. 5.2: Galactic binaries, simplified to one time-domain
channel of quasi-monochromatic sinusoids), at the five sizes the benchmark and
the tests use.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

PULSE, SINUSOID, PULSE_LINAMP = 0, 1, 2
SCHED_ROUNDS, SCHED_MIXTURE = 0, 1
MODEL_D = {PULSE: 3, SINUSOID: 4, PULSE_LINAMP: 1}

# priors of the pulse model: A ~ U[0.5,2], t0 ~ U[0.05,0.95], w ~ logU[0.005,0.05]
PULSE_LO = (0.5, 0.05, 0.005, 0.0)
PULSE_HI = (2.0, 0.95, 0.05, 0.0)
PULSE_LOGMASK = 0b100
# sinusoid: f ~ U[3.000, 3.005] mHz, fdot ~ U[0, 1e-16] Hz/s, phi0 ~ U[0, 2pi)
GB_F_LO, GB_F_HI = 3.000e-3, 3.005e-3
GB_FDOT_HI = 1e-16


@dataclasses.dataclass
class Problem:
    d: np.ndarray            # float64 samples
    t_origin: float
    dt: float
    sigma: float
    n1: int = 0              # first not-yet-assimilated sample
    truth: Optional[np.ndarray] = None   # [K_true][D] injected parameters
    lo: Optional[tuple] = None           # per-problem prior bounds (sinusoid bands)
    hi: Optional[tuple] = None

    @property
    def n(self) -> int:
        return int(self.d.shape[0])


@dataclasses.dataclass
class Workload:
    name: str
    model: int
    kmax: int
    P: int                    # particles per problem
    problems: List[Problem]
    lo: tuple = (0.0, 0.0, 0.0, 0.0)
    hi: tuple = (0.0, 0.0, 0.0, 0.0)
    logmask: int = 0
    n_mut: int = 5
    max_depth: int = 6
    alpha: float = 0.5
    p_nuts: float = 0.0
    p_birth: float = 0.5
    p_death: float = 0.5
    schedule: int = SCHED_ROUNDS
    seed: int = 0
    amp_mean: float = 1.0
    amp_sd: float = 1.0
    fixed_tw: Optional[np.ndarray] = None   # LINAMP: [kmax][2]
    kmin: int = 0             # K prior U{kmin..kmax}
    birth_proposal: int = 0   # 0: births from the prior; 1: population mixture
    birth_prior_weight: float = 0.2   # prior weight of the population mixture
    channels: int = 1         # sinusoids: 2 = channels A and E, data [A samples, E samples]
    resp: tuple = (1.0, 0.0, 1.0, 0.0)   # (r_A, delta_A, r_E, delta_E)
    problem_base: int = 0     # index of problems[0] in a larger set (a shard of it)
    wrapmask: int = 0         # bit d: parameter d is periodic on [lo, hi) (a phase)

    @property
    def D(self) -> int:
        return MODEL_D[self.model]

    def bounds(self, b: int):
        """Prior bounds for problem b (sinusoid bands carry their own)."""
        pr = self.problems[b]
        return (pr.lo or self.lo, pr.hi or self.hi)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


def _pulse_signal(t, truth):
    s = np.zeros_like(t)
    for A, t0, w in truth:
        s += A * np.exp(-((t - t0) ** 2) / (2.0 * w * w))
    return s


def _sin_phase(t, f, fd, p0):
    return 2.0 * math.pi * f * t + math.pi * fd * t * t + p0


def pulse_problem(rng, n, k_true, sigma=0.1, span_n=None, noise=True) -> Problem:
    """Pulses on t_n = n / span_n (span_n defaults to n): A, t0, w from the priors."""
    span_n = span_n or n
    u = rng.random((k_true, 3))
    A = PULSE_LO[0] + (PULSE_HI[0] - PULSE_LO[0]) * u[:, 0]
    t0 = PULSE_LO[1] + (PULSE_HI[1] - PULSE_LO[1]) * u[:, 1]
    w = np.exp(math.log(PULSE_LO[2]) + (math.log(PULSE_HI[2]) - math.log(PULSE_LO[2])) * u[:, 2])
    truth = np.stack([A, t0, w], axis=1)
    t = np.arange(n, dtype=np.float64) / span_n
    d = _pulse_signal(t, truth)
    if noise:
        d = d + sigma * rng.standard_normal(n)
    return Problem(d=d, t_origin=0.0, dt=1.0 / span_n, sigma=sigma, truth=truth)


def gb_amp_bounds(n, dt, sigma, f_c):
    """log-uniform amplitude prior on [A(rho=5), A(rho=60)], A(rho) = rho sigma / ||cos||."""
    t = np.arange(n, dtype=np.float64) * dt
    norm = math.sqrt(float(np.sum(np.cos(2.0 * math.pi * f_c * t) ** 2)))
    return 5.0 * sigma / norm, 60.0 * sigma / norm


def sinusoid_problem(rng, n, k_true, dt=15.0, sigma=1.0, f_lo=GB_F_LO, f_hi=GB_F_HI,
                     noise=True) -> Problem:
    """Quasi-monochromatic sinusoids with per-source SNR ~ U[10, 40] (time-domain rho); white
    noise of level sigma unless noise=False (the paper's example data are noise-free)."""
    t = np.arange(n, dtype=np.float64) * dt
    f = f_lo + (f_hi - f_lo) * rng.random(k_true)
    fd = GB_FDOT_HI * rng.random(k_true)
    p0 = 2.0 * math.pi * rng.random(k_true)
    rho = 10.0 + 30.0 * rng.random(k_true)
    d = np.zeros(n)
    A = np.empty(k_true)
    for k in range(k_true):
        c = np.cos(_sin_phase(t, f[k], fd[k], p0[k]))
        A[k] = rho[k] * sigma / math.sqrt(float(np.sum(c * c)))
        d += A[k] * c
    noise_draw = rng.standard_normal(n)   # drawn either way: the stream is the same
    if noise:
        d = d + sigma * noise_draw
    a_lo, a_hi = gb_amp_bounds(n, dt, sigma, 0.5 * (f_lo + f_hi))
    truth = np.stack([A, f, fd, p0], axis=1)
    return Problem(d=d, t_origin=0.0, dt=dt, sigma=sigma, truth=truth,
                   lo=(a_lo, f_lo, 0.0, 0.0), hi=(a_hi, f_hi, GB_FDOT_HI, 2.0 * math.pi))


# Two noise-orthogonal channels A and E (Sec. 5.2), flat PSD, noise-free: channel c sees
# r_c A cos(phi(t) + delta_c).  The simplified synthetic response used here (the real one
# needs the LISA response, not available) gives E 0.8 of A's sensitivity in quadrature.
AE_RESP = (1.0, 0.0, 0.8, 0.5 * math.pi)


def ae_problem(rng, n, k_true, dt=15.0, sigma=1.0, f_lo=GB_F_LO, f_hi=GB_F_HI,
               resp=AE_RESP, noise=False) -> Problem:
    """Two-channel sinusoids, noise-free, rho^2 = sum_c (h_c | h_c) ~ U[10, 40]^2 per source
    (flat PSD: the frequency-domain inner product equals sum_n a_n b_n / sigma^2 with
    sigma^2 = S / (2 dt)); data [channel A samples, channel E samples]."""
    t = np.arange(n, dtype=np.float64) * dt
    f = f_lo + (f_hi - f_lo) * rng.random(k_true)
    fd = GB_FDOT_HI * rng.random(k_true)
    p0 = 2.0 * math.pi * rng.random(k_true)
    rho = 10.0 + 30.0 * rng.random(k_true)
    d = np.zeros(2 * n)
    A = np.empty(k_true)
    for k in range(k_true):
        ca = resp[0] * np.cos(_sin_phase(t, f[k], fd[k], p0[k] + resp[1]))
        ce = resp[2] * np.cos(_sin_phase(t, f[k], fd[k], p0[k] + resp[3]))
        A[k] = rho[k] * sigma / math.sqrt(float(np.sum(ca * ca) + np.sum(ce * ce)))
        d[:n] += A[k] * ca
        d[n:] += A[k] * ce
    if noise:   # white noise of the flat PSD (the paper's example is noise-free)
        d = d + sigma * rng.standard_normal(2 * n)
    a_lo, a_hi = gb_amp_bounds(n, dt, sigma, 0.5 * (f_lo + f_hi))
    truth = np.stack([A, f, fd, p0], axis=1)
    return Problem(d=d, t_origin=0.0, dt=dt, sigma=sigma, truth=truth,
                   lo=(a_lo, f_lo, 0.0, 0.0), hi=(a_hi, f_hi, GB_FDOT_HI, 2.0 * math.pi))


def ae_workload(name, n, k_true, kmax, P, seed, resp=AE_RESP, noise=False, **kw) -> Workload:
    """Galactic-binary band in channels A and E (n samples per channel)."""
    rng = _rng(seed)
    pr = ae_problem(rng, n, k_true, resp=resp, noise=noise)
    return Workload(name=name, model=SINUSOID, kmax=kmax, P=P, problems=[pr], lo=pr.lo,
                    hi=pr.hi, logmask=0b0001, seed=seed, channels=2, resp=tuple(resp), **kw)


def pulse_workload(name, n, k_true, kmax, P, seed, sigma=0.1, n_problems=1, **kw) -> Workload:
    rng = _rng(seed)
    probs = [pulse_problem(rng, n, k_true, sigma) for _ in range(n_problems)]
    return Workload(name=name, model=PULSE, kmax=kmax, P=P, problems=probs, lo=PULSE_LO,
                    hi=PULSE_HI, logmask=PULSE_LOGMASK, seed=seed, **kw)


def sinusoid_workload(name, n, k_true, kmax, P, seed, noise=True, **kw) -> Workload:
    rng = _rng(seed)
    pr = sinusoid_problem(rng, n, k_true, noise=noise)
    return Workload(name=name, model=SINUSOID, kmax=kmax, P=P, problems=[pr], lo=pr.lo,
                    hi=pr.hi, logmask=0b0001, seed=seed, **kw)


# ---------------------------------------------------------------------------
# The five benchmark workloads (data seeds 1001 to 1005)
# ---------------------------------------------------------------------------
def pulse_n1024_k3(seed=1001) -> Workload:
    """Gaussian-pulse sum, N=1024 on [0,1], K_true=3, sigma=0.1, K~U{0..10}, P=512."""
    return pulse_workload("pulse_n1024_k3_p512", 1024, 3, 10, 512, seed)


def pulse_k20(seed=1002, P=8192, n=16384) -> Workload:
    """Gaussian-pulse sum at scale: N=16384, K_true=20, K_max=40, P=8192."""
    return pulse_workload(f"pulse_n{n}_k20_p{P}", n, 20, 40, P, seed)


def gb_band_k10(seed=1003, P=4096, n=1 << 18) -> Workload:
    """Galactic-binary band: N=2^18 at dt=15 s, sigma=1, K_true=10, K_max=30, P=4096."""
    return sinusoid_workload(f"gb_n{n}_k10_p{P}", n, 10, 30, P, seed)


def assimilation_pulse_k14(seed=1004, P=16384, n_full=1 << 19) -> Workload:
    """Assimilation: pulses on t_n = n/2^19, K_true=14, data arrive as 2^17, 2^18, 2^19."""
    rng = _rng(seed)
    pr = pulse_problem(rng, n_full, 14, 0.1, span_n=n_full)
    return Workload(name=f"assim_pulse_n{n_full}_k14_p{P}", model=PULSE, kmax=40, P=P,
                    problems=[pr], lo=PULSE_LO, hi=PULSE_HI, logmask=PULSE_LOGMASK, seed=seed)


# The paper's own pulse example (Sec. 5.1): 10 Gaussian pulses in 200 s of noise-free data,
# uniform priors on (A, mu, width) that also serve as the birth proposal, K in [1, 10],
# 6000 particles, alpha = 0.9, mixture moves NUTS / birth / death = 0.6 / 0.2 / 0.2, and data
# arriving in segments 20 s longer each time.  Not given there, so chosen here: 10 samples per
# second, a likelihood sigma of 0.05, A in [0.5, 2], width in [1, 6] s, and the injected
# values below (one pulse near 150 s, as in its segment-count discussion).
PAPER_PULSE_LO = (0.5, 0.0, 1.0, 0.0)
PAPER_PULSE_HI = (2.0, 200.0, 6.0, 0.0)
PAPER_PULSE_MU = (14.0, 31.0, 47.0, 63.0, 79.0, 96.0, 112.0, 127.0, 151.0, 178.0)


def paper_pulse_workload(P=6000, seed=2001, rate=10.0, sigma=0.05, n_mut=5) -> Workload:
    """Noise-free 10-pulse signal on t_n = n / rate, n < 200 rate."""
    rng = _rng(seed)
    k = len(PAPER_PULSE_MU)
    A = PAPER_PULSE_LO[0] + (PAPER_PULSE_HI[0] - PAPER_PULSE_LO[0]) * rng.random(k)
    w = 1.5 + 3.0 * rng.random(k)
    truth = np.stack([A, np.array(PAPER_PULSE_MU), w], axis=1)
    n = int(round(200.0 * rate))
    t = np.arange(n, dtype=np.float64) / rate
    pr = Problem(d=_pulse_signal(t, truth), t_origin=0.0, dt=1.0 / rate, sigma=sigma, truth=truth)
    return Workload(name=f"paper_pulses_200s_p{P}", model=PULSE, kmax=k, P=P, problems=[pr],
                    lo=PAPER_PULSE_LO, hi=PAPER_PULSE_HI, logmask=0, n_mut=n_mut, max_depth=6,
                    alpha=0.9, p_nuts=0.6, p_birth=0.2, p_death=0.2, schedule=SCHED_MIXTURE,
                    seed=seed, kmin=1)


def gb_bands(seed=1005, n_bands=64, P=2048, log2n=(14, 18)) -> Workload:
    """64 independent GB bands with disjoint 5 uHz windows, N_b = round(2^U[14,18])."""
    rng = _rng(seed)
    probs = []
    for b in range(n_bands):
        n = int(round(2.0 ** rng.uniform(*log2n)))
        k_true = int(rng.integers(1, 16))
        f_lo = GB_F_LO + 5e-6 * b
        probs.append(sinusoid_problem(rng, n, k_true, f_lo=f_lo, f_hi=f_lo + 5e-6))
    return Workload(name=f"gb_batched_{n_bands}x{P}", model=SINUSOID, kmax=30, P=P,
                    problems=probs, lo=probs[0].lo, hi=probs[0].hi, logmask=0b0001, seed=seed)


def linamp_workload(n=256, k=3, P=256, seed=7, sigma=0.1, amp_mean=1.0, amp_sd=1.0) -> Workload:
    """Linear-Gaussian test model: fixed pulse positions/widths, Gaussian amplitude prior."""
    rng = _rng(seed)
    t0 = np.linspace(0.2, 0.8, k)
    w = np.full(k, 0.05)
    A = amp_mean + amp_sd * rng.standard_normal(k)
    t = np.arange(n, dtype=np.float64) / n
    d = _pulse_signal(t, np.stack([A, t0, w], 1)) + sigma * rng.standard_normal(n)
    pr = Problem(d=d, t_origin=0.0, dt=1.0 / n, sigma=sigma, truth=A[:, None])
    return Workload(name=f"linamp_n{n}_k{k}", model=PULSE_LINAMP, kmax=k, P=P, problems=[pr],
                    amp_mean=amp_mean, amp_sd=amp_sd, fixed_tw=np.stack([t0, w], 1), seed=seed)


# ---------------------------------------------------------------------------
# Frozen populations (benchmarks and parity cases)
# ---------------------------------------------------------------------------
def _logit(u):
    return np.log(u) - np.log1p(-u)


def prior_population(wl: Workload, seed: int, P_total: Optional[int] = None):
    """K ~ U{kmin..kmax}; every coordinate z ~ logistic (theta ~ its prior)."""
    rng = _rng(seed)
    P_total = P_total or wl.P * len(wl.problems)
    K = rng.integers(wl.kmin, wl.kmax + 1, size=P_total).astype(np.int32)
    u = rng.random((P_total, wl.kmax, wl.D)).clip(1e-12, 1 - 1e-12)
    z = _logit(u)
    for d in range(wl.D):
        if wl.wrapmask >> d & 1:          # periodic: z is the position on one period
            z[..., d] = u[..., d]
    z[np.arange(wl.kmax)[None, :] >= K[:, None]] = 0.0
    return z, K


def theta_to_z(wl: Workload, b: int, theta: np.ndarray) -> np.ndarray:
    """Inverse coordinate map, used only to place frozen populations near the injection."""
    lo, hi = wl.bounds(b)
    z = np.empty_like(theta)
    for d in range(wl.D):
        if wl.logmask >> d & 1:
            u = (np.log(theta[..., d]) - math.log(lo[d])) / (math.log(hi[d]) - math.log(lo[d]))
        else:
            u = (theta[..., d] - lo[d]) / (hi[d] - lo[d])
        if wl.wrapmask >> d & 1:
            z[..., d] = u - np.floor(u)
        else:
            z[..., d] = _logit(np.clip(u, 1e-9, 1 - 1e-9))
    return z


def posterior_like_population(wl: Workload, seed: int):
    """K_p = K_true + U{-1,0,1} (clipped), components = injected values + 1% jitter."""
    rng = _rng(seed)
    zs, Ks = [], []
    for b, pr in enumerate(wl.problems):
        kt = pr.truth.shape[0]
        K = np.clip(kt + rng.integers(-1, 2, size=wl.P), 0, min(wl.kmax, kt)).astype(np.int32)
        z = np.zeros((wl.P, wl.kmax, wl.D))
        ztrue = theta_to_z(wl, b, pr.truth)
        for i in range(wl.P):
            perm = rng.permutation(kt)[: K[i]]
            z[i, : K[i]] = ztrue[perm] * (1.0 + 0.01 * rng.standard_normal((K[i], wl.D)))
        zs.append(z)
        Ks.append(K)
    return np.concatenate(zs), np.concatenate(Ks)
