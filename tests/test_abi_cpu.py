"""Host-only checks of the C ABI: the library loads, exports every declared entry
point, and validates configurations without touching a GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2609_17674_b300 import capi, synth
from paper_2609_17674_b300.sampler import make_config

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tsmc.h")).read()
    return sorted(set(re.findall(r"^(?:tsmc_status|const char\*)\s+(tsmc_\w+)\(", src, re.M)))


def test_library_exports_every_declared_symbol():
    L = capi.lib()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(capi.SIGNATURES)


def test_header_is_plain_c_with_a_typed_context(tmp_path):
    """The header compiles as C11; the context handle is an opaque struct pointer, so
    passing any other pointer where a context is expected is a compile error."""
    import subprocess

    inc = os.path.join(ROOT, "include")
    good = tmp_path / "good.c"
    good.write_text('#include "tsmc.h"\n'
                    'int f(tsmc_ctx* c) { return (int)tsmc_sync(c) + (int)tsmc_destroy(c); }\n')
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I", inc, "-c", str(good),
                           "-o", str(tmp_path / "good.o")])
    bad = tmp_path / "bad.c"
    bad.write_text('#include "tsmc.h"\n'
                   'int f(tsmc_config* c) { return (int)tsmc_sync(c); }\n')
    r = subprocess.run(["gcc", "-std=c11", "-Werror=incompatible-pointer-types", "-I", inc,
                        "-c", str(bad), "-o", str(tmp_path / "bad.o")], capture_output=True)
    assert r.returncode != 0


def test_workspace_bytes_and_config_validation():
    L = capi.lib()
    wl = synth.pulse_k20()
    cfg = make_config(wl, capi.MIXED)
    cap = np.array([wl.problems[0].n], dtype=np.int64)
    nb = C.c_size_t(0)
    assert L.tsmc_workspace_bytes(C.byref(cfg), cap.ctypes.data, C.byref(nb)) == capi.OK
    # two population copies of z dominate: 2 * P * kmax * D * 8 bytes
    assert nb.value >= 2 * 8192 * 40 * 3 * 8
    bad = make_config(wl, capi.MIXED)
    bad.kmax = 0
    assert L.tsmc_workspace_bytes(C.byref(bad), cap.ctypes.data, C.byref(nb)) == capi.EINVAL
    bad = make_config(wl, capi.MIXED)
    bad.max_depth = 11
    assert L.tsmc_workspace_bytes(C.byref(bad), cap.ctypes.data, C.byref(nb)) == capi.EINVAL
    bad = make_config(wl, capi.MIXED)
    bad.threads = 48
    assert L.tsmc_workspace_bytes(C.byref(bad), cap.ctypes.data, C.byref(nb)) == capi.EINVAL
    neg = np.array([-5], dtype=np.int64)
    assert L.tsmc_workspace_bytes(C.byref(cfg), neg.ctypes.data, C.byref(nb)) == capi.EINVAL


def test_particle_shard_configuration_rules():
    """particles_global: at least the local count, the local block inside it, no population
    birth proposal (it would be built from one shard); particle_base only when sharded."""
    L = capi.lib()
    wl = synth.pulse_n1024_k3()
    cap = np.array([1024], dtype=np.int64)
    nb = C.c_size_t(0)

    def status(**kw):
        cfg = make_config(wl, capi.FP64)
        for k, v in kw.items():
            setattr(cfg, k, v)
        return L.tsmc_workspace_bytes(C.byref(cfg), cap.ctypes.data, C.byref(nb))

    assert status(particles_global=2048, particle_base=1024) == capi.OK
    assert status(particles_global=256) == capi.EINVAL          # fewer than the local 512
    assert status(particles_global=1000, particle_base=600) == capi.EINVAL
    assert status(particle_base=5) == capi.EINVAL
    assert status(particles_global=2048, birth_proposal=1) == capi.EINVAL
    assert status(fused_rounds=2) == capi.EINVAL


def test_periodic_parameter_configuration_rules():
    """wrap_mask: bits below the model's D only; not with the linear-amplitude model or the
    population birth proposal (its kernel density is not periodic)."""
    L = capi.lib()
    cap = np.array([4096], dtype=np.int64)
    nb = C.c_size_t(0)

    def status(wl, **kw):
        cfg = make_config(wl, capi.MIXED)
        for k, v in kw.items():
            setattr(cfg, k, v)
        return L.tsmc_workspace_bytes(C.byref(cfg), cap.ctypes.data, C.byref(nb))

    ws = synth.sinusoid_workload("t", 4096, 3, 8, 64, 1)
    wp = synth.pulse_workload("t", 4096, 3, 8, 64, 1)
    assert status(ws, wrap_mask=0b1000) == capi.OK
    assert status(ws, wrap_mask=0b1111) == capi.OK
    assert status(ws, wrap_mask=0b10000) == capi.EINVAL        # sinusoids have 4 parameters
    assert status(wp, wrap_mask=0b100) == capi.OK
    assert status(wp, wrap_mask=0b1000) == capi.EINVAL         # pulses have 3
    assert status(ws, wrap_mask=0b1000, birth_proposal=1, birth_prior_weight=0.2) == capi.EINVAL
    assert status(synth.linamp_workload(), wrap_mask=1) == capi.EINVAL
    ws.wrapmask = 0b1000
    assert make_config(ws, capi.MIXED).wrap_mask == 0b1000


def test_create_rejects_misaligned_workspace_without_device_work():
    L = capi.lib()
    wl = synth.pulse_n1024_k3()
    cfg = make_config(wl, capi.FP64)
    cap = np.array([1024], dtype=np.int64)
    h = C.c_void_p()
    assert L.tsmc_create(C.byref(cfg), cap.ctypes.data, 0x1001, 1 << 30, None, C.byref(h)) == capi.EINVAL
    assert L.tsmc_create(C.byref(cfg), cap.ctypes.data, 0x100000, 16, None, C.byref(h)) == capi.ENOMEM


def _ws_status(cfg, n):
    cap = np.array([n], dtype=np.int64)
    nb = C.c_size_t(0)
    return capi.lib().tsmc_workspace_bytes(C.byref(cfg), cap.ctypes.data, C.byref(nb))


# (workload, field, value, expected status): every rule of the configuration check, with the
# values just inside each bound accepted
_PULSE = synth.pulse_n1024_k3
_AE = lambda: synth.ae_workload("t", 1024, 2, 4, 16, 1)   # noqa: E731
CFG_CASES = [
    (_PULSE, "model", 3, capi.EINVAL),
    (_PULSE, "precision", 2, capi.EINVAL),
    (_PULSE, "n_problems", 0, capi.EINVAL),
    (_PULSE, "particles", 0, capi.EINVAL),
    (_PULSE, "kmin", -1, capi.EINVAL),
    (_PULSE, "kmin", 11, capi.EINVAL),          # above kmax = 10
    (_PULSE, "kmin", 10, capi.OK),
    (_PULSE, "max_depth", 0, capi.EINVAL),
    (_PULSE, "max_depth", 10, capi.OK),
    (_PULSE, "n_mut", -1, capi.EINVAL),
    (_PULSE, "alpha", 0.0, capi.EINVAL),
    (_PULSE, "alpha", 1.5, capi.EINVAL),
    (_PULSE, "alpha", 1.0, capi.OK),
    (_PULSE, "threads", 16, capi.EINVAL),
    (_PULSE, "threads", 288, capi.EINVAL),
    (_PULSE, "threads", 256, capi.OK),
    (_PULSE, "threads", 32, capi.OK),
    (_PULSE, "samples_per_thread", 8, capi.EINVAL),
    (_PULSE, "samples_per_thread", 16, capi.OK),
    (_PULSE, "pulse_window", 2, capi.EINVAL),
    (_PULSE, "birth_proposal", 2, capi.EINVAL),
    (_PULSE, "channels", 2, capi.EINVAL),       # two channels are for sinusoids only
    (_PULSE, "channels", 3, capi.EINVAL),
    (_AE, "channels", 2, capi.OK),
]


@pytest.mark.parametrize("mk,field,value,want", CFG_CASES)
def test_config_rules(mk, field, value, want):
    wl = mk()
    cfg = make_config(wl, capi.MIXED)
    setattr(cfg, field, value)
    assert _ws_status(cfg, wl.problems[0].n) == want


def test_config_rules_birth_proposal_and_response():
    wl = synth.pulse_n1024_k3()
    cfg = make_config(wl, capi.MIXED)
    cfg.birth_proposal = 1
    for w, want in ((0.0, capi.EINVAL), (1.5, capi.EINVAL), (float("nan"), capi.EINVAL),
                    (1.0, capi.OK), (0.1, capi.OK)):
        cfg.birth_prior_weight = w
        assert _ws_status(cfg, 1024) == want, w
    ae = synth.ae_workload("t", 1024, 2, 4, 16, 1)
    for q, v in ((0, 0.0), (2, -1.0), (1, float("inf")), (3, float("nan"))):
        cfg = make_config(ae, capi.MIXED)
        cfg.response[q] = v
        assert _ws_status(cfg, 1024) == capi.EINVAL, (q, v)
    cfg = make_config(ae, capi.MIXED)
    cfg.schedule = capi.SCHED_ROUNDS     # birth and death both needed in every round
    cfg.p_birth = 0.0
    assert _ws_status(cfg, 1024) == capi.EINVAL


def test_make_config_maps_the_workload():
    ae = synth.ae_workload("t", 1024, 2, 4, 16, 1)
    cfg = make_config(ae, capi.FP64)
    assert cfg.channels == 2 and cfg.model == capi.SINUSOID
    assert list(cfg.response) == pytest.approx(list(ae.resp))
    pw = synth.paper_pulse_workload(P=600)
    cfg = make_config(pw, capi.MIXED)
    assert cfg.kmin == 1 and cfg.kmax == pw.kmax and cfg.particles == 600
    assert cfg.schedule == capi.SCHED_MIXTURE     # the paper's mixture of moves
    assert cfg.alpha == pytest.approx(0.9)


def test_sample_capacity_bounds():
    """Capacities in [1, 2^24] (sample indices exact in FP32 and 32-bit in the loops)."""
    cfg = make_config(synth.pulse_n1024_k3(), capi.MIXED)
    for n, want in ((1, capi.OK), (1 << 24, capi.OK), ((1 << 24) + 1, capi.EINVAL),
                    (0, capi.EINVAL)):
        assert _ws_status(cfg, n) == want, n
