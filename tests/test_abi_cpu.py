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


def test_workspace_bytes_and_config_validation():
    L = capi.lib()
    wl = synth.config2()
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


def test_create_rejects_misaligned_workspace_without_device_work():
    L = capi.lib()
    wl = synth.config1()
    cfg = make_config(wl, capi.FP64)
    cap = np.array([1024], dtype=np.int64)
    h = C.c_void_p()
    assert L.tsmc_create(C.byref(cfg), cap.ctypes.data, 0x1001, 1 << 30, None, C.byref(h)) == capi.EINVAL
    assert L.tsmc_create(C.byref(cfg), cap.ctypes.data, 0x100000, 16, None, C.byref(h)) == capi.ENOMEM
