"""The C-ABI library builds for sm_103a, loads and exports what include/me.h
declares; host-only entry points behave (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_0806_0689_gb300 import build, me

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "me.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(me_[a-z_]+)\s*\(", text)))


def test_library_builds_and_exports_header():
    path = build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert "me_estimate" in declared and "me_init" in declared
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    # the binding knows every declared entry point
    assert sorted(me.EXPORTS) == declared


def test_binding_loads():
    L = me.load()
    assert L.me_estimate is not None


def test_stats_from_sums_host_arithmetic():
    L = me.load()
    st = me.Stats()
    sums = np.array([300, 900, 70, 3, 5 * 2 ** 24, 10, 100, 1], dtype=np.uint64)
    assert L.me_stats_from_sums(ctypes.c_void_p(sums.ctypes.data), ctypes.byref(st)) == me.ME_OK
    assert st.mad == 3.0 and st.mse == 9.0 and st.nsp == 7.0
    assert abs(st.psnr - 10 * np.log10(255.0 ** 2 / 9.0)) < 1e-12
    assert st.distance == 0.5 and st.probability == 0.3
    zero = np.array([0, 0, 0, 0, 0, 4, 64, 0], dtype=np.uint64)
    assert L.me_stats_from_sums(ctypes.c_void_p(zero.ctypes.data), ctypes.byref(st)) == me.ME_OK
    assert st.psnr == 100.0 and st.distance == 0.0
    bad = np.zeros(8, dtype=np.uint64)
    assert L.me_stats_from_sums(ctypes.c_void_p(bad.ctypes.data), ctypes.byref(st)) == me.ME_ERR_ARG


def test_null_context_is_rejected():
    L = me.load()
    assert L.me_estimate(None, None, None, 16, 16, 16, 7, 1, None, None, None, None) == me.ME_ERR_ARG
    assert L.me_estimate_batch(None, None, 0, 16, 1, None) == me.ME_ERR_ARG
    assert L.me_last_error(None) == b"null context"


def test_init_without_device_fails_loudly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    L = me.load()
    h = ctypes.c_void_p()
    assert L.me_init(ctypes.byref(h), 0, None) == me.ME_ERR_CUDA
    with pytest.raises(me.MeError):
        me.Context(0)
