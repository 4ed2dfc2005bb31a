"""The C-ABI library loads and exports every symbol include/bap.h declares; argument checks
that need no device (no compute call is made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_0805_1827_gb300 as bap
from bap_workloads import spec_max_call

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "bap.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(bap_[a-z0-9_]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["bap_create", "bap_fit_boundary", "bap_fit_classifier", "bap_price",
              "bap_debug_continuation", "bap_destroy", "bap_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    L = bap.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert set(bap.EXPORTED) <= set(_declared())
    assert "sm_103a" in bap.version()


def test_rejects_bad_models_before_touching_a_device():
    L = bap.lib()
    spec = spec_max_call(2, 90.0)
    bad_rho = np.array([[1.0, 0.5], [0.4, 1.0]])
    keep = [np.ascontiguousarray(a, dtype=np.float64) for a in
            (spec.S0, spec.sigma, spec.delta, bad_rho)]
    dp = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    m = bap._Model(2, dp(keep[0]), dp(keep[1]), dp(keep[2]), dp(keep[3]), 0.05, 100.0, 3.0, 9,
                   None, 0, None)
    h = ctypes.c_void_p()
    assert L.bap_create(ctypes.byref(m), ctypes.byref(h)) == bap.BAP_EINVAL
    assert b"symmetric" in L.bap_last_error()
    m.rho = dp(np.ascontiguousarray(spec.rho))
    m.d = 11
    assert L.bap_create(ctypes.byref(m), ctypes.byref(h)) == bap.BAP_EINVAL
    m.d = 2
    m.n_dates = 0
    assert L.bap_create(ctypes.byref(m), ctypes.byref(h)) == bap.BAP_EINVAL
    assert L.bap_create(None, ctypes.byref(h)) == bap.BAP_EINVAL


def test_rng_hook_rejects_bad_sizes():
    L = bap.lib()
    assert L.bap_debug_rng(0, 1, 0, 0, 0, 0, 10, None, None) == bap.BAP_EINVAL
    assert L.bap_debug_rng(0, 1, 0, 0, 0, 4, 0, None, None) == bap.BAP_EINVAL


def test_no_cpu_fallback_without_a_device():
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if has_gpu:
        pytest.skip("a CUDA device is present")
    with pytest.raises(bap.BapError) as e:
        bap.Option(spec_max_call(2, 90.0))
    assert e.value.status == bap.BAP_ECUDA
