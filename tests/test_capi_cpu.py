"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/*.h declares, and rejects bad arguments before any
CUDA call."""
from __future__ import annotations

import ctypes
import glob
import os
import re

import numpy as np
import pytest

import __graft_entry__
from paper_2105_06676_gb300 import _capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return _capi.lib()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(stencil_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_core_entry_points():
    names = declared_functions()
    for core in ("stencil_plan", "stencil_run", "stencil_destroy", "stencil_status",
                 "stencil_strerror", "stencil_symbol_power", "stencil_run_host"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_cover_header():
    bound = {name for name, _, _ in _capi.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_strerror_names_every_code(lib):
    for code, name in _capi.STATUS.items():
        msg = lib.stencil_strerror(code)
        assert msg and msg.decode() != "unknown status code", name
    assert lib.stencil_strerror(12345).decode() == "unknown status code"


def _plan(lib, dims, radius, boundary=0, precision=1, weights=None):
    d = (ctypes.c_int64 * len(dims))(*dims)
    if weights is None:
        weights = np.full(max(1, 2 * radius + 1) ** len(dims), 0.1)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    h = ctypes.c_void_p()
    rc = lib.stencil_plan(ctypes.byref(h), len(dims), d, radius,
                          w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), boundary, precision)
    return rc, h


@pytest.mark.parametrize("dims,radius,boundary,precision,code", [
    ((), 1, 0, 1, -1),                  # ndim 0
    ((8, 8, 8, 8), 1, 0, 1, -1),        # ndim 4
    ((16,), -1, 0, 1, -1),              # negative radius
    ((16,), 4, 0, 1, -1),               # radius above the supported maximum
    ((16,), 1, 3, 1, -1),               # unknown boundary
    ((16,), 1, 0, 7, -1),               # unknown precision
    ((2,), 0, 0, 1, -1),                # axis shorter than 4
    ((4,), 2, 0, 1, -1),                # axis shorter than 2r+1
    ((22,), 1, 0, 1, -7),               # a prime factor above 7 (n = 11)
    ((15,), 1, 0, 1, -7),               # odd last axis (real rows pack pairs)
    ((12,), 1, 1, 1, -7),               # mixed radix: periodic plans only
    ((12,), 1, 2, 1, -7),
    ((96, 64), 1, 0, 2, -7),            # mixed radix: no tensor-core DFTs
    ((8, 2 * 9 * 1024), 1, 0, 1, -7),   # mixed-radix rows above 8192 complex values
    ((1 << 25,), 1, 0, 1, -7),          # beyond the 1-D limit of 2^24
    ((8, 1 << 16), 1, 0, 1, -7),        # beyond the single-CTA row limit
])
def test_plan_rejects_bad_arguments(lib, dims, radius, boundary, precision, code):
    if len(dims) == 0:
        h = ctypes.c_void_p()
        w = np.zeros(3)
        rc = lib.stencil_plan(ctypes.byref(h), 0, (ctypes.c_int64 * 1)(8), 1,
                              w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0, 1)
    else:
        rc, h = _plan(lib, dims, radius, boundary, precision)
    assert rc == code
    assert not h.value


def test_implicit_and_vector_plans_reject_bad_arguments(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    w = np.full(9, 0.1)
    h = ctypes.c_void_p()
    d2 = (ctypes.c_int64 * 2)(64, 64)
    # implicit: null weights, tensor-core precision, a mixed-radix axis
    assert lib.stencil_plan_implicit(ctypes.byref(h), 2, d2, 1, w.ctypes.data_as(dp), None, 1) == -1
    assert lib.stencil_plan_implicit(ctypes.byref(h), 2, (ctypes.c_int64 * 2)(256, 256), 1,
                                     w.ctypes.data_as(dp), w.ctypes.data_as(dp), 2) == -7
    assert lib.stencil_plan_implicit(ctypes.byref(h), 2, (ctypes.c_int64 * 2)(60, 64), 1,
                                     w.ctypes.data_as(dp), w.ctypes.data_as(dp), 1) == -7
    long1d = (ctypes.c_int64 * 1)(1 << 20)   # n1 x n2 passes take no multiplier table
    w1 = np.full(3, 0.3)
    assert lib.stencil_plan_implicit(ctypes.byref(h), 1, long1d, 1, w1.ctypes.data_as(dp),
                                     w1.ctypes.data_as(dp), 1) == -7
    # vector: 0 or 5 fields, a tensor-core precision, non-finite weights
    wv = np.full(4 * 9, 0.1)
    assert lib.stencil_plan_vector(ctypes.byref(h), 2, d2, 1, 0, wv.ctypes.data_as(dp), 1) == -1
    assert lib.stencil_plan_vector(ctypes.byref(h), 2, d2, 1, 5, wv.ctypes.data_as(dp), 1) == -1
    assert lib.stencil_plan_vector(ctypes.byref(h), 2, (ctypes.c_int64 * 2)(256, 256), 1, 2,
                                   wv.ctypes.data_as(dp), 3) == -7
    wv[20] = np.inf
    assert lib.stencil_plan_vector(ctypes.byref(h), 2, d2, 1, 2, wv.ctypes.data_as(dp), 1) == -1
    assert not h.value


def test_plan_rejects_null_and_nonfinite(lib):
    d = (ctypes.c_int64 * 1)(16)
    w = np.array([0.25, 0.5, 0.25])
    wp = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.stencil_plan(None, 1, d, 1, wp, 0, 1) == -1
    h = ctypes.c_void_p()
    assert lib.stencil_plan(ctypes.byref(h), 1, d, 1, None, 0, 1) == -1
    bad = np.array([0.25, np.nan, 0.25])
    assert lib.stencil_plan(ctypes.byref(h), 1, d, 1,
                            bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 0, 1) == -1


def test_null_plan_calls_are_rejected(lib):
    assert lib.stencil_run(None, None, 1, None) == -1
    assert lib.stencil_run_host(None, None, None, 1, None) == -1
    assert lib.stencil_status(None, None) == -1
    assert lib.stencil_destroy(None) == -1
    assert lib.stencil_symbol_power(None, 1, None, None) == -1
    assert lib.stencil_plan_set_cutoff(None, 8) == -1
    assert lib.stencil_plan_set_schedule(None, 0) == -1
    assert lib.stencil_plan_autotune(None, None, 5, None, None, 0) == -1
    assert lib.stencil_profile_enable(None, 1) == -1
    assert lib.stencil_prepare(None, 5, None) == -1
    assert lib.stencil_plan_set_weights(None, 1, None) == -1


def test_size_limits_and_workspace(lib):
    assert lib.stencil_max_axis(2, 1, 1) >= 8192
    assert lib.stencil_max_axis(2, 1, 0) >= 8192
    assert lib.stencil_max_axis(4, 1, 0) == 0
    # 1-D: up to 2^24 in both precisions (n1 x n2 passes beyond one CTA)
    assert lib.stencil_max_axis(1, 1, 0) == 1 << 24
    assert lib.stencil_max_axis(1, 0, 0) == 1 << 24
    d = (ctypes.c_int64 * 2)(4096, 4096)
    # half spectrum 4096 x (2048 + 1 padded to 2064) complex float, plus the
    # repeated-T multiplier table (blocked layout; sized for the row-major one
    # an implicit plan keeps)
    assert lib.stencil_workspace_bytes(2, d, 1, 0, 1) == 2 * 4096 * 2064 * 8
    assert lib.stencil_workspace_bytes(2, d, 1, 1, 1) == 4096 * 2064 * 8
    d1 = (ctypes.c_int64 * 1)(4096)
    # 1-D periodic FP64 held by one CTA: no half spectrum, the (2048 + 1)-entry
    # multiplier table kept for a repeated T; zero Dirichlet keeps no such table
    assert lib.stencil_workspace_bytes(1, d1, 1, 0, 0) == 2049 * 16
    assert lib.stencil_workspace_bytes(1, d1, 1, 1, 0) == 0
    # 3-D periodic FP32: half spectrum plus the table laid out like it
    d3 = (ctypes.c_int64 * 3)(64, 32, 128)
    assert lib.stencil_workspace_bytes(3, d3, 1, 0, 1) == 2 * 64 * 32 * 80 * 8
    assert lib.stencil_workspace_bytes(3, d3, 1, 1, 1) == 64 * 32 * 80 * 8
    assert lib.stencil_profile_kind_name(0).decode() == "rows_r2c"
    assert lib.stencil_profile_kind_name(999) is None
