"""ctypes declarations of the C ABI in include/stencilfft.h (argument marshalling only).

Loading fails loudly when libstencilfft.so has not been built: there is no
CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes
import os
import threading

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libstencilfft.so")

STENCIL_PERIODIC = 0
STENCIL_ZERO_DIRICHLET = 1
STENCIL_NEUMANN = 2
STENCIL_FP64 = 0
STENCIL_FP32 = 1
STENCIL_FP32_GEMM_BF16 = 2
STENCIL_FP32_GEMM_FP16 = 3
STENCIL_FP32_GEMM_BF16X3 = 4

STATUS = {
    0: "STENCIL_OK", -1: "STENCIL_EINVAL", -2: "STENCIL_ENOMEM", -3: "STENCIL_ECUDA",
    -4: "STENCIL_ETIMEOUT", -5: "STENCIL_ENONFINITE", -6: "STENCIL_EQUEUEFULL",
    -7: "STENCIL_EUNSUPPORTED",
}

# (name, restype, argtypes) for every entry point the header declares.
_c = ctypes
_vp = _c.c_void_p
_i64p = _c.POINTER(_c.c_int64)
_dp = _c.POINTER(_c.c_double)
SIGNATURES = [
    ("stencil_plan", _c.c_int, [_c.POINTER(_vp), _c.c_int, _i64p, _c.c_int, _dp, _c.c_int, _c.c_int]),
    ("stencil_plan_implicit", _c.c_int, [_c.POINTER(_vp), _c.c_int, _i64p, _c.c_int, _dp, _dp,
                                         _c.c_int]),
    ("stencil_plan_vector", _c.c_int, [_c.POINTER(_vp), _c.c_int, _i64p, _c.c_int, _c.c_int, _dp,
                                       _c.c_int]),
    ("stencil_run", _c.c_int, [_vp, _vp, _c.c_int64, _vp]),
    ("stencil_run_host", _c.c_int, [_vp, _vp, _vp, _c.c_int64, _vp]),
    ("stencil_symbol_power", _c.c_int, [_vp, _c.c_int64, _vp, _vp]),
    ("stencil_prepare", _c.c_int, [_vp, _c.c_int64, _vp]),
    ("stencil_plan_set_weights", _c.c_int, [_vp, _c.c_int, _c.POINTER(_c.c_double)]),
    ("stencil_status", _c.c_int, [_vp, _vp]),
    ("stencil_destroy", _c.c_int, [_vp]),
    ("stencil_strerror", _c.c_char_p, [_c.c_int]),
    ("stencil_cuda_error_name", _c.c_char_p, []),
    ("stencil_max_axis", _c.c_int64, [_c.c_int, _c.c_int, _c.c_int]),
    ("stencil_workspace_bytes", _c.c_size_t, [_c.c_int, _i64p, _c.c_int, _c.c_int, _c.c_int]),
    ("stencil_plan_set_cutoff", _c.c_int, [_vp, _c.c_int64]),
    ("stencil_plan_set_schedule", _c.c_int, [_vp, _c.c_int]),
    ("stencil_plan_autotune", _c.c_int, [_vp, _vp, _c.c_int64, _vp, _c.POINTER(_c.c_double), _c.c_int]),
    ("stencil_plan_set_pass_variant", _c.c_int, [_vp, _c.c_int]),
    ("stencil_profile_enable", _c.c_int, [_vp, _c.c_int]),
    ("stencil_profile_read", _c.c_int, [_vp, _c.POINTER(_c.c_double), _i64p, _c.c_int]),
    ("stencil_profile_kind_name", _c.c_char_p, [_c.c_int]),
    ("stencil_periodic_run_noalloc", _c.c_int, [_c.c_int, _i64p, _c.c_int, _dp, _c.c_int, _vp,
                                                 _c.c_int64, _vp]),
    ("stencil_noalloc_scratch_bytes", _c.c_size_t, []),
    ("stencil_debug_schedule", _c.c_int64, [_c.c_int, _i64p, _c.c_int, _c.c_int64, _c.c_int64,
                                            _i64p, _c.c_int64]),
    ("stencil_debug_schedule_reach", _c.c_int64, [_c.c_int, _i64p, _c.c_int, _c.POINTER(_c.c_int),
                                                  _c.c_int64, _c.c_int64, _i64p, _c.c_int64]),
    ("stencil_debug_face_reach", _c.c_int, [_c.c_int, _c.c_int, _dp, _c.POINTER(_c.c_int)]),
]

class StencilRequest(ctypes.Structure):
    _fields_ = [("ndim", _c.c_int), ("dims", _c.c_int64 * 3), ("radius", _c.c_int),
                ("weights", _dp), ("boundary", _c.c_int), ("precision", _c.c_int),
                ("T", _c.c_int64), ("grid", _vp)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", _c.c_uint64), ("completed", _c.c_uint64), ("failed", _c.c_uint64),
                ("max_in_flight", _c.c_int), ("batched_launches", _c.c_uint64),
                ("batched_requests", _c.c_uint64), ("bytes_in_use", _c.c_size_t),
                ("peak_bytes", _c.c_size_t), ("budget_bytes", _c.c_size_t)]


SIGNATURES += [
    ("stencil_server_create", _c.c_int, [_c.POINTER(_vp), _c.c_size_t, _c.c_int, _c.c_int]),
    ("stencil_server_submit", _c.c_int, [_vp, _c.POINTER(StencilRequest), _c.POINTER(_c.c_uint64)]),
    ("stencil_server_poll", _c.c_int, [_vp, _c.c_uint64, _c.POINTER(_c.c_int),
                                       _c.POINTER(_c.c_double)]),
    ("stencil_server_wait", _c.c_int, [_vp, _c.c_uint64, _c.c_double, _c.POINTER(_c.c_double)]),
    ("stencil_server_stats", _c.c_int, [_vp, _c.POINTER(ServerStats)]),
    ("stencil_server_destroy", _c.c_int, [_vp]),
    ("stencil_batch_smem_bytes", _c.c_size_t, [_c.c_int, _i64p, _c.c_int]),
    ("stencil_batch_create", _c.c_int, [_c.POINTER(_vp), _c.c_int, _c.c_int]),
    ("stencil_batch_run", _c.c_int, [_vp, _c.c_int, _c.POINTER(StencilRequest), _vp]),
    ("stencil_batch_status", _c.c_int, [_vp, _vp]),
    ("stencil_batch_destroy", _c.c_int, [_vp]),
]

_lock = threading.Lock()
_lib = None


class StencilError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = lib().stencil_strerror(code).decode() if _lib is not None else STATUS.get(code, "?")
        super().__init__(f"{where}: {STATUS.get(code, code)} ({msg})")


def lib():
    """The loaded library; raises if it was never built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            handle = ctypes.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
    return _lib


def check(code: int, where: str) -> None:
    if code != 0:
        if code in (-2, -3):   # ENOMEM / ECUDA: name the CUDA error behind it
            cuda = lib().stencil_cuda_error_name()
            where = f"{where} [{cuda.decode() if cuda else '?'}]"
        raise StencilError(code, where)
