"""ctypes wrapper and gcc build step for the C nested-loop oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring). The C source
``stencil_loop.c`` is the plain definition of the stencil evolution
(paper Sec. 1 "Problem Specification", Fig. "looping-code").
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stencil_loop.c")
_LIB_PATH = os.path.join(_HERE, "liboracle_loop.so")
_lock = threading.Lock()
_lib = None


def oracle_library_path() -> str:
    return _LIB_PATH


def build_oracle_library(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, no FP contraction, portable flags).

    ``-ffp-contract=off`` keeps every multiply and add separately rounded, so the
    oracle gives the same bits on x86_64 and aarch64.
    """
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
           _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build_oracle_library()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.oracle_stencil_loop.restype = ctypes.c_int
            lib.oracle_stencil_loop.argtypes = [
                ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.c_int,
                ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_int64,
                ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                ctypes.c_int]
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def oracle_threads() -> int:
    """Threads an OpenMP region of the oracle uses by default."""
    return int(_load().oracle_max_threads())


def stencil_loop(a0: np.ndarray, weights: np.ndarray, T: int,
                 boundary: str = "periodic", nthreads: int = 0) -> np.ndarray:
    """a_T by T sequential applications of the stencil (FP64).

    a0       : grid, shape (l_1, ..., l_d), d in 1..3, row-major.
    weights  : stencil coefficients over [-r, r]^d, shape (2r+1,)*d; entry
               (m_1+r, ..., m_d+r) multiplies a_t[i + m].
    boundary : "periodic" (indices wrap, paper Sec. 1), "dirichlet" (cells
               outside the grid read 0) or "neumann" (reflecting: index -1-k
               reads cell k, index l+k reads cell l-1-k).
    """
    a0 = np.ascontiguousarray(a0, dtype=np.float64)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    d = a0.ndim
    if w.ndim != d or len(set(w.shape)) != 1 or w.shape[0] % 2 != 1:
        raise ValueError("weights must have shape (2r+1,)*ndim")
    r = (w.shape[0] - 1) // 2
    codes = {"periodic": 0, "dirichlet": 1, "neumann": 2}
    if boundary not in codes:
        raise ValueError("boundary must be 'periodic', 'dirichlet' or 'neumann'")
    if T < 0:
        raise ValueError("T must be >= 0")
    dims = (ctypes.c_int64 * d)(*a0.shape)
    out = np.empty_like(a0)
    rc = _load().oracle_stencil_loop(
        d, dims, r, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        codes[boundary], int(T),
        a0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_stencil_loop failed with code {rc}")
    return out
