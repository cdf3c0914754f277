"""Thin Python binding over libstencilfft.so (argument marshalling only).

Every step of a solve runs in the library's CUDA kernels. PyTorch is used for
device memory and streams: a grid is a CUDA tensor, the stream is
``torch.cuda.current_stream()`` unless one is given.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi

_BOUNDARY = {"periodic": _capi.STENCIL_PERIODIC, "dirichlet": _capi.STENCIL_ZERO_DIRICHLET,
             "zero_dirichlet": _capi.STENCIL_ZERO_DIRICHLET, "neumann": _capi.STENCIL_NEUMANN}
_PRECISION = {"fp64": _capi.STENCIL_FP64, "fp32": _capi.STENCIL_FP32,
              # FP32 grids with the strided-axis radix-16 DFTs on the tensor cores
              "fp32_gemm_bf16": _capi.STENCIL_FP32_GEMM_BF16,
              "fp32_gemm_fp16": _capi.STENCIL_FP32_GEMM_FP16,
              "fp32_gemm_bf16x3": _capi.STENCIL_FP32_GEMM_BF16X3}


def _stream_ptr(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def max_axis(ndim: int, precision: str, axis: int) -> int:
    return int(_capi.lib().stencil_max_axis(ndim, _PRECISION[precision], axis))


def workspace_bytes(dims, radius: int, boundary: str, precision: str) -> int:
    d = (ctypes.c_int64 * len(dims))(*[int(x) for x in dims])
    return int(_capi.lib().stencil_workspace_bytes(len(dims), d, int(radius),
                                                  _BOUNDARY[boundary], _PRECISION[precision]))


class StencilPlan:
    """A plan for advancing grids of one shape by one stencil (stencil_plan)."""

    def __init__(self, dims, weights, boundary: str = "periodic", precision: str = "fp32",
                 implicit_weights=None):
        """implicit_weights: Q of an implicit stencil Q a_{t+1} = S a_t (weights
        then hold S; periodic, fp32 or fp64: stencil_plan_implicit)."""
        w = np.ascontiguousarray(weights, dtype=np.float64)
        dims = tuple(int(x) for x in dims)
        if w.ndim != len(dims) or len(set(w.shape)) != 1 or w.shape[0] % 2 != 1:
            raise ValueError("weights must have shape (2r+1,)*ndim")
        self.dims = dims
        self.radius = (w.shape[0] - 1) // 2
        self.boundary = boundary
        self.precision = precision
        self.weights = w
        self._handle = ctypes.c_void_p()
        d = (ctypes.c_int64 * len(dims))(*dims)
        dp = ctypes.POINTER(ctypes.c_double)
        if implicit_weights is None:
            rc = _capi.lib().stencil_plan(ctypes.byref(self._handle), len(dims), d, self.radius,
                                          w.ctypes.data_as(dp), _BOUNDARY[boundary],
                                          _PRECISION[precision])
            _capi.check(rc, "stencil_plan")
        else:
            q = np.ascontiguousarray(implicit_weights, dtype=np.float64)
            if q.shape != w.shape:
                raise ValueError("implicit_weights must have the shape of weights")
            if boundary != "periodic":
                raise ValueError("implicit stencils are periodic")
            self.implicit_weights = q
            rc = _capi.lib().stencil_plan_implicit(ctypes.byref(self._handle), len(dims), d,
                                                   self.radius, w.ctypes.data_as(dp),
                                                   q.ctypes.data_as(dp), _PRECISION[precision])
            _capi.check(rc, "stencil_plan_implicit")

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == "fp64" else torch.float32

    @property
    def handle(self):
        return self._handle

    def set_weights(self, weights) -> None:
        """Replace the stencil, keeping the plan's tables and workspace
        (stencil_plan_set_weights)."""
        w = np.ascontiguousarray(weights, dtype=np.float64)
        if w.ndim != len(self.dims) or len(set(w.shape)) != 1 or w.shape[0] % 2 != 1:
            raise ValueError("weights must have shape (2r+1,)*ndim")
        r = (w.shape[0] - 1) // 2
        _capi.check(_capi.lib().stencil_plan_set_weights(
            self._handle, r, w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
            "stencil_plan_set_weights")
        self.radius = r
        self.weights = w

    def set_cutoff(self, cutoff: int) -> None:
        _capi.check(_capi.lib().stencil_plan_set_cutoff(self._handle, int(cutoff)),
                    "stencil_plan_set_cutoff")

    def autotune(self, grid, T: int, stream=None) -> dict:
        """Time the zero-Dirichlet schedules, or the periodic pass variants, for T
        on a copy of `grid` (CUDA tensor, unchanged) and keep the fastest
        (stencil_plan_autotune)."""
        if self.boundary == "periodic":
            names = ["blocked_tma", "rowmajor_tma", "register_1024", "register_512"]
        else:
            names = ["recursive", "loop", "recursive_half_cutoff", "recursive_double_cutoff",
                     "cluster"]
        ms = (ctypes.c_double * len(names))()
        rc = _capi.lib().stencil_plan_autotune(self._handle, ctypes.c_void_p(grid.data_ptr()), int(T),
                                               _stream_ptr(stream), ms, len(names))
        if rc < 0:
            _capi.check(rc, "stencil_plan_autotune")
        return {"chosen": names[rc], "ms": {n: ms[i] for i, n in enumerate(names) if ms[i] >= 0}}

    def set_pass_variant(self, variant: int) -> None:
        """Periodic pass variant 0..3 (-1: default), stencil_plan_set_pass_variant."""
        _capi.check(_capi.lib().stencil_plan_set_pass_variant(self._handle, int(variant)),
                    "stencil_plan_set_pass_variant")

    def set_schedule(self, mode: str) -> None:
        """Zero-Dirichlet schedule: "auto", "recursive", "loop" or "cluster"
        (stencil_plan_set_schedule)."""
        code = {"auto": 0, "recursive": 1, "loop": 2, "cluster": 3}[mode]
        _capi.check(_capi.lib().stencil_plan_set_schedule(self._handle, code),
                    "stencil_plan_set_schedule")

    def prepare(self, T: int, stream=None) -> None:
        """Per-T set-up ahead of the first run (stencil_prepare): afterwards runs
        with this T allocate nothing and do not synchronise."""
        _capi.check(_capi.lib().stencil_prepare(self._handle, int(T), _stream_ptr(stream)),
                    "stencil_prepare")

    def run(self, grid, T: int, stream=None):
        """Advance a CUDA tensor of shape dims in place by T steps (async); returns it."""
        if not grid.is_cuda or grid.dtype != self.dtype or tuple(grid.shape) != self.dims \
                or not grid.is_contiguous():
            raise ValueError(f"grid must be a contiguous CUDA {self.dtype} tensor of shape {self.dims}")
        rc = _capi.lib().stencil_run(self._handle, ctypes.c_void_p(grid.data_ptr()), int(T),
                                     _stream_ptr(stream))
        _capi.check(rc, "stencil_run")
        return grid

    def run_host(self, host_in, T: int, host_out=None, stream=None):
        """End-to-end solve of a host (CPU) tensor (stencil_run_host): pinned input and
        output are read and written in place by the GPU, other buffers go through
        a device copy; synchronises."""
        import torch
        if host_in.is_cuda or host_in.dtype != self.dtype or tuple(host_in.shape) != self.dims:
            raise ValueError("host_in must be a CPU tensor of the plan's shape and dtype")
        host_in = host_in.contiguous()
        if host_out is None:
            host_out = torch.empty_like(host_in)
        rc = _capi.lib().stencil_run_host(self._handle, ctypes.c_void_p(host_in.data_ptr()),
                                          ctypes.c_void_p(host_out.data_ptr()), int(T),
                                          _stream_ptr(stream))
        _capi.check(rc, "stencil_run_host")
        return host_out

    def symbol_power(self, T: int, stream=None):
        """Lambda^T on the half spectrum, complex128 CUDA tensor (stencil_symbol_power)."""
        import torch
        shape = self.dims[:-1] + (self.dims[-1] // 2 + 1,)
        out = torch.empty(shape + (2,), dtype=torch.float64, device="cuda")
        rc = _capi.lib().stencil_symbol_power(self._handle, int(T), ctypes.c_void_p(out.data_ptr()),
                                              _stream_ptr(stream))
        _capi.check(rc, "stencil_symbol_power")
        return torch.view_as_complex(out)

    def profile(self, enable: bool = True) -> None:
        """Bracket every kernel launch of later runs with CUDA events (stencil_profile_enable)."""
        _capi.check(_capi.lib().stencil_profile_enable(self._handle, int(bool(enable))),
                    "stencil_profile_enable")

    def profile_read(self) -> dict:
        """{kernel kind: (total ms, launches)} since the last read (synchronises)."""
        nk = 32
        ms = (ctypes.c_double * nk)()
        cnt = (ctypes.c_int64 * nk)()
        _capi.check(_capi.lib().stencil_profile_read(self._handle, ms, cnt, nk), "stencil_profile_read")
        out = {}
        for k in range(nk):
            name = _capi.lib().stencil_profile_kind_name(k)
            if name is None:
                break
            if cnt[k]:
                out[name.decode()] = (float(ms[k]), int(cnt[k]))
        return out

    def status(self, stream=None) -> int:
        """Synchronise and return the latched status code (0 or a negative code)."""
        return int(_capi.lib().stencil_status(self._handle, _stream_ptr(stream)))

    def close(self):
        if self._handle:
            _capi.lib().stencil_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class VectorStencilPlan:
    """m coupled fields on a periodic grid (stencil_plan_vector): weights of
    shape (m, m, 2r+1, ..., 2r+1), block (i, j) taking field j into field i."""

    def __init__(self, dims, weights, precision: str = "fp32"):
        w = np.ascontiguousarray(weights, dtype=np.float64)
        dims = tuple(int(x) for x in dims)
        if w.ndim != len(dims) + 2 or w.shape[0] != w.shape[1] or len(set(w.shape[2:])) != 1 \
                or w.shape[2] % 2 != 1:
            raise ValueError("weights must have shape (m, m) + (2r+1,)*ndim")
        self.dims = dims
        self.nfields = w.shape[0]
        self.radius = (w.shape[2] - 1) // 2
        self.precision = precision
        self.weights = w
        self._handle = ctypes.c_void_p()
        d = (ctypes.c_int64 * len(dims))(*dims)
        rc = _capi.lib().stencil_plan_vector(ctypes.byref(self._handle), len(dims), d, self.radius,
                                             self.nfields,
                                             w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             _PRECISION[precision])
        _capi.check(rc, "stencil_plan_vector")

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.precision == "fp64" else torch.float32

    @property
    def handle(self):
        return self._handle

    def run(self, fields, T: int, stream=None):
        """Advance a contiguous CUDA tensor of shape (m, *dims) in place by T steps (async)."""
        shape = (self.nfields,) + self.dims
        if not fields.is_cuda or fields.dtype != self.dtype or tuple(fields.shape) != shape \
                or not fields.is_contiguous():
            raise ValueError(f"fields must be a contiguous CUDA {self.dtype} tensor of shape {shape}")
        rc = _capi.lib().stencil_run(self._handle, ctypes.c_void_p(fields.data_ptr()), int(T),
                                     _stream_ptr(stream))
        _capi.check(rc, "stencil_run")
        return fields

    def status(self, stream=None) -> int:
        return int(_capi.lib().stencil_status(self._handle, _stream_ptr(stream)))

    def close(self):
        if self._handle:
            _capi.lib().stencil_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(grid, weights, T: int, boundary: str = "periodic", stream=None):
    """One-shot solve of a CUDA tensor in place (builds and frees a plan)."""
    precision = "fp32" if str(grid.dtype) == "torch.float32" else "fp64"
    plan = StencilPlan(tuple(grid.shape), weights, boundary, precision)
    try:
        plan.run(grid, T, stream)
        import torch
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
    finally:
        plan.close()
    return grid


class BatchExecutor:
    """Small periodic solves of mixed shapes in one persistent launch
    (stencil_batch_*): every request a CUDA tensor solved in place with its own
    weights and T."""

    def __init__(self, capacity: int, precision: str = "fp32"):
        self.precision = precision
        self._h = ctypes.c_void_p()
        _capi.check(_capi.lib().stencil_batch_create(ctypes.byref(self._h), int(capacity),
                                                     _PRECISION[precision]),
                    "stencil_batch_create")

    @staticmethod
    def smem_bytes(dims, precision: str = "fp32") -> int:
        d = (ctypes.c_int64 * len(dims))(*[int(x) for x in dims])
        return int(_capi.lib().stencil_batch_smem_bytes(len(dims), d, _PRECISION[precision]))

    def run(self, grids, weights, Ts, stream=None):
        """Enqueue one batch: grids (CUDA tensors), weights and T per request."""
        n = len(grids)
        reqs = (_capi.StencilRequest * n)()
        keep = []
        for i, (g, w, T) in enumerate(zip(grids, weights, Ts)):
            w = np.ascontiguousarray(w, dtype=np.float64)
            keep.append(w)
            r = reqs[i]
            r.ndim = g.dim()
            for a in range(g.dim()):
                r.dims[a] = int(g.shape[a])
            r.radius = (w.shape[0] - 1) // 2
            r.weights = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            r.boundary = _capi.STENCIL_PERIODIC
            r.precision = _capi.STENCIL_FP32 if str(g.dtype) == "torch.float32" else _capi.STENCIL_FP64
            r.T = int(T)
            r.grid = ctypes.c_void_p(g.data_ptr())
        rc = _capi.lib().stencil_batch_run(self._h, n, reqs, _stream_ptr(stream))
        _capi.check(rc, "stencil_batch_run")
        return grids

    def status(self, stream=None) -> int:
        return int(_capi.lib().stencil_batch_status(self._h, _stream_ptr(stream)))

    def close(self):
        if self._h:
            _capi.lib().stencil_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StencilServer:
    """Continuous-batching request server (stencil_server_*).

    submit() takes a CUDA tensor that the caller keeps alive and untouched until
    its ticket completes; the solve runs in place on the server's own streams,
    so every write to the tensor must have completed before submit().
    """

    def __init__(self, hbm_budget_bytes: int, max_slots: int = 8, queue_capacity: int = 4096):
        self._h = ctypes.c_void_p()
        _capi.check(_capi.lib().stencil_server_create(ctypes.byref(self._h), int(hbm_budget_bytes),
                                                      int(max_slots), int(queue_capacity)),
                    "stencil_server_create")
        self._keep = {}

    def submit(self, grid, weights, T: int, boundary: str = "periodic") -> int:
        """Queue grid (CUDA tensor, solved in place); returns the ticket or raises."""
        w = np.ascontiguousarray(weights, dtype=np.float64)
        r = _capi.StencilRequest()
        r.ndim = grid.dim()
        for a in range(grid.dim()):
            r.dims[a] = int(grid.shape[a])
        r.radius = (w.shape[0] - 1) // 2
        r.weights = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        r.boundary = _BOUNDARY[boundary]
        r.precision = _capi.STENCIL_FP32 if str(grid.dtype) == "torch.float32" else _capi.STENCIL_FP64
        r.T = int(T)
        r.grid = ctypes.c_void_p(grid.data_ptr())
        t = ctypes.c_uint64()
        rc = _capi.lib().stencil_server_submit(self._h, ctypes.byref(r), ctypes.byref(t))
        _capi.check(rc, "stencil_server_submit")
        self._keep[t.value] = grid
        return t.value

    def try_submit(self, grid, weights, T: int, boundary: str = "periodic"):
        """Like submit(), but returns the status code instead of raising (0: queued)."""
        try:
            return 0, self.submit(grid, weights, T, boundary)
        except _capi.StencilError as e:
            return e.code, None

    def poll(self, ticket: int):
        """(done, status, latency_s)."""
        done = ctypes.c_int()
        lat = ctypes.c_double()
        rc = _capi.lib().stencil_server_poll(self._h, int(ticket), ctypes.byref(done), ctypes.byref(lat))
        if done.value:
            self._keep.pop(ticket, None)
        return bool(done.value), int(rc), float(lat.value)

    def wait(self, ticket: int, timeout_s: float = 60.0):
        """Block until done; returns (status, latency_s)."""
        lat = ctypes.c_double()
        rc = _capi.lib().stencil_server_wait(self._h, int(ticket), float(timeout_s), ctypes.byref(lat))
        self._keep.pop(ticket, None)
        return int(rc), float(lat.value)

    def stats(self) -> dict:
        st = _capi.ServerStats()
        _capi.check(_capi.lib().stencil_server_stats(self._h, ctypes.byref(st)), "stencil_server_stats")
        return {name: getattr(st, name) for name, _ in st._fields_}

    def close(self):
        if self._h:
            _capi.lib().stencil_server_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
