"""The allocation-free periodic entry point against the planned one.

stencil_periodic_run_noalloc serves callers that cannot allocate device memory
when they solve (a latency-critical loop that cannot pay cudaMalloc's implicit
device synchronisation, or a program whose allocator already holds the device
memory): it takes its scratch from one fixed device array inside the library.
Two calls in a row with different shapes and precisions reuse that array and
must each match stencil_plan + stencil_run within the solver's tolerance.
This file is collected last so that a failure here comes after every other
test has run.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_2105_06676_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-4}
PREC = {"fp64": 0, "fp32": 1}


def _lib():
    import __graft_entry__
    from paper_2105_06676_gb300 import _capi
    __graft_entry__.build()
    return _capi.lib()


def _noalloc(lib, grid, w, T, precision):
    dims = tuple(grid.shape)
    d = (ctypes.c_int64 * len(dims))(*dims)
    wf = np.ascontiguousarray(w, dtype=np.float64)
    r = (wf.shape[0] - 1) // 2
    stream = torch.cuda.current_stream()
    return lib.stencil_periodic_run_noalloc(
        len(dims), d, r, wf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), PREC[precision],
        ctypes.c_void_p(grid.data_ptr()), int(T), ctypes.c_void_p(stream.cuda_stream))


def _planned(a0, w, T, precision):
    from paper_2105_06676_gb300 import StencilPlan
    dt = torch.float32 if precision == "fp32" else torch.float64
    g = torch.tensor(a0, dtype=dt, device="cuda")
    plan = StencilPlan(a0.shape, w, "periodic", precision)
    plan.run(g, T)
    assert plan.status() == 0
    plan.close()
    return g.double().cpu().numpy()


CALLS = [
    ((512, 256), wl.weights_star(2, 0.6, 0.1), 1000, "fp32"),
    ((128, 256), wl.weights_random_box(2, 2, 3), 77, "fp64"),
    ((4096,), wl.weights_1d([0.25, 0.5, 0.25]), 1000, "fp64"),     # 1-D: no half-spectrum scratch
    ((64, 64, 64), wl.weights_star(3, 0.4, 0.1), 200, "fp32"),     # 3-D: three passes per direction
]


def test_noalloc_matches_planned_run_twice():
    # two calls in a row on each shape (the array keeps the previous call's
    # contents), each against stencil_plan + stencil_run
    lib = _lib()
    for dims, w, T, precision in CALLS + CALLS:
        a0 = wl.grid_uniform(dims, 11 + T)
        dt = torch.float32 if precision == "fp32" else torch.float64
        g = torch.tensor(a0, dtype=dt, device="cuda")
        assert _noalloc(lib, g, w, T, precision) == 0
        torch.cuda.synchronize()
        got = g.double().cpu().numpy()
        ref = _planned(a0, w, T, precision)
        err = np.max(np.abs(got - ref)) / np.max(np.abs(a0))
        assert err <= TOL[precision], (dims, precision, err)


def test_noalloc_calls_leave_free_device_memory_unchanged():
    # after one call per shape (kernel code loaded), further calls of every shape
    # take no device memory: the free-memory figure does not move
    lib = _lib()
    grids = []
    for dims, w, T, precision in CALLS:
        dt = torch.float32 if precision == "fp32" else torch.float64
        g = torch.tensor(wl.grid_uniform(dims, 5), dtype=dt, device="cuda")
        assert _noalloc(lib, g, w, T, precision) == 0
        grids.append(g)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for g, (dims, w, T, precision) in zip(grids, CALLS):
        assert _noalloc(lib, g, w, T + 1, precision) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_rejects_sizes_beyond_its_scratch():
    lib = _lib()
    assert lib.stencil_noalloc_scratch_bytes() == 32 << 20
    g = torch.zeros((4096, 4096), dtype=torch.float32, device="cuda")
    rc = _noalloc(lib, g, wl.weights_star(2, 0.6, 0.1), 10, "fp32")
    assert rc == -7       # STENCIL_EUNSUPPORTED: the half spectrum needs 67 MB
    np.testing.assert_array_equal(g.cpu().numpy(), 0.0)
