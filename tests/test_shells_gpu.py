"""l-shell regions on the GPU (appendix "l-shell Spatial Grid Decomposition"):
zero-Dirichlet and reflecting solves of stencils that reach further towards
some faces than towards others (upwind, leaning, anisotropic), whose
RecursiveBoundary regions are cut per face by the plan's toward-reach,
against the loop oracle. Tolerance relative to
max|a_0|: 1e-10 (FP64), 2e-4 (FP32)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import ell_shells as es
from paper_2105_06676_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-4}


def _support(nd, r, offsets, seed):
    rng = np.random.default_rng(seed)
    w = np.zeros((2 * r + 1,) * nd)
    for m in offsets:
        w[tuple(mm + r for mm in m)] = 0.2 + rng.random()
    return w / w.sum()


STENCILS = {
    "upwind1d": (1, 1, [(-1,), (0,)]),
    "lean1d": (1, 2, [(-1,), (0,), (2,)]),
    "upwind2d": (2, 1, [(0, 0), (-1, 0), (0, -1)]),
    "downwind2d": (2, 1, [(0, 0), (1, 0), (0, 1), (1, 1)]),
    "aniso2d": (2, 2, [(0, 0), (-2, 0), (2, 0), (0, -1), (0, 1), (1, 1)]),
    "lean2d": (2, 3, [(0, 0), (-1, 0), (3, 0), (0, 2), (0, -1), (1, -1)]),
    "upwind3d": (3, 1, [(0, 0, 0), (-1, 0, 0), (0, -1, 0), (0, 0, 1), (-1, 0, 1)]),
}


def run_gpu(a0, w, T, boundary, precision, schedule=None, cutoff=None):
    from paper_2105_06676_gb300 import StencilPlan
    dt = torch.float32 if precision == "fp32" else torch.float64
    g = torch.tensor(a0, dtype=dt, device="cuda")
    plan = StencilPlan(a0.shape, w, boundary, precision)
    if schedule is not None:
        plan.set_schedule(schedule)
    if cutoff is not None:
        plan.set_cutoff(cutoff)
    plan.run(g, T)
    rc = plan.status()
    plan.close()
    assert rc == 0, f"device status {rc}"
    return g.double().cpu().numpy()


def err_rel(got, ref, a0):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(a0)))


CASES = [
    ("upwind1d", (4096,), 700), ("upwind1d", (256,), 90), ("lean1d", (8192,), 900),
    ("upwind2d", (256, 256), 60), ("upwind2d", (512, 128), 150), ("downwind2d", (256, 512), 77),
    ("aniso2d", (256, 256), 40), ("lean2d", (512, 512), 33), ("upwind3d", (64, 64, 64), 20),
    ("upwind3d", (32, 64, 128), 31),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("boundary", ["dirichlet", "neumann"])
@pytest.mark.parametrize("schedule", [None, "recursive"])
@pytest.mark.parametrize("name,dims,T", CASES)
def test_shells_match_loop(name, dims, T, schedule, boundary, precision):
    nd, r, offs = STENCILS[name]
    w = _support(nd, r, offs, 50 + T)
    a0 = wl.grid_uniform(dims, 51 + T)
    got = run_gpu(a0, w, T, boundary, precision, schedule)
    ref = oracle.stencil_loop(a0, w, T, boundary)
    assert err_rel(got, ref, a0) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("cutoff", [2, 5])
def test_shells_small_cutoffs(cutoff, precision):
    # deep recursion: many levels of per-face strips and bands
    nd, r, offs = STENCILS["lean2d"]
    w = _support(nd, r, offs, 60)
    a0 = wl.grid_uniform((128, 256), 61)
    for T in (7, 40, 111):
        got = run_gpu(a0, w, T, "dirichlet", precision, "recursive", cutoff)
        assert err_rel(got, oracle.stencil_loop(a0, w, T, "dirichlet"), a0) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_upwind_shells_at_2048(precision):
    # 2048^2 first-order upwind stencil, T = 600, against the loop
    nd, r, offs = STENCILS["upwind2d"]
    w = _support(nd, r, offs, 62)
    dims, T = (2048, 2048), 600
    a0 = wl.grid_uniform(dims, 63)
    got = run_gpu(a0, w, T, "dirichlet", precision)
    ref = oracle.stencil_loop(a0, w, T, "dirichlet")
    assert err_rel(got, ref, a0) <= TOL[precision]
    # two faces only: the boundary reaches (2048 - 600)^2 cells fewer than a
    # symmetric stencil's frame would cover
    ell = es.arrival_time(dims, es.face_reach(w))
    assert np.count_nonzero(ell > T) == (2048 - 600) ** 2


def test_new_weights_with_another_reach_rebuild_the_schedule():
    from paper_2105_06676_gb300 import StencilPlan
    import ctypes
    from paper_2105_06676_gb300 import _capi
    dims, T = (256, 256), 50
    up = _support(2, 1, STENCILS["upwind2d"][2], 64)
    down = _support(2, 1, STENCILS["downwind2d"][2], 65)
    a0 = wl.grid_uniform(dims, 66)
    plan = StencilPlan(dims, up, "dirichlet", "fp64")
    g = torch.tensor(a0, device="cuda")
    plan.run(g, T)
    assert err_rel(g.cpu().numpy(), oracle.stencil_loop(a0, up, T, "dirichlet"), a0) <= 1e-10
    dp = ctypes.POINTER(ctypes.c_double)
    assert _capi.lib().stencil_plan_set_weights(plan.handle, 1, down.ctypes.data_as(dp)) == 0
    for _ in range(2):   # eager run, then the captured graph
        g = torch.tensor(a0, device="cuda")
        plan.run(g, T)
        assert err_rel(g.cpu().numpy(), oracle.stencil_loop(a0, down, T, "dirichlet"), a0) <= 1e-10
    assert plan.status() == 0
    plan.close()
