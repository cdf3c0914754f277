"""Parity of the reflecting-boundary (zero-flux Neumann) CUDA path with the
oracle: RecursiveBoundary's periodic strip solves keep only cells the boundary
cannot reach (paper Sec. 5.1), so the same schedule with a mirroring base case
gives the reflecting solve. Against the C loop oracle with mirror ghosts on
small and medium grids, and against the periodic solve of the even extension
(symmetric stencils) at 2048^2. Tolerance relative to max|a_0|: 1e-10 (FP64),
2e-4 (FP32)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2105_06676_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-4}


def run_gpu(a0, w, T, precision, cutoff=None, schedule=None):
    from paper_2105_06676_gb300 import StencilPlan
    dt = torch.float32 if precision == "fp32" else torch.float64
    g = torch.tensor(a0, dtype=dt, device="cuda")
    plan = StencilPlan(a0.shape, w, "neumann", precision)
    if cutoff is not None:
        plan.set_cutoff(cutoff)
    if schedule is not None:
        plan.set_schedule(schedule)
    plan.run(g, T)
    rc = plan.status()
    plan.close()
    assert rc == 0, f"device status {rc}"
    return g.double().cpu().numpy()


def err_rel(got, ref, a0):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(a0)))


CASES = [
    ((64,), 1), ((256,), 2), ((4096,), 1), ((32,), 3),
    ((32, 32), 1), ((64, 128), 1), ((128, 64), 2), ((256, 256), 1), ((64, 64), 3),
    ((16, 16, 16), 1), ((32, 16, 64), 1), ((16, 16, 32), 2),
]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("dims,r", CASES)
@pytest.mark.parametrize("T", [1, 2, 7, 13, 64, 200])
@pytest.mark.parametrize("cutoff", [None, 2, 5])
def test_neumann_matches_loop(dims, r, T, cutoff, precision):
    n = int(np.prod(dims))
    if n * T > 2e8:
        pytest.skip("loop oracle too slow for this combination")
    w = wl.weights_random_box(len(dims), r, 31 + T)     # not symmetric
    a0 = wl.grid_uniform(dims, 5 + T)
    ref = oracle.stencil_loop(a0, w, T, "neumann")
    got = run_gpu(a0, w, T, precision, cutoff)
    assert err_rel(got, ref, a0) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("schedule", ["recursive", "loop"])
@pytest.mark.parametrize("dims,r,T", [((512, 256), 1, 150), ((64, 64, 64), 1, 40), ((8192,), 2, 700)])
def test_neumann_schedules_match_loop(dims, r, T, schedule, precision):
    w = wl.weights_random_box(len(dims), r, 7)
    a0 = wl.grid_uniform(dims, 8)
    ref = oracle.stencil_loop(a0, w, T, "neumann")
    got = run_gpu(a0, w, T, precision, schedule=schedule)
    assert err_rel(got, ref, a0) <= TOL[precision]


def _even_extension(a):
    for ax in range(a.ndim):
        a = np.concatenate([a, np.flip(a, axis=ax)], axis=ax)
    return a


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_neumann_even_extension_full_size_2d(precision):
    # a stencil symmetric along both axes: reflecting on l equals the periodic
    # solve of the half-sample even extension on 2 l (no loop oracle needed)
    dims, T = (2048, 2048), 1000
    w = np.array([[0.05, 0.1, 0.05], [0.15, 0.3, 0.15], [0.05, 0.1, 0.05]])
    a0 = wl.grid_uniform(dims, 19)
    ref = oracle.stencil_fft_periodic(_even_extension(a0), w, T, workers=8)[:dims[0], :dims[1]]
    got = run_gpu(a0, w, T, precision)
    assert err_rel(got, ref, a0) <= TOL[precision]
    # mass is conserved (symmetric weights summing to 1)
    assert abs(got.sum() - a0.sum()) / a0.sum() <= TOL[precision]


def test_neumann_differs_from_dirichlet():
    # the condition reaches the result: reflecting keeps mass, zero Dirichlet loses it
    from paper_2105_06676_gb300 import StencilPlan
    dims, T = (128, 128), 300
    w = wl.weights_star(2, 0.6, 0.1)
    a0 = wl.grid_uniform(dims, 20)
    neu = run_gpu(a0, w, T, "fp64")
    plan = StencilPlan(dims, w, "dirichlet", "fp64")
    g = torch.tensor(a0, device="cuda")
    plan.run(g, T)
    plan.close()
    dir_ = g.cpu().numpy()
    assert abs(neu.sum() - a0.sum()) / a0.sum() < 1e-12
    assert dir_.sum() < 0.9 * a0.sum()
