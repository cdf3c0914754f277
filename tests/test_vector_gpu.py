"""Vector-valued fields on the GPU (stencil_plan_vector) against the oracle
(appendix "Supporting Vector Valued Fields"): the plain m-field loop on small
grids, the spectral oracle with the matrix of symbols at larger ones, the
affine example and a leapfrog recurrence written out."""
from __future__ import annotations

import numpy as np
import pytest
import torch

import oracle
from oracle import vector_fields as vf
from paper_2105_06676_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-4}


def _delta(ndim):
    w = np.zeros((3,) * ndim)
    w[(1,) * ndim] = 1.0
    return w


def _weights(m, ndim, seed, r=1):
    # non-negative blocks, every field's row of blocks summing to 1: the
    # coupled evolution is a convex combination (no growth)
    rng = np.random.default_rng(seed)
    w = rng.random((m, m) + (2 * r + 1,) * ndim)
    w /= w.sum(axis=tuple(range(1, w.ndim)), keepdims=True)
    return w


def _run(dims, W, T, precision, seed=51):
    from paper_2105_06676_gb300 import VectorStencilPlan
    m = W.shape[0]
    a0 = np.stack([wl.grid_uniform(dims, seed + i) for i in range(m)])
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = VectorStencilPlan(dims, W, precision)
    g = torch.tensor(a0, dtype=dt, device="cuda")
    plan.run(g, T)
    assert plan.status() == 0
    out = g.double().cpu().numpy()
    plan.close()
    return a0, out


def _err(got, ref, a0):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(a0)), np.max(np.abs(ref))))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("m,dims,T", [(2, (64,), 9), (3, (32, 16), 5), (2, (16, 8, 32), 3), (4, (16, 16), 7),
                                      (1, (32, 64), 11)])
def test_vector_matches_loop(precision, m, dims, T):
    W = _weights(m, len(dims), 60 + m)
    a0, out = _run(dims, W, T, precision)
    assert _err(out, vf.vector_loop(a0, W, T), a0) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("m,dims,T", [(2, (4096,), 1000), (2, (512, 512), 300), (3, (256, 1024), 40),
                                      (2, (64, 32, 128), 100), (2, (1024, 1024), 5000)])
def test_vector_matches_spectral_oracle(precision, m, dims, T):
    W = _weights(m, len(dims), 70 + m)
    a0, out = _run(dims, W, T, precision)
    assert _err(out, vf.stencil_fft_periodic_vector(a0, W, T), a0) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_vector_one_field_is_the_scalar_solve(precision):
    from paper_2105_06676_gb300 import StencilPlan
    dims, T = (256, 512), 77
    w = wl.weights_random_box(2, 2, 80)
    a0, out = _run(dims, w[None, None], T, precision)
    plan = StencilPlan(dims, w, "periodic", precision)
    g = torch.tensor(a0[0], dtype=torch.float64 if precision == "fp64" else torch.float32, device="cuda")
    plan.run(g, T)
    plan.close()
    assert _err(out[0], g.double().cpu().numpy(), a0) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_vector_affine_stencil(precision):
    # a_{t+1} = A a_t + c as fields (a, c): a_T = A^T a_0 + T c (sum(A) = 1)
    from paper_2105_06676_gb300 import VectorStencilPlan
    dims, T, c = (256, 256), 60, 0.25
    A = wl.weights_random_box(2, 1, 81)
    W = np.zeros((2, 2, 3, 3))
    W[0, 0], W[0, 1], W[1, 1] = A, _delta(2), _delta(2)
    a0 = wl.grid_uniform(dims, 82)
    x0 = np.stack([a0, np.full_like(a0, c)])
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = VectorStencilPlan(dims, W, precision)
    g = torch.tensor(x0, dtype=dt, device="cuda")
    plan.run(g, T)
    assert plan.status() == 0
    plan.close()
    got = g.double().cpu().numpy()
    want = oracle.stencil_loop(a0, A, T, "periodic") + T * c
    assert np.max(np.abs(got[0] - want)) / np.max(np.abs(want)) <= TOL[precision]
    assert np.max(np.abs(got[1] - c)) / c <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_vector_leapfrog_wave(precision):
    # u_{t+1} = 2 u_t - u_{t-1} + k^2 L u_t as fields (u_t, u_{t-1})
    from paper_2105_06676_gb300 import VectorStencilPlan
    l, k2, T = 1024, 0.3, 200
    L = np.array([1.0, -2.0, 1.0])
    W = np.zeros((2, 2, 3))
    W[0, 0] = 2 * _delta(1) + k2 * L
    W[0, 1] = -_delta(1)
    W[1, 0] = _delta(1)
    u0 = np.sin(2 * np.pi * 3 * np.arange(l) / l) + 0.05 * wl.grid_uniform((l,), 83)
    prev, cur = u0.copy(), u0.copy()
    for _ in range(T):
        lap = np.roll(cur, -1) + np.roll(cur, 1) - 2 * cur
        prev, cur = cur, 2 * cur - prev + k2 * lap
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = VectorStencilPlan((l,), W, precision)
    g = torch.tensor(np.stack([u0, u0]), dtype=dt, device="cuda")
    plan.run(g, T)
    assert plan.status() == 0
    plan.close()
    got = g.double().cpu().numpy()
    scale = max(np.max(np.abs(u0)), np.max(np.abs(cur)))
    assert np.max(np.abs(got[0] - cur)) / scale <= TOL[precision] * 10
    assert np.max(np.abs(got[1] - prev)) / scale <= TOL[precision] * 10
