"""Implicit stencils Q a_{t+1} = S a_t on the GPU (stencil_plan_implicit)
against the oracle (appendix "Supporting Implicit Stencils"): the spectral
oracle with Lambda_R = Lambda_Q^+ Lambda_S, the dense pseudoinverse definition
on small grids, and the implicit equation's residual at full size."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

import oracle
from oracle import implicit as imp
from paper_2105_06676_gb300 import _capi
from paper_2105_06676_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-4}


def _delta(ndim):
    w = np.zeros((3,) * ndim)
    w[(1,) * ndim] = 1.0
    return w


def _laplacian(ndim):
    L = np.zeros((3,) * ndim)
    c = (1,) * ndim
    L[c] = -2.0 * ndim
    for a in range(ndim):
        for s in (0, 2):
            idx = list(c)
            idx[a] = s
            L[tuple(idx)] = 1.0
    return L


def _crank_nicolson(ndim, nu):
    return _delta(ndim) + 0.5 * nu * _laplacian(ndim), _delta(ndim) - 0.5 * nu * _laplacian(ndim)


def _general_pair(ndim, seed):
    # non-symmetric S and Q = 1.3 I - 0.3 B (B a non-negative box summing to
    # 1): Re Lambda_Q >= 1, so |Lambda_R| <= |Lambda_S| <= 1 and nothing grows
    S = wl.weights_random_box(ndim, 1, seed)
    Q = -0.3 * wl.weights_random_box(ndim, 1, seed + 1000)
    Q[(1,) * ndim] += 1.3
    return S, Q


def _run(dims, S, Q, T, precision):
    from paper_2105_06676_gb300 import StencilPlan
    a0 = wl.grid_uniform(dims, 31)
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = StencilPlan(dims, S, "periodic", precision, implicit_weights=Q)
    g = torch.tensor(a0, dtype=dt, device="cuda")
    plan.run(g, T)
    assert plan.status() == 0
    out = g.double().cpu().numpy()
    plan.close()
    return a0, out


def _err(got, ref, a0):
    return float(np.max(np.abs(got - ref)) / max(np.max(np.abs(a0)), np.max(np.abs(ref))))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("dims", [(64,), (4096,), (256, 128), (1024, 512), (32, 16, 64)])
@pytest.mark.parametrize("kind", ["cn", "general"])
@pytest.mark.parametrize("T", [1, 13, 400])
def test_implicit_matches_spectral_oracle(precision, dims, kind, T):
    S, Q = _crank_nicolson(len(dims), 1.7) if kind == "cn" else _general_pair(len(dims), 41)
    a0, out = _run(dims, S, Q, T, precision)
    ref = imp.stencil_fft_periodic_implicit(a0, S, Q, T)
    assert _err(out, ref, a0) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_implicit_small_grid_matches_dense_pseudoinverse(precision):
    dims, T = (16, 8), 9
    S, Q = _general_pair(2, 42)
    a0, out = _run(dims, S, Q, T, precision)
    assert _err(out, imp.implicit_dense(a0, S, Q, T), a0) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_implicit_singular_q_projects_out_its_null_space(precision):
    # Q = -Laplacian, S = identity: Lambda_Q(0) = 0 drops the mean
    dims, T = (128, 64), 2
    Q = -_laplacian(2)
    a0, out = _run(dims, _delta(2), Q, T, precision)
    ref = imp.stencil_fft_periodic_implicit(a0, _delta(2), Q, T)
    assert _err(out, ref, a0) <= TOL[precision]
    assert abs(out.mean()) <= TOL[precision] * np.max(np.abs(ref))


def test_implicit_result_satisfies_the_equation_at_full_size():
    # 2048^2 FP64: Q a_{T+1} = S a_T with Q and S applied by the loop oracle
    from paper_2105_06676_gb300 import StencilPlan
    dims, T = (2048, 2048), 50
    S, Q = _crank_nicolson(2, 2.5)
    a0 = wl.grid_uniform(dims, 33)
    plan = StencilPlan(dims, S, "periodic", "fp64", implicit_weights=Q)
    outs = []
    for t in (T, T + 1):
        g = torch.tensor(a0, device="cuda")
        plan.run(g, t)
        outs.append(g.cpu().numpy())
    assert plan.status() == 0
    plan.close()
    lhs = oracle.stencil_loop(outs[1], Q, 1, "periodic")
    rhs = oracle.stencil_loop(outs[0], S, 1, "periodic")
    assert np.max(np.abs(lhs - rhs)) / np.max(np.abs(a0)) <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_implicit_new_T_rebuilds_the_table(precision):
    from paper_2105_06676_gb300 import StencilPlan
    dims = (128, 256)
    S, Q = _general_pair(2, 43)
    a0 = wl.grid_uniform(dims, 34)
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = StencilPlan(dims, S, "periodic", precision, implicit_weights=Q)
    outs = {}
    for T in (7, 7, 30, 7, 0):
        g = torch.tensor(a0, dtype=dt, device="cuda")
        plan.run(g, T)
        outs.setdefault(T, []).append(g.double().cpu().numpy())
    assert plan.status() == 0
    plan.close()
    np.testing.assert_array_equal(outs[7][0], outs[7][1])
    np.testing.assert_array_equal(outs[7][0], outs[7][2])
    np.testing.assert_array_equal(outs[0][0], a0.astype(np.float32 if precision == "fp32" else np.float64))
    for T in (7, 30):
        assert _err(outs[T][0], imp.stencil_fft_periodic_implicit(a0, S, Q, T), a0) <= TOL[precision]


def test_implicit_symbol_power_table():
    # stencil_symbol_power returns Lambda_R^T (FP64) for implicit plans
    from paper_2105_06676_gb300 import StencilPlan
    dims, T = (32, 64), 5
    S, Q = _general_pair(2, 44)
    plan = StencilPlan(dims, S, "periodic", "fp64", implicit_weights=Q)
    got = plan.symbol_power(T).cpu().numpy()
    plan.close()
    want = oracle.symbol_power(imp.implicit_symbol(S, Q, dims), T)[:, : dims[1] // 2 + 1]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12 * np.max(np.abs(want)))


def test_implicit_rejects_what_it_does_not_cover():
    lib = _capi.lib()
    S, Q = _crank_nicolson(1, 1.0)
    h = ctypes.c_void_p()
    dp = ctypes.POINTER(ctypes.c_double)
    long1d = (ctypes.c_int64 * 1)(1 << 20)
    rc = lib.stencil_plan_implicit(ctypes.byref(h), 1, long1d, 1, S.ctypes.data_as(dp),
                                   Q.ctypes.data_as(dp), _capi.STENCIL_FP32)
    assert rc == -7   # STENCIL_EUNSUPPORTED: n1 x n2 passes take no table
    from paper_2105_06676_gb300 import StencilPlan
    S2, Q2 = _crank_nicolson(2, 1.0)
    plan = StencilPlan((64, 64), S2, "periodic", "fp32", implicit_weights=Q2)
    rc = lib.stencil_plan_set_weights(plan.handle, 1, S2.ctypes.data_as(dp))
    assert rc == -7
    plan.close()
