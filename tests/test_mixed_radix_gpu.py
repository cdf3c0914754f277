"""Mixed-radix periodic solves (axis lengths with prime factors 2, 3, 5, 7; the
paper's 8000^2 and 800^3 grids, Sec. 6 Tab. "experimental-results") against
the oracle: the loop on small grids, the numpy StencilFFT-P at medium sizes,
and Fourier-mode closed forms at the paper's full sizes. Tolerance relative to
max|a_0|: 1e-10 (FP64), 2e-4 (FP32)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import vector_fields as vf
from paper_2105_06676_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-4}


def run_gpu(a0, w, T, precision):
    from paper_2105_06676_gb300 import StencilPlan
    dt = torch.float32 if precision == "fp32" else torch.float64
    g = torch.tensor(a0, dtype=dt, device="cuda")
    plan = StencilPlan(a0.shape, w, "periodic", precision)
    plan.run(g, T)
    rc = plan.status()
    plan.close()
    assert rc == 0, f"device status {rc}"
    return g.double().cpu().numpy()


def err_rel(got, ref, a0):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(a0)))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("dims,r", [((30,), 1), ((1000,), 1), ((2058,), 2), ((6,), 1), ((12, 10), 1),
                                    ((96, 80), 1), ((80, 96), 2), ((64, 90), 1), ((20, 30, 42), 1),
                                    ((16, 18, 10), 1), ((14, 32, 40), 1)])
@pytest.mark.parametrize("T", [1, 3, 40])
def test_mixed_matches_loop(dims, r, T, precision):
    w = wl.weights_random_box(len(dims), r, 90 + T)
    a0 = wl.grid_uniform(dims, 91)
    got = run_gpu(a0, w, T, precision)
    assert err_rel(got, oracle.stencil_loop(a0, w, T, "periodic"), a0) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("dims,T", [((4000,), 5000), ((800, 1000), 300), ((1000, 800), 1000),
                                    ((120, 126, 250), 50), ((7000, 60), 9)])
def test_mixed_matches_spectral_oracle(dims, T, precision):
    w = wl.weights_random_box(len(dims), 1, 92)
    a0 = wl.grid_uniform(dims, 93)
    got = run_gpu(a0, w, T, precision)
    ref = oracle.stencil_fft_periodic(a0, w, T, workers=8)
    assert err_rel(got, ref, a0) <= TOL[precision]


def _cos_modes(dims, ks, amps):
    a = np.full(dims, 0.5)
    axes = np.meshgrid(*[np.arange(l) for l in dims], indexing="ij", sparse=True)
    for k, c in zip(ks, amps):
        ph = sum(2 * np.pi * kk * x / l for kk, x, l in zip(k, axes, dims))
        a = a + c * np.cos(ph)
    return a


def _star_symbol(k, dims, center, nb):
    return center + sum(2 * nb * np.cos(2 * np.pi * kk / l) for kk, l in zip(k, dims))


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("dims,T,center,nb", [((8000, 8000), 100000, 0.6, 0.1),
                                              ((800, 800, 800), 10000, 0.4, 0.1)])
def test_mixed_paper_sizes_fourier_modes(dims, T, center, nb, precision):
    # the paper's seidel2d / heat3d sizes: a constant plus cosine modes of a
    # symmetric star stencil evolve in closed form, a_T = 0.5 (sum w)^T +
    # sum c lambda(k)^T cos(2 pi k.x / l)
    if precision == "fp64" and len(dims) == 3:
        pytest.skip("800^3 FP64 needs 8 GB of grid and spectrum; FP32 covers the size")
    w = wl.weights_star(len(dims), center, nb)
    ks = [(1,) * len(dims), (3, 2, 1)[: len(dims)], (20, 7, 5)[: len(dims)]]
    amps = [0.3, 0.2, 0.1]
    a0 = _cos_modes(dims, ks, amps)
    want = _cos_modes(dims, ks, [c * _star_symbol(k, dims, center, nb) ** T for k, c in zip(ks, amps)])
    got = run_gpu(a0, w, T, precision)
    assert err_rel(got, want, a0) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_mixed_vector_fields(precision):
    from paper_2105_06676_gb300 import VectorStencilPlan
    dims, T, m = (60, 90), 11, 2
    rng = np.random.default_rng(94)
    W = rng.random((m, m, 3, 3))
    W /= W.sum(axis=(1, 2, 3), keepdims=True)
    a0 = np.stack([wl.grid_uniform(dims, 95 + i) for i in range(m)])
    plan = VectorStencilPlan(dims, W, precision)
    g = torch.tensor(a0, dtype=torch.float64 if precision == "fp64" else torch.float32, device="cuda")
    plan.run(g, T)
    assert plan.status() == 0
    plan.close()
    assert err_rel(g.double().cpu().numpy(), vf.vector_loop(a0, W, T), a0) <= TOL[precision]


def test_mixed_symbol_power():
    from paper_2105_06676_gb300 import StencilPlan
    dims, T = (30, 40), 7
    w = wl.weights_random_box(2, 1, 96)
    plan = StencilPlan(dims, w, "periodic", "fp64")
    got = plan.symbol_power(T).cpu().numpy()
    plan.close()
    want = oracle.symbol_power(oracle.symbol_closed_form(w, dims), T)[:, : dims[1] // 2 + 1]
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
