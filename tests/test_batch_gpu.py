"""The mixed-shape batch executor (stencil_batch_*) against the oracle: one
persistent launch over requests of different dimension, shape, radius,
weights and T, each element-wise against the loop (small T) or the numpy
StencilFFT-P, and against the same request solved alone by a plan."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2105_06676_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-4}


def _mixed_requests(count, seed, precision):
    rng = np.random.default_rng(seed)
    shapes = [(64,), (4096,), (8, 8), (32, 64), (64, 16), (128, 32), (16, 16, 16), (8, 32, 16),
              (4, 4, 4), (256,), (16, 128)]
    reqs = []
    for i in range(count):
        dims = shapes[rng.integers(len(shapes))]
        r = int(rng.integers(0, 4))
        r = min(r, (min(dims) - 1) // 2)
        w = wl.weights_random_box(len(dims), r, seed * 1000 + i)
        T = int(10 ** rng.uniform(0, 3.5))
        a0 = wl.grid_uniform(dims, seed * 1000 + 500 + i)
        reqs.append((dims, w, T, a0))
    return reqs


def _run_batch(reqs, precision, capacity=None):
    from paper_2105_06676_gb300 import BatchExecutor
    dt = torch.float32 if precision == "fp32" else torch.float64
    ex = BatchExecutor(capacity or len(reqs), precision)
    grids = [torch.tensor(a0, dtype=dt, device="cuda") for (_, _, _, a0) in reqs]
    ex.run(grids, [w for (_, w, _, _) in reqs], [T for (_, _, T, _) in reqs])
    assert ex.status() == 0
    ex.close()
    return [g.double().cpu().numpy() for g in grids]


def err_rel(got, ref, a0):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(a0)))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("count,seed", [(1, 1), (7, 2), (40, 3), (400, 4)])
def test_batch_matches_oracle(precision, count, seed):
    reqs = _mixed_requests(count, seed, precision)
    outs = _run_batch(reqs, precision)
    for (dims, w, T, a0), got in zip(reqs, outs):
        ref = oracle.stencil_fft_periodic(a0, w, T)
        assert err_rel(got, ref, a0) <= TOL[precision], (dims, w.shape, T)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_small_T_against_loop(precision):
    reqs = [(d, wl.weights_random_box(len(d), 1, 7 + i), T, wl.grid_uniform(d, 9 + i))
            for i, (d, T) in enumerate([((64,), 3), ((16, 32), 5), ((8, 8, 16), 2), ((32, 8), 0)])]
    outs = _run_batch(reqs, precision)
    for (dims, w, T, a0), got in zip(reqs, outs):
        assert err_rel(got, oracle.stencil_loop(a0, w, T, "periodic"), a0) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_equals_single_plan_solves(precision):
    from paper_2105_06676_gb300 import StencilPlan
    reqs = _mixed_requests(12, 5, precision)
    outs = _run_batch(reqs, precision)
    dt = torch.float32 if precision == "fp32" else torch.float64
    for (dims, w, T, a0), got in zip(reqs, outs):
        plan = StencilPlan(dims, w, "periodic", precision)
        g = torch.tensor(a0, dtype=dt, device="cuda")
        plan.run(g, T)
        plan.close()
        assert err_rel(got, g.double().cpu().numpy(), a0) <= TOL[precision]


def test_batch_repeated_runs_and_limits():
    from paper_2105_06676_gb300 import BatchExecutor
    assert BatchExecutor.smem_bytes((64, 128), "fp32") > 0
    assert BatchExecutor.smem_bytes((256, 256), "fp32") == 0     # beyond one CTA's spectrum
    assert BatchExecutor.smem_bytes((48, 64), "fp32") == 0       # not a power of two
    ex = BatchExecutor(8, "fp32")
    w = wl.weights_star(2, 0.6, 0.1)
    a0 = wl.grid_uniform((32, 32), 11)
    g = torch.tensor(a0, dtype=torch.float32, device="cuda")
    for _ in range(3):
        ex.run([g], [w], [10])
    assert ex.status() == 0
    ex.close()
    ref = oracle.stencil_fft_periodic(a0, w, 30)
    assert err_rel(g.double().cpu().numpy(), ref, a0) <= 2e-4
