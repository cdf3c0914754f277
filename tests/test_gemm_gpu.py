"""The tensor-core DFT variants (precision fp32_gemm_bf16 / _fp16 / _bf16x3):
every radix-16 butterfly of the strided-axis transforms is a tcgen05 GEMM.
The split-operand variant must meet the FP32 tolerance (2e-4 relative to
max|a_0|); the single-term variants carry their operand rounding (bf16 2^-9,
fp16 2^-12 per stage) and are held to looser bounds derived from it: a few
stages per transform, two transforms per axis, errors adding in quadrature
at worst linearly -> 3e-2 for bf16, 4e-3 for fp16."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2105_06676_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BOUND = {"fp32_gemm_bf16x3": 2e-4, "fp32_gemm_fp16": 4e-3, "fp32_gemm_bf16": 3e-2}


def run(a0, w, T, precision):
    from paper_2105_06676_gb300 import StencilPlan
    g = torch.tensor(a0, dtype=torch.float32, device="cuda")
    plan = StencilPlan(a0.shape, w, "periodic", precision)
    plan.run(g, T)
    rc = plan.status()
    plan.close()
    assert rc == 0, f"device status {rc}"
    return g.double().cpu().numpy()


def err_rel(got, ref, a0):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(a0)))


@pytest.mark.parametrize("precision", list(BOUND))
@pytest.mark.parametrize("dims,r", [((256, 64), 1), ((512, 256), 2), ((256, 256, 16), 1),
                                    ((4096, 32), 1), ((1024, 512), 3)])
@pytest.mark.parametrize("T", [1, 9, 500])
def test_gemm_variant_vs_oracle(precision, dims, r, T):
    w = wl.weights_random_box(len(dims), r, 7 + T)
    a0 = wl.grid_uniform(dims, 8 + T)
    n = int(np.prod(dims))
    ref = oracle.stencil_loop(a0, w, T, "periodic") if n * T <= 5e7 else \
        oracle.stencil_fft_periodic(a0, w, T)
    assert err_rel(run(a0, w, T, precision), ref, a0) <= BOUND[precision]


@pytest.mark.parametrize("precision", list(BOUND))
def test_gemm_variant_star7_512_cube_vs_spectral_oracle(precision):
    wk = wl.star3d_512("fp32")
    a0 = wk.grid()
    ref = oracle.stencil_fft_periodic(a0, wk.weights, wk.T)
    assert err_rel(run(a0, wk.weights, wk.T, precision), ref, a0) <= BOUND[precision]


def test_gemm_variant_fourier_mode_exact_decay():
    # a single mode of a symmetric stencil decays by lambda(k)^T: checks the
    # transform's orientation and scaling through the tensor-core stages
    dims, T = (512, 512), 40
    w = wl.weights_star(2, 0.6, 0.1)
    k = (5, 9)
    a0 = wl.fourier_mode(dims, k)
    lam = 0.6 + 0.2 * np.cos(2 * np.pi * k[0] / dims[0]) + 0.2 * np.cos(2 * np.pi * k[1] / dims[1])
    assert err_rel(run(a0, w, T, "fp32_gemm_bf16x3"), lam ** T * a0, a0) <= 2e-4


def test_gemm_rejects_unsupported_shapes():
    from paper_2105_06676_gb300 import StencilPlan, StencilError
    w2 = wl.weights_star(2, 0.6, 0.1)
    for dims, boundary in [((128, 64), "periodic"), ((8192, 64), "periodic"),
                           ((512, 512), "dirichlet")]:
        with pytest.raises(StencilError):
            StencilPlan(dims, w2, boundary, "fp32_gemm_bf16")
    with pytest.raises(StencilError):
        StencilPlan((4096,), np.array([0.25, 0.5, 0.25]), "periodic", "fp32_gemm_bf16")


def test_abandoned_tensor_core_wait_reports_timeout_and_plan_recovers(monkeypatch):
    # With the test hook the tensor-core kernel issues no MMA, so its first
    # bounded wait runs out (about 2 s): the CTA records the timeout, issues and
    # waits on nothing more, releases its tensor memory and returns. The host
    # reads STENCIL_ETIMEOUT; the context stays usable and the next solve (hook
    # off) is correct.
    import time
    from paper_2105_06676_gb300 import StencilPlan
    dims, T = (256, 64), 30           # 3 CTAs: every one of them times out once
    w = wl.weights_star(2, 0.6, 0.1)
    a0 = wl.grid_uniform(dims, 3)
    plan = StencilPlan(dims, w, "periodic", "fp32_gemm_bf16x3")
    g = torch.tensor(a0, dtype=torch.float32, device="cuda")
    monkeypatch.setenv("STENCILFFT_TEST_SKIP_MMA_COMMIT", "1")
    t0 = time.perf_counter()
    plan.run(g, T)
    rc = plan.status()
    elapsed = time.perf_counter() - t0
    monkeypatch.delenv("STENCILFFT_TEST_SKIP_MMA_COMMIT")
    assert rc == -4, rc               # STENCIL_ETIMEOUT
    assert elapsed < 30.0
    g = torch.tensor(a0, dtype=torch.float32, device="cuda")
    plan.run(g, T)
    assert plan.status() == 0
    ref = oracle.stencil_loop(a0, w, T)
    assert err_rel(g.double().cpu().numpy(), ref, a0) <= BOUND["fp32_gemm_bf16x3"]
    plan.close()
