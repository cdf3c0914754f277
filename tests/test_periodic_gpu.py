"""Parity of the periodic CUDA path (StencilFFT-P) with the CPU oracle.

Tolerance (relative to max|a_0|): 1e-10 for FP64 plans, 2e-4 for FP32 plans.
Small and medium cases compare every element with the nested-loop oracle;
the full-size grids compare with the oracle's numpy StencilFFT-P (itself pinned
to the loop) and with closed forms that hold at any size.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2105_06676_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-4}


def run_gpu(a0, w, T, precision, boundary="periodic", cutoff=None):
    from paper_2105_06676_gb300 import StencilPlan
    dt = torch.float32 if precision == "fp32" else torch.float64
    g = torch.tensor(a0, dtype=dt, device="cuda")
    plan = StencilPlan(a0.shape, w, boundary, precision)
    if cutoff is not None:
        plan.set_cutoff(cutoff)
    plan.run(g, T)
    rc = plan.status()
    plan.close()
    assert rc == 0, f"device status {rc}"
    return g.double().cpu().numpy()


def err_rel(got, ref, a0):
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(a0)))


SMALL = [
    ((4,), "sym", 1), ((8,), "asym", 1), ((64,), "sym", 1), ((256,), "asym", 2), ((4096,), "sym", 1),
    ((8, 8), "sym", 1), ((16, 32), "asym", 1), ((64, 128), "asym", 2), ((256, 64), "sym", 1),
    ((128, 16), "asym", 1), ((8, 8, 8), "sym", 1), ((16, 8, 32), "asym", 1), ((32, 32, 16), "asym", 2),
]


def weights_for(ndim, kind, r, seed):
    if kind == "sym":
        w = wl.weights_random_box(ndim, r, seed)
        return 0.5 * (w + np.flip(w))            # symmetric under m -> -m: real symbol
    return wl.weights_random_box(ndim, r, seed)  # general: complex symbol


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("dims,kind,r", SMALL)
@pytest.mark.parametrize("T", [1, 2, 3, 7, 64, 1000])
def test_periodic_matches_loop(dims, kind, r, T, precision):
    if max(dims) < 2 * r + 1:
        pytest.skip("grid smaller than the stencil")
    n = int(np.prod(dims))
    if n * T > 3e8:
        pytest.skip("loop oracle too slow for this combination")
    w = weights_for(len(dims), kind, r, 11 + T)
    a0 = wl.grid_uniform(dims, 5 + T)
    ref = oracle.stencil_loop(a0, w, T)
    got = run_gpu(a0, w, T, precision)
    assert err_rel(got, ref, a0) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_T_zero_leaves_grid_unchanged(precision):
    a0 = wl.grid_uniform((32, 16), 3)
    got = run_gpu(a0, wl.weights_star(2, 0.6, 0.1), 0, precision)
    np.testing.assert_array_equal(got, a0.astype(np.float32 if precision == "fp32" else np.float64))


def test_worked_example_symbol_and_matrix():
    # appendix "Stencil Matrix Example": weights (-2, 1, 3) on 4 cells
    from paper_2105_06676_gb300 import StencilPlan
    w = np.array([-2.0, 1.0, 3.0])
    plan = StencilPlan((4,), w, "periodic", "fp64")
    lam = plan.symbol_power(1).cpu().numpy()
    np.testing.assert_allclose(lam, [2, 1 + 5j, 0], atol=1e-14)
    lam3 = plan.symbol_power(3).cpu().numpy()
    np.testing.assert_allclose(lam3, np.array([2, 1 + 5j, 0]) ** 3, atol=1e-12)
    plan.close()
    S = np.stack([run_gpu(np.eye(4)[j], w, 1, "fp64") for j in range(4)], axis=1)
    np.testing.assert_allclose(S, [[1, 3, 0, -2], [-2, 1, 3, 0], [0, -2, 1, 3], [3, 0, -2, 1]],
                               atol=1e-12)


@pytest.mark.parametrize("dims,r", [((64,), 1), ((16, 32), 2), ((8, 16, 32), 1), ((4096, 64), 1)])
@pytest.mark.parametrize("T", [0, 1, 5, 1000, 10000])
def test_symbol_power_table_matches_oracle(dims, r, T):
    from paper_2105_06676_gb300 import StencilPlan
    w = wl.weights_random_signed(len(dims), r, 3 + T)
    w = w / np.abs(w).sum()                   # |lambda| <= 1: lambda^T stays finite
    plan = StencilPlan(dims, w, "periodic", "fp64")
    got = plan.symbol_power(T).cpu().numpy()
    plan.close()
    lam = oracle.symbol_closed_form(w, dims)
    half = lam[..., : dims[-1] // 2 + 1]
    ref = oracle.symbol_power(half, T)
    # first-order error bound of a T-th power: T |lam|^(T-1) |d lam| + T eps |lam|^T,
    # with |d lam| <= eps * sum|w| * (number of terms)
    eps = np.finfo(np.float64).eps
    a = np.abs(half)
    dlam = 16 * eps * np.abs(w).sum()
    bound = (max(T, 1) * (a ** max(T - 1, 0) * dlam + 16 * eps * a ** T)) + 1e-300
    assert np.all(np.abs(got - ref) <= bound)


# -------------------------------------------------------------------------
# full-size grids of the benchmark workloads
# -------------------------------------------------------------------------
def test_heat1d_4096_full_size_fp64():
    wk = wl.heat1d_4096()
    a0 = wk.grid()
    ref = oracle.stencil_loop(a0, wk.weights, wk.T)
    got = run_gpu(a0, wk.weights, wk.T, "fp64")
    assert err_rel(got, ref, a0) <= 1e-10


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_star2d_4096_full_size_vs_spectral_oracle(precision):
    wk = wl.star2d_4096(precision)
    a0, ks, amps = wl.grid_with_modes(wk.dims, wk.grid_seed, 3002)
    for T in (1, 10, 100, wk.T):
        ref = oracle.stencil_fft_periodic(a0, wk.weights, T)
        got = run_gpu(a0, wk.weights, T, precision)
        assert err_rel(got, ref, a0) <= TOL[precision], T


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_star2d_4096_fourier_modes_closed_form(precision):
    # a pure mode sin(k.x) scales by lambda(k)^T with lambda = 0.6 + 0.2 cos + 0.2 cos
    wk = wl.star2d_4096(precision)
    l = wk.dims[0]
    ks, _ = wl.seeded_modes(2, 3002)
    for k in ks + [(l // 2, l // 2), (64, 0)]:
        a0 = wl.fourier_mode(wk.dims, k, 0.2)
        lam = 0.6 + 0.2 * np.cos(2 * np.pi * k[0] / l) + 0.2 * np.cos(2 * np.pi * k[1] / l)
        got = run_gpu(a0, wk.weights, wk.T, precision)
        assert err_rel(got, lam ** wk.T * a0, a0) <= TOL[precision], k


def test_star2d_4096_T1_loop_sample_fp32():
    wk = wl.star2d_4096("fp32")
    a0 = wk.grid()
    ref = oracle.stencil_loop(a0, wk.weights, 3)
    got = run_gpu(a0, wk.weights, 3, "fp32")
    assert err_rel(got, ref, a0) <= 2e-4


def test_star2d_mass_conservation_fp32():
    wk = wl.star2d_4096("fp32")
    a0 = wk.grid()
    got = run_gpu(a0, wk.weights, wk.T, "fp32")
    assert abs(got.mean() - a0.astype(np.float32).astype(np.float64).mean()) < 2e-4


def test_star3d_512_full_size_fp32():
    wk = wl.star3d_512("fp32")
    a0 = wk.grid()
    # T = 2 against the loop on the full grid
    ref = oracle.stencil_loop(a0, wk.weights, 2)
    got = run_gpu(a0, wk.weights, 2, "fp32")
    assert err_rel(got, ref, a0) <= 2e-4
    # T = 1000 on pure modes (closed form) and the mean (mass)
    l = wk.dims[0]
    for k in [(1, 2, 3), (5, 0, 9), (256, 256, 256)]:
        m = wl.fourier_mode(wk.dims, k, 0.3)
        lam = 0.4 + sum(0.2 * np.cos(2 * np.pi * kk / l) for kk in k)
        gotm = run_gpu(m, wk.weights, wk.T, "fp32")
        assert err_rel(gotm, lam ** wk.T * m, m) <= 2e-4, k
    full = run_gpu(a0, wk.weights, wk.T, "fp32")
    assert abs(full.mean() - a0.mean()) < 2e-4


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_run_host_matches_device_run(precision):
    from paper_2105_06676_gb300 import StencilPlan
    dims, T = (256, 128), 77
    w = wl.weights_random_box(2, 1, 9)
    a0 = wl.grid_uniform(dims, 4)
    dt = torch.float32 if precision == "fp32" else torch.float64
    plan = StencilPlan(dims, w, "periodic", precision)
    host = torch.tensor(a0, dtype=dt).pin_memory()
    out = plan.run_host(host, T)
    dev = torch.tensor(a0, dtype=dt, device="cuda")
    plan.run(dev, T)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.numpy(), dev.cpu().numpy())
    plan.close()


def test_nonfinite_output_is_reported():
    from paper_2105_06676_gb300 import StencilPlan
    dims = (64, 64)
    w = wl.weights_star(2, 3.0, 1.0)          # |lambda| up to 7: lambda^T overflows
    plan = StencilPlan(dims, w, "periodic", "fp32")
    g = torch.ones(dims, dtype=torch.float32, device="cuda")
    plan.run(g, 100000)
    assert plan.status() == -5
    assert plan.status() == 0                 # latch cleared
    plan.close()


def test_profile_counts_launches():
    from paper_2105_06676_gb300 import StencilPlan
    dims = (128, 256)
    plan = StencilPlan(dims, wl.weights_star(2, 0.6, 0.1), "periodic", "fp32")
    g = torch.tensor(wl.grid_uniform(dims, 1), dtype=torch.float32, device="cuda")
    plan.profile(True)
    for _ in range(3):
        plan.run(g, 10)
    prof = plan.profile_read()
    assert {k: v[1] for k, v in prof.items()} == {"rows_r2c": 3, "cols_fused": 3, "rows_c2r": 3}
    assert all(v[0] > 0 for v in prof.values())
    plan.close()


# 1-D axes longer than one CTA holds (FP32 above 2^15, FP64 above 2^14): the
# packed sequence runs as n1 x n2 passes with the spectrum in k1 + n1 k2 order.
LONG_1D = [(1 << 15, "fp64"), (1 << 16, "fp32"), (1 << 16, "fp64"), (1 << 17, "fp32"),
           (1 << 19, "fp32"), (1 << 20, "fp64")]


@pytest.mark.parametrize("L,precision", LONG_1D)
@pytest.mark.parametrize("kind,r", [("sym", 1), ("asym", 2), ("asym", 3)])
@pytest.mark.parametrize("T", [1, 7, 100])
def test_long_1d_matches_loop(L, precision, kind, r, T):
    if L * T > 2e7:
        pytest.skip("loop oracle too slow for this combination")
    w = weights_for(1, kind, r, 40 + r + T)
    a0 = wl.grid_uniform((L,), 11 + T)
    ref = oracle.stencil_loop(a0, w, T, "periodic")
    assert err_rel(run_gpu(a0, w, T, precision), ref, a0) <= TOL[precision]


@pytest.mark.parametrize("L,precision", [(1 << 21, "fp32"), (1 << 22, "fp64"), (1 << 24, "fp32")])
@pytest.mark.parametrize("T", [3, 1000, 100000])
def test_long_1d_full_size_vs_spectral_oracle(L, precision, T):
    w = weights_for(1, "asym", 2, 77)
    a0 = wl.grid_uniform((L,), 5)
    ref = oracle.stencil_fft_periodic(a0, w, T)
    assert err_rel(run_gpu(a0, w, T, precision), ref, a0) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_long_1d_fourier_mode_closed_form(precision):
    # a_0 = cos(2 pi k x / L) with symmetric weights: a_T = lambda(k)^T a_0, lambda real
    L, T = 1 << 22, 5000
    w = np.array([0.2, 0.6, 0.2])
    x = np.arange(L)
    got = []
    for k in (1, 37, L // 2 - 3):
        a0 = np.cos(2 * np.pi * k * x / L)
        lam = 0.6 + 0.4 * np.cos(2 * np.pi * k / L)
        got.append(err_rel(run_gpu(a0, w, T, precision), lam ** T * a0, a0))
    assert max(got) <= TOL[precision]


def test_long_1d_nyquist_and_mean():
    # the Nyquist mode (-1)^x and the mean survive exactly as lambda(L/2)^T and 1
    L, T = 1 << 18, 9
    w = np.array([0.1, 0.7, 0.2])
    x = np.arange(L)
    a0 = 0.5 + (-1.0) ** x
    lam_nyq = 0.7 - 0.1 - 0.2
    ref = 0.5 + lam_nyq ** T * (-1.0) ** x
    assert err_rel(run_gpu(a0, w, T, "fp64"), ref, a0) <= 1e-12


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_gemm_bf16x3"])
@pytest.mark.parametrize("dims", [(256, 128), (32, 16, 64), (512, 256, 8)])
def test_run_host_in_place_on_pinned_memory(precision, dims):
    # both buffers pinned: the first and last passes address host memory directly;
    # one pinned and one pageable: the staging-copy path. Same kernels, same bits.
    from paper_2105_06676_gb300 import StencilPlan
    if precision.startswith("fp32_gemm") and min(dims[:-1]) < 256:
        pytest.skip("tensor-core variant needs strided axes >= 256")
    T = 31
    w = wl.weights_random_box(len(dims), 1, 12)
    a0 = wl.grid_uniform(dims, 13)
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = StencilPlan(dims, w, "periodic", precision)
    dev = torch.tensor(a0, dtype=dt, device="cuda")
    plan.run(dev, T)
    torch.cuda.synchronize()
    want = dev.cpu().numpy()
    src = torch.tensor(a0, dtype=dt).pin_memory()
    direct = plan.run_host(src, T, torch.empty_like(src).pin_memory())
    staged = plan.run_host(src, T, torch.empty_like(src))
    aliased = src.clone().pin_memory()
    plan.run_host(aliased, T, aliased)
    assert plan.status() == 0
    plan.close()
    np.testing.assert_array_equal(direct.numpy(), want)
    np.testing.assert_array_equal(staged.numpy(), want)
    np.testing.assert_array_equal(aliased.numpy(), want)
    tol = 1e-10 if precision == "fp64" else 2e-4
    assert err_rel(want, oracle.stencil_loop(a0, w, T, "periodic"), a0) <= tol


@pytest.mark.parametrize("dims,precision", [((4096,), "fp64"), ((1024,), "fp32"), ((64, 32, 128), "fp32"),
                                            ((32, 16, 64), "fp64")])
def test_repeated_T_uses_cached_multipliers_same_result(dims, precision):
    # the second run with the same T builds the Lambda^T table, the third reads
    # it: every run must give the same bits, and a new T or new weights must
    # not reuse it
    from paper_2105_06676_gb300 import StencilPlan
    w = wl.weights_random_box(len(dims), 1, 21)
    a0 = wl.grid_uniform(dims, 22)
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = StencilPlan(dims, w, "periodic", precision)
    outs = []
    for T in (37, 37, 37, 38, 37):
        g = torch.tensor(a0, dtype=dt, device="cuda")
        plan.run(g, T)
        outs.append(g.cpu().numpy())
    assert plan.status() == 0
    plan.close()
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])
    np.testing.assert_array_equal(outs[0], outs[4])
    tol = 1e-10 if precision == "fp64" else 2e-4
    assert err_rel(outs[3], oracle.stencil_loop(a0, w, 38, "periodic"), a0) <= tol
    assert err_rel(outs[2], oracle.stencil_loop(a0, w, 37, "periodic"), a0) <= tol


# Strided axes of 512..4096 points (the persistent TMA-fed column passes: tiles
# of 8192 complex values = 8192 / n columns, the last tile ragged) against the
# loop, element by element; 3-D shapes put the long axis first (fused pass with
# a mid axis) and second (forward / inverse passes over outer slabs).
TMA_SHAPES = [((512, 64), "asym", 1), ((1024, 32), "sym", 1), ((2048, 16), "asym", 2),
              ((4096, 16), "asym", 1), ((4096, 64), "sym", 2), ((512, 16, 8), "asym", 1),
              ((16, 512, 8), "asym", 1), ((8, 1024, 16), "sym", 2), ((512, 512, 4), "asym", 1)]


@pytest.mark.parametrize("dims,kind,r", TMA_SHAPES)
@pytest.mark.parametrize("T", [1, 3, 50])
def test_long_strided_axes_match_loop(dims, kind, r, T):
    w = weights_for(len(dims), kind, r, 40 + r)
    a0 = wl.grid_uniform(dims, 900 + T)
    ref = oracle.stencil_loop(a0, w, T, "periodic")
    got = run_gpu(a0, w, T, "fp32")
    assert err_rel(got, ref, a0) <= TOL["fp32"]


@pytest.mark.parametrize("dims", [(4096, 256), (1024, 64, 32)])
def test_long_strided_axes_repeated_T_and_large_T(dims):
    # T = 10^4 against the numpy method (itself pinned to the loop), twice in a
    # row (the 3-D plan switches to its cached multiplier table on the repeat)
    w = wl.weights_star(len(dims), 0.6 if len(dims) == 2 else 0.4, 0.1)
    a0 = wl.grid_with_modes(dims, 77, 3)[0]
    ref = oracle.stencil_fft_periodic(a0, w, 10000)
    from paper_2105_06676_gb300 import StencilPlan
    plan = StencilPlan(dims, w, "periodic", "fp32")
    for _ in range(2):
        g = torch.tensor(a0, dtype=torch.float32, device="cuda")
        plan.run(g, 10000)
        assert plan.status() == 0
        assert err_rel(g.double().cpu().numpy(), ref, a0) <= TOL["fp32"]
    plan.close()


@pytest.mark.parametrize("dims,precision", [((64, 32, 128), "fp32"), ((4096,), "fp64"),
                                            ((256, 128), "fp32")])
def test_prepared_T_first_run_uses_the_table_and_matches(dims, precision):
    # stencil_prepare builds the multiplier table for T (3-D, one-CTA 1-D) ahead
    # of time: the first run then reads it; the result is the one an unprepared
    # run gives, within the tolerance, and matches the loop
    from paper_2105_06676_gb300 import StencilPlan
    w = weights_for(len(dims), "asym", 1, 8)
    a0 = wl.grid_uniform(dims, 31)
    T = 57
    ref = oracle.stencil_loop(a0, w, T)
    dt = torch.float32 if precision == "fp32" else torch.float64
    plan = StencilPlan(dims, w, "periodic", precision)
    plan.prepare(T)
    g = torch.tensor(a0, dtype=dt, device="cuda")
    plan.run(g, T)
    assert plan.status() == 0
    assert err_rel(g.double().cpu().numpy(), ref, a0) <= TOL[precision]
    plan.close()


@pytest.mark.parametrize("boundary", ["periodic", "dirichlet"])
def test_set_weights_reuses_the_plan(boundary):
    # one plan, several stencils (including a radius change): each run matches
    # a fresh plan's loop result
    from paper_2105_06676_gb300 import StencilPlan
    dims = (64, 128)
    a0 = wl.grid_uniform(dims, 71)
    plan = StencilPlan(dims, wl.weights_random_box(2, 1, 1), boundary, "fp64")
    for i, r in enumerate((1, 2, 1)):
        w = wl.weights_random_box(2, r, 80 + i)
        plan.set_weights(w)
        g = torch.tensor(a0, dtype=torch.float64, device="cuda")
        plan.run(g, 37)
        assert plan.status() == 0
        ref = oracle.stencil_loop(a0, w, 37, boundary)
        assert err_rel(g.cpu().numpy(), ref, a0) <= TOL["fp64"]
    plan.close()


@pytest.mark.parametrize("dims,precision", [((4096, 4096), "fp32"), ((512, 1024), "fp32"),
                                            ((128, 64, 256), "fp32"), ((1024, 1024), "fp64")])
def test_periodic_autotune_variants_agree_and_choice_sticks(dims, precision):
    # every pass variant gives the oracle's result; the fastest is kept by the
    # plan and by later plans of the same shape
    from paper_2105_06676_gb300 import StencilPlan
    T = 333
    w = wl.weights_random_box(len(dims), 1, 61)
    a0 = wl.grid_uniform(dims, 62)
    dt = torch.float64 if precision == "fp64" else torch.float32
    g = torch.tensor(a0, dtype=dt, device="cuda")
    plan = StencilPlan(dims, w, "periodic", precision)
    res = plan.autotune(g, T)
    assert res["chosen"] in res["ms"] and len(res["ms"]) == 4
    np.testing.assert_array_equal(g.cpu().numpy(), a0.astype(np.float32 if precision == "fp32" else np.float64))
    plan.run(g, T)
    assert plan.status() == 0
    got = g.double().cpu().numpy()
    plan.close()
    ref = oracle.stencil_fft_periodic(a0, w, T, workers=8)
    tol = 1e-10 if precision == "fp64" else 2e-4
    assert err_rel(got, ref, a0) <= tol
    plan2 = StencilPlan(dims, w, "periodic", precision)
    g2 = torch.tensor(a0, dtype=dt, device="cuda")
    plan2.run(g2, T)
    plan2.close()
    np.testing.assert_array_equal(g2.double().cpu().numpy(), got)


@pytest.mark.parametrize("variant", [0, 1, 2, 3])
@pytest.mark.parametrize("dims,precision", [((4096, 2048), "fp32"), ((1024, 512), "fp32"),
                                            ((64, 128, 256), "fp32"), ((512, 256), "fp64")])
def test_periodic_pass_variants_match_oracle(variant, dims, precision):
    from paper_2105_06676_gb300 import StencilPlan
    T = 77
    w = wl.weights_random_box(len(dims), 1, 63)
    a0 = wl.grid_uniform(dims, 64)
    dt = torch.float64 if precision == "fp64" else torch.float32
    plan = StencilPlan(dims, w, "periodic", precision)
    plan.set_pass_variant(variant)
    g = torch.tensor(a0, dtype=dt, device="cuda")
    plan.run(g, T)
    assert plan.status() == 0
    plan.close()
    ref = oracle.stencil_fft_periodic(a0, w, T, workers=8)
    tol = 1e-10 if precision == "fp64" else 2e-4
    assert err_rel(g.double().cpu().numpy(), ref, a0) <= tol
