"""Pins for the oracle: checks against what the paper and mathematics fix.

None of these retype the oracle's own formulas. They use the matrix the paper
prints, explicitly assembled shift-operator matrices raised to a power by
LAPACK/BLAS, exact rational arithmetic, textbook closed forms for Fourier
modes, invariants (mass, maximum principle, composition, shift equivariance),
the method of images, and numpy's eigenvalue routine. The last section plants
plausible mistakes in copies of oracle functions and shows that a pin fails.
"""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import (boundary_distance, dft_naive, first_column, recursive_boundary,
                    stencil_fft_aperiodic, stencil_fft_periodic, stencil_loop,
                    symbol_closed_form, symbol_multi_fft, symbol_power)
from paper_2105_06676_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# helpers that build things independently of the oracle
# --------------------------------------------------------------------------
def read_worked_example():
    w, rows = None, []
    with open(os.path.join(GOLDEN, "worked_example_stencil_matrix.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            if key == "weights":
                w = np.array([float(v) for v in vals])
            elif key == "row":
                rows.append([float(v) for v in vals])
    return w, np.array(rows)


def shift_power(n: int, m: int, periodic: bool) -> np.ndarray:
    """Matrix P_m with (P_m a)[i] = a[i + m] (wrapping, or zero outside).

    Built from the paper's right shift X (X[i, j] = delta_{i, j+1}, Sec. 4):
    P_m = X^(-m). For zero Dirichlet the shift drops what leaves the grid.
    """
    if periodic:
        X = np.roll(np.eye(n), 1, axis=0)          # X[i, j] = 1 iff i = j + 1 (mod n)
        Xinv = X.T
    else:
        X = np.eye(n, k=-1)                         # truncated right shift
        Xinv = X.T
    if m >= 0:
        return np.linalg.matrix_power(Xinv, m)
    return np.linalg.matrix_power(X, -m)


def dense_operator(weights: np.ndarray, dims, periodic: bool) -> np.ndarray:
    """S = sum_m w[m] P^(1)_{m_1} (x) ... (x) P^(d)_{m_d} (Kronecker products)."""
    r = (weights.shape[0] - 1) // 2
    n = int(np.prod(dims))
    S = np.zeros((n, n))
    for m in np.ndindex(*weights.shape):
        op = np.ones((1, 1))
        for mi, l in zip(m, dims):
            op = np.kron(op, shift_power(l, mi - r, periodic))
        S += weights[m] * op
    return S


def rel_err(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


# --------------------------------------------------------------------------
# 1. the worked example the paper prints (appendix "Stencil Matrix Example")
# --------------------------------------------------------------------------
def check_worked_example_matrix(loop_fn) -> bool:
    w, S_printed = read_worked_example()
    cols = []
    for j in range(4):
        e = np.zeros(4)
        e[j] = 1.0
        cols.append(loop_fn(e, w, 1, "periodic"))
    return np.array_equal(np.stack(cols, axis=1), S_printed)


def check_worked_example_symbol(symbol_fn) -> bool:
    """Fourier modes v_k[j] = exp(2 pi i jk / 4) satisfy S v_k = lambda(k) v_k."""
    w, S_printed = read_worked_example()
    lam = symbol_fn(w, (4,))
    j = np.arange(4)
    ok = True
    for k in range(4):
        v = np.exp(2j * np.pi * j * k / 4)
        ok &= np.allclose(S_printed @ v, lam[k] * v, atol=1e-12)
    return bool(ok)


def test_worked_example_matrix_from_loop():
    assert check_worked_example_matrix(stencil_loop)


def test_worked_example_first_column():
    w, S_printed = read_worked_example()
    np.testing.assert_array_equal(first_column(w, (4,)), S_printed[:, 0])


@pytest.mark.parametrize("fn", [symbol_multi_fft, symbol_closed_form])
def test_worked_example_symbol_eigvecs(fn):
    assert check_worked_example_symbol(fn)


def test_worked_example_symbol_is_eigenvalue_set():
    w, S_printed = read_worked_example()
    lam = symbol_multi_fft(w, (4,))
    eig = np.linalg.eigvals(S_printed)
    key = lambda z: (round(z.real, 9), round(z.imag, 9))
    assert sorted(map(key, lam)) == sorted(map(key, eig))
    # the values the eigenvector check implies, in DFT order k = 0..3
    np.testing.assert_allclose(lam, [2, 1 + 5j, 0, 1 - 5j], atol=1e-12)


# --------------------------------------------------------------------------
# 2. dense brute force: S^T a_0 with S assembled from shift matrices
# --------------------------------------------------------------------------
DENSE_CASES = [
    ((16,), 1, "periodic", 7), ((16,), 2, "periodic", 33), ((13,), 1, "dirichlet", 9),
    ((12,), 2, "dirichlet", 25), ((6, 5), 1, "periodic", 11), ((6, 7), 1, "dirichlet", 6),
    ((5, 5), 2, "periodic", 4), ((4, 3, 5), 1, "periodic", 5), ((3, 4, 4), 1, "dirichlet", 3),
    ((64,), 1, "periodic", 1000), ((64,), 1, "dirichlet", 200),
]


@pytest.mark.parametrize("dims,r,boundary,T", DENSE_CASES)
def test_loop_matches_dense_matrix_power(dims, r, boundary, T):
    w = wl.weights_random_signed(len(dims), r, seed=17 + T) * 0.5
    if boundary == "dirichlet" or T > 50:
        w = wl.weights_random_box(len(dims), r, seed=19 + T)      # keep powers bounded
    a0 = wl.grid_uniform(dims, seed=7 + T)
    S = dense_operator(w, dims, boundary == "periodic")
    ref = (np.linalg.matrix_power(S, T) @ a0.ravel()).reshape(dims)
    got = stencil_loop(a0, w, T, boundary)
    assert rel_err(got, ref) < 1e-12


# --------------------------------------------------------------------------
# 3. exact rationals: dyadic weights and inputs stay exact in FP64
# --------------------------------------------------------------------------
def _rational_evolve_1d(a, w, T, periodic):
    n, r = len(a), (len(w) - 1) // 2
    for _ in range(T):
        b = []
        for i in range(n):
            acc = Fraction(0)
            for m in range(-r, r + 1):
                j = i + m
                if periodic:
                    j %= n
                elif j < 0 or j >= n:
                    continue
                acc += w[m + r] * a[j]
            b.append(acc)
        a = b
    return a


@pytest.mark.parametrize("periodic", [True, False])
def test_loop_exact_with_dyadic_rationals(periodic):
    w = [Fraction(1, 4), Fraction(1, 2), Fraction(1, 4)]
    rng = np.random.default_rng(3)
    a = [Fraction(int(v), 1024) for v in rng.integers(0, 1024, size=10)]
    T = 18
    exact = _rational_evolve_1d(a, w, T, periodic)
    got = stencil_loop(np.array([float(x) for x in a]), np.array([float(x) for x in w]), T,
                       "periodic" if periodic else "dirichlet")
    assert [Fraction(float(v)) for v in got] == exact


# --------------------------------------------------------------------------
# 4. Fourier modes: textbook closed forms
# --------------------------------------------------------------------------
def test_heat1d_fourier_mode_closed_form():
    # (0.25, 0.5, 0.25) acting on cos(theta x) multiplies it by cos^2(theta/2)
    n, T = 64, 300
    x = np.arange(n)
    for k in (1, 3, 10, 32):
        theta = 2 * np.pi * k / n
        a0 = np.cos(theta * x + 0.3)
        expect = np.cos(theta / 2) ** (2 * T) * a0
        for fn in (lambda a: stencil_loop(a, wl.weights_1d([0.25, 0.5, 0.25]), T),
                   lambda a: stencil_fft_periodic(a, wl.weights_1d([0.25, 0.5, 0.25]), T)):
            assert np.max(np.abs(fn(a0) - expect)) < 1e-12


def test_asymmetric_1d_fourier_mode_closed_form():
    # a_{t+1}[i] = p a[i-1] + q a[i] + s a[i+1] on cos(theta x): the mode rotates by
    # arg(mu) and scales by |mu| with mu = p e^{-i theta} + q + s e^{+i theta}
    p, q, s = 0.2, 0.5, 0.3
    n, T = 48, 40
    x = np.arange(n)
    for k in (1, 5, 11):
        theta = 2 * np.pi * k / n
        mu = p * np.exp(-1j * theta) + q + s * np.exp(1j * theta)
        a0 = np.cos(theta * x)
        expect = np.abs(mu) ** T * np.cos(theta * x + T * np.angle(mu))
        got = stencil_loop(a0, np.array([p, q, s]), T)
        assert np.max(np.abs(got - expect)) < 1e-12
        got = stencil_fft_periodic(a0, np.array([p, q, s]), T)
        assert np.max(np.abs(got - expect)) < 1e-12


def test_star2d_fourier_mode_closed_form():
    # 5-point (0.6 centre, 0.1 neighbours): sin(k.x) scales by 0.6 + 0.2 cos t1 + 0.2 cos t2
    dims, T = (32, 16), 57
    w = wl.weights_star(2, 0.6, 0.1)
    for k in ((1, 2), (5, 3), (16, 8)):
        a0 = wl.fourier_mode(dims, k, phase=0.4)
        lam = 0.6 + 0.2 * np.cos(2 * np.pi * k[0] / dims[0]) + 0.2 * np.cos(2 * np.pi * k[1] / dims[1])
        expect = lam ** T * a0
        assert np.max(np.abs(stencil_loop(a0, w, T) - expect)) < 1e-12
        assert np.max(np.abs(stencil_fft_periodic(a0, w, T) - expect)) < 1e-12


def test_star3d_fourier_mode_closed_form():
    dims, T = (8, 8, 16), 21
    w = wl.weights_star(3, 0.4, 0.1)
    k = (1, 3, 5)
    a0 = wl.fourier_mode(dims, k)
    lam = 0.4 + sum(0.2 * np.cos(2 * np.pi * kk / l) for kk, l in zip(k, dims))
    assert np.max(np.abs(stencil_loop(a0, w, T) - lam ** T * a0)) < 1e-12
    assert np.max(np.abs(stencil_fft_periodic(a0, w, T) - lam ** T * a0)) < 1e-12


# --------------------------------------------------------------------------
# 5. invariants
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dims", [(50,), (12, 9), (5, 6, 7)])
def test_mass_and_max_principle_periodic(dims):
    w = wl.weights_random_box(len(dims), 1, seed=5)
    a0 = wl.grid_uniform(dims, 9)
    for fn in (stencil_loop, stencil_fft_periodic):
        aT = fn(a0, w, 37)
        assert abs(aT.sum() - a0.sum()) < 1e-10 * a0.size
        assert aT.min() >= a0.min() - 1e-12 and aT.max() <= a0.max() + 1e-12


@pytest.mark.parametrize("dims", [(40,), (10, 14), (6, 5, 7)])
def test_dirichlet_positivity_and_mass_decay(dims):
    w = wl.weights_random_box(len(dims), 1, seed=6)
    a = wl.grid_uniform(dims, 10)
    amax, mass = a.max(), a.sum()
    for _ in range(6):
        a = stencil_loop(a, w, 3, "dirichlet")
        assert a.min() >= 0.0 and a.max() <= amax + 1e-15
        assert a.sum() <= mass + 1e-12
        mass = a.sum()


def test_composition_and_shift_equivariance():
    dims = (12, 10)
    w = wl.weights_random_signed(2, 1, 4) * 0.3
    a0 = wl.grid_uniform(dims, 11)
    a5 = stencil_loop(a0, w, 5)
    a3 = stencil_loop(stencil_loop(a0, w, 2), w, 3)
    assert rel_err(a3, a5) < 1e-13
    shifted = np.roll(a0, (3, -2), axis=(0, 1))
    assert rel_err(stencil_loop(shifted, w, 5), np.roll(a5, (3, -2), axis=(0, 1))) < 1e-13
    # Dirichlet composes too
    d5 = stencil_loop(a0, w, 5, "dirichlet")
    d23 = stencil_loop(stencil_loop(a0, w, 2, "dirichlet"), w, 3, "dirichlet")
    assert rel_err(d23, d5) < 1e-13


def test_T_zero_is_identity():
    a0 = wl.grid_uniform((9, 4), 1)
    w = wl.weights_random_box(2, 2, 1)
    for b in ("periodic", "dirichlet"):
        np.testing.assert_array_equal(stencil_loop(a0, w, 0, b), a0)
    np.testing.assert_allclose(stencil_fft_periodic(a0, w, 0), a0, atol=1e-15)


# --------------------------------------------------------------------------
# 6. method of images: zero Dirichlet = periodic solve of the odd extension
# --------------------------------------------------------------------------
def _odd_extend(a, axis):
    n = a.shape[axis]
    zero = np.zeros_like(np.take(a, [0], axis=axis))
    return np.concatenate([zero, a, zero, -np.flip(a, axis=axis)], axis=axis), n


def test_method_of_images_1d():
    w = np.array([0.3, 0.4, 0.3])
    a0 = wl.grid_uniform((37,), 12)
    ext, n = _odd_extend(a0, 0)
    for T in (1, 17, 200):
        per = stencil_loop(ext, w, T)[1:n + 1]
        assert rel_err(stencil_loop(a0, w, T, "dirichlet"), per) < 1e-12


def test_method_of_images_2d():
    # reflection-symmetric in each axis separately
    w = np.array([[0.05, 0.1, 0.05], [0.15, 0.3, 0.15], [0.05, 0.1, 0.05]])
    a0 = wl.grid_uniform((13, 9), 13)
    ext, n0 = _odd_extend(a0, 0)
    ext, n1 = _odd_extend(ext, 1)
    for T in (3, 40):
        per = stencil_loop(ext, w, T)[1:n0 + 1, 1:n1 + 1]
        assert rel_err(stencil_loop(a0, w, T, "dirichlet"), per) < 1e-12


def test_method_of_images_2d_threaded_fft_primitive():
    # the same pin through scipy.fft with threads as the Multi-FFT primitive
    # (used for the full-size odd extensions, 2 (l + 1) = 2 * 3 * 2731 points)
    w = np.array([[0.05, 0.1, 0.05], [0.15, 0.3, 0.15], [0.05, 0.1, 0.05]])
    a0 = wl.grid_uniform((13, 9), 14)
    ext, n0 = _odd_extend(a0, 0)
    ext, n1 = _odd_extend(ext, 1)
    for T in (3, 40):
        per = stencil_fft_periodic(ext, w, T, workers=2)[1:n0 + 1, 1:n1 + 1]
        assert rel_err(stencil_loop(a0, w, T, "dirichlet"), per) < 1e-12
        np.testing.assert_allclose(per, stencil_fft_periodic(ext, w, T)[1:n0 + 1, 1:n1 + 1],
                                   rtol=0, atol=1e-13)


# --------------------------------------------------------------------------
# 7. spectral pieces: symbol, DFT convention, repeated squaring
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dims,r", [((8,), 1), ((16,), 2), ((6, 10), 1), ((8, 4, 6), 1), ((5, 5), 2)])
def test_symbol_closed_form_equals_multi_fft(dims, r):
    w = wl.weights_random_signed(len(dims), r, 21)
    np.testing.assert_allclose(symbol_closed_form(w, dims), symbol_multi_fft(w, dims), atol=1e-12)


def test_symbol_eigenvectors_of_dense_operator_2d():
    dims = (4, 6)
    w = wl.weights_random_signed(2, 1, 2)
    S = dense_operator(w, dims, True)
    lam = symbol_multi_fft(w, dims)
    i0, i1 = np.meshgrid(np.arange(dims[0]), np.arange(dims[1]), indexing="ij")
    for k in np.ndindex(*dims):
        v = np.exp(2j * np.pi * (k[0] * i0 / dims[0] + k[1] * i1 / dims[1])).ravel()
        np.testing.assert_allclose(S @ v, lam[k] * v, atol=1e-12)


def test_dft_convention():
    n = 16
    delta = np.zeros(n)
    delta[0] = 1.0
    np.testing.assert_allclose(dft_naive(delta), np.ones(n), atol=1e-14)
    j = np.arange(n)
    for k0 in (1, 5):
        X = dft_naive(np.exp(2j * np.pi * k0 * j / n))   # w^(+k0 j) lands in bin k0
        expect = np.zeros(n, complex)
        expect[k0] = n
        np.testing.assert_allclose(X, expect, atol=1e-12)
    x = wl.grid_uniform((n,), 4)
    np.testing.assert_allclose(np.fft.fft(x), dft_naive(x), atol=1e-12)


@pytest.mark.parametrize("T", [0, 1, 2, 3, 7, 64, 1000, 10000, 65535, 65536])
def test_symbol_power_matches_complex_power(T):
    rng = np.random.default_rng(T + 1)
    lam = rng.uniform(-1, 1, 200) + 1j * rng.uniform(-1, 1, 200)
    lam /= np.maximum(1.0, np.abs(lam))
    lam = np.concatenate([lam, [0.0, 1.0, -1.0, 1j]])
    ref = np.array([complex(z) ** T if T > 0 else 1.0 + 0j for z in lam])
    # both sides round differently; relative error of a T-th power grows like T * eps
    rtol = max(1e-13, 8 * T * np.finfo(np.float64).eps)
    np.testing.assert_allclose(symbol_power(lam, T), ref, rtol=rtol, atol=1e-300)


def test_symbol_power_special_values():
    lam = np.array([0.0, 2.0, -0.5j])
    np.testing.assert_array_equal(symbol_power(lam, 0), np.ones(3))
    assert symbol_power(lam, 5)[0] == 0
    assert symbol_power(lam, 10)[1] == 1024.0


# --------------------------------------------------------------------------
# 8. the paper's method (numpy) against the definition (loop)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dims,r,T", [((64,), 1, 1000), ((50,), 2, 77), ((16, 12), 1, 31),
                                      ((9, 10), 2, 5), ((6, 8, 5), 1, 13)])
def test_stencil_fft_periodic_matches_loop(dims, r, T):
    w = wl.weights_random_box(len(dims), r, 31)
    a0 = wl.grid_uniform(dims, 32)
    assert rel_err(stencil_fft_periodic(a0, w, T), stencil_loop(a0, w, T)) < 1e-12


RB_CASES = [
    ((40,), 1, T, c) for T in (1, 2, 3, 5, 7, 13, 19) for c in (2, 3, 8)
] + [
    ((64,), 2, 13, 2), ((64,), 2, 45, 4), ((30,), 1, 45, 2),        # sigma T >= l/2
    ((24, 20), 1, 9, 2), ((24, 20), 1, 13, 3), ((18, 26), 2, 6, 2),
    ((32, 32), 1, 32, 4), ((8, 40), 1, 11, 2),                      # rectangular
    ((10, 12, 9), 1, 5, 2), ((12, 12, 12), 1, 7, 3),
]


@pytest.mark.parametrize("dims,r,T,cutoff", RB_CASES)
def test_stencil_fft_aperiodic_matches_dirichlet_loop(dims, r, T, cutoff):
    w = wl.weights_random_box(len(dims), r, 41 + T)
    a0 = wl.grid_uniform(dims, 42)
    got = stencil_fft_aperiodic(a0, w, T, cutoff)
    assert rel_err(got, stencil_loop(a0, w, T, "dirichlet")) < 1e-12


def test_recursive_boundary_only_needs_its_input_region():
    # RecursiveBoundary(T) reads a_0 only at dist <= 2 sigma T
    dims, T, r = (48,), 9, 1
    w = wl.weights_random_box(1, r, 3)
    a0 = wl.grid_uniform(dims, 5)
    dist = boundary_distance(dims)
    junk = np.where(dist <= 2 * r * T, a0, 1e6)
    out = recursive_boundary(junk, w, T, 2)
    ref = stencil_loop(a0, w, T, "dirichlet")
    keep = dist <= r * T
    assert rel_err(out[keep], ref[keep]) < 1e-12


def test_interior_equals_periodic():
    dims, T = (30, 28), 6
    w = wl.weights_random_box(2, 1, 8)
    a0 = wl.grid_uniform(dims, 8)
    inner = boundary_distance(dims) > T
    assert rel_err(stencil_loop(a0, w, T, "dirichlet")[inner], stencil_loop(a0, w, T)[inner]) < 1e-13


def test_boundary_distance_geometry():
    d = boundary_distance((5,))
    np.testing.assert_array_equal(d, [1, 2, 3, 2, 1])
    d = boundary_distance((4, 6))
    assert d[0].tolist() == [1] * 6 and d[1].tolist() == [1, 2, 2, 2, 2, 1]


# --------------------------------------------------------------------------
# 9. planted mistakes: a pin fails for each
# --------------------------------------------------------------------------
def _loop_flipped_weights(a, w, T, b="periodic"):
    return stencil_loop(a, np.flip(w), T, b)


def _loop_one_step_short(a, w, T, b="periodic"):
    return stencil_loop(a, w, max(T - 1, 0), b)


def _symbol_wrong_sign(w, dims):
    return np.conj(symbol_closed_form(w, dims))


def _first_column_no_negation(w, dims):
    s = np.zeros(dims)
    r = (w.shape[0] - 1) // 2
    for m in np.ndindex(*w.shape):
        s[tuple((mi - r) % l for mi, l in zip(m, dims))] += w[m]
    return s


def test_planted_flipped_weights_fails_worked_example():
    assert not check_worked_example_matrix(_loop_flipped_weights)


def test_planted_off_by_one_T_fails_worked_example():
    assert not check_worked_example_matrix(lambda a, w, T, b: _loop_one_step_short(a, w, T, b))


def test_planted_symbol_sign_fails_eigvec_pin():
    assert not check_worked_example_symbol(_symbol_wrong_sign)
    assert not check_worked_example_symbol(lambda w, d: np.fft.fftn(_first_column_no_negation(w, d)))


def test_planted_dropped_power_iteration_fails():
    lam = np.array([0.9 + 0.1j, 0.5])
    T = 10
    good = symbol_power(lam, T)
    bad = symbol_power(lam, T // 2) ** 2 * lam    # an extra factor: T+1
    assert not np.allclose(bad, good)


def test_planted_rb_keep_range_fails():
    # widening the Step-2 keep range past sigma*T must break the aperiodic result
    dims, T = (40,), 11
    w = wl.weights_random_box(1, 1, 3)
    a0 = wl.grid_uniform(dims, 4)
    dist = boundary_distance(dims)
    ref = stencil_loop(a0, w, T, "dirichlet")
    center = stencil_fft_periodic(a0, w, T)
    res = np.where(dist > T - 2, center, recursive_boundary(a0, w, T, 2))  # wrong split
    assert rel_err(res, ref) > 1e-6


def test_oracle_threads_reported():
    assert oracle.oracle_threads() >= 1
