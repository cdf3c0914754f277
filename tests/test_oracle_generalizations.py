"""Pins of the oracle's generalisations (CPU): implicit stencils (appendix
"Supporting Implicit Stencils"), vector-valued fields (appendix "Supporting
Vector Valued Fields") and the reflecting boundary of the loop and of
RecursiveBoundary (Sec. 5.1). Each function is checked against something other
than itself: the explicit loop, dense matrices, textbook identities (even
extension, leapfrog recurrence), closed forms and invariants; planted mistakes
fail them."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import implicit as imp
from oracle import vector_fields as vf
from paper_2105_06676_gb300 import workloads as wl


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
    d, L = _delta(ndim), _laplacian(ndim)
    return d + 0.5 * nu * L, d - 0.5 * nu * L    # S, Q


# ---------------------------------------------------------------- implicit


@pytest.mark.parametrize("dims", [(32,), (8, 12)])
def test_implicit_with_identity_q_is_the_explicit_loop(dims):
    w = wl.weights_random_box(len(dims), 1, 3)
    a0 = wl.grid_uniform(dims, 4)
    want = oracle.stencil_loop(a0, w, 9, "periodic")
    np.testing.assert_allclose(imp.stencil_fft_periodic_implicit(a0, w, _delta(len(dims)), 9), want,
                               rtol=0, atol=1e-13)
    np.testing.assert_allclose(imp.implicit_dense(a0, w, _delta(len(dims)), 9), want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("dims,T", [((32,), 1), ((32,), 50), ((8, 12), 7)])
def test_implicit_dense_pseudoinverse_matches_spectral(dims, T):
    S, Q = _crank_nicolson(len(dims), 0.8)
    a0 = wl.grid_uniform(dims, 5)
    np.testing.assert_allclose(imp.stencil_fft_periodic_implicit(a0, S, Q, T),
                               imp.implicit_dense(a0, S, Q, T), rtol=0, atol=1e-12)


def test_implicit_result_satisfies_the_implicit_equation():
    # Q a_{t+1} = S a_t, with Q and S applied by the explicit loop oracle
    S, Q = _crank_nicolson(2, 1.3)
    a0 = wl.grid_uniform((32, 32), 6)
    aT = imp.stencil_fft_periodic_implicit(a0, S, Q, 20)
    aT1 = imp.stencil_fft_periodic_implicit(a0, S, Q, 21)
    lhs = oracle.stencil_loop(aT1, Q, 1, "periodic")
    rhs = oracle.stencil_loop(aT, S, 1, "periodic")
    assert np.max(np.abs(lhs - rhs)) < 1e-12
    # a planted mistake: the ratio inverted (Lambda_S^+ Lambda_Q) breaks it
    lam_bad = imp.implicit_symbol(Q, S, a0.shape)
    bad = lambda T: np.fft.ifftn(oracle.symbol_power(lam_bad, T) * np.fft.fftn(a0)).real
    lhs_b = oracle.stencil_loop(bad(21), Q, 1, "periodic")
    rhs_b = oracle.stencil_loop(bad(20), S, 1, "periodic")
    assert np.max(np.abs(lhs_b - rhs_b)) > 1e-3


def test_implicit_fourier_mode_closed_form():
    S, Q = _crank_nicolson(1, 0.6)
    l, k, T = 64, 5, 30
    x = np.arange(l)
    a0 = np.cos(2 * np.pi * k * x / l)
    lam = lambda w: sum(w[m + 1] * np.cos(2 * np.pi * m * k / l) for m in (-1, 0, 1))
    want = (lam(S) / lam(Q)) ** T * a0
    np.testing.assert_allclose(imp.stencil_fft_periodic_implicit(a0, S, Q, T), want, rtol=0, atol=1e-13)


def test_implicit_singular_q_drops_its_null_space():
    # Q = -Laplacian (Lambda_Q(0) = 0), S = identity: a_1 = Q^+ a_0 has zero
    # mean and Q a_1 = a_0 - mean(a_0) (the pseudoinverse on the range of Q)
    Q = -_laplacian(1)
    a0 = wl.grid_uniform((48,), 7)
    a1 = imp.stencil_fft_periodic_implicit(a0, _delta(1), Q, 1)
    assert abs(a1.mean()) < 1e-14
    np.testing.assert_allclose(oracle.stencil_loop(a1, Q, 1, "periodic"), a0 - a0.mean(), rtol=0,
                               atol=1e-12)
    # Q^+ amplifies the lowest nonzero mode ~58-fold per step: compare relative
    got = imp.stencil_fft_periodic_implicit(a0, _delta(1), Q, 3)
    dense = imp.implicit_dense(a0, _delta(1), Q, 3)
    assert np.max(np.abs(got - dense)) <= 1e-10 * np.max(np.abs(dense))


def test_implicit_zero_threshold_reading():
    assert imp.zero_threshold(np.array([-1.0, 2.0, -1.0])) == 4.0 * 2.0 ** -40
    lam = imp.implicit_symbol(_delta(1), -_laplacian(1), (16,))
    assert lam[0] == 0 and np.all(lam[1:] != 0)


# ------------------------------------------------------------ vector fields


def _random_vector_weights(m, ndim, seed, sum_to=1.0):
    rng = np.random.default_rng(seed)
    w = rng.random((m, m) + (3,) * ndim)
    w /= w.sum(axis=tuple(range(1, w.ndim)), keepdims=True) / sum_to
    return w


@pytest.mark.parametrize("T", [0, 1, 2, 3, 17, 100])
def test_matrix_power_by_squaring(T):
    rng = np.random.default_rng(T)
    lam = (rng.standard_normal((5, 3, 3)) + 1j * rng.standard_normal((5, 3, 3))) * 0.5
    want = np.stack([np.linalg.matrix_power(x, T) for x in lam])
    np.testing.assert_allclose(vf.matrix_power_sq(lam, T), want, rtol=1e-12, atol=1e-300)


def test_vector_decoupled_fields_are_scalar_solves():
    w1 = wl.weights_random_box(2, 1, 8)
    w2 = wl.weights_star(2, 0.4, 0.15)
    W = np.zeros((2, 2, 3, 3))
    W[0, 0], W[1, 1] = w1, w2
    a0 = np.stack([wl.grid_uniform((12, 10), 9), wl.grid_uniform((12, 10), 10)])
    want = np.stack([oracle.stencil_loop(a0[0], w1, 15, "periodic"),
                     oracle.stencil_loop(a0[1], w2, 15, "periodic")])
    np.testing.assert_allclose(vf.vector_loop(a0, W, 15), want, rtol=0, atol=1e-13)
    np.testing.assert_allclose(vf.stencil_fft_periodic_vector(a0, W, 15), want, rtol=0, atol=1e-13)


def test_vector_loop_is_the_block_matrix_power():
    W = _random_vector_weights(2, 1, 11)
    l, T = 8, 6
    a0 = np.stack([wl.grid_uniform((l,), 12), wl.grid_uniform((l,), 13)])
    blocks = [[imp.stencil_matrix(W[i, j], (l,)) for j in range(2)] for i in range(2)]
    M = np.block(blocks)
    want = (np.linalg.matrix_power(M, T) @ a0.reshape(-1)).reshape(a0.shape)
    np.testing.assert_allclose(vf.vector_loop(a0, W, T), want, rtol=0, atol=1e-13)


@pytest.mark.parametrize("m,dims,T", [(2, (16, 16), 1), (2, (16, 16), 40), (3, (8, 6, 10), 5), (3, (64,), 33)])
def test_vector_spectral_matches_loop(m, dims, T):
    W = _random_vector_weights(m, len(dims), 14 + m)
    a0 = np.stack([wl.grid_uniform(dims, 20 + i) for i in range(m)])
    np.testing.assert_allclose(vf.stencil_fft_periodic_vector(a0, W, T), vf.vector_loop(a0, W, T),
                               rtol=0, atol=1e-12)


def test_vector_affine_stencil_example():
    # appendix example: a_{t+1} = A a_t + c as two fields (a, c): S00 = A,
    # S01 = S11 = identity, S10 = 0; with sum(A) = 1 a constant c stays c, so
    # a_T = A^T a_0 + T c
    A = wl.weights_random_box(2, 1, 15)
    W = np.zeros((2, 2, 3, 3))
    W[0, 0], W[0, 1], W[1, 1] = A, _delta(2), _delta(2)
    c, T = 0.37, 25
    a0 = wl.grid_uniform((10, 14), 16)
    x0 = np.stack([a0, np.full_like(a0, c)])
    want = oracle.stencil_loop(a0, A, T, "periodic") + T * c
    np.testing.assert_allclose(vf.stencil_fft_periodic_vector(x0, W, T)[0], want, rtol=0, atol=1e-12)
    np.testing.assert_allclose(vf.vector_loop(x0, W, T)[1], c, rtol=0, atol=1e-14)


def test_vector_fields_carry_two_time_levels_leapfrog():
    # the wave equation u_{t+1} = 2 u_t - u_{t-1} + k^2 L u_t (a stencil that
    # reads two past steps) as fields (u_t, u_{t-1}): S00 = 2 I + k^2 L,
    # S01 = -I, S10 = I, S11 = 0; against the recurrence written out
    k2, T = 0.2, 40
    L = _laplacian(1)
    W = np.zeros((2, 2, 3))
    W[0, 0] = 2 * _delta(1) + k2 * L
    W[0, 1] = -_delta(1)
    W[1, 0] = _delta(1)
    u0 = np.sin(2 * np.pi * np.arange(32) / 32) + 0.1 * wl.grid_uniform((32,), 17)
    um1 = u0.copy()
    prev, cur = um1, u0
    for _ in range(T):
        lap = np.roll(cur, -1) + np.roll(cur, 1) - 2 * cur
        prev, cur = cur, 2 * cur - prev + k2 * lap
    got = vf.stencil_fft_periodic_vector(np.stack([u0, um1]), W, T)
    np.testing.assert_allclose(got[0], cur, rtol=0, atol=1e-11)
    np.testing.assert_allclose(got[1], prev, rtol=0, atol=1e-11)


def test_vector_planted_transpose_fails():
    # reading block (i, j) as field i -> field j is caught by the loop
    W = _random_vector_weights(2, 1, 18)
    a0 = np.stack([wl.grid_uniform((24,), 19), wl.grid_uniform((24,), 20)])
    good = vf.vector_loop(a0, W, 7)
    bad = vf.stencil_fft_periodic_vector(a0, np.swapaxes(W, 0, 1), 7)
    assert np.max(np.abs(good - bad)) > 1e-3


# --------------------------------------------------------- reflecting boundary


def _even_extension(a):
    for ax in range(a.ndim):
        a = np.concatenate([a, np.flip(a, axis=ax)], axis=ax)
    return a


@pytest.mark.parametrize("dims,r", [((17,), 1), ((17,), 2), ((9, 12), 1), ((6, 5, 7), 1), ((10, 9), 2)])
def test_neumann_loop_is_the_periodic_even_extension(dims, r):
    # a stencil symmetric along every axis keeps the half-sample even extension
    # even, so reflecting ghosts on l equal the periodic solve on 2 l (DCT-II
    # symmetry)
    rng = np.random.default_rng(21)
    half = rng.random((r + 1,) * len(dims))
    w = half
    for ax in range(len(dims)):
        w = np.concatenate([np.flip(w, axis=ax)[tuple(slice(0, r) if a == ax else slice(None)
                                                      for a in range(len(dims)))], w], axis=ax)
    w /= w.sum()
    a0 = wl.grid_uniform(dims, 22)
    T = 13
    ext = oracle.stencil_loop(_even_extension(a0), w, T, "periodic")
    want = ext[tuple(slice(0, l) for l in dims)]
    got = oracle.stencil_loop(a0, w, T, "neumann")
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)
    assert abs(got.sum() - a0.sum()) < 1e-10          # mass is conserved
    # one step against numpy's half-sample padding ("symmetric": ghost -1-k =
    # cell k); the whole-sample reflection ("reflect": ghost -k = cell k) is a
    # planted mistake that differs
    def padded_step(mode):
        p = np.pad(a0, r, mode=mode)
        out = np.zeros(dims)
        for m in np.ndindex(*w.shape):
            out += w[m] * p[tuple(slice(mi, mi + l) for mi, l in zip(m, dims))]
        return out
    one = oracle.stencil_loop(a0, w, 1, "neumann")
    np.testing.assert_allclose(padded_step("symmetric"), one, rtol=0, atol=1e-14)
    assert np.max(np.abs(padded_step("reflect") - one)) > 1e-6


@pytest.mark.parametrize("dims,r,T,cutoff", [((40,), 1, 13, 2), ((40,), 2, 9, 3), ((24, 30), 1, 8, 2),
                                             ((20, 22), 1, 5, 8), ((12, 10, 14), 1, 4, 2)])
def test_recursive_boundary_with_reflecting_base_case_matches_loop(dims, r, T, cutoff):
    # the recursion's periodic solves keep only cells the boundary cannot
    # reach, so the same recursion with a reflecting base case is exact; the
    # weights need not be symmetric
    w = wl.weights_random_box(len(dims), r, 23)
    a0 = wl.grid_uniform(dims, 24)
    got = oracle.stencil_fft_aperiodic(a0, w, T, cutoff, boundary="neumann")
    want = oracle.stencil_loop(a0, w, T, "neumann")
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-12)
    dirichlet = oracle.stencil_loop(a0, w, T, "dirichlet")
    assert np.max(np.abs(want - dirichlet)) > 1e-3     # the condition matters here
