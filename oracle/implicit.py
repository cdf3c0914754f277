"""Implicit stencils Q a_{t+1} = S a_t on periodic grids, in numpy FP64
(oracle; test infrastructure only).

Paper appendix "Supporting Implicit Stencils" (Sec. 4.2 "Implicit Stencils"):
diagonalise both explicit stencils by the DFT, Lambda_Q = F Q F^-1 and
Lambda_S = F S F^-1, take the pseudoinverse of Lambda_Q elementwise
(1 / Lambda_Q[k] where Lambda_Q[k] != 0, else 0) and evolve with the explicit
stencil R whose symbol is Lambda_R = Lambda_Q^+ Lambda_S: a_{t+1} = R a_t then
satisfies Q a_{t+1} = S a_t wherever Q is invertible.

Reading of "Lambda_Q[k] != 0" in floating point: a symbol value counts as zero
when |Lambda_Q[k]| <= 2^-40 * sum|q| (rounding of the FP64 sum is near
2^-52 * sum|q|; any symbol a realistic Q takes on grids of at most 2^24 cells
is far above the threshold).

Both stencils use the correlation form of the explicit solver:
(S a)[i] = sum_m w_S[m] a[i + m], the same for Q.
"""
from __future__ import annotations

import numpy as np

from .spectral import _fftn, _ifftn, symbol_closed_form, symbol_power

ZERO_REL = 2.0 ** -40


def zero_threshold(weights_q: np.ndarray) -> float:
    """|Lambda_Q| at or below this counts as zero (the reading above)."""
    return ZERO_REL * float(np.sum(np.abs(np.asarray(weights_q, dtype=np.float64))))


def stencil_matrix(weights: np.ndarray, dims) -> np.ndarray:
    """The dense N x N periodic stencil matrix: row i holds w[m] in column
    (i + m) mod l (the plain definition of Sec. 1, "Problem Specification")."""
    w = np.asarray(weights, dtype=np.float64)
    dims = tuple(int(x) for x in dims)
    r = (w.shape[0] - 1) // 2
    N = int(np.prod(dims))
    M = np.zeros((N, N))
    for i in np.ndindex(*dims):
        row = np.ravel_multi_index(i, dims)
        for m in np.ndindex(*w.shape):
            j = tuple((ia + mi - r) % l for ia, mi, l in zip(i, m, dims))
            M[row, np.ravel_multi_index(j, dims)] += w[m]
    return M


def implicit_dense(a0: np.ndarray, weights_s: np.ndarray, weights_q: np.ndarray, T: int) -> np.ndarray:
    """The plain definition on small grids: T steps of a_{t+1} = Q^+ S a_t with
    dense matrices and numpy's Moore-Penrose pseudoinverse (singular values at
    or below the zero threshold dropped; for a circulant Q they are |Lambda_Q|)."""
    a0 = np.asarray(a0, dtype=np.float64)
    S = stencil_matrix(weights_s, a0.shape)
    Q = stencil_matrix(weights_q, a0.shape)
    smax = np.linalg.norm(Q, 2)
    rcond = zero_threshold(weights_q) / smax if smax > 0 else 1.0
    R = np.linalg.pinv(Q, rcond=rcond) @ S
    a = a0.reshape(-1).copy()
    for _ in range(int(T)):
        a = R @ a
    return a.reshape(a0.shape)


def implicit_symbol(weights_s: np.ndarray, weights_q: np.ndarray, dims) -> np.ndarray:
    """Lambda_R = Lambda_Q^+ Lambda_S over the full spectrum (appendix
    "Supporting Implicit Stencils"), closed-form symbols."""
    lam_s = symbol_closed_form(weights_s, dims)
    lam_q = symbol_closed_form(weights_q, dims)
    inv = np.zeros_like(lam_q)
    nz = np.abs(lam_q) > zero_threshold(weights_q)
    inv[nz] = 1.0 / lam_q[nz]
    return inv * lam_s


def stencil_fft_periodic_implicit(a0: np.ndarray, weights_s: np.ndarray, weights_q: np.ndarray,
                                  T: int, workers=None) -> np.ndarray:
    """StencilFFT-P with Lambda_R in place of Lambda: Steps 1-4 of Fig.
    "stencil-fft-algorithm-dD" (forward Multi-FFT, repeated squaring, pointwise
    product, inverse Multi-FFT)."""
    a0 = np.asarray(a0, dtype=np.float64)
    lam = implicit_symbol(weights_s, weights_q, a0.shape)
    x = _fftn(a0, workers)
    V = symbol_power(lam, T)
    return _ifftn(V * x, workers).real
