"""Vector-valued fields on periodic grids, in numpy FP64 (oracle; test
infrastructure only).

Paper Sec. 4.2 "Vector-Valued Fields" and appendix "Supporting Vector Valued
Fields": m scalar fields evolve as

    a^(i)_{t+1} = sum_j S^(i,j) a^(j)_t,

each S^(i,j) a periodic stencil (correlation form, (S a)[x] = sum_k w_ij[k]
a[x + k]). Diagonalised by the DFT, every wave vector k carries an m x m matrix
Lambda(k) with entries Lambda_ij(k) = symbol of w_ij; T steps apply Lambda(k)^T,
found by repeated squaring of the matrix of stencils (Q = R R reads off two
steps from one).

Weights: an array of shape (m, m, 2r+1, ..., 2r+1); block (i, j) is the
stencil that takes field j into field i.
"""
from __future__ import annotations

import numpy as np

from .spectral import _fftn, _ifftn, symbol_closed_form


def vector_loop(a0: np.ndarray, weights: np.ndarray, T: int) -> np.ndarray:
    """The plain definition: T sequential steps, each field the sum over source
    fields and offsets of w_ij[k] times the source field shifted by k (periodic
    wrap); a0 has shape (m, *dims)."""
    a = np.asarray(a0, dtype=np.float64).copy()
    w = np.asarray(weights, dtype=np.float64)
    m = w.shape[0]
    r = (w.shape[2] - 1) // 2
    d = a.ndim - 1
    for _ in range(int(T)):
        b = np.zeros_like(a)
        for i in range(m):
            for j in range(m):
                for k in np.ndindex(*w.shape[2:]):
                    if w[(i, j) + k] == 0.0:
                        continue
                    shift = tuple(-(kk - r) for kk in k)   # b[x] += w[k] a[x + k]
                    b[i] += w[(i, j) + k] * np.roll(a[j], shift, axis=tuple(range(d)))
        a = b
    return a


def symbol_matrix(weights: np.ndarray, dims) -> np.ndarray:
    """Lambda(k) for every k: shape (*dims, m, m), Lambda_ij = symbol of w_ij."""
    w = np.asarray(weights, dtype=np.float64)
    m = w.shape[0]
    dims = tuple(int(x) for x in dims)
    lam = np.zeros(dims + (m, m), dtype=np.complex128)
    for i in range(m):
        for j in range(m):
            lam[..., i, j] = symbol_closed_form(w[i, j], dims)
    return lam


def matrix_power_sq(lam: np.ndarray, T: int) -> np.ndarray:
    """Lambda^T per wave vector by repeated squaring over the bits of T (the
    appendix: 'swap out sequential squaring of Lambda with a sequential squaring
    of a matrix of stencils'); T = 0 gives the identity."""
    if T < 0:
        raise ValueError("T must be >= 0")
    m = lam.shape[-1]
    V = np.broadcast_to(np.eye(m, dtype=np.complex128), lam.shape).copy()
    sq = lam.copy()
    R = int(T)
    while R > 0:
        if R & 1:
            V = V @ sq
        R >>= 1
        if R:
            sq = sq @ sq
    return V


def stencil_fft_periodic_vector(a0: np.ndarray, weights: np.ndarray, T: int,
                                workers=None) -> np.ndarray:
    """StencilFFT-P for m fields: forward Multi-FFT of every field, y(k) =
    Lambda(k)^T x(k), inverse Multi-FFT (Fig. "stencil-fft-algorithm-dD" with
    the matrix power of the appendix)."""
    a0 = np.asarray(a0, dtype=np.float64)
    m = a0.shape[0]
    dims = a0.shape[1:]
    x = np.stack([_fftn(a0[i], workers) for i in range(m)], axis=-1)   # (*dims, m)
    V = matrix_power_sq(symbol_matrix(weights, dims), T)
    y = np.einsum("...ij,...j->...i", V, x)
    return np.stack([_ifftn(y[..., i], workers).real for i in range(m)])
