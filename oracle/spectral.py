"""StencilFFT-P, step by step, in numpy FP64 (oracle; test infrastructure only).

Follows the paper's periodic algorithm in its own order and notation
(Sec. 4 "1-D Explicit Stencil Algorithm" and Fig. "stencil-fft-algorithm-dD";
d-D form in the appendix "Supporting d-D Spatial Grids"):

    Step 1  Lambda <- Multi-FFT(s),  x <- Multi-FFT(a_0)
    Step 2  V <- Lambda^T by repeated squaring over the bits of T
    Step 3  y <- V * x  (pointwise)
    Step 4  a_T <- Inverse-Multi-FFT(y)

DFT convention (Sec. 4, "Reformulating the Final Data"): the forward transform
is unnormalised, F[i,j] = w^(-ij) with w = exp(2 pi i / l), and the inverse
carries the 1/N. numpy's ``fft.fftn`` / ``fft.ifftn`` use exactly this
convention; they serve as the library Multi-FFT primitive.

The stencil is stored as the first column s of the circulant matrix S (Sec. 4,
"we will store only the first column"). With the update
a_{t+1}[i] = sum_m w[m] a_t[i+m], entry S[i, i+m] = w[m], so s[(-m) mod l] = w[m].
"""
from __future__ import annotations

import numpy as np


def _radius(weights: np.ndarray) -> int:
    return (weights.shape[0] - 1) // 2


def first_column(weights: np.ndarray, dims) -> np.ndarray:
    """First column s of the circulant stencil matrix S, as a grid of shape dims.

    Sec. 4 ("Mathematical Formulation": S = sum_i S[i,0] X^i; store only the
    first column). s[(-m) mod l] = w[m] for every offset m in [-r, r]^d.
    """
    w = np.asarray(weights, dtype=np.float64)
    dims = tuple(int(x) for x in dims)
    r = _radius(w)
    s = np.zeros(dims, dtype=np.float64)
    for m in np.ndindex(*w.shape):
        offset = tuple(mi - r for mi in m)
        idx = tuple((-o) % l for o, l in zip(offset, dims))
        s[idx] += w[m]
    return s


def _fftn(x, workers):
    """The library Multi-FFT primitive: numpy, or scipy.fft with `workers` threads
    (same convention: unnormalised forward, 1/N on the inverse)."""
    if workers is None:
        return np.fft.fftn(x)
    import scipy.fft
    return scipy.fft.fftn(x, workers=workers)


def _ifftn(x, workers):
    if workers is None:
        return np.fft.ifftn(x)
    import scipy.fft
    return scipy.fft.ifftn(x, workers=workers)


def symbol_multi_fft(weights: np.ndarray, dims, workers=None) -> np.ndarray:
    """Lambda = Multi-FFT(s): the eigenvalues of S (Step 1, Eq. final_data).

    Appendix "Proof of Eigenvalue-FFT Relation": Lambda[k] = (F s)[k].
    """
    return _fftn(first_column(weights, dims), workers)


def symbol_closed_form(weights: np.ndarray, dims) -> np.ndarray:
    """Lambda[k] = sum_m w[m] exp(+2 pi i sum_d m_d k_d / l_d), evaluated directly.

    This is (F s)[k] written out with s[(-m) mod l] = w[m]
    (Appendix "Proof of Eigenvalue-FFT Relation"): sum_j s[j] w^(-jk) with
    j = -m gives w^(+mk).
    """
    w = np.asarray(weights, dtype=np.float64)
    dims = tuple(int(x) for x in dims)
    r = _radius(w)
    grids = np.meshgrid(*[np.arange(l, dtype=np.float64) for l in dims],
                        indexing="ij")
    lam = np.zeros(dims, dtype=np.complex128)
    for m in np.ndindex(*w.shape):
        phase = np.zeros(dims, dtype=np.float64)
        for axis, (mi, l) in enumerate(zip(m, dims)):
            phase += (mi - r) * grids[axis] / l
        lam += w[m] * np.exp(2j * np.pi * phase)
    return lam


def symbol_power(lam: np.ndarray, T: int) -> np.ndarray:
    """V = Lambda^T elementwise by repeated squaring (Step 2).

    Sec. 4: Lambda^T = product over the set bits b_i of T of Lambda^(2^i);
    Fig. "stencil-fft-algorithm-dD" keeps V (running product, all ones at the
    start), R (remaining exponent, all T) and Squares (Lambda^(2^k)) and loops
    k = 0 .. log T. The loop runs floor(log2 T) + 1 times; T = 0 gives V = 1.
    """
    if T < 0:
        raise ValueError("T must be >= 0")
    lam = np.asarray(lam, dtype=np.complex128)
    V = np.ones_like(lam)
    R = int(T)
    squares = lam.copy()
    n_iter = R.bit_length()  # floor(log2 T) + 1 for T >= 1, 0 for T == 0
    for _ in range(n_iter):
        if R % 2 == 1:
            V = V * squares
            R -= 1
        R //= 2
        squares = squares * squares
    return V


def stencil_fft_periodic(a0: np.ndarray, weights: np.ndarray, T: int,
                         workers=None) -> np.ndarray:
    """StencilFFT-P (Fig. "stencil-fft-algorithm-dD"): a_T = F^-1 Lambda^T F a_0.

    `workers` selects scipy.fft with that many threads as the Multi-FFT
    primitive (large grids); the steps are the same."""
    a0 = np.asarray(a0, dtype=np.float64)
    lam = symbol_multi_fft(weights, a0.shape, workers)   # Step 1 (i)
    x = _fftn(a0, workers)                               # Step 1 (ii)
    V = symbol_power(lam, T)                             # Step 2
    del lam
    y = V * x                                            # Step 3
    del V, x
    return _ifftn(y, workers).real                       # Step 4 (real grid)


def dft_naive(x: np.ndarray) -> np.ndarray:
    """O(n^2) 1-D DFT by the defining sum X[k] = sum_j x[j] exp(-2 pi i jk/n).

    Sec. 4 DFT matrix F[i,j] = w^(-ij). Used only to pin the library FFT
    convention on small inputs.
    """
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[0]
    j = np.arange(n)
    F = np.exp(-2j * np.pi * np.outer(j, j) / n)
    return F @ x
