"""RecursiveBoundary over l-shells (oracle; test infrastructure only).

Appendix "l-shell Spatial Grid Decomposition": the regions of RecursiveBoundary
(Sec. 5.2, Fig. "stencil-fft-algorithm-1D-aperiodic") are described by the time
at which the boundary's influence first reaches a cell instead of by the
distance to the boundary, so that stencils reaching further along one axis
than another, or further to one side than the other (upwind), get narrower
regions.

Notation (per face F = (axis d, side): side 0 is the face just below index 0,
side 1 the face just above index l_d - 1):
  delta_F(i)  the distance of cell i to F: i_d + 1 (side 0), l_d - i_d (side 1);
  a_F         the toward-reach: the largest offset towards F among the nonzero
              weights (weight (m + r) multiplies a_t[i + m]; side 0 looks at
              -m_d, side 1 at +m_d), 0 if none;
  b_F         the away-reach: the toward-reach of the opposite face of d.
After t steps a cell depends on the cells up to t a_F closer to F and up to
t b_F farther from it, so the boundary has reached exactly the cells with
delta_F <= a_F t for some F: the l-shell of cell i is
  ell(i) = min over faces with a_F > 0 of ceil(delta_F(i) / a_F).

Reading. The appendix keeps the figure's ranges and reads them in units of ell
with sigma = 1. That fixes what the boundary changes (a kept cell needs
ell > T_k), but a periodic solve must also hold every cell the kept cells'
dependence cones reach, and a cone reaches b_F T_k away from F, which is more
than a_F T_k when the stencil leans away from the face. Written per face, with
"some F" ranging over the faces with a_F > 0 (a face no offset looks towards
never reaches any cell and takes part in no region):
  RecursiveBoundary(T): input  some F: delta_F <= (a_F + b_F) T,
                        output ell <= T;
  Step 1: periodic solve for T1 of the input region, kept on ell > T1 and
          some F: delta_F <= a_F T + b_F T2; recursive call for T1 on some F:
          delta_F <= (a_F + b_F) T1, kept on ell <= T1;
  Step 2: periodic solve for T2 of the time-T1 region some F: delta_F <=
          a_F T + b_F T2, kept on T2 < ell <= T; recursive call for T2, kept
          on ell <= T2;
  base case (T < cutoff): the loop with the boundary's ghosts on the input
          region for T steps, kept on ell <= T.
With a_F = b_F = sigma on every face these are the main body's ranges
(delta_F <= 2 sigma T, sigma T1 < dist <= sigma T + sigma T2, ...). Odd T
splits as T1 = floor(T/2), T2 = T - T1, as in recursive_boundary.py.
"""
from __future__ import annotations

import numpy as np

from .spectral import stencil_fft_periodic
from .stencil_loop import stencil_loop


def face_reach(weights: np.ndarray) -> np.ndarray:
    """Toward-reach a_F per face, shape (ndim, 2): [d, 0] low face, [d, 1] high face."""
    w = np.asarray(weights, dtype=np.float64)
    r = (w.shape[0] - 1) // 2
    reach = np.zeros((w.ndim, 2), dtype=np.int64)
    nz = np.argwhere(w != 0.0) - r          # offsets m of the nonzero weights
    for d in range(w.ndim):
        if len(nz):
            reach[d, 0] = max(0, int(-nz[:, d].min()))
            reach[d, 1] = max(0, int(nz[:, d].max()))
    return reach


def face_distances(dims) -> np.ndarray:
    """delta_F(i) for every face, shape (ndim, 2, *dims)."""
    dims = tuple(int(x) for x in dims)
    grids = np.meshgrid(*[np.arange(l) for l in dims], indexing="ij")
    out = np.empty((len(dims), 2) + dims, dtype=np.int64)
    for d, (g, l) in enumerate(zip(grids, dims)):
        out[d, 0] = g + 1
        out[d, 1] = l - g
    return out


def arrival_time(dims, reach) -> np.ndarray:
    """ell(i): the step at which the boundary's influence first reaches cell i
    (a large sentinel where no face reaches it)."""
    delta = face_distances(dims)
    ell = np.full(tuple(int(x) for x in dims), np.iinfo(np.int64).max // 4, dtype=np.int64)
    for d in range(len(dims)):
        for s in range(2):
            a = int(reach[d][s])
            if a > 0:
                ell = np.minimum(ell, -(-delta[d, s] // a))
    return ell


def _within(delta, reach, width) -> np.ndarray:
    """Cells with delta_F <= width(a_F, b_F) for some face with a_F > 0."""
    m = np.zeros(delta.shape[2:], dtype=bool)
    nd = delta.shape[0]
    for d in range(nd):
        for s in range(2):
            a, b = int(reach[d][s]), int(reach[d][1 - s])
            if a > 0:
                m |= delta[d, s] <= width(a, b)
    return m


def recursive_boundary_shells(a: np.ndarray, weights: np.ndarray, T: int, cutoff: int = 8,
                              boundary: str = "dirichlet", reach=None) -> np.ndarray:
    """RecursiveBoundary on l-shells: from a on the input region of T, the grid
    at time +T on ell <= T (other cells of the result are not meaningful)."""
    if cutoff < 2:
        raise ValueError("cutoff must be >= 2")
    a = np.asarray(a, dtype=np.float64)
    reach = face_reach(weights) if reach is None else np.asarray(reach)
    delta = face_distances(a.shape)
    ell = arrival_time(a.shape, reach)

    def region(width):
        return _within(delta, reach, width)

    if T < cutoff:
        inp = np.where(region(lambda fa, fb: (fa + fb) * T), a, 0.0)
        return stencil_loop(inp, weights, T, boundary)
    T1 = T // 2
    T2 = T - T1
    result = np.zeros_like(a)
    # Step 1: periodic solve of the input region for T1 steps
    A12 = np.where(region(lambda fa, fb: (fa + fb) * T), a, 0.0)
    B23 = stencil_fft_periodic(A12, weights, T1)
    keep = (ell > T1) & region(lambda fa, fb: fa * T + fb * T2)
    result[keep] = B23[keep]
    # Step 1: recursive call for T1
    A1 = np.where(region(lambda fa, fb: (fa + fb) * T1), a, 0.0)
    B1 = recursive_boundary_shells(A1, weights, T1, cutoff, boundary, reach)
    keep = ell <= T1
    result[keep] = B1[keep]
    # Step 2: periodic solve of the time-T1 region for T2 steps
    B123 = np.where(region(lambda fa, fb: fa * T + fb * T2), result, 0.0)
    out = np.zeros_like(a)
    C2 = stencil_fft_periodic(B123, weights, T2)
    keep = (ell > T2) & (ell <= T)
    out[keep] = C2[keep]
    # Step 2: recursive call for T2
    B12 = np.where(region(lambda fa, fb: (fa + fb) * T2), B123, 0.0)
    C1 = recursive_boundary_shells(B12, weights, T2, cutoff, boundary, reach)
    keep = ell <= T2
    out[keep] = C1[keep]
    return out


def stencil_fft_aperiodic_shells(a0: np.ndarray, weights: np.ndarray, T: int, cutoff: int = 8,
                                 boundary: str = "dirichlet") -> np.ndarray:
    """StencilFFT-A on l-shells: cells with ell > T from the periodic solve of the
    whole grid (their cones meet no face), the others from RecursiveBoundary."""
    a0 = np.asarray(a0, dtype=np.float64)
    reach = face_reach(weights)
    ell = arrival_time(a0.shape, reach)
    result = np.empty_like(a0)
    interior = ell > T
    if interior.any():
        center = stencil_fft_periodic(a0, weights, T)
        result[interior] = center[interior]
    if (~interior).any():
        near = recursive_boundary_shells(a0, weights, T, cutoff, boundary, reach)
        result[~interior] = near[~interior]
    return result


def upwind_dirichlet_closed_form(a0: np.ndarray, p, T: int, cells) -> np.ndarray:
    """a_T at the given cells for the 2-D stencil p0 a[i] + p1 a[i - e0] +
    p2 a[i - e1] on a zero-Dirichlet grid (closed form, no recursion).

    The stencil looks only towards the two low faces, so the grid evolves as
    the free-space problem with a0 extended by zeros below index 0 (those
    cells read only cells further below, all zero, and stay zero; the high
    faces are never read). The T-fold convolution power of the stencil is
    the trinomial distribution K_T(dx, dy) = T! / (k! dx! dy!) p0^k p1^dx
    p2^dy with k = T - dx - dy, so
        a_T(i, j) = sum over 0 <= dx <= i, 0 <= dy <= j of K_T(dx, dy) a0(i - dx, j - dy),
    evaluated in FP64 through log-gamma."""
    from scipy.special import gammaln
    a0 = np.asarray(a0, dtype=np.float64)
    dx = np.arange(T + 1)[:, None]
    dy = np.arange(T + 1)[None, :]
    k = T - dx - dy
    kc = np.maximum(k, 0)
    logK = (gammaln(T + 1) - gammaln(kc + 1) - gammaln(dx + 1) - gammaln(dy + 1)
            + kc * np.log(p[0]) + dx * np.log(p[1]) + dy * np.log(p[2]))
    K = np.where(k >= 0, np.exp(logK), 0.0)
    out = []
    for i, j in cells:
        mi, mj = min(i, T), min(j, T)
        win = a0[i - mi:i + 1, j - mj:j + 1][::-1, ::-1]
        out.append(float(np.sum(K[:mi + 1, :mj + 1] * win)))
    return np.array(out)
