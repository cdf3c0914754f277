"""StencilFFT-A and RecursiveBoundary in numpy FP64 (oracle; test infrastructure only).

Follows Sec. 5 ("Correcting Final Values in the Boundary's Region of
Influence") and Fig. "stencil-fft-algorithm-1D-aperiodic" in the paper's
order. The boundary condition is zero Dirichlet (cells outside the grid read
0) or reflecting (zero-flux Neumann: the ghost at index -1-k mirrors cell k).
Sec. 5.1 describes which cells a boundary condition changes, not how: the
periodic solves keep only cells whose dependence cone never reaches the
boundary, so the condition enters through the base-case loop alone.

Notation. dist(i) = min over axes of min(i_d + 1, l_d - i_d): the boundary
lies just outside a[0] and a[l-1] (Sec. 5.2, the 1-D and 2-D region
descriptions), so the outermost cells have dist 1. A[a < dist <= b] is the set
of cells of A with dist in (a, b]. sigma is the stencil radius, so after t steps
the boundary influences exactly the cells with dist <= sigma t (Sec. 5.1).

Readings taken where the paper is ambiguous:
  * odd T (the paper writes T/2 and Delta = sigma T / 2): split T = T1 + T2
    with T1 = floor(T/2), T2 = T - T1. Step 1 keeps sigma T1 < dist <=
    sigma T + sigma T2; Step 2 keeps sigma T2 < dist <= sigma T. For even T
    these are the paper's (Delta, 3 Delta] and (Delta, 2 Delta].
  * the recursive call's input: cells with dist <= 2 sigma T_k (the paper
    writes "< 2 Delta" in Step 1 and "<= 2 Delta" in Step 2; the recursion's
    own contract needs <=).
  * "Periodic(s, A, l_1..l_d, T/2)" is the periodic solver applied to the whole
    grid shape with every cell outside the region A set to 0: it is correct on
    the kept cells because their dependence cone (radius sigma T_k) neither
    leaves the region nor crosses the grid boundary.
  * the base case (T < cutoff) evolves the cells with dist <= 2 sigma T by the
    plain loop with the boundary's ghosts for T steps and keeps dist <= sigma T. The
    cutoff must be >= 2 (with cutoff 1, T = 1 would split into T1 = 0,
    T2 = 1 and never terminate).
"""
from __future__ import annotations

import numpy as np

from .spectral import stencil_fft_periodic
from .stencil_loop import stencil_loop


def boundary_distance(dims) -> np.ndarray:
    """dist(i) = min_d min(i_d + 1, l_d - i_d) (Sec. 5.2 region geometry)."""
    dims = tuple(int(x) for x in dims)
    grids = np.meshgrid(*[np.arange(l) for l in dims], indexing="ij")
    dist = None
    for g, l in zip(grids, dims):
        dd = np.minimum(g + 1, l - g)
        dist = dd if dist is None else np.minimum(dist, dd)
    return dist


def _sigma(weights: np.ndarray) -> int:
    return (np.asarray(weights).shape[0] - 1) // 2


def recursive_boundary(a: np.ndarray, weights: np.ndarray, T: int,
                       cutoff: int = 8, dist: np.ndarray | None = None,
                       boundary: str = "dirichlet") -> np.ndarray:
    """RecursiveBoundary: from a at dist <= 2 sigma T, the grid at time +T on dist <= sigma T.

    Returns a full-shape array; only the cells with dist <= sigma T are
    meaningful.
    """
    if cutoff < 2:
        raise ValueError("cutoff must be >= 2")
    a = np.asarray(a, dtype=np.float64)
    if dist is None:
        dist = boundary_distance(a.shape)
    sigma = _sigma(weights)
    # Base case: iterate the loop on the cells within 2 Delta = sigma T.
    if T < cutoff:
        region = np.where(dist <= 2 * sigma * T, a, 0.0)
        return stencil_loop(region, weights, T, boundary)
    T1 = T // 2
    T2 = T - T1
    result = np.zeros_like(a)
    # Step 1 (1): periodic solve of A12 = a[dist <= 2 sigma T] for T1 steps.
    A12 = np.where(dist <= 2 * sigma * T, a, 0.0)
    B23 = stencil_fft_periodic(A12, weights, T1)
    keep = (dist > sigma * T1) & (dist <= sigma * T + sigma * T2)
    result[keep] = B23[keep]
    # Step 1 (2): recursive call on A1 = a[dist <= 2 sigma T1].
    A1 = np.where(dist <= 2 * sigma * T1, a, 0.0)
    B1 = recursive_boundary(A1, weights, T1, cutoff, dist, boundary)
    keep = dist <= sigma * T1
    result[keep] = B1[keep]
    # B123: time-T1 data on dist <= sigma T + sigma T2.
    B123 = np.where(dist <= sigma * T + sigma * T2, result, 0.0)
    out = np.zeros_like(a)
    # Step 2 (1): periodic solve of B123 for T2 steps, keep sigma T2 < dist <= sigma T.
    C2 = stencil_fft_periodic(B123, weights, T2)
    keep = (dist > sigma * T2) & (dist <= sigma * T)
    out[keep] = C2[keep]
    # Step 2 (2): recursive call on B12 = B[dist <= 2 sigma T2].
    B12 = np.where(dist <= 2 * sigma * T2, B123, 0.0)
    C1 = recursive_boundary(B12, weights, T2, cutoff, dist, boundary)
    keep = dist <= sigma * T2
    out[keep] = C1[keep]
    return out


def stencil_fft_aperiodic(a0: np.ndarray, weights: np.ndarray, T: int,
                          cutoff: int = 8, boundary: str = "dirichlet") -> np.ndarray:
    """StencilFFT-A: interior from StencilFFT-P, boundary region from RecursiveBoundary.

    Fig. "stencil-fft-algorithm-1D-aperiodic": result[dist > 2 Delta] comes
    from the periodic solve of the whole grid, result[dist <= 2 Delta] from
    RecursiveBoundary, with 2 Delta = sigma T.
    """
    a0 = np.asarray(a0, dtype=np.float64)
    dist = boundary_distance(a0.shape)
    sigma = _sigma(weights)
    result = np.empty_like(a0)
    interior = dist > sigma * T
    if interior.any():
        center = stencil_fft_periodic(a0, weights, T)
        result[interior] = center[interior]
    near = recursive_boundary(a0, weights, T, cutoff, dist, boundary)
    result[~interior] = near[~interior]
    return result
