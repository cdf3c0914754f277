"""Seeded synthetic inputs for the stencil solves (grids, weights, request streams).

This module only draws numbers: it holds none of the method's arithmetic, so
the GPU path and the CPU oracle can both consume its output.

The workloads mirror the shapes of the paper's benchmarks (Sec. 6,
Tab. "benchmarks": 3-point 1-D heat, 5-point 2-D, 9-point 2-D box, 7-point
3-D) with synthetic coefficients, since the paper does not list them.
Grids are uniform[0, 1) in FP64; the FP32 path receives the same values
rounded to nearest.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def grid_uniform(dims, seed: int) -> np.ndarray:
    """uniform[0, 1) FP64 grid of shape dims from numpy's default_rng(seed)."""
    rng = np.random.default_rng(seed)
    return rng.random(tuple(int(x) for x in dims), dtype=np.float64)


def weights_star(ndim: int, center: float, neighbour: float) -> np.ndarray:
    """Radius-1 star stencil: center weight plus one weight on the 2*ndim axis neighbours."""
    w = np.zeros((3,) * ndim, dtype=np.float64)
    c = (1,) * ndim
    w[c] = center
    for axis in range(ndim):
        for side in (0, 2):
            idx = list(c)
            idx[axis] = side
            w[tuple(idx)] = neighbour
    return w


def weights_1d(values) -> np.ndarray:
    return np.asarray(values, dtype=np.float64)


def weights_random_box(ndim: int, radius: int, seed: int) -> np.ndarray:
    """Box stencil of radius r with uniform[0, 1) weights normalised to sum 1."""
    rng = np.random.default_rng(seed)
    w = rng.random((2 * radius + 1,) * ndim, dtype=np.float64)
    return w / w.sum()


def weights_random_signed(ndim: int, radius: int, seed: int) -> np.ndarray:
    """Box stencil with weights uniform in [-1, 1) (no symmetry, no normalisation)."""
    rng = np.random.default_rng(seed)
    return rng.random((2 * radius + 1,) * ndim, dtype=np.float64) * 2.0 - 1.0


def fourier_mode(dims, k, phase: float = 0.0) -> np.ndarray:
    """sin(2 pi k.x / l + phase) sampled on the grid (a test input, not a transform)."""
    dims = tuple(int(x) for x in dims)
    grids = np.meshgrid(*[np.arange(l, dtype=np.float64) for l in dims], indexing="ij")
    arg = np.zeros(dims, dtype=np.float64)
    for g, l, kk in zip(grids, dims, k):
        arg += 2.0 * np.pi * kk * g / l
    return np.sin(arg + phase)


def seeded_modes(ndim: int, seed: int, count: int = 3, kmax: int = 16):
    """count wave vectors with components in [1, kmax] and amplitudes in [0.1, 1)."""
    rng = np.random.default_rng(seed)
    ks = [tuple(int(v) for v in rng.integers(1, kmax + 1, size=ndim)) for _ in range(count)]
    amps = [float(v) for v in rng.uniform(0.1, 1.0, size=count)]
    return ks, amps


def grid_with_modes(dims, seed: int, mode_seed: int, count: int = 3, kmax: int = 16):
    """uniform[0, 1) grid plus `count` seeded Fourier modes; returns (grid, ks, amps)."""
    a = grid_uniform(dims, seed)
    ks, amps = seeded_modes(len(dims), mode_seed, count, kmax)
    for k, c in zip(ks, amps):
        a = a + c * fourier_mode(dims, k)
    return a, ks, amps


@dataclasses.dataclass(frozen=True)
class Workload:
    """One stencil solve: grid shape, stencil weights, steps, boundary, precision."""
    name: str
    dims: tuple
    weights: np.ndarray = dataclasses.field(compare=False, repr=False)
    T: int
    boundary: str          # "periodic" | "dirichlet"
    precision: str         # "fp64" | "fp32"
    grid_seed: int

    @property
    def radius(self) -> int:
        return (self.weights.shape[0] - 1) // 2

    @property
    def n_cells(self) -> int:
        return int(math.prod(self.dims))

    def grid(self) -> np.ndarray:
        return grid_uniform(self.dims, self.grid_seed)


def heat1d_4096() -> Workload:
    """1-D periodic 3-point heat stencil (0.25, 0.5, 0.25), l = 4096, T = 1000, FP64."""
    return Workload("heat1d_periodic_4096_T1000", (4096,), weights_1d([0.25, 0.5, 0.25]),
                    1000, "periodic", "fp64", 1001)


def star2d_4096(precision: str = "fp32") -> Workload:
    """2-D periodic 5-point stencil (center 0.6, neighbours 0.1), 4096^2, T = 10000."""
    return Workload(f"star5_2d_periodic_4096x4096_T10000_{precision}", (4096, 4096),
                    weights_star(2, 0.6, 0.1), 10000, "periodic", precision, 1002)


def star3d_512(precision: str = "fp32") -> Workload:
    """3-D periodic 7-point stencil (center 0.4, neighbours 0.1), 512^3, T = 1000."""
    return Workload(f"star7_3d_periodic_512x512x512_T1000_{precision}", (512, 512, 512),
                    weights_star(3, 0.4, 0.1), 1000, "periodic", precision, 1003)


def box2d_8192_dirichlet() -> Workload:
    """2-D zero-Dirichlet 9-point box, random nonnegative weights summing to 1, 8192^2, T = 4096."""
    return Workload("box9_2d_dirichlet_8192x8192_T4096_fp32", (8192, 8192),
                    weights_random_box(2, 1, 2004), 4096, "dirichlet", "fp32", 1004)


@dataclasses.dataclass
class Request:
    """One solve request of the mixed serving stream."""
    rid: int
    arrival_s: float
    dims: tuple
    weights: np.ndarray
    T: int
    boundary: str
    grid_seed: int


def mixed_stream(n_requests: int, rate_per_s: float, seed: int = 5000,
                 max_1d_log2: int = 24, max_2d_log2: int = 13, max_3d_log2: int = 8):
    """Poisson-arrival stream of mixed solves.

    1-D l = 2^U{12..max_1d_log2}, 2-D per-axis 2^U{6..max_2d_log2}, 3-D per-axis
    2^U{4..max_3d_log2}; T = floor(10^U[1, 5]); periodic / zero-Dirichlet 50/50;
    radius 1 or 2 box with uniform[0, 1) weights normalised to sum 1.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n_requests):
        t += float(rng.exponential(1.0 / rate_per_s))
        nd = int(rng.integers(1, 4))
        if nd == 1:
            dims = (1 << int(rng.integers(12, max_1d_log2 + 1)),)
        elif nd == 2:
            dims = tuple(1 << int(rng.integers(6, max_2d_log2 + 1)) for _ in range(2))
        else:
            dims = tuple(1 << int(rng.integers(4, max_3d_log2 + 1)) for _ in range(3))
        T = int(math.floor(10.0 ** rng.uniform(1.0, 5.0)))
        boundary = "periodic" if rng.random() < 0.5 else "dirichlet"
        radius = int(rng.integers(1, 3))
        w = rng.random((2 * radius + 1,) * nd, dtype=np.float64)
        w = w / w.sum()
        out.append(Request(rid, t, dims, w, T, boundary, int(rng.integers(0, 2**31))))
    return out
