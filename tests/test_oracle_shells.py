"""Pins of the l-shell RecursiveBoundary oracle (appendix "l-shell Spatial
Grid Decomposition") against what the mathematics fixes: hand-counted reaches,
the arrival time of the boundary's influence by brute force, the plain loop
(zero Dirichlet and reflecting) for biased, upwind and anisotropic stencils,
the main body's RecursiveBoundary for symmetric stencils, and a planted
mistake (the appendix's ranges without the away-reach) that the loop exposes."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import ell_shells as es
from paper_2105_06676_gb300 import workloads as wl


def _support(nd, r, offsets, seed):
    """Non-negative weights on the given offsets (sum 1), in a (2r+1)^nd box."""
    rng = np.random.default_rng(seed)
    w = np.zeros((2 * r + 1,) * nd)
    for m in offsets:
        w[tuple(mm + r for mm in m)] = 0.2 + rng.random()
    return w / w.sum()


UPWIND_2D = [(0, 0), (-1, 0), (0, -1)]                     # first-order upwind, flow to +x, +y
LEAN_1D = [(-1,), (0,), (2,)]                               # reaches 1 left, 2 right
ANISO_2D = [(0, 0), (-2, 0), (2, 0), (0, -1), (0, 1), (1, 1)]
UPWIND_3D = [(0, 0, 0), (-1, 0, 0), (0, -1, 0), (0, 0, 1), (-1, 0, 1)]
LEAN_2D = [(0, 0), (-1, 0), (3, 0), (0, 2), (0, -1), (1, -1)]

STENCILS = {
    "upwind2d": (2, 1, UPWIND_2D),
    "lean1d": (1, 2, LEAN_1D),
    "aniso2d": (2, 2, ANISO_2D),
    "upwind3d": (3, 1, UPWIND_3D),
    "lean2d": (2, 3, LEAN_2D),
}


def test_face_reach_hand_counted():
    w = _support(1, 2, LEAN_1D, 0)
    np.testing.assert_array_equal(es.face_reach(w), [[1, 2]])
    w = _support(2, 1, UPWIND_2D, 0)
    np.testing.assert_array_equal(es.face_reach(w), [[1, 0], [1, 0]])
    w = _support(2, 2, ANISO_2D, 0)
    np.testing.assert_array_equal(es.face_reach(w), [[2, 2], [1, 1]])
    w = _support(3, 1, UPWIND_3D, 0)
    np.testing.assert_array_equal(es.face_reach(w), [[1, 0], [1, 0], [0, 1]])
    # a symmetric box reaches r towards every face
    np.testing.assert_array_equal(es.face_reach(wl.weights_random_box(3, 2, 1)), [[2, 2]] * 3)


def _brute_arrival(dims, w, tmax):
    """First step at which cell i depends on anything outside the grid: embed
    the grid in a zero pad wider than every cone, evolve once with the pad at
    0 and once at 1 (non-negative weights, nonzero centre: the difference is
    positive exactly where some path of offsets leaves the grid)."""
    r = (w.shape[0] - 1) // 2
    pad = r * tmax + 1
    big = tuple(l + 2 * pad for l in dims)
    inner = tuple(slice(pad, pad + l) for l in dims)
    x0 = np.zeros(big)
    x0[inner] = 1.0
    x1 = np.ones(big)
    out = np.full(dims, tmax + 1)
    for t in range(1, tmax + 1):
        x0 = oracle.stencil_loop(x0, w, 1, "periodic")
        x1 = oracle.stencil_loop(x1, w, 1, "periodic")
        hit = (x1[inner] - x0[inner]) > 0
        out = np.where(hit & (out > tmax), t, out)
    return out


@pytest.mark.parametrize("name,dims", [("lean1d", (23,)), ("upwind2d", (9, 12)), ("aniso2d", (14, 10)),
                                       ("upwind3d", (6, 7, 5)), ("lean2d", (13, 11))])
def test_arrival_time_by_brute_force(name, dims):
    nd, r, offs = STENCILS[name]
    w = _support(nd, r, offs, 3)
    tmax = 6
    got = np.minimum(es.arrival_time(dims, es.face_reach(w)), tmax + 1)
    np.testing.assert_array_equal(got, _brute_arrival(dims, w, tmax))


CASES = [("lean1d", (64,), T) for T in (1, 4, 9, 20, 31)] + [
    ("upwind2d", (32, 32), 9), ("upwind2d", (32, 16), 21), ("upwind2d", (16, 64), 40),
    ("aniso2d", (32, 32), 7), ("aniso2d", (64, 16), 12), ("lean2d", (32, 32), 5),
    ("lean2d", (64, 64), 11), ("upwind3d", (16, 16, 16), 6), ("upwind3d", (16, 8, 16), 11),
]


@pytest.mark.parametrize("boundary", ["dirichlet", "neumann"])
@pytest.mark.parametrize("cutoff", [2, 3, 8])
@pytest.mark.parametrize("name,dims,T", CASES)
def test_shells_match_loop(name, dims, T, cutoff, boundary):
    nd, r, offs = STENCILS[name]
    w = _support(nd, r, offs, 10 + T)
    a0 = wl.grid_uniform(dims, 20 + T)
    got = es.stencil_fft_aperiodic_shells(a0, w, T, cutoff, boundary)
    ref = oracle.stencil_loop(a0, w, T, boundary)
    assert np.max(np.abs(got - ref)) / np.max(np.abs(a0)) < 1e-12


@pytest.mark.parametrize("dims,r,T", [((64,), 1, 13), ((32, 32), 1, 9), ((64, 32), 2, 7),
                                      ((16, 16, 16), 1, 5)])
def test_symmetric_stencils_take_the_main_body_regions(dims, r, T):
    # a_F = b_F = sigma: the same regions as the distance-based recursion
    w = wl.weights_random_box(len(dims), r, 40 + T)
    a0 = wl.grid_uniform(dims, 41)
    for c in (2, 4):
        got = es.stencil_fft_aperiodic_shells(a0, w, T, c)
        ref = oracle.stencil_fft_aperiodic(a0, w, T, c)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)


def test_upwind_regions_are_narrower():
    # an upwind stencil is reached from two faces only: its boundary region is
    # a quarter of the symmetric box's frame or less
    dims, T = (64, 64), 8
    w = _support(2, 1, UPWIND_2D, 5)
    frame_shells = np.count_nonzero(es.arrival_time(dims, es.face_reach(w)) <= T)
    frame_box = np.count_nonzero(oracle.boundary_distance(dims) <= T)
    assert frame_shells < 0.55 * frame_box


def _literal_reading(a, w, T, cutoff, reach, boundary="dirichlet"):
    """Planted mistake: the figure's ranges in units of ell alone (input ell <=
    2T, Step 1 keeps T1 < ell <= T + T2, ...), no allowance for the away-reach."""
    ell = es.arrival_time(a.shape, reach)
    if T < cutoff:
        return oracle.stencil_loop(np.where(ell <= 2 * T, a, 0.0), w, T, boundary)
    T1 = T // 2
    T2 = T - T1
    res = np.zeros_like(a)
    B = oracle.stencil_fft_periodic(np.where(ell <= 2 * T, a, 0.0), w, T1)
    k = (ell > T1) & (ell <= T + T2)
    res[k] = B[k]
    B1 = _literal_reading(np.where(ell <= 2 * T1, a, 0.0), w, T1, cutoff, reach, boundary)
    res[ell <= T1] = B1[ell <= T1]
    B123 = np.where(ell <= T + T2, res, 0.0)
    out = np.zeros_like(a)
    C = oracle.stencil_fft_periodic(B123, w, T2)
    k = (ell > T2) & (ell <= T)
    out[k] = C[k]
    C1 = _literal_reading(np.where(ell <= 2 * T2, B123, 0.0), w, T2, cutoff, reach, boundary)
    out[ell <= T2] = C1[ell <= T2]
    return out


def test_ranges_without_the_away_reach_are_wrong():
    # the stencil reaches 2 cells away from the low face but 1 towards it: a
    # kept cell's cone leaves the region the literal ranges hand to the solve
    nd, r, offs = STENCILS["lean1d"]
    w = _support(nd, r, offs, 6)
    a0 = wl.grid_uniform((128,), 7)
    T = 24
    ref = oracle.stencil_loop(a0, w, T, "dirichlet")
    reach = es.face_reach(w)
    ell = es.arrival_time(a0.shape, reach)
    lit = _literal_reading(a0, w, T, 4, reach)
    near = ell <= T
    assert np.max(np.abs(lit[near] - ref[near])) > 1e-3
    good = es.recursive_boundary_shells(a0, w, T, 4)
    assert np.max(np.abs(good[near] - ref[near])) < 1e-12


@pytest.mark.parametrize("dims,T", [((128, 96), 57), ((64, 200), 150), ((40, 40), 100)])
def test_upwind_closed_form_matches_loop(dims, T):
    w = np.zeros((3, 3))
    w[1, 1], w[0, 1], w[1, 0] = 0.5, 0.3, 0.2
    a0 = wl.grid_uniform(dims, 70 + T)
    ref = oracle.stencil_loop(a0, w, T, "dirichlet")
    rng = np.random.default_rng(T)
    cells = [(0, 0), (dims[0] - 1, dims[1] - 1)] + [
        (int(rng.integers(dims[0])), int(rng.integers(dims[1]))) for _ in range(20)]
    got = es.upwind_dirichlet_closed_form(a0, (0.5, 0.3, 0.2), T, cells)
    np.testing.assert_allclose(got, [ref[c] for c in cells], rtol=0, atol=1e-13)
