"""Host-side check of the zero-Dirichlet schedule (no GPU).

The library exports the RecursiveBoundary schedule it would launch
(stencil_debug_schedule). This test executes that schedule with numpy
stand-ins for each kernel -- gather, periodic solve of a strip box (the
oracle's StencilFFT-P), masked scatter, temporally blocked base-case tiles
(the oracle's loop on the tile's input box) -- and compares the result with
the zero-Dirichlet loop oracle. A wrong strip width, keep range, offset,
face mask, odd-T split or base-tile cover fails here on the CPU.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import __graft_entry__
import oracle
from oracle import ell_shells as es
from paper_2105_06676_gb300 import _capi
from paper_2105_06676_gb300 import workloads as wl


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    return _capi.lib()


def fetch_schedule(lib, dims, r, T, cutoff, reach=None):
    d = (ctypes.c_int64 * len(dims))(*dims)
    if reach is None:
        n = lib.stencil_debug_schedule(len(dims), d, r, T, cutoff, None, 0)
        assert n > 0
        buf = (ctypes.c_int64 * n)()
        assert lib.stencil_debug_schedule(len(dims), d, r, T, cutoff, buf, n) == n
        return list(buf)
    rc = (ctypes.c_int * (2 * len(dims)))(*[int(x) for x in np.asarray(reach).ravel()])
    n = lib.stencil_debug_schedule_reach(len(dims), d, r, rc, T, cutoff, None, 0)
    assert n > 0
    buf = (ctypes.c_int64 * n)()
    assert lib.stencil_debug_schedule_reach(len(dims), d, r, rc, T, cutoff, buf, n) == n
    return list(buf)


def decode(v):
    ops, i = [], 0
    while i < len(v):
        kind = v[i]
        if kind == 1:
            step, Tk, level, n = v[i + 1:i + 5]
            i += 5
            strips = []
            for _ in range(n):
                f = v[i:i + 26]
                i += 26
                strips.append(dict(bdims=f[0:3], off=f[3:6], valid=f[6:9], perm=f[9:12],
                                   lo=f[12:18], hi=f[18:24], face_axis=f[24], face_side=f[25]))
            ops.append(("solve", step, Tk, level, strips))
        elif kind == 2:
            ops.append(("scatter", v[i + 1]))
            i += 2
        elif kind in (4, 5, 6):
            ops.append(("loop", v[i + 1]))
            i += 2
        elif kind == 3:
            Tb, wout, n = v[i + 1], v[i + 2:i + 8], v[i + 8]
            i += 9
            tiles = []
            for _ in range(n):
                f = v[i:i + 6]
                i += 6
                tiles.append((f[0::2], f[1::2]))
            ops.append(("base", Tb, tiles, wout))
        else:
            raise AssertionError(f"bad op {kind}")
    return ops


def region_slices(s, nd):
    """Grid slices of a strip: grid axis perm[a] spans valid[a] cells from off."""
    sl = [None] * nd
    for a in range(nd):
        ga = s["perm"][a]
        sl[ga] = slice(s["off"][ga], s["off"][ga] + s["valid"][a])
    return tuple(sl)


def _near(delta, bound):
    """Cells within bound[f] of some face f (delta: face_distances, faces 2a + side)."""
    m = np.zeros(delta.shape[2:], dtype=bool)
    for a in range(delta.shape[0]):
        for s in range(2):
            m |= delta[a, s] <= bound[2 * a + s]
    return m


def emulate(a0, w, T, ops, boundary="dirichlet"):
    """Replay the exported schedule with numpy stand-ins for each kernel. The
    interior (cells the boundary cannot reach in T steps) comes from the
    periodic solve of the whole input, as the solver does. The boundary
    condition enters only through the loops: a base-case tile is evolved by
    the oracle's loop on its input box with that condition's ghosts (on a
    side of the box inside the grid any ghost value is harmless: the kept
    cells lie a full halo away from it)."""
    dims = a0.shape
    nd = a0.ndim
    r = (w.shape[0] - 1) // 2
    delta = es.face_distances(dims)
    X = a0.copy()
    loop = any(op[0] == "loop" for op in ops)
    interior = es.arrival_time(dims, es.face_reach(w)) > T
    Z = oracle.stencil_fft_periodic(a0, w, T) if interior.any() and not loop else None
    stash = {}
    for op in ops:
        if op[0] == "loop":
            X = oracle.stencil_loop(X, w, op[1], boundary)
            continue
        if op[0] == "solve":
            _, step, Tk, level, strips = op
            out = []
            for s in strips:
                perm = s["perm"][:nd]
                bd = tuple(s["bdims"][:nd])
                S = np.zeros(bd)
                # box axis a is grid axis perm[a]: the box holds the region transposed
                region = X[region_slices(s, nd)]
                valid = tuple(slice(0, s["valid"][a]) for a in range(nd))
                S[valid] = np.transpose(region, perm)
                out.append(oracle.stencil_fft_periodic(S, np.transpose(w, perm), Tk))
            stash[step] = (strips, out)
        elif op[0] == "scatter":
            strips, out = stash.pop(op[1])
            for s, S in zip(strips, out):
                perm = s["perm"][:nd]
                inv = np.argsort(perm)
                valid = tuple(slice(0, s["valid"][a]) for a in range(nd))
                back = np.transpose(S[valid], inv)
                sl_grid = region_slices(s, nd)
                dl = delta[(slice(None), slice(None)) + sl_grid]
                m = ~_near(dl, s["lo"])
                fa = s["face_axis"]
                if fa >= 0:
                    f = 2 * fa + s["face_side"]
                    m &= dl[fa, s["face_side"]] <= s["hi"][f]
                else:
                    m &= _near(dl, s["hi"])
                sub = X[sl_grid]
                sub[m] = back[m]
        else:
            _, Tb, tiles, wout = op
            h = r * Tb
            Y = X.copy()
            for lo, hi in tiles:
                lo, hi = lo[:nd], hi[:nd]
                ilo = [max(lo[a] - h, 0) for a in range(nd)]
                ihi = [min(hi[a] + h, dims[a]) for a in range(nd)]
                sub = X[tuple(slice(ilo[a], ihi[a]) for a in range(nd))]
                res = oracle.stencil_loop(sub, w, Tb, boundary)
                osl = tuple(slice(lo[a], hi[a]) for a in range(nd))
                rsl = tuple(slice(lo[a] - ilo[a], hi[a] - ilo[a]) for a in range(nd))
                m = _near(delta[(slice(None), slice(None)) + osl], wout)
                Y[osl][m] = res[rsl][m]
            cover = _near(delta, wout)
            X[cover] = Y[cover]
    if Z is not None:
        X[interior] = Z[interior]
    return X


CASES = [
    ((64,), 1, T, c) for T in (1, 2, 3, 5, 7, 13, 19, 40) for c in (2, 3, 8)
] + [
    ((256,), 2, 50, 4), ((64,), 2, 45, 0), ((32,), 1, 45, 2), ((1024,), 1, 300, 0),
    ((32, 32), 1, 9, 2), ((32, 16), 1, 13, 3), ((64, 32), 2, 6, 2), ((16, 64), 1, 11, 4),
    ((64, 64), 1, 32, 0), ((128, 64), 1, 40, 8), ((16, 16, 16), 1, 5, 2), ((32, 16, 8), 1, 7, 3),
    ((16, 16, 32), 1, 10, 0),
]


@pytest.mark.parametrize("dims,r,T,cutoff", CASES)
def test_schedule_reproduces_dirichlet_loop(lib, dims, r, T, cutoff):
    w = wl.weights_random_box(len(dims), r, 100 + T)
    a0 = wl.grid_uniform(dims, 7 + T)
    ops = decode(fetch_schedule(lib, dims, r, T, cutoff))
    got = emulate(a0, w, T, ops)
    ref = oracle.stencil_loop(a0, w, T, "dirichlet")
    assert np.max(np.abs(got - ref)) / np.max(np.abs(a0)) < 1e-11


def test_schedule_structure(lib):
    ops = decode(fetch_schedule(lib, (8192, 8192), 1, 4096, 32))
    solves = [o for o in ops if o[0] == "solve"]
    bases = [o for o in ops if o[0] == "base"]
    # T = 4096 halves down to 16 < 32: 256 leaves, 255 internal nodes x 2 solves
    assert len(bases) == 256 and len(solves) == 510
    assert all(o[1] == 16 for o in bases)
    # the top two levels are whole-grid solves, deeper ones four face strips,
    # the vertical two gathered transposed (face-normal axis first)
    assert all(len(o[4]) == 1 for o in solves if o[3] <= 1)
    assert all(len(o[4]) == 4 for o in solves if o[3] >= 2)
    for o in solves:
        if o[3] >= 2:
            assert [s["perm"][:2] for s in o[4]] == [[0, 1], [0, 1], [1, 0], [1, 0]]
            assert len({tuple(s["bdims"]) for s in o[4]}) == 1
    # every scatter follows its solve
    seen = set()
    for o in ops:
        if o[0] == "solve":
            seen.add(o[1])
        elif o[0] == "scatter":
            assert o[1] in seen


def test_schedule_rejects_bad_arguments(lib):
    d = (ctypes.c_int64 * 1)(64)
    assert lib.stencil_debug_schedule(1, d, 0, 5, 0, None, 0) == -1
    assert lib.stencil_debug_schedule(1, d, 1, 0, 0, None, 0) == -1
    assert lib.stencil_debug_schedule(1, d, 1, 5, 1, None, 0) == -1
    d12 = (ctypes.c_int64 * 1)(12)
    assert lib.stencil_debug_schedule(1, d12, 1, 5, 0, None, 0) == -1


def test_auto_mode_picks_the_loop_when_everything_is_boundary(lib):
    # sigma T far beyond the grid: every cell feels the boundary, FFTs cannot help
    ops = decode(fetch_schedule(lib, (16, 16), 1, 5000, 0))
    assert ops and all(o[0] == "loop" for o in ops) and sum(o[1] for o in ops) == 5000
    # a larger grid may take base leaves over the whole grid instead (the same
    # loop in other chunks), but never an FFT solve
    ops = decode(fetch_schedule(lib, (32, 32), 3, 20000, 0))
    assert ops and all(o[0] in ("loop", "base") for o in ops)
    ops = decode(fetch_schedule(lib, (16, 16, 16), 1, 300, 0))
    assert ops == [("loop", 300)]
    # the benchmark regime stays recursive
    ops = decode(fetch_schedule(lib, (8192, 8192), 1, 4096, 0))
    assert any(o[0] == "solve" for o in ops)


@pytest.mark.parametrize("dims,r,T", [((32, 32), 2, 300), ((16, 16, 16), 1, 40), ((128,), 1, 900)])
def test_auto_loop_schedule_reproduces_dirichlet_loop(lib, dims, r, T):
    w = wl.weights_random_box(len(dims), r, 5)
    a0 = wl.grid_uniform(dims, 6)
    ops = decode(fetch_schedule(lib, dims, r, T, 0))
    got = emulate(a0, w, T, ops)
    ref = oracle.stencil_loop(a0, w, T, "dirichlet")
    assert np.max(np.abs(got - ref)) < 1e-11


# automatic cutoff with r = 2, 3 (bounded by the leaves' halo recomputation)
CASES_AUTO_R = [((128, 128), 2, 40), ((256, 64), 3, 30), ((32, 32, 32), 2, 12), ((512,), 3, 200),
                ((128, 256), 2, 75)]


@pytest.mark.parametrize("dims,r,T", CASES_AUTO_R)
def test_recursive_schedule_with_automatic_cutoff_reproduces_loop(lib, dims, r, T):
    w = wl.weights_random_box(len(dims), r, 200 + T)
    a0 = wl.grid_uniform(dims, 9 + T)
    # cutoff 0 lets the model also pick the loop; the recursion is forced by
    # asking for the automatic cutoff's value explicitly below
    for cutoff in (0, auto_cutoff_value(dims, r)):
        ops = decode(fetch_schedule(lib, dims, r, T, cutoff))
        got = emulate(a0, w, T, ops)
        ref = oracle.stencil_loop(a0, w, T, "dirichlet")
        assert np.max(np.abs(got - ref)) / np.max(np.abs(a0)) < 1e-11


def auto_cutoff_value(dims, r, elem=4):
    """The automatic base-case cutoff's rule restated: the largest T_b + 1 whose
    halo h = r T_b leaves tiles at least 2h wide within the shared-memory
    budget of 150 KB per two buffers (side of the budget's cube / square)."""
    d = len(dims)
    side = (150 * 1024 / (2 * elem)) ** (1.0 / d)
    tb = int((side - 2 * r) / (4 * r))
    return max(2, min({1: 256, 2: 64, 3: 8}[d], tb + 1))


@pytest.mark.parametrize("dims,r,T", [((8192, 8192), 1, 4096), ((4096, 256), 2, 7004),
                                      ((2048, 2048), 3, 500), ((512, 2048), 2, 1000),
                                      ((64, 64, 64), 1, 40)])
def test_automatic_cutoff_keeps_leaf_halos_small(lib, dims, r, T):
    # every leaf of the automatic schedule satisfies 4 r T_b + 2 r <= side of
    # the shared-memory budget, so a tile can be twice its halo wide (a cutoff
    # chosen only by "the tile fits" gives 1-cell tiles with halos of 60+)
    ops = decode(fetch_schedule(lib, dims, r, T, auto_cutoff_value(dims, r)))
    leaves = [o for o in ops if o[0] == "base"]
    assert leaves
    side = (150 * 1024 / 8) ** (1.0 / len(dims))
    for _, Tb, _tiles, _wout in leaves:
        assert 4 * r * Tb + 2 * r <= side


# ---------------------------------------------------------------------------
# l-shell regions (appendix "l-shell Spatial Grid Decomposition"): stencils
# that reach further towards some faces than towards others
# ---------------------------------------------------------------------------
def _support(nd, r, offsets, seed):
    rng = np.random.default_rng(seed)
    w = np.zeros((2 * r + 1,) * nd)
    for m in offsets:
        w[tuple(mm + r for mm in m)] = 0.2 + rng.random()
    return w / w.sum()


SHELL_STENCILS = {
    "upwind1d": (1, 1, [(-1,), (0,)]),
    "lean1d": (1, 2, [(-1,), (0,), (2,)]),
    "upwind2d": (2, 1, [(0, 0), (-1, 0), (0, -1)]),
    "aniso2d": (2, 2, [(0, 0), (-2, 0), (2, 0), (0, -1), (0, 1), (1, 1)]),
    "lean2d": (2, 3, [(0, 0), (-1, 0), (3, 0), (0, 2), (0, -1), (1, -1)]),
    "upwind3d": (3, 1, [(0, 0, 0), (-1, 0, 0), (0, -1, 0), (0, 0, 1), (-1, 0, 1)]),
}

SHELL_CASES = [("upwind1d", (64,), T, c) for T in (1, 5, 13, 40, 63, 90) for c in (2, 3, 8)] + [
    ("lean1d", (128,), 31, 4), ("lean1d", (256,), 70, 0), ("lean1d", (64,), 21, 3),
    ("upwind2d", (64, 64), 40, 4), ("upwind2d", (32, 64), 21, 3), ("upwind2d", (128, 32), 100, 8),
    ("aniso2d", (64, 32), 9, 2), ("aniso2d", (128, 64), 20, 4), ("lean2d", (64, 64), 9, 3),
    ("lean2d", (128, 128), 17, 0), ("upwind3d", (16, 16, 32), 9, 2), ("upwind3d", (32, 16, 16), 14, 3),
]


@pytest.mark.parametrize("name,dims,T,cutoff", SHELL_CASES)
def test_shell_schedule_reproduces_dirichlet_loop(lib, name, dims, T, cutoff):
    nd, r, offs = SHELL_STENCILS[name]
    w = _support(nd, r, offs, 300 + T)
    a0 = wl.grid_uniform(dims, 301 + T)
    ops = decode(fetch_schedule(lib, dims, r, T, cutoff, es.face_reach(w)))
    got = emulate(a0, w, T, ops)
    ref = oracle.stencil_loop(a0, w, T, "dirichlet")
    assert np.max(np.abs(got - ref)) / np.max(np.abs(a0)) < 1e-11


def test_symmetric_reach_gives_the_distance_schedule(lib):
    for dims, r, T, c in [((8192, 8192), 1, 4096, 32), ((64, 32), 2, 6, 2), ((16, 16, 16), 1, 5, 2)]:
        assert fetch_schedule(lib, dims, r, T, c) == fetch_schedule(lib, dims, r, T, c,
                                                                    [r] * (2 * len(dims)))


def test_upwind_schedule_touches_only_the_upwind_faces(lib):
    # flow towards +x and +y: only the low faces (0 and 2) are ever reached, so
    # strips and base-case bands sit on those two faces alone
    ops = decode(fetch_schedule(lib, (4096, 4096), 1, 1024, 16, [1, 0, 1, 0]))
    strips = [s for o in ops if o[0] == "solve" for s in o[4]]
    assert strips and all(s["face_axis"] == -1 or s["face_side"] == 0 for s in strips)
    assert sum(1 for s in strips if s["face_axis"] >= 0) > 0
    for o in ops:
        if o[0] == "base":
            assert o[3][1] == 0 and o[3][3] == 0
            # every tile lies in a low band: lo of its normal axis is 0
            assert all(min(lo[0], lo[1]) == 0 for lo, _hi in o[2])
    # half the strips of the symmetric schedule
    sym = decode(fetch_schedule(lib, (4096, 4096), 1, 1024, 16))
    n_sym = sum(len(o[4]) for o in sym if o[0] == "solve")
    assert len(strips) < 0.6 * n_sym


def test_reach_arguments_are_checked(lib):
    d = (ctypes.c_int64 * 2)(64, 64)
    bad = [[0, 0, 0, 0], [2, 0, 0, 0], [-1, 1, 1, 1]]
    for reach in bad:
        rc = (ctypes.c_int * 4)(*reach)
        assert lib.stencil_debug_schedule_reach(2, d, 1, rc, 5, 0, None, 0) == -1


def _plan_reach(lib, w):
    nd = w.ndim
    r = (w.shape[0] - 1) // 2
    out = (ctypes.c_int * (2 * nd))()
    wc = np.ascontiguousarray(w, dtype=np.float64)
    assert lib.stencil_debug_face_reach(nd, r, wc.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out) == 0
    return np.array(list(out)).reshape(nd, 2)


def test_plan_face_reach_matches_the_oracle(lib):
    # the reach a plan derives from its weights (the l-shell regions' input)
    # against the oracle's, on random sparse supports of every dimension and radius
    rng = np.random.default_rng(400)
    for nd in (1, 2, 3):
        for r in (0, 1, 2, 3):
            for _ in range(25):
                w = rng.random((2 * r + 1,) * nd) * (rng.random((2 * r + 1,) * nd) < 0.3)
                np.testing.assert_array_equal(_plan_reach(lib, w), es.face_reach(w))
    for name, (nd, r, offs) in SHELL_STENCILS.items():
        w = _support(nd, r, offs, 401)
        np.testing.assert_array_equal(_plan_reach(lib, w), es.face_reach(w))


def test_plan_reach_drives_the_schedule_end_to_end(lib):
    # weights -> the library's reach -> the library's schedule -> replay == loop
    nd, r, offs = SHELL_STENCILS["lean2d"]
    w = _support(nd, r, offs, 402)
    a0 = wl.grid_uniform((64, 128), 403)
    T = 13
    ops = decode(fetch_schedule(lib, (64, 128), r, T, 3, _plan_reach(lib, w)))
    got = emulate(a0, w, T, ops)
    assert np.max(np.abs(got - oracle.stencil_loop(a0, w, T, "dirichlet"))) / np.max(np.abs(a0)) < 1e-11


def test_face_reach_rejects_bad_arguments(lib):
    w = np.ones(3)
    out = (ctypes.c_int * 2)()
    dp = w.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.stencil_debug_face_reach(0, 1, dp, out) == -1
    assert lib.stencil_debug_face_reach(1, 4, dp, out) == -1
    assert lib.stencil_debug_face_reach(1, 1, None, out) == -1


NEUMANN_CASES = [(None, (64,), 1, 40, 3), (None, (32, 64), 1, 21, 3), (None, (64, 32), 2, 9, 2),
                 (None, (16, 16, 32), 1, 7, 2), ("upwind1d", (64,), 1, 33, 3),
                 ("lean2d", (64, 64), 3, 9, 3), ("upwind2d", (64, 32), 1, 30, 4),
                 ("upwind3d", (16, 32, 16), 1, 11, 3)]


@pytest.mark.parametrize("name,dims,r,T,cutoff", NEUMANN_CASES)
def test_schedule_reproduces_reflecting_loop(lib, name, dims, r, T, cutoff):
    # the reflecting boundary runs the same schedule; only the base-case loop
    # changes its ghosts
    if name is None:
        w = wl.weights_random_box(len(dims), r, 500 + T)
        reach = None
    else:
        nd, r, offs = SHELL_STENCILS[name]
        w = _support(nd, r, offs, 500 + T)
        reach = es.face_reach(w)
    a0 = wl.grid_uniform(dims, 501 + T)
    ops = decode(fetch_schedule(lib, dims, r, T, cutoff, reach))
    assert any(o[0] == "solve" for o in ops)
    got = emulate(a0, w, T, ops, "neumann")
    ref = oracle.stencil_loop(a0, w, T, "neumann")
    assert np.max(np.abs(got - ref)) / np.max(np.abs(a0)) < 1e-11
