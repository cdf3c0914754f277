"""Host logic of bench.py that needs no GPU: the DRAM-traffic record is used
only while the kernel sources are the ones it was measured on, the FFT flop
count of the FP64 line, the whole-job value."""
from __future__ import annotations

import json
import math

import pytest

import bench


def test_traffic_record_matches_current_kernel_sources():
    # the committed record was taken on the committed kernels
    with open(bench.TRAFFIC_FILE) as fh:
        rec = json.load(fh)
    assert rec["source_sha256"] == bench.kernel_source_hash()
    for kind in ("cols_fused", "rows_r2c", "rows_c2r"):
        assert bench.kernel_traffic(kind) == rec["bytes_per_launch"][kind] > 0


def test_traffic_is_withheld_once_the_kernels_change(tmp_path, monkeypatch):
    with open(bench.TRAFFIC_FILE) as fh:
        rec = json.load(fh)
    rec["source_sha256"] = "0" * 64                 # taken on other kernels
    f = tmp_path / "traffic.json"
    f.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.kernel_traffic("cols_fused") is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.json"))
    assert bench.kernel_traffic("cols_fused") is None


def test_fft_flop_count_of_the_2d_solve():
    # 4096 rows of 2048-point transforms and 2049 columns of 4096-point
    # transforms, forward and inverse, 5 n log2 n each
    want = 2 * 4096 * 5 * 2048 * 11 + 2 * 2049 * 5 * 4096 * 12
    assert bench.fft2d_flops((4096, 4096)) == pytest.approx(want)
    assert bench.fft2d_flops((16, 32)) == pytest.approx(
        2 * 16 * 5 * 16 * math.log2(16) + 2 * 17 * 5 * 16 * math.log2(16))


def test_job_value_counts_every_rank():
    assert bench.job_value(4096 * 4096, 10000, 4, 0.2) == pytest.approx(
        4 * 4096 * 4096 * 10000 / 0.2e-3)


# ---------------------------------------------------------------------------
# algorithmic bytes of the zero-Dirichlet schedule (the Dirichlet roofline)
# ---------------------------------------------------------------------------
def _schedule(dims, r, T, cutoff, reach=None):
    import ctypes

    from paper_2105_06676_gb300 import _capi
    lib = _capi.lib()
    d = (ctypes.c_int64 * len(dims))(*dims)
    rc = None if reach is None else (ctypes.c_int * (2 * len(dims)))(*reach)
    n = lib.stencil_debug_schedule_reach(len(dims), d, r, rc, T, cutoff, None, 0)
    buf = (ctypes.c_int64 * n)()
    lib.stencil_debug_schedule_reach(len(dims), d, r, rc, T, cutoff, buf, n)
    return bench._decode_schedule(list(buf))


@pytest.mark.parametrize("dims,r,T,cutoff,reach", [((64, 64), 1, 21, 3, None), ((128, 64), 2, 17, 2, None),
                                                   ((64, 128), 1, 40, 4, [1, 0, 1, 0]),
                                                   ((128, 128), 3, 9, 3, [1, 3, 2, 1])])
def test_kept_cell_count_matches_the_keep_rule(dims, r, T, cutoff, reach):
    import numpy as np
    import __graft_entry__
    __graft_entry__.build()
    g = np.meshgrid(*[np.arange(l) for l in dims], indexing="ij")
    delta = [[g[a] + 1, dims[a] - g[a]] for a in range(2)]
    for o in _schedule(dims, r, T, cutoff, reach):
        if o[0] != "solve":
            continue
        for s in o[2]:
            clear = np.ones(dims, dtype=bool)
            near = np.zeros(dims, dtype=bool)
            for a in range(2):
                for side in range(2):
                    clear &= delta[a][side] > s["lo"][2 * a + side]
                    near |= delta[a][side] <= s["hi"][2 * a + side]
            if s["face_axis"] >= 0:
                f = 2 * s["face_axis"] + s["face_side"]
                near = delta[s["face_axis"]][s["face_side"]] <= s["hi"][f]
            assert bench._kept_cells(dims, s) == int(np.count_nonzero(clear & near))


@pytest.mark.parametrize("dims,r,T,cutoff,reach", [((256, 256), 1, 40, 8, None), ((256, 128), 2, 30, 4, None),
                                                   ((256, 256), 1, 60, 8, [1, 0, 1, 0])])
def test_base_case_bytes_cover_each_frame_once(dims, r, T, cutoff, reach):
    # the tiles of a leaf partition its frame: their output cells add up to
    # the frame (cells within wout of some face), each written once
    import numpy as np
    import __graft_entry__
    __graft_entry__.build()
    g = np.meshgrid(*[np.arange(l) for l in dims], indexing="ij")
    for o in _schedule(dims, r, T, cutoff, reach):
        if o[0] != "base":
            continue
        _, Tb, tiles, wout = o
        frame = np.zeros(dims, dtype=bool)
        for a in range(2):
            frame |= (g[a] + 1 <= wout[2 * a]) | (dims[a] - g[a] <= wout[2 * a + 1])
        covered = np.zeros(dims, dtype=np.int64)
        for lo, hi in tiles:
            covered[lo[0]:hi[0], lo[1]:hi[1]] += 1
        assert np.all(covered[frame] == 1)


def test_dirichlet_bytes_of_the_bench_solve():
    # 8192^2, r = 1, T = 4096 with the solver's own cutoff: every kind has
    # bytes, the three FFT passes move the same half spectrum
    import __graft_entry__
    __graft_entry__.build()
    b = bench.dirichlet_algorithmic_bytes((8192, 8192), 1, 4096)
    assert set(b) == {"gather", "rows_r2c", "cols_fused", "rows_c2r", "scatter", "base_loop"}
    assert all(v > 0 for v in b.values())
    assert b["rows_r2c"] == b["rows_c2r"]
    assert bench.dirichlet_algorithmic_bytes((16, 16, 16), 1, 5) is None
