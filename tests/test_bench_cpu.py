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
