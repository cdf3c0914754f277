"""The N > 1 path of bench.py (replicas only: every rank solves its own copy;
the job's time is the slowest rank's, its value counts every rank's updates),
run as two gloo ranks on the CPU."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [0.25, 0.4][rank]                     # rank 1 is the slow one
    job = bench.max_over_ranks(ms, world)
    out[rank] = (job, bench.job_value(4096 * 4096, 10000, world, job))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_report_the_slowest_time_and_the_whole_job():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]
    job, value = res[0]
    assert job == pytest.approx(0.4)
    assert value == pytest.approx(2 * 4096 * 4096 * 10000 / 0.4e-3)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(0.3, 1) == 0.3
    assert bench.job_value(10, 5, 1, 2.0) == pytest.approx(25_000.0)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import argparse

    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(steps=1, warmup=0, ref_steps_per_sample=1)
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""
