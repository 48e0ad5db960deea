"""bench.py's multi-rank aggregation (replicas, max over ranks) with two gloo
ranks on the CPU: no GPU, no collective on the data path."""

from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = [120.0, 80.0][rank]
    out[rank] = (bench.max_over_ranks(ms, world, "cpu"), bench.job_rate(world, 1000, 5, bench.max_over_ranks(ms, world, "cpu")))
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        ms, rate = out[r]
        assert ms == 120.0
        assert rate == pytest.approx(2 * 1000 * 5 / 0.120 / 1e6)


def test_single_rank_passthrough():
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5
    assert bench.job_rate(1, 10**6, 2, 1000.0) == pytest.approx(2.0)
