"""Host logic of the multi-GPU benchmark on CPU (gloo, world size 2).

The path has no exchange step: under torchrun every rank runs an independent replica
of the workload, and the whole-job value is the units of all ranks over the slowest
rank's time.  These tests run that reduction over two gloo processes, and check that
the reference arm does its work on rank 0 only."""
from __future__ import annotations

import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 1 + r seconds for 8 units
        value, t = bench.aggregate_rate(1.0 + rank, 8, world, dist, "cpu")
        out[rank] = (value, t)
    finally:
        dist.destroy_process_group()


def test_replica_throughput_uses_the_slowest_rank():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        value, t = out[rank]
        assert t == pytest.approx(2.0)              # max over ranks
        assert value == pytest.approx(2 * 8 / 2.0)  # all ranks' units / slowest time


def test_single_rank_needs_no_process_group():
    assert bench.aggregate_rate(4.0, 10, 1) == (2.5, 4.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class Args:
        workload = "uniform4096"
        warmup, steps, ref_budget = 0, 1, 0.1
    bench.run_reference(Args(), rank=1, world=2)   # returns at once, prints nothing
    assert capsys.readouterr().out == ""
