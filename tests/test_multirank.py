"""The N-GPU form of the benchmark on CPU (gloo, world size 2): every rank
runs its own replica on its own inputs (weak scaling, no collective on the
data path); the job's step time is the slowest rank's, its throughput the
units of all ranks over that time; only rank 0 reports, and the reference
arm does its work on rank 0 only."""
import io
import os
import socket
import contextlib

import numpy as np
import pytest
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r took 10 + r ms per step and 3 + 2r ms of aggregation
        ms, agg = bench.max_over_ranks([10.0 + rank, 3.0 + 2 * rank], world)
        value = bench.job_throughput(1_000_000, world, ms)
        # each rank's replica has its own inputs (seed = rank)
        w = bench._gen("ungrouped_1m", rank, 4096)
        dist.barrier()
        out[rank] = (ms, agg, value, int(w.keys[:64].sum()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_sum_the_units():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][:3] == res[1][:3]
    ms, agg, value, _ = res[0]
    assert ms == 11.0 and agg == 5.0
    assert value == pytest.approx(2 * 1_000_000 / 0.011)
    assert res[0][3] != res[1][3]                      # independent replicas, distinct inputs


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"ref_rows": 1000, "warmup": 0, "steps": 1, "workload": "ungrouped_1m", "gpus": 2})()
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.run_reference(args) == 0
    assert buf.getvalue() == ""


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks([4.0, 2.0], 1) == [4.0, 2.0]
    assert bench.job_throughput(500, 1, 2.0) == pytest.approx(250_000.0)
