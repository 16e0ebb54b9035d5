"""The multi-process path of the benchmark on the CPU (gloo, world size 2).

The solver path does not shard across GPUs ("replicas only"): under torchrun every rank solves
its own copy of the workload on its own GPU and the only exchange is the timing reduction.  Here
two gloo ranks on the host run that reduction with different local results, and rank 0 checks
the whole-job throughput: the units of all ranks over the slowest rank's time.  The reference
arm runs on rank 0 only.
"""
import argparse
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench

MS = [120.0, 150.0]
UNITS = [3000, 3300]


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        value, ms, units = bench.replica_throughput(torch, dist, world, MS[rank], UNITS[rank], "cpu")
        out.put((rank, value, ms, units))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_throughput_is_total_units_over_slowest_rank():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    expect = sum(UNITS) / (max(MS) * 1e-3)
    for rank, value, ms, units in res:
        assert ms == max(MS) and units == sum(UNITS)
        assert value == pytest.approx(expect, rel=1e-15)


def test_single_process_is_a_plain_division():
    value, ms, units = bench.replica_throughput(torch, None, 1, 250.0, 1000, "cpu")
    assert (value, ms, units) == (1000 / 0.25, 250.0, 1000.0)


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(workload="c1", warmup=3, steps=1, ref_budget=1.0, gpus=2)
    bench.run_reference(args)
    assert capsys.readouterr().out == ""
