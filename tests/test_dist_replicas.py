"""Multi-rank bookkeeping of the benchmark (replicas, no data-path
collective), run as two gloo ranks on the CPU.

Each rank times its own replica of the step; the job's time is the slowest
rank's, and the throughput counts the units of every rank (weak scaling).
The reference arm runs on rank 0 only; the other ranks exit without work.
"""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    r, w, local = bench.dist_env()
    assert (r, w, local) == (rank, world, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 2.0 + 3.0 * rank  # rank 1 is the slow replica
        bench.replica_barrier(world)
        ms = bench.replica_max(ms_local, world, torch.device("cpu"))
        units = 1000
        out[rank] = (ms, bench.replica_throughput(units, world, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank_and_count_all_units():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    for rank in range(world):
        ms, value = out[rank]
        assert ms == pytest.approx(5.0)
        assert value == pytest.approx(world * 1000 / 5e-3)


def test_single_rank_is_the_identity():
    import bench
    assert bench.replica_max(3.5, 1, None) == 3.5
    assert bench.replica_throughput(10, 1, 2.0) == pytest.approx(5000.0)


def _reference_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    class Args:
        steps, warmup = 1, 1

    if rank != 0:
        # a non-zero rank returns at once, without building the workload
        called = []
        orig = bench.workload
        bench.workload = lambda *a, **k: called.append(1) or orig(*a, **k)
        bench.run_reference(Args())
        out[rank] = len(called)


def test_reference_arm_runs_on_rank_zero_only():
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_reference_rank, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    assert out[1] == 0
