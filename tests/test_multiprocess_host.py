"""The N > 1 path of bench.py on CPU: one process per replica, world size 2
over gloo.  The path has no exchange step (replicas only), so the only
cross-rank operations are the barrier and the max over ranks of the timed
region; the whole-job value counts every replica's cells.  The reference arm
runs on rank 0 alone."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t = bench.max_over_ranks(1.5 + rank, dist, "cpu")  # rank 1 is the slowest
        out[rank] = t
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    assert dict(out) == {0: 2.5, 1: 2.5}


def test_replica_value_counts_every_rank():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.0, None, "cpu") == 3.0
    # 2 replicas of 1000 cells, 10 steps each, slowest rank 0.5 s
    assert bench.replica_throughput(1000, 10, 2, 0.5) == pytest.approx(40000.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        workload, steps, warmup, gpus = "density8", 1, 0, 2

    assert bench.run_reference(A, rank=1, world=2) is None
    assert capsys.readouterr().out == ""
