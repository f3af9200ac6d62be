"""The benchmark's multi-rank host logic on CPU ranks (gloo, 127.0.0.1): the
job's time is the slowest rank's, the whole-job throughput counts every
rank's cells, and the reference arm runs and prints on rank 0 only."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.max_over_ranks(10.0 + 3.0 * rank, world, "cpu")
    q.put((rank, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 13.0, 1: 13.0}


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(7.5, 1, "cpu") == 7.5


def test_whole_job_throughput_counts_every_rank():
    import bench
    # two ranks, 1,048,576 cells each, 50 steps, slowest rank 100 ms
    assert bench.whole_job_mlups(1 << 20, 50, 2, 100.0) == pytest.approx(2 * (1 << 20) * 50 / 0.1 / 1e6)


def test_reference_arm_is_silent_off_rank_zero(capsys):
    import argparse

    import bench
    args = argparse.Namespace(workload="gas_thread", steps=1, warmup=3, gpus=2)
    bench.run_reference(args, 1)
    assert capsys.readouterr().out == ""
