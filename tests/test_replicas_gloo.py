"""The multi-GPU form of the benchmark: one process per GPU, each an independent replica of the
workload (the hot path has no exchange step), joined only by a barrier before the timed region
and the maximum of the ranks' times after it; `value` is the units of all replicas over that
time ("weak" scaling). These tests run the same aggregation with two gloo ranks on the CPU, and
check that the oracle's reference arm does its work on rank 0 alone.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        r, w, local = bench.dist_env()
        seconds = 1.5 + rank  # the ranks finish at different times
        slowest = bench.max_over_ranks(seconds, torch.device("cpu"), w)
        rate = bench.replica_rate(w, 1000.0, slowest)
        dist.barrier()
        q.put((rank, r, w, local, slowest, rate))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank_and_the_whole_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, r, w, local, slowest, rate in got:
        assert (r, w, local) == (rank, 2, rank)
        assert slowest == 2.5  # every rank sees the slowest rank's time
        assert rate == 2 * 1000.0 / 2.5  # units of both replicas over that time


def test_one_process_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(3.0, torch.device("cpu"), 1) == 3.0
    assert bench.replica_rate(1, 500.0, 2.0) == 250.0


def test_reference_arm_works_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun with N > 1 the oracle's reference arm runs and prints on rank 0; the other
    ranks exit at once with status 0 and print nothing."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2", "--steps", "3",
                                      "--warmup", "1"])
    assert bench.main() == 0
    assert capsys.readouterr().out == ""
