"""bench.py's host logic for N > 1 ranks (one process per GPU, independent
replicas), checked on two gloo ranks on the CPU: per-rank times reduce to the
slowest rank's, the whole-job rate counts every rank's units over that time,
and the reference arm prints from rank 0 only."""
import argparse
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, queue):
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            init_method="tcp://127.0.0.1:%d" % port)
    try:
        # rank r reports times (1 + r, 10 - r): the slowest rank's are (2, 10)
        vals = bench.max_over_ranks([1.0 + rank, 10.0 - rank], world, torch.device("cpu"))
        queue.put((rank, vals))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    queue = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, queue)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(queue.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert got[0] == got[1] == [2.0, 10.0]


def test_one_rank_passes_times_through():
    assert bench.max_over_ranks([1.5, 2.5], 1, None) == [1.5, 2.5]


def test_whole_job_rate_counts_every_rank():
    # 2 ranks x 3 units each in 0.5 s (the slowest rank's time) = 12 units/s
    assert bench.whole_job_rate(3.0, 2, 0.5) == 12.0


def test_reference_arm_prints_on_rank_zero_only(capsys):
    args = argparse.Namespace(steps=1, warmup=0, precision=0)
    bench.run_reference(args, 2, 1)        # rank 1 of 2: no work, no line
    assert capsys.readouterr().out == ""
