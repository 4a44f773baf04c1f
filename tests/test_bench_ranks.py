"""The multi-rank path of bench.py on CPU: two gloo ranks, each timing its
own replica, agree on the slowest rank's timings, and the whole-job value
counts every rank's pairs (replicas only: the method has no exchange step)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r is slower in the first timing, faster in the second
        got = bench.max_over_ranks([1.0 + rank, 5.0 - rank, 0.5], world, "cpu")
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_timing():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(q.get(timeout=10) for _ in range(world))
    assert res[0] == res[1] == [2.0, 5.0, 0.5]


def test_single_rank_and_whole_job_value():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.0], 1, "cpu") == [3.0, 4.0]
    # 2 replicas of 1e6 pairs, 10 steps in 2 s: 1e7 pairs/s
    assert bench.replica_throughput(2, 1_000_000, 10, 2.0) == 1e7
