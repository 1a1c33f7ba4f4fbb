"""The benchmark's multi-rank host logic on CPU: two gloo ranks, a barrier
and the max-over-ranks time reduction; the whole-job value of weak scaling."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    barrier, max_over_ranks = bench.rank_helpers(dist)
    barrier()
    t = max_over_ranks(1.5 + rank)  # rank r "took" 1.5 + r seconds
    q.put((rank, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    mp = pytest.importorskip("torch.multiprocessing")
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == {0: 2.5, 1: 2.5}


def test_whole_job_value_is_weak_scaling_aggregate():
    import bench
    one = bench.whole_job_value(1, 8e8, 10, 2.0)
    assert one == pytest.approx(4.0)
    assert bench.whole_job_value(4, 8e8, 10, 2.0) == pytest.approx(4 * one)


def test_single_process_helpers_are_noops():
    import bench
    barrier, mx = bench.rank_helpers(None)
    barrier()
    assert mx(3.25) == 3.25
