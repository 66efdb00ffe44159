"""Replica timing of bench.py on two gloo ranks (CPU).

The operator does not shard: with N GPUs the bench runs N independent replicas, and
the only exchange is the timing.  Every rank must see the slowest rank's step time,
and the whole-job throughput counts the dofs of all ranks at that time.
"""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        ms = bench.reduce_max(10.0 + 5.0 * rank, world, "cpu")
        q.put((rank, ms, bench.whole_job_gdofs(25350, world, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    assert all(ms == 15.0 for _, ms, _ in res)
    assert all(v == pytest.approx(2 * 25350 / 15e-3 / 1e9) for _, _, v in res)


def test_one_rank_is_the_identity():
    import bench

    assert bench.reduce_max(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_gdofs(1000, 1, 1.0) == pytest.approx(1e-3)
