"""Replica scaling logic of bench.py on CPU: two gloo ranks, each its own file,
the job timed by its slowest rank (no collective on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        slowest = bench.max_over_ranks(times[rank], dist)
        q.put((rank, slowest, bench.rank_seed(2, rank)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_and_own_files():
    import bench
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    times = [1.5, 2.5]
    procs = [ctx.Process(target=_rank, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.5, 2.5]              # every rank sees the max
    assert out[0][2] != out[1][2]                          # distinct input files
    rate = bench.job_rate(8 << 30, 5, 2, 2.5)
    assert rate == pytest.approx(2 * 5 * (8 << 30) / 2.5 / 1e9)


def test_single_rank_passes_through():
    import bench
    assert bench.max_over_ranks(3.0, None) == 3.0
    assert bench.job_rate(10 ** 9, 1, 1, 1.0) == pytest.approx(1.0)
