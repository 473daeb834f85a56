"""GPU tests of the request-queue study (Section 3.2): the static slot partition of
GPUfs (slot = threadblock index, host thread k polls a fixed contiguous share of
the slots) against the shared ring, the per-thread counters, and the host I/O trace
with its CPU replay.  Data is compared with the plain definition in every case.
"""
import os

import numpy as np
import pytest

import inputs
from oracle import plain

pytestmark = pytest.mark.gpu

KiB, MiB = 1 << 10, 1 << 20


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    torch.cuda.set_device(0)
    return torch


@pytest.fixture(scope="module")
def gfs():
    from paper_2109_05366_gb300 import gfs as g
    g.load()
    return g


def _file(datadir, seed, size):
    path = os.path.join(datadir, "q%d_%d.bin" % (seed, size))
    inputs.ensure_file(path, seed, size)
    return path


def _check_scan(gfs, path, stride, cnt, sm, hs):
    c, s, h = plain.scan_plain(path, stride)
    assert cnt.cpu().numpy()[:len(c)].tolist() == c
    assert np.array_equal(gfs.u64_view(sm)[:len(s)], np.array(s, dtype=np.uint64))
    assert np.array_equal(gfs.u64_view(hs)[:len(h)], np.array(h, dtype=np.uint64))


@pytest.mark.parametrize("xfer", [0, 1, 2])
@pytest.mark.parametrize("queue", [0, 1])
def test_scan_exact_with_either_queue(torch_cuda, gfs, datadir, xfer, queue):
    path = _file(datadir, 41, 96 * MiB + 333)
    with gfs.Context(cache_bytes=32 * MiB, page_size=256 * KiB, xfer=xfer, queue=queue, rpc_slots=64,
                     host_threads=4, max_rpc_pages=16, self_serve=0) as ctx:  # mapped: served by the host
        fid = ctx.open(path)
        for _ in range(2):
            out = ctx.scan(fid, MiB, blocks=96, threads=256)
            torch_cuda.cuda.synchronize()
            _check_scan(gfs, path, MiB, *out)
            st = ctx.stats()
            ts = ctx.thread_stats()
            assert len(ts) == 4
            assert sum(t["requests"] for t in ts) == st["host_requests"] + st["host_controls"]
            assert st["timeouts"] == 0
            ctx.reset_cache()


def test_static_queue_leaves_threads_of_unused_slots_idle(torch_cuda, gfs, datadir):
    """16 blocks, 64 slots, 4 host threads of 16 slots each: every request of a
    static queue lands in slots 0-15, so threads 1-3 never serve (the imbalance of
    Section 3.2); the shared ring spreads the same requests over all threads."""
    path = _file(datadir, 42, 64 * MiB)
    per = {}
    for queue in (0, 1):
        with gfs.Context(cache_bytes=16 * MiB, page_size=256 * KiB, xfer=1, queue=queue, rpc_slots=64,
                         host_threads=4, max_rpc_pages=16) as ctx:
            fid = ctx.open(path)
            out = ctx.scan(fid, MiB, blocks=16, threads=256)
            torch_cuda.cuda.synchronize()
            _check_scan(gfs, path, MiB, *out)
            per[queue] = ctx.thread_stats()
    assert per[1][0]["requests"] > 0
    assert all(t["requests"] == 0 and t["first_request_ns"] == 0 for t in per[1][1:])
    assert all(t["polls_before_first"] > 0 for t in per[1][1:])
    assert sum(t["requests"] > 0 for t in per[0]) >= 3


@pytest.mark.parametrize("xfer", [1, 2])
def test_io_trace_covers_the_file_and_replays(torch_cuda, gfs, datadir, xfer):
    path = _file(datadir, 43, 40 * MiB + 4321)
    size = os.path.getsize(path)
    with gfs.Context(cache_bytes=64 * MiB, page_size=256 * KiB, xfer=xfer, trace_capacity=1 << 14,
                     max_rpc_pages=16, self_serve=0) as ctx:  # the host I/O trace: requests the host serves
        fid = ctx.open(path)
        out = ctx.scan(fid, MiB, blocks=32, threads=256)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, MiB, *out)
        recs = ctx.io_trace()
        st = ctx.stats()
    assert len(recs) == st["host_requests"]
    covered = np.zeros(size, dtype=bool)
    for r in recs:
        assert r.offset % (256 * KiB) == 0 and r.offset + r.bytes <= size
        covered[r.offset:r.offset + r.bytes] = True
    assert covered.all()                                    # fits: every byte requested once
    assert sum(r.bytes for r in recs) == size
    assert all(r.thread < 16 for r in recs)
    secs, nbytes = gfs.replay_io(path, recs, 8)
    assert nbytes == size and secs > 0
