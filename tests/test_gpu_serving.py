"""Serving (continuous batching) against the oracle: every request's checksum is
the plain definition's, and identical alone and in the mix."""
import os

import numpy as np
import pytest

import inputs
from oracle import plain

pytestmark = pytest.mark.gpu

KiB, MiB = 1 << 10, 1 << 20


def _files(datadir, n):
    from paper_2109_05366_gb300 import serving
    sizes = serving.log_uniform_sizes(n, 20, 25, seed=55)  # 1 MiB .. 32 MiB
    paths = []
    for i, sz in enumerate(sizes):
        p = os.path.join(datadir, "serve_%d_%d.bin" % (i, sz))
        inputs.ensure_file(p, 1000 + i, sz)
        paths.append(p)
    return paths


def _oracle(path, off, ln):
    fd = os.open(path, os.O_RDONLY)
    try:
        n, data = plain.gread_plain(fd, os.path.getsize(path), off, ln)
    finally:
        os.close(fd)
    return n, plain.byte_sum(data), plain.pos_hash(data, off)


@pytest.mark.parametrize("xfer,mode", [(2, 0), (1, 0), (0, 0), (2, 1)])
def test_serving_mix_equals_alone_and_oracle(datadir, xfer, mode):
    import torch
    from paper_2109_05366_gb300 import gfs, serving
    torch.cuda.set_device(0)
    paths = _files(datadir, 10)
    with gfs.Context(cache_bytes=24 * MiB, page_size=512 * KiB, xfer=xfer, mode=mode, max_rpc_pages=16,
                     max_streams=1024) as ctx:
        fids = [ctx.open(p) for p in paths]
        reqs = []
        for i, (fid, p) in enumerate(zip(fids, paths)):
            size = os.path.getsize(p)
            off = (i * 12345) % max(size // 3, 1)
            reqs.append((fid, off, size - off + (7 if i % 3 == 0 else 0)))   # some run past EOF
        reqs.append((fids[0], os.path.getsize(paths[0]) + 5, 100))          # entirely past EOF
        reqs.append((fids[1], 0, 0))                                         # empty
        stream = torch.cuda.Stream()
        ctx.serve_start(ctas=24, threads=256, unit_bytes=MiB, max_requests=8, queue_slots=64,
                        units_in_flight=2, frame_budget=16, stream=stream)
        try:
            mix, t0 = serving.run(ctx, reqs, timeout_s=60)
            alone = [serving.run(ctx, [r], timeout_s=60)[0][0] for r in reqs]
        finally:
            ctx.serve_stop()
        for i, (fid, off, ln) in enumerate(reqs):
            n, s, h = _oracle(paths[fids.index(fid)], off, ln)
            for res in (mix[i], alone[i]):
                assert res["status"] == 0
                assert res["bytes"] == n and res["sum"] == s and res["hash"] == h
        st = ctx.stats()
        assert st["timeouts"] == 0 and st["eio"] == 0


def test_serving_poisson_arrivals(datadir):
    import torch
    from paper_2109_05366_gb300 import gfs, serving
    torch.cuda.set_device(0)
    paths = _files(datadir, 10)
    with gfs.Context(cache_bytes=64 * MiB, page_size=512 * KiB, xfer=2, max_rpc_pages=16) as ctx:
        fids = [ctx.open(p) for p in paths]
        reqs = [(fid, 0, os.path.getsize(p)) for fid, p in zip(fids, paths)] * 2
        arrivals = serving.poisson_arrivals(len(reqs), 200.0, seed=5)
        ctx.serve_start(ctas=64, threads=256, unit_bytes=MiB, max_requests=16, queue_slots=64)
        try:
            res, t0 = serving.run(ctx, reqs, arrivals, timeout_s=60)
        finally:
            ctx.serve_stop()
        summ = serving.summarize(res, t0)
        assert summ["errors"] == 0 and summ["requests"] == len(reqs)
        for i, (fid, off, ln) in enumerate(reqs):
            n, s, h = _oracle(paths[fids.index(fid)], off, ln)
            assert (res[i]["bytes"], res[i]["sum"], res[i]["hash"]) == (n, s, h)
