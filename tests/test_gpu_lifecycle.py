"""Contexts come and go without leaking: device memory, files and host threads.

A serving process opens a context per job or per tenant; whatever one context took
(cache frames, the metadata arena, pinned staging, the request ring, mapped files,
the host I/O threads) must be given back when it shuts down, whatever transfer it
used and whether or not it scanned.  Every scan is checked against the oracle's plain
definition.
"""
import os
import numpy as np
import pytest

import inputs
from oracle import plain

pytestmark = pytest.mark.gpu

KiB, MiB, GiB = 1 << 10, 1 << 20, 1 << 30


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


def _fds():
    return len(os.listdir("/proc/self/fd"))


def _tasks():  # every thread of the process, the library's native I/O threads included
    return len(os.listdir("/proc/self/task"))


def test_contexts_give_everything_back(torch_cuda, gfs, datadir):
    torch = torch_cuda
    path = os.path.join(datadir, "life_%d.bin" % (48 * MiB + 11))
    inputs.ensure_file(path, 51, 48 * MiB + 11)
    want = plain.scan_plain(path, MiB)
    out = tuple(torch.empty(len(want[0]), dtype=torch.int64, device="cuda") for _ in range(3))
    torch.cuda.synchronize()

    def one(xfer, scan):
        with gfs.Context(cache_bytes=GiB, page_size=256 * KiB, xfer=xfer, max_rpc_pages=16) as ctx:
            fid = ctx.open(path)
            if scan:
                ctx.scan(fid, MiB, blocks=64, out=out)
                torch.cuda.synchronize()
                assert out[0].cpu().tolist() == want[0]
                assert np.array_equal(gfs.u64_view(out[1]), np.array(want[1], dtype=np.uint64))
                assert np.array_equal(gfs.u64_view(out[2]), np.array(want[2], dtype=np.uint64))

    one(2, True)  # first use loads the library and the CUDA context
    torch.cuda.synchronize()
    free0, tasks0, fds0 = torch.cuda.mem_get_info()[0], _tasks(), _fds()
    for rep in range(6):
        for xfer in (0, 1, 2):
            one(xfer, scan=rep % 2 == 0)
    torch.cuda.synchronize()
    free1, tasks1, fds1 = torch.cuda.mem_get_info()[0], _tasks(), _fds()
    # each context held > 1 GiB of device memory: eighteen of them leaking would show
    assert free1 >= free0 - 64 * MiB, (free0, free1)
    assert tasks1 <= tasks0 + 2, (tasks0, tasks1)  # 16 I/O threads per context would show
    assert fds1 <= fds0 + 2, (fds0, fds1)


@pytest.mark.parametrize("xfers", [(2, 2), (2, 1), (1, 0)])
def test_two_contexts_scan_at_once(torch_cuda, gfs, datadir, xfers):
    """Two tenants: two contexts (each its own cache, ring and I/O threads) scan their own
    files on two streams at the same time; both results equal the oracle's."""
    torch = torch_cuda
    paths = []
    for k, size in enumerate((40 * MiB + 3, 56 * MiB + 4097)):
        p = os.path.join(datadir, "two_%d_%d.bin" % (k, size))
        inputs.ensure_file(p, 60 + k, size)
        paths.append(p)
    wants = [plain.scan_plain(p, MiB) for p in paths]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    ctxs = [gfs.Context(cache_bytes=16 * MiB, page_size=256 * KiB, xfer=x, max_rpc_pages=16) for x in xfers]
    try:
        fids = [c.open(p) for c, p in zip(ctxs, paths)]
        outs = [c.scan(f, MiB, blocks=48, stream=s) for c, f, s in zip(ctxs, fids, streams)]
        torch.cuda.synchronize()
        for out, want, c in zip(outs, wants, ctxs):
            assert out[0].cpu().numpy()[:len(want[0])].tolist() == want[0]
            assert np.array_equal(gfs.u64_view(out[1])[:len(want[1])], np.array(want[1], dtype=np.uint64))
            assert np.array_equal(gfs.u64_view(out[2])[:len(want[2])], np.array(want[2], dtype=np.uint64))
            st = c.stats()
            assert st["timeouts"] == 0 and st["eio"] == 0 and st["enomem"] == 0
    finally:
        for c in ctxs:
            c.shutdown()
