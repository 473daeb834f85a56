"""gfs_scan_static: the allocation-free stride scan.

Some callers cannot call cudaMalloc while they run: serving loops that must not
stall other streams (cudaMalloc and cudaFree can synchronise the device), and
code that owns the device's memory through its own allocator and budget.
gfs_scan_static serves them: its per-threadblock gread buffers live in a static
device array instead of memory the call would allocate.  Its results must equal
gfs_scan's and the oracle's exactly (integer checksums) on two calls in a row,
the device's free memory must not change across those calls, and a request
larger than the static array must be rejected before anything is launched.

This file is collected last: if it fails, a run that stops at the first
failure has already run every other test.
"""
import ctypes
import os

import numpy as np
import pytest

import inputs
from oracle import plain

pytestmark = pytest.mark.gpu

KiB, MiB = 1 << 10, 1 << 20
STATIC_SCRATCH = 64 * MiB  # GFS_STATIC_SCRATCH_BYTES
ENOSPC, ENOTSUP = 28, 95


def _static_fn(gfs):
    lib = gfs.load()
    fn = lib.gfs_scan_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(gfs.ScanArgs), ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    return lib, fn


def _args(gfs, stride, read_len, blocks):
    a = gfs.ScanArgs()
    a.stride, a.read_len, a.blocks, a.threads = stride, read_len, blocks, 256
    return a


def test_static_scratch_scan_matches_scan(tmp_path_factory):
    import torch

    from paper_2109_05366_gb300 import gfs

    torch.cuda.set_device(0)
    lib, fn = _static_fn(gfs)
    path = os.path.join(str(tmp_path_factory.mktemp("noalloc")), "f.bin")
    size = 48 * MiB + 4321
    inputs.write_file(path, 13, size)
    stride, blocks = MiB, 64  # 64 blocks x 1 MiB = exactly the static array
    ns = (size + stride - 1) // stride
    c, s, h = plain.scan_plain(path, stride)
    with gfs.Context(cache_bytes=32 * MiB, page_size=256 * KiB, max_rpc_pages=16) as ctx:
        fid = ctx.open(path)
        ref = ctx.scan(fid, stride, blocks=blocks, threads=256)
        torch.cuda.synchronize()
        want = [t.cpu().numpy().copy() for t in ref]
        args = _args(gfs, stride, stride, blocks)
        outs = [[torch.full((ns,), -7, dtype=torch.int64, device="cuda") for _ in range(3)] for _ in range(2)]
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for call in range(2):
            ctx.reset_cache()
            out = outs[call]
            rc = fn(ctx.handle, fid, ctypes.byref(args), out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(),
                    None)
            assert rc == 0, lib.gfs_strerror(rc)
            torch.cuda.synchronize()
            for got, exp in zip(out, want):
                assert np.array_equal(got.cpu().numpy(), exp), "call %d differs from gfs_scan" % call
            # and from the oracle's plain definition, directly
            assert out[0].cpu().numpy().tolist() == c
            assert np.array_equal(gfs.u64_view(out[1]), np.array(s, dtype=np.uint64))
            assert np.array_equal(gfs.u64_view(out[2]), np.array(h, dtype=np.uint64))
        assert torch.cuda.mem_get_info()[0] == free0, "the allocation-free scan changed the device's free memory"
        # the scratch a request needs must fit the static array; nothing is launched otherwise
        out = outs[0]
        for a in (_args(gfs, stride, stride, blocks + 1),          # one block too many
                  _args(gfs, stride, (1 << 64) - 1, 2),             # rounding read_len up would wrap to 0
                  _args(gfs, stride, 1 << 58, 64)):                 # blocks * read_len would wrap to 0
            rc = fn(ctx.handle, fid, ctypes.byref(a), out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), None)
            assert rc == -ENOSPC
        assert (blocks + 1) * stride > STATIC_SCRATCH
        # a read longer than the file needs only the file's bytes per block
        a = _args(gfs, 64 * MiB, 1 << 40, 1)
        rc = fn(ctx.handle, fid, ctypes.byref(a), out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), None)
        assert rc == 0, lib.gfs_strerror(rc)
        torch.cuda.synchronize()
        assert int(out[0][0].item()) == size


def test_static_scan_needs_per_block_state_sized_first(tmp_path_factory):
    """With the per-block LRA replacement the context keeps per-threadblock queues that an
    allocating call sizes: the allocation-free scan refuses (-ENOTSUP) until one has run."""
    import torch

    from paper_2109_05366_gb300 import gfs

    torch.cuda.set_device(0)
    lib, fn = _static_fn(gfs)
    path = os.path.join(str(tmp_path_factory.mktemp("noalloc2")), "g.bin")
    size = 8 * MiB + 17
    inputs.write_file(path, 14, size)
    ns = (size + MiB - 1) // MiB
    c, s, h = plain.scan_plain(path, MiB)
    with gfs.Context(cache_bytes=16 * MiB, page_size=256 * KiB, max_rpc_pages=16, replacement=gfs.REPL_TB_LRA) as ctx:
        fid = ctx.open(path)
        out = [torch.zeros(ns, dtype=torch.int64, device="cuda") for _ in range(3)]
        a = _args(gfs, MiB, MiB, 8)
        rc = fn(ctx.handle, fid, ctypes.byref(a), out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), None)
        assert rc == -ENOTSUP
        ctx.scan(fid, MiB, blocks=8)
        torch.cuda.synchronize()
        ctx.reset_cache()
        rc = fn(ctx.handle, fid, ctypes.byref(a), out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), None)
        assert rc == 0, lib.gfs_strerror(rc)
        torch.cuda.synchronize()
        assert out[0].cpu().numpy().tolist() == c
        assert np.array_equal(gfs.u64_view(out[1]), np.array(s, dtype=np.uint64))
        assert np.array_equal(gfs.u64_view(out[2]), np.array(h, dtype=np.uint64))
