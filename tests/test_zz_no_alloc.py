"""gfs_scan_static: the allocation-free stride scan.

Some callers cannot call cudaMalloc while they run (serving loops that must not
stall other streams, code that owns the device memory through its own
allocator).  gfs_scan_static serves them: its per-threadblock gread buffers live
in a static device array instead of memory the call would allocate.  Its
results must equal gfs_scan's exactly (integer checksums) on two calls in a
row, and a request larger than the static array must be rejected.
"""
import ctypes
import os

import numpy as np
import pytest

import inputs

pytestmark = pytest.mark.gpu

KiB, MiB = 1 << 10, 1 << 20
STATIC_SCRATCH = 64 * MiB  # GFS_STATIC_SCRATCH_BYTES
ENOSPC = 28


def test_static_scratch_scan_matches_scan(tmp_path_factory):
    import torch

    from paper_2109_05366_gb300 import gfs

    torch.cuda.set_device(0)
    lib = gfs.load()
    fn = lib.gfs_scan_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(gfs.ScanArgs), ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]

    path = os.path.join(str(tmp_path_factory.mktemp("noalloc")), "f.bin")
    size = 48 * MiB + 4321
    inputs.write_file(path, 13, size)
    stride, blocks = MiB, 64  # 64 blocks x 1 MiB = exactly the static array
    ns = (size + stride - 1) // stride
    with gfs.Context(cache_bytes=32 * MiB, page_size=256 * KiB, max_rpc_pages=16) as ctx:
        fid = ctx.open(path)
        ref = ctx.scan(fid, stride, blocks=blocks, threads=256)
        torch.cuda.synchronize()
        want = [t.cpu().numpy().copy() for t in ref]
        args = gfs.ScanArgs()
        args.stride, args.read_len, args.blocks, args.threads = stride, stride, blocks, 256
        for call in range(2):
            ctx.reset_cache()
            out = [torch.full((ns,), -7, dtype=torch.int64, device="cuda") for _ in range(3)]
            rc = fn(ctx.handle, fid, ctypes.byref(args), out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(),
                    None)
            assert rc == 0, lib.gfs_strerror(rc)
            torch.cuda.synchronize()
            for got, exp in zip(out, want):
                assert np.array_equal(got.cpu().numpy(), exp), "call %d differs from gfs_scan" % call
        # the scratch a request needs must fit the static array
        big = gfs.ScanArgs()
        big.stride, big.read_len, big.blocks, big.threads = stride, stride, blocks + 1, 256
        rc = fn(ctx.handle, fid, ctypes.byref(big), out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), None)
        assert rc == -ENOSPC
        assert (blocks + 1) * stride > STATIC_SCRATCH
