"""Application-shaped streams through the read path against the oracle:
float32 row dot products within the gamma_n bound on identical delivered bytes
(stripe checksums exact), and an exact histogram of Zipf int32 values."""
import os

import numpy as np
import pytest

import inputs
from oracle import apps, plain

pytestmark = pytest.mark.gpu

KiB, MiB = 1 << 10, 1 << 20


def _stripe_checksums(path, rows, cols, stripe_rows):
    fd = os.open(path, os.O_RDONLY)
    size = os.path.getsize(path)
    sums, hashes = [], []
    try:
        for r0 in range(0, rows, stripe_rows):
            off = r0 * cols * 4
            n, data = plain.gread_plain(fd, size, off, min(stripe_rows, rows - r0) * cols * 4)
            sums.append(plain.byte_sum(data))
            hashes.append(plain.pos_hash(data, off))
    finally:
        os.close(fd)
    return sums, hashes


@pytest.mark.parametrize("xfer", [0, 1, 2])
@pytest.mark.parametrize("rows,cols,stripe_rows,read_len", [
    (512, 32768, 128, MiB),           # the 32768-column shape, 1 MiB = 8 rows per gread
    (300, 2048, 128, 32 * KiB),       # ragged last stripe
])
def test_rowdot_within_bound(datadir, xfer, rows, cols, stripe_rows, read_len):
    import torch
    from paper_2109_05366_gb300 import gfs
    torch.cuda.set_device(0)
    path = os.path.join(datadir, "mat_%d_%d.f32" % (rows, cols))
    inputs.ensure_typed(path, "f32", 7, rows * cols)
    vec = inputs.f32_values(8, cols) if cols <= 4096 else None
    if vec is None:
        vp = os.path.join(datadir, "vec_%d.f32" % cols)
        inputs.ensure_typed(vp, "f32", 8, cols)
        vec = np.fromfile(vp, dtype=np.float32)
    with gfs.Context(cache_bytes=32 * MiB, page_size=256 * KiB, xfer=xfer, max_rpc_pages=16) as ctx:
        fid = ctx.open(path)
        d_vec = torch.from_numpy(vec).cuda()
        out, ssum, shash, status = ctx.rowdot(fid, rows, cols, d_vec, stripe_rows, read_len, blocks=64)
        torch.cuda.synchronize()
        assert status.item() == 0
        got = out.cpu().numpy().astype(np.float64)
    ref, ab = apps.rowdot(path, rows, cols, vec)
    bound = apps.gamma(cols) * ab
    assert np.all(np.abs(got - ref) <= bound), float(np.max(np.abs(got - ref) / np.maximum(bound, 1e-30)))
    s, h = _stripe_checksums(path, rows, cols, stripe_rows)
    assert np.array_equal(gfs.u64_view(ssum), np.array(s, dtype=np.uint64))
    assert np.array_equal(gfs.u64_view(shash), np.array(h, dtype=np.uint64))


@pytest.mark.parametrize("xfer", [0, 1, 2])
@pytest.mark.parametrize("nbins", [1 << 20, 3000])
def test_histogram_exact(datadir, xfer, nbins):
    import torch
    from paper_2109_05366_gb300 import gfs
    torch.cuda.set_device(0)
    n = 32 * MiB + 1000
    path = os.path.join(datadir, "zipf_%d.i32" % n)
    inputs.ensure_typed(path, "zipf", 9, n, nbins=1 << 20, s=1.1)
    with gfs.Context(cache_bytes=32 * MiB, page_size=512 * KiB, xfer=xfer, max_rpc_pages=16) as ctx:
        fid = ctx.open(path)
        hist, sums, status = ctx.histogram(fid, nbins=nbins, read_len=MiB, blocks=96)
        torch.cuda.synchronize()
        assert status.item() == 0
        got = hist.cpu().numpy().view(np.uint32).astype(np.uint64)
        s = gfs.u64_view(sums)
    want, outside = apps.histogram(path, nbins)
    assert np.array_equal(got, want)
    assert int(s[1]) == outside
    with open(path, "rb") as f:
        assert int(s[0]) == plain.byte_sum(f.read())
