"""Parity at the full sizes of the benchmark workloads.

Every delivered byte is checked through the per-stride checksums (count, byte
sum, position hash) against the oracle's plain definition computed on all host
cores (oracle/pool.py), stride for stride, bit-exact:

* the 8 GiB file through a 1 GiB cache (512 KiB pages, 296 threadblocks, 1 MiB
  strides; the configuration the benchmark times), with every transfer, with
  and without the fused consumer, readahead and on-demand;
* the 16 GiB file through a 2 GiB cache at the three tuned points of the
  autotuner (64 KiB, 1 MiB and 16 MiB strides);
* the 32768 x 32768 float32 matrix (4 GiB): every row's dot product within
  gamma_n * sum |a_i b_i| of the float64 value, stripe checksums exact;
* the 8 GiB Zipf int32 file: the 2^20-bin histogram exactly equal to the
  oracle's counts.
"""
import json
import os

import numpy as np
import pytest

import inputs
from oracle import apps, pool

pytestmark = pytest.mark.gpu

KiB, MiB, GiB = 1 << 10, 1 << 20, 1 << 30
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


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


def _check(gfs, want, out, what):
    c, s, h = want
    got_c = out[0].cpu().numpy()[:len(c)]
    bad = np.nonzero(got_c != np.array(c, dtype=np.int64))[0]
    assert bad.size == 0, "%s: %d strides with wrong counts, first %d" % (what, bad.size, bad[0])
    for name, got, exp in (("sum", out[1], s), ("hash", out[2], h)):
        g = gfs.u64_view(got)[:len(exp)]
        bad = np.nonzero(g != np.array(exp, dtype=np.uint64))[0]
        assert bad.size == 0, "%s: %d strides with a wrong %s, first %d" % (what, bad.size, name, bad[0])


# ------------------------------------------------ 8 GiB file, 1 GiB cache
CFG2 = dict(size=8 * GiB, seed=2, page=512 * KiB, cache=GiB, blocks=296, stride=MiB)


@pytest.fixture(scope="module")
def cfg2_file(datadir):
    path = os.path.join(datadir, "full_cfg2_%d.bin" % CFG2["size"])
    inputs.ensure_file(path, CFG2["seed"], CFG2["size"])
    return path


@pytest.fixture(scope="module")
def cfg2_oracle(cfg2_file):
    return pool.scan_plain_parallel(cfg2_file, CFG2["stride"])


@pytest.mark.parametrize("xfer,mode", [(2, 0), (2, 1), (1, 0), (0, 0)])
def test_cfg2_full_size_exact(torch_cuda, gfs, cfg2_file, cfg2_oracle, xfer, mode):
    torch = torch_cuda
    npages = CFG2["size"] // CFG2["page"]
    ns = CFG2["size"] // CFG2["stride"]
    with gfs.Context(cache_bytes=CFG2["cache"], page_size=CFG2["page"], mode=mode, xfer=xfer, max_rpc_pages=16,
                     rpc_slots=512, debug_counts=1) as ctx:
        fid = ctx.open(cfg2_file)
        out = tuple(torch.full((ns,), -1, dtype=torch.int64, device="cuda") for _ in range(3))
        for fused in ((False, True) if mode == 0 and xfer == 2 else (False,)):
            ctx.reset_cache()
            ctx.scan(fid, CFG2["stride"], blocks=CFG2["blocks"], threads=256, fused=fused, out=out)
            torch.cuda.synchronize()
            _check(gfs, cfg2_oracle, out, "xfer %d mode %d fused %d" % (xfer, mode, fused))
            st = ctx.stats()
            counts = ctx.fetch_counts(npages)
            assert st["timeouts"] == 0 and st["eio"] == 0 and st["enomem"] == 0
            # streaming with the demand reserve: every page fetched exactly once
            assert (counts == 1).all() and st["pages_fetched"] == npages
            if mode == 1:
                assert st["rpcs"] == npages


# ------------------------------------------------ 16 GiB file, 2 GiB cache, the tuned points
@pytest.fixture(scope="module")
def cfg3_file(datadir):
    path = os.path.join(datadir, "full_cfg3_%d.bin" % (16 * GiB))
    inputs.ensure_file(path, 3, 16 * GiB)
    return path


def _tuned():
    with open(os.path.join(ROOT, "paper_2109_05366_gb300", "tuned", "gb300_cfg3.json")) as f:
        return {int(k): v for k, v in json.load(f)["best_by_stride"].items()}


@pytest.mark.parametrize("stride", [64 * KiB, MiB, 16 * MiB])
def test_cfg3_tuned_points_exact(torch_cuda, gfs, cfg3_file, stride):
    torch = torch_cuda
    pt = _tuned()[stride]
    want = pool.scan_plain_parallel(cfg3_file, stride)
    ns = len(want[0])
    page = pt["page_size"]
    with gfs.Context(cache_bytes=2 * GiB, page_size=page, ra_cap_pages=pt["ra_cap_pages"], rpc_slots=pt["rpc_slots"],
                     max_rpc_pages=min(256, max(16, pt["ra_cap_pages"] + stride // page + 1)),
                     max_streams=4096) as ctx:
        fid = ctx.open(cfg3_file)
        out = tuple(torch.full((ns,), -1, dtype=torch.int64, device="cuda") for _ in range(3))
        ctx.scan(fid, stride, blocks=pt["blocks"], threads=256, out=out)
        torch.cuda.synchronize()
        _check(gfs, want, out, "stride %d" % stride)
        st = ctx.stats()
        assert st["timeouts"] == 0 and st["eio"] == 0 and st["enomem"] == 0


# ------------------------------------------------ application streams at full size
def test_cfg4a_rowdot_full_size(torch_cuda, gfs, datadir):
    torch = torch_cuda
    rows = cols = 32768
    mpath = os.path.join(datadir, "full_mat_%d.f32" % rows)
    vpath = os.path.join(datadir, "full_vec_%d.f32" % cols)
    inputs.ensure_typed(mpath, "f32", 7, rows * cols)
    inputs.ensure_typed(vpath, "f32", 8, cols)
    vec = np.fromfile(vpath, dtype=np.float32)
    with gfs.Context(cache_bytes=GiB, page_size=512 * KiB, max_rpc_pages=16, rpc_slots=512) as ctx:
        fid = ctx.open(mpath)
        out, ssum, shash, status = ctx.rowdot(fid, rows, cols, torch.from_numpy(vec).cuda(), 128, MiB, blocks=296)
        torch.cuda.synchronize()
        assert status.item() == 0
        got = out.cpu().numpy().astype(np.float64)
        ss, sh = gfs.u64_view(ssum), gfs.u64_view(shash)
    ref, ab = apps.rowdot(mpath, rows, cols, vec)
    bound = apps.gamma(cols) * ab
    over = np.nonzero(np.abs(got - ref) > bound)[0]
    assert over.size == 0, "%d rows outside the bound, first %d" % (over.size, over[0])
    stripe = 128 * cols * 4
    c, s, h = pool.scan_plain_parallel(mpath, stripe)
    assert np.array_equal(ss[:len(s)], np.array(s, dtype=np.uint64))
    assert np.array_equal(sh[:len(h)], np.array(h, dtype=np.uint64))


def test_cfg4b_histogram_full_size(torch_cuda, gfs, datadir):
    torch = torch_cuda
    n = 1 << 31
    zpath = os.path.join(datadir, "full_zipf.i32")
    inputs.ensure_typed(zpath, "zipf", 9, n, nbins=1 << 20, s=1.1)
    with gfs.Context(cache_bytes=GiB, page_size=512 * KiB, max_rpc_pages=16, rpc_slots=512) as ctx:
        fid = ctx.open(zpath)
        hist, sums, status = ctx.histogram(fid, 1 << 20, MiB, blocks=296)
        torch.cuda.synchronize()
        assert status.item() == 0
        got = hist.cpu().numpy().view(np.uint32).astype(np.uint64)
        s = gfs.u64_view(sums)
    want, outside = apps.histogram(zpath, 1 << 20)
    assert int(want.sum()) + outside == n
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, "%d bins differ, first %d" % (bad.size, bad[0])
    assert int(s[1]) == outside
    assert int(s[0]) == pool.range_checksums(zpath, 0, 4 * n)[1]
