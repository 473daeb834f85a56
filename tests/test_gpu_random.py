"""GPU tests of small random reads and of a mixed workload (Section 3.1: the collage
application reads 4 KB tiles at data-dependent places while it reads a base picture
sequentially; Section 4.4: the RANDOM hint turns readahead off for a file).

Every delivered byte is compared with the file (plain definition of a read).  With the
RANDOM hint the policy must issue one page per request and no readahead; in a cache the
file fits, it then fetches exactly the distinct pages the reads touch.
"""
import os
import random

import numpy as np
import pytest

import inputs

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
    path = os.path.join(datadir, "r%d_%d.bin" % (seed, size))
    inputs.ensure_file(path, seed, size)
    return path


def _tiles(size, n, seed, page):
    """n tile reads: most 4 KiB at 4 KiB-aligned offsets, some unaligned or crossing a page."""
    rng = random.Random(seed)
    offs, lens = [], []
    for i in range(n):
        if i % 8 == 7:
            offs.append(rng.randrange(size))
            lens.append(rng.choice([1, 3000, 4096, page + 5]))
        else:
            offs.append(rng.randrange(size // (4 * KiB)) * 4 * KiB)
            lens.append(4 * KiB)
    return offs, lens


def _read_many(torch, gfs, ctx, fid, offs, lens, blocks=64, stream=None, threads=256):
    dsts, pos = [], 0
    for ln in lens:
        dsts.append(pos)
        pos += (ln + 255) // 256 * 256
    d_off = torch.tensor(offs, dtype=torch.int64, device="cuda")
    d_len = torch.tensor(lens, dtype=torch.int64, device="cuda")
    d_dst = torch.tensor(dsts, dtype=torch.int64, device="cuda")
    d_buf = torch.zeros(max(pos, 1), dtype=torch.uint8, device="cuda")
    d_ret = torch.full((len(offs),), -999, dtype=torch.int64, device="cuda")
    if stream is not None:  # the inputs were written on the current stream
        stream.wait_stream(torch.cuda.current_stream())
    ctx.read_many(fid, d_off, d_len, d_dst, d_buf, d_ret, blocks=blocks, threads=threads, stream=stream)
    return dsts, d_buf, d_ret


def _check(ref, offs, lens, dsts, d_buf, d_ret):
    ret = d_ret.cpu().numpy()
    buf = d_buf.cpu().numpy()
    for i in range(len(offs)):
        want = ref[offs[i]:offs[i] + lens[i]]
        assert ret[i] == len(want)
        assert np.array_equal(buf[dsts[i]:dsts[i] + len(want)], want)


def _touched(offs, lens, size, page):
    pages = set()
    for o, n in zip(offs, lens):
        end = min(o + n, size)
        if o < end:
            pages.update(range(o // page, (end - 1) // page + 1))
    return pages


@pytest.mark.parametrize("xfer,blocks,threads", [(0, 64, 256), (1, 64, 256), (2, 64, 256), (0, 1216, 128),
                                                  (2, 1216, 128)])
def test_small_pages_random_hint_fetches_only_touched_pages(torch_cuda, gfs, datadir, xfer, blocks, threads):
    torch = torch_cuda
    P = 4 * KiB
    size = 32 * MiB + 999
    path = _file(datadir, 31, size)
    ref = np.fromfile(path, dtype=np.uint8)
    offs, lens = _tiles(size, 3000, 7, P)
    with gfs.Context(cache_bytes=64 * MiB, page_size=P, xfer=xfer, max_rpc_pages=64, ra_cap_pages=63) as ctx:
        fid = ctx.open(path)
        ctx.fadvise(fid, gfs.ADV_RANDOM)
        dsts, d_buf, d_ret = _read_many(torch, gfs, ctx, fid, offs, lens, blocks=blocks, threads=threads)
        torch.cuda.synchronize()
        _check(ref, offs, lens, dsts, d_buf, d_ret)
        st = ctx.stats()
    assert st["ra_pages_sync"] == 0 and st["ra_pages_async"] == 0
    assert st["rpcs"] == st["pages_fetched"]                      # one page per request
    assert st["pages_fetched"] == len(_touched(offs, lens, size, P))  # fits: each touched page once
    assert st["evictions"] == 0 and st["timeouts"] == 0


def test_readahead_on_random_reads_fetches_more_than_the_hint(torch_cuda, gfs, datadir):
    torch = torch_cuda
    P = 4 * KiB
    size = 8 * MiB
    path = _file(datadir, 32, size)
    ref = np.fromfile(path, dtype=np.uint8)
    offs, lens = _tiles(size, 1500, 8, P)  # dense: many reads land next to a present page
    fetched = {}
    for advice in (gfs.ADV_NORMAL, gfs.ADV_RANDOM):
        with gfs.Context(cache_bytes=64 * MiB, page_size=P, max_rpc_pages=64, ra_cap_pages=63) as ctx:
            fid = ctx.open(path)
            ctx.fadvise(fid, advice)
            dsts, d_buf, d_ret = _read_many(torch, gfs, ctx, fid, offs, lens)
            torch.cuda.synchronize()
            _check(ref, offs, lens, dsts, d_buf, d_ret)
            fetched[advice] = ctx.stats()
    assert fetched[gfs.ADV_RANDOM]["pages_fetched"] == len(_touched(offs, lens, size, P))
    assert fetched[gfs.ADV_NORMAL]["pages_fetched"] > fetched[gfs.ADV_RANDOM]["pages_fetched"]
    assert fetched[gfs.ADV_NORMAL]["ra_pages_sync"] + fetched[gfs.ADV_NORMAL]["ra_pages_async"] > 0


@pytest.mark.parametrize("xfer", [0, 2])
@pytest.mark.parametrize("page", [4 * KiB, 64 * KiB])
def test_mixed_sequential_and_random_streams_exact(torch_cuda, gfs, datadir, xfer, page):
    """A sequential scan of one file and random tiles of another, on two streams at once,
    through one cache smaller than the two files."""
    torch = torch_cuda
    seq = _file(datadir, 33, 24 * MiB + 17)
    rnd = _file(datadir, 34, 40 * MiB + 5)
    ref = np.fromfile(rnd, dtype=np.uint8)
    offs, lens = _tiles(os.path.getsize(rnd), 4000, 9, page)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    with gfs.Context(cache_bytes=16 * MiB, page_size=page, xfer=xfer, max_rpc_pages=64,
                     ra_cap_pages=min(63, MiB // page)) as ctx:
        fs, fr = ctx.open(seq), ctx.open(rnd)
        ctx.fadvise(fr, gfs.ADV_RANDOM)
        out = ctx.scan(fs, MiB, blocks=24, fused=True, stream=s1)
        dsts, d_buf, d_ret = _read_many(torch, gfs, ctx, fr, offs, lens, blocks=24, stream=s2)
        torch.cuda.synchronize()
        _check(ref, offs, lens, dsts, d_buf, d_ret)
        from oracle import plain
        c, s, h = plain.scan_plain(seq, MiB)
        assert out[0].cpu().numpy()[:len(c)].tolist() == c
        assert np.array_equal(gfs.u64_view(out[1])[:len(s)], np.array(s, dtype=np.uint64))
        assert np.array_equal(gfs.u64_view(out[2])[:len(h)], np.array(h, dtype=np.uint64))
        assert ctx.stats()["timeouts"] == 0


@pytest.mark.parametrize("cache_mib,blocks,threads", [
    (64, 296, 256),    # 1024 frames (scanned whole)
    (256, 296, 256),   # 4096 frames (scanned by windows)
    (256, 1216, 128),  # eight blocks per SM: the <256, 4> instance of the read kernel
])
@pytest.mark.parametrize("xfer", [0, 2])
def test_thrashing_random_reads_many_blocks(torch_cuda, gfs, datadir, xfer, cache_mib, blocks, threads):
    """4 KiB reads at random places of a file 8x-32x the cache, 64 KiB pages, 296 or 1216
    blocks: every miss needs the demand fallback (no page is ever consumed whole).  Every
    read must succeed with the file's bytes: a reader waiting on its pinned page may see
    an evictor's transient claim, and a gread may evict pages other greads allocated
    after it started."""
    torch = torch_cuda
    P, R = 64 * KiB, 4 * KiB
    size = 2048 * MiB if cache_mib == 256 else 512 * MiB
    path = _file(datadir, 35, size)
    n = 1 << 15
    rng = np.random.default_rng(5)
    offs = rng.integers(0, size // R, size=n, dtype=np.int64) * R
    with gfs.Context(cache_bytes=cache_mib * MiB, page_size=P, xfer=xfer, max_rpc_pages=17, ra_cap_pages=15,
                     rpc_slots=512, timeout_ns=5 * 10**9) as ctx:
        fid = ctx.open(path)
        d_off = torch.from_numpy(offs).cuda()
        d_len = torch.full((n,), R, dtype=torch.int64, device="cuda")
        d_dst = torch.arange(n, dtype=torch.int64, device="cuda") * R
        d_buf = torch.zeros(n * R, dtype=torch.uint8, device="cuda")
        d_ret = torch.full((n,), -999, dtype=torch.int64, device="cuda")
        ctx.read_many(fid, d_off, d_len, d_dst, d_buf, d_ret, blocks=blocks, threads=threads)
        torch.cuda.synchronize()
        st = ctx.stats()
        ret = d_ret.cpu().numpy()
        got = d_buf.cpu().numpy().reshape(n, R)
    ref = np.memmap(path, dtype=np.uint8, mode="r").reshape(-1, R)
    assert (ret == R).all(), dict(zip(*np.unique(ret[ret != R], return_counts=True)))
    assert np.array_equal(got, ref[offs // R])
    assert st["enomem"] == 0 and st["timeouts"] == 0 and st["eio"] == 0
    assert st["unconsumed_evictions"] > 0
