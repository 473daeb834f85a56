"""GPU parity: the CUDA read path through the C ABI against the CPU oracle.

Data (counts, per-stride byte sums and position hashes, delivered bytes) must
be bit-exact.  In serialized mode (one gread at a time in stride order, each
waiting for its requests) the GPU's RPC and eviction logs must equal the
oracle's entry for entry; in concurrent mode the policy has several correct
outcomes and only its invariants are checked.
"""
import os
import random

import numpy as np
import pytest

import inputs
from oracle import plain, policy

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
    path = os.path.join(datadir, "x%d_%d.bin" % (seed, size))
    inputs.ensure_file(path, seed, size)
    return path


def _check_scan(gfs, path, stride, cnt, sm, hs, read_len=None):
    c, s, h = plain.scan_plain(path, stride, read_len)
    assert cnt.cpu().numpy().tolist() == c
    assert np.array_equal(gfs.u64_view(sm)[:len(s)], np.array(s, dtype=np.uint64))
    assert np.array_equal(gfs.u64_view(hs)[:len(h)], np.array(h, dtype=np.uint64))
# ------------------------------------------------ 64 MiB file, 128 MiB cache (fits), 256 KiB pages, 64 blocks

# ------------------------------------------------ config 1: 64 MiB, fits the cache
XFERS = [0, 1, 2]  # GFS_XFER_DMA, GFS_XFER_PULL, GFS_XFER_MAPPED


@pytest.mark.parametrize("xfer", XFERS)
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("fused", [False, True])
def test_config1_scan_exact(torch_cuda, gfs, datadir, mode, fused, xfer):
    path = _file(datadir, 1, 64 * MiB)
    with gfs.Context(cache_bytes=128 * MiB, page_size=256 * KiB, mode=mode, debug_counts=1, xfer=xfer,
                     max_rpc_pages=16) as ctx:
        fid = ctx.open(path)
        for rep in range(2):
            out = ctx.scan(fid, 1 * MiB, blocks=64, threads=256, fused=fused)
            torch_cuda.cuda.synchronize()
            _check_scan(gfs, path, MiB, *out)
            st = ctx.stats()
            counts = ctx.fetch_counts(256)
            assert st["pages_fetched"] == 256 and (counts == 1).all()  # fits: each page once
            assert st["evictions"] == 0 and st["timeouts"] == 0 and st["eio"] == 0
            if mode == 1:
                assert st["rpcs"] == 256                                  # one page per request
            ctx.reset_cache()


def test_config1_second_pass_hits(torch_cuda, gfs, datadir):
    path = _file(datadir, 1, 64 * MiB)
    with gfs.Context(cache_bytes=128 * MiB, page_size=256 * KiB) as ctx:
        fid = ctx.open(path)
        ctx.scan(fid, MiB, blocks=64)
        out = ctx.scan(fid, MiB, blocks=64)  # everything cached now
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, MiB, *out)
        st = ctx.stats()
        assert st["pages_fetched"] == 256 and st["misses"] <= 256


# ------------------------------------------------ serialized: exact policy logs
@pytest.mark.parametrize("xfer", XFERS)
@pytest.mark.parametrize("size,page,frames,blocks,stride,ra_cap,mode,async_ra", [
    (64 * MiB, 256 * KiB, 512, 64, MiB, 8, 0, 1),          # config-1 shape
    (64 * MiB + 12345, 512 * KiB, 16, 8, MiB, 8, 0, 1),    # config-2 shape, file 8x cache, ragged tail
    (24 * MiB, 256 * KiB, 24, 6, 512 * KiB, 2, 0, 1),
    (16 * MiB + 7, 64 * KiB, 40, 4, 192 * KiB, 8, 0, 0),   # sync readahead only
    (8 * MiB, 128 * KiB, 10, 4, 256 * KiB, 8, 1, 1),       # on-demand
    # small pages: greads take runs of cached pages, released in page order
    (4 * MiB + 5, 4 * KiB, 256, 4, 64 * KiB, 8, 0, 1),
    (2 * MiB + 3, 16 * KiB, 48, 4, 128 * KiB, 4, 0, 1),
    (3 * MiB + 7, 4 * KiB, 200, 6, 40 * KiB + 4, 15, 0, 0),  # runs start and end inside pages
    (2 * MiB, 4 * KiB, 128, 4, 64 * KiB, 8, 1, 1),           # on-demand
])
def test_serialized_logs_match_oracle(torch_cuda, gfs, datadir, size, page, frames, blocks, stride, ra_cap, mode,
                                      async_ra, xfer):
    path = _file(datadir, 2, size)
    reserve = policy.default_reserve(blocks, stride, page)
    with gfs.Context(cache_bytes=frames * page, page_size=page, mode=mode, ra_cap_pages=ra_cap, async_ra=async_ra,
                     trace_capacity=1 << 16, reserve_frames=reserve, max_rpc_pages=16, xfer=xfer) as ctx:
        fid = ctx.open(path)
        out = ctx.scan(fid, stride, blocks=blocks, threads=256, serialize=True)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, stride, *out)
        rpc, ev, nr, ne = ctx.trace()
    sim, res = policy.run_scan(path, page, frames, stride, blocks, mode=("ondemand" if mode else "readahead"),
                               ra_cap=ra_cap, reserve=reserve, async_ra=bool(async_ra), max_rpc_pages=16)
    assert nr == len(sim.rpc_log) and ne == len(sim.evict_log)
    assert rpc == sim.rpc_log
    assert ev == sim.evict_log


@pytest.mark.parametrize("xfer", XFERS)
@pytest.mark.parametrize("size,frames,blocks,stride,ra_cap", [
    (6 * MiB + 5, 1024, 3, MiB, 255),     # 256-page demand runs, file larger than the cache
    (3 * MiB + 7, 2048, 2, 64 * KiB, 255),  # readahead windows growing to 256 pages, file fits
])
def test_serialized_logs_at_the_largest_request(torch_cuda, gfs, datadir, size, frames, blocks, stride, ra_cap, xfer):
    """Requests of up to 256 pages (the largest a request holds): runs of frames taken,
    evicted and installed in eight rounds of 32 lanes; the logs still equal the oracle's."""
    page = 4 * KiB
    path = _file(datadir, 2, size)
    reserve = policy.default_reserve(blocks, stride, page)
    with gfs.Context(cache_bytes=frames * page, page_size=page, mode=0, ra_cap_pages=ra_cap, trace_capacity=1 << 16,
                     reserve_frames=reserve, max_rpc_pages=256, xfer=xfer) as ctx:
        fid = ctx.open(path)
        out = ctx.scan(fid, stride, blocks=blocks, threads=256, serialize=True)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, stride, *out)
        rpc, ev, nr, ne = ctx.trace()
    sim, res = policy.run_scan(path, page, frames, stride, blocks, mode="readahead", ra_cap=ra_cap, reserve=reserve,
                               max_rpc_pages=256)
    assert max(n for _, _, n, _ in sim.rpc_log) >= 200  # the shape reaches the largest requests
    assert nr == len(sim.rpc_log) and ne == len(sim.evict_log)
    assert rpc == sim.rpc_log
    assert ev == sim.evict_log


@pytest.mark.parametrize("xfer", XFERS)
@pytest.mark.parametrize("size,page,frames,blocks,stride,read_len,ra_cap,fused", [
    (72 * MiB + 7, 2 * MiB, 16, 4, 4 * MiB, 4 * MiB, 4, False),    # 2 MiB pages, file 2.3x the cache
    (72 * MiB + 7, 2 * MiB, 16, 4, 4 * MiB, 4 * MiB, 4, True),     # the same with the fused consumer
    (160 * MiB + 5, 64 << 20, 4, 2, 16 * MiB, 16 * MiB, 2, False),  # the largest page: four reads per page
])
def test_serialized_logs_at_the_largest_pages(torch_cuda, gfs, datadir, size, page, frames, blocks, stride, read_len,
                                             ra_cap, fused, xfer):
    path = _file(datadir, 2, size)
    reserve = policy.default_reserve(blocks, read_len, page)
    with gfs.Context(cache_bytes=frames * page, page_size=page, mode=0, ra_cap_pages=ra_cap, trace_capacity=1 << 16,
                     reserve_frames=reserve, max_rpc_pages=16, xfer=xfer) as ctx:
        fid = ctx.open(path)
        out = ctx.scan(fid, stride, read_len=read_len, blocks=blocks, threads=256, serialize=True, fused=fused)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, stride, *out, read_len=read_len)
        rpc, ev, nr, ne = ctx.trace()
    sim, res = policy.run_scan(path, page, frames, stride, blocks, read_len=read_len, mode="readahead", ra_cap=ra_cap,
                               reserve=reserve, max_rpc_pages=16)
    assert nr == len(sim.rpc_log) and ne == len(sim.evict_log)
    assert rpc == sim.rpc_log
    assert ev == sim.evict_log


@pytest.mark.parametrize("xfer", [1, 2])
@pytest.mark.parametrize("mode", [0, 1])
def test_serialized_least_recently_allocated_beyond_1024_frames(torch_cuda, gfs, datadir, mode, xfer):
    """Above 1024 frames concurrent greads take the demand fallback's victim from a window
    of the cache; one gread at a time takes the exact least recently allocated frame of the
    whole cache, as the oracle does.  Reads of a page and 100 bytes of the next leave every
    second page unconsumed, so the fallback runs hundreds of times (1100 frames)."""
    page, frames, blocks, stride, read_len = 4 * KiB, 1100, 4, 8 * KiB, 4 * KiB + 100
    path = _file(datadir, 33, 3000 * page + 17)
    reserve = policy.default_reserve(blocks, stride, page)
    with gfs.Context(cache_bytes=frames * page, page_size=page, mode=mode, xfer=xfer, trace_capacity=1 << 16,
                     reserve_frames=reserve, max_rpc_pages=16) as ctx:
        fid = ctx.open(path)
        out = ctx.scan(fid, stride, read_len=read_len, blocks=blocks, threads=256, serialize=True)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, stride, *out, read_len=read_len)
        rpc, ev, nr, ne = ctx.trace()
        st = ctx.stats()
    sim, res = policy.run_scan(path, page, frames, stride, blocks, mode=("ondemand" if mode else "readahead"),
                               read_len=read_len, reserve=reserve, max_rpc_pages=16)
    assert sim.stats.unconsumed_evictions > 300 and st["unconsumed_evictions"] == sim.stats.unconsumed_evictions
    assert nr == len(sim.rpc_log) and ne == len(sim.evict_log)
    assert rpc == sim.rpc_log
    assert ev == sim.evict_log


# ------------------------------------------------ concurrent: larger than the cache
@pytest.mark.parametrize("xfer", XFERS)
@pytest.mark.parametrize("page", [4 * KiB, 16 * KiB])
def test_small_pages_streaming_and_cached_exact(torch_cuda, gfs, datadir, page, xfer):
    """Small pages through a cache 4x smaller than the file, many blocks (runs of pages
    still being filled, readahead marks inside runs), then a file that fits, read twice
    (the second scan is all runs of cached pages)."""
    big = _file(datadir, 13, 64 * MiB + 4097)
    with gfs.Context(cache_bytes=16 * MiB, page_size=page, xfer=xfer, max_rpc_pages=64,
                     ra_cap_pages=min(63, MiB // page)) as ctx:
        fid = ctx.open(big)
        for fused in (False, True):
            out = ctx.scan(fid, 256 * KiB, blocks=48, threads=256, fused=fused)
            torch_cuda.cuda.synchronize()
            _check_scan(gfs, big, 256 * KiB, *out)
        st = ctx.stats()
        assert st["timeouts"] == 0 and st["eio"] == 0 and st["enomem"] == 0
    small = _file(datadir, 14, 6 * MiB + 333)
    with gfs.Context(cache_bytes=16 * MiB, page_size=page, xfer=xfer, max_rpc_pages=64,
                     ra_cap_pages=min(63, MiB // page)) as ctx:
        fid = ctx.open(small)
        for _ in range(2):
            out = ctx.scan(fid, 96 * KiB + 8, blocks=32, threads=256, fused=True)
            torch_cuda.cuda.synchronize()
            _check_scan(gfs, small, 96 * KiB + 8, *out)
        st = ctx.stats()
        assert st["pages_fetched"] == (6 * MiB + 333 + page - 1) // page  # fits: every page once
        assert st["timeouts"] == 0 and st["eio"] == 0



@pytest.mark.parametrize("xfer", [1, 2])
@pytest.mark.parametrize("page", [4 * KiB, 16 * KiB])
def test_overlapping_greads_race_for_the_same_pages_exact(torch_cuda, gfs, datadir, xfer, page):
    """Greads of 256 KiB every 16 KiB: sixteen blocks read every page at about the same
    time, so runs being installed meet pages other greads map meanwhile (the request is cut
    there and the pages after it are requested on their own).  Every stride stays exact and
    every page is fetched.  The loser of a contested page gives its frame back, keyless, to
    the returned-frame ring, which is taken before any consumed page is evicted: the file
    fits, so (almost) no page is read twice.  (When lost frames went to the consumed FIFO
    instead, 0-13 % of the pages were evicted and read again, as the races fell.)"""
    size = 12 * MiB + 333
    path = _file(datadir, 34, size)
    npages = (size + page - 1) // page
    with gfs.Context(cache_bytes=32 * MiB, page_size=page, xfer=xfer, max_rpc_pages=64, ra_cap_pages=63,
                     debug_counts=1) as ctx:
        fid = ctx.open(path)
        cuts = refetched = 0
        for rep in range(3):
            ctx.reset_cache()
            out = ctx.scan(fid, 16 * KiB, read_len=256 * KiB, blocks=128, threads=256, fused=rep == 1)
            torch_cuda.cuda.synchronize()
            _check_scan(gfs, path, 16 * KiB, *out, read_len=256 * KiB)
            st = ctx.stats()
            assert st["timeouts"] == 0 and st["eio"] == 0 and st["enomem"] == 0
            counts = ctx.fetch_counts(npages)
            assert (counts >= 1).all() and counts.sum() <= npages + npages // 100
            cuts += st["run_cuts"]
            refetched += int(counts.sum()) - npages
        print("requests cut by a concurrent install:", cuts, "pages fetched again:", refetched, "of", 3 * npages)


@pytest.mark.parametrize("xfer", XFERS)
@pytest.mark.parametrize("threads", [256, 512])
def test_streaming_big_file_exact(torch_cuda, gfs, datadir, threads, xfer):
    size, page, cache, blocks = 256 * MiB + 4096 * 3, 512 * KiB, 32 * MiB, 48
    path = _file(datadir, 3, size)
    with gfs.Context(cache_bytes=cache, page_size=page, debug_counts=1, xfer=xfer, max_rpc_pages=16) as ctx:
        fid = ctx.open(path)
        out = ctx.scan(fid, MiB, blocks=blocks, threads=threads)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, MiB, *out)
        st = ctx.stats()
        npages = (size + page - 1) // page
        counts = ctx.fetch_counts(npages)
        assert st["timeouts"] == 0 and st["eio"] == 0 and st["enomem"] == 0
        assert (counts >= 1).all()
        assert st["evictions"] >= npages - cache // page


@pytest.mark.parametrize("xfer", XFERS)
@pytest.mark.parametrize("stride,read_len,page", [
    (MiB + 16, MiB + 16, 256 * KiB),     # stride not a page multiple
    (700 * KiB + 3, 300 * KiB + 5, 64 * KiB),  # odd offsets: unaligned copy path
    (64 * KiB, 64 * KiB, 2 * MiB),       # 32 blocks share one page
    (3 * MiB, 2 * MiB + 1, 1 * MiB),
    (100 * KiB + 3, 50 * KiB + 7, 4 * KiB),  # runs of small pages from unaligned offsets
    (256 * KiB, 256 * KiB, 16 * KiB),
])
def test_ragged_strides_exact(torch_cuda, gfs, datadir, stride, read_len, page, xfer):
    size = 40 * MiB + 999
    path = _file(datadir, 4, size)
    with gfs.Context(cache_bytes=16 * MiB if page < 2 * MiB else 32 * MiB, page_size=page, xfer=xfer,
                     max_rpc_pages=16) as ctx:
        fid = ctx.open(path)
        out = ctx.scan(fid, stride, read_len=read_len, blocks=32, threads=128)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, stride, *out, read_len=read_len)


# ------------------------------------------------ independent greads
@pytest.mark.parametrize("xfer", XFERS)
@pytest.mark.parametrize("mode,advice", [(0, 0), (1, 0), (0, 2)])
def test_random_reads_exact(torch_cuda, gfs, datadir, mode, advice, xfer):
    torch = torch_cuda
    size = 12 * MiB + 77
    path = _file(datadir, 5, size)
    ref = np.fromfile(path, dtype=np.uint8)
    rng = random.Random(mode * 10 + advice)
    n = 400
    offs = [rng.randrange(size + 3 * 65536) for _ in range(n)]
    lens = [rng.choice([0, 1, 17, 4096, 65536, 200000, 1 << 20]) for _ in range(n)]
    dsts, pos = [], 0
    for ln in lens:
        dsts.append(pos)
        pos += (ln + 255) // 256 * 256
    with gfs.Context(cache_bytes=4 * MiB, page_size=64 * KiB, mode=mode, xfer=xfer, max_rpc_pages=32) as ctx:
        fid = ctx.open(path)
        if advice:
            ctx.fadvise(fid, advice)
        d_off = torch.tensor(offs, dtype=torch.int64, device="cuda")
        d_len = torch.tensor(lens, dtype=torch.int64, device="cuda")
        d_dst = torch.tensor(dsts, dtype=torch.int64, device="cuda")
        d_buf = torch.zeros(max(pos, 1), dtype=torch.uint8, device="cuda")
        d_ret = torch.full((n,), -999, dtype=torch.int64, device="cuda")
        ctx.read_many(fid, d_off, d_len, d_dst, d_buf, d_ret, blocks=24, threads=256)
        torch.cuda.synchronize()
        ret = d_ret.cpu().numpy()
        buf = d_buf.cpu().numpy()
    for i in range(n):
        want = ref[offs[i]:offs[i] + lens[i]] if offs[i] < size else ref[:0]
        assert ret[i] == len(want)
        assert np.array_equal(buf[dsts[i]:dsts[i] + len(want)], want)


@pytest.mark.parametrize("xfer", XFERS)
def test_edge_cases(torch_cuda, gfs, datadir, xfer):
    torch = torch_cuda
    empty = os.path.join(datadir, "empty.bin")
    open(empty, "wb").close()
    small = _file(datadir, 6, 100)
    with gfs.Context(cache_bytes=MiB, page_size=64 * KiB, xfer=xfer) as ctx:
        fe = ctx.open(empty)
        assert ctx.fstat(fe).size == 0
        cnt, sm, hs = ctx.scan_host(fe, 4096, blocks=4)
        assert len(cnt) == 0
        fs = ctx.open(small)
        cnt, sm, hs = ctx.scan_host(fs, 64, blocks=4, threads=128)
        c, s, h = plain.scan_plain(small, 64)
        assert cnt.tolist() == c and sm.tolist() == s and hs.tolist() == h
        d = torch.zeros(4, dtype=torch.int64, device="cuda")
        r = torch.zeros(4, dtype=torch.int64, device="cuda")
        buf = torch.zeros(4096, dtype=torch.uint8, device="cuda")
        ctx.read_many(fs, torch.tensor([100, 99, 0, 5000], device="cuda"),
                      torch.tensor([10, 10, 0, 1], device="cuda"), d, buf, r, blocks=2, threads=128)
        torch.cuda.synchronize()
        assert r.cpu().tolist() == [0, 1, 0, 0]
        with pytest.raises(gfs.GfsError):
            ctx.scan(7, 4096)
        with pytest.raises(gfs.GfsError):
            ctx.open(os.path.join(datadir, "does-not-exist"))


@pytest.mark.parametrize("xfer", XFERS)
def test_host_read_errors_surface_as_eio(torch_cuda, gfs, datadir, xfer):
    size = 16 * MiB
    path = _file(datadir, 7, size)
    with gfs.Context(cache_bytes=32 * MiB, page_size=256 * KiB, timeout_ns=5 * 10**9, xfer=xfer) as ctx:
        fid = ctx.open(path)
        ctx.set_faults(eio_every=5)
        cnt, sm, hs = ctx.scan_host(fid, MiB, blocks=8)
        c, s, h = plain.scan_plain(path, MiB)
        bad = [i for i in range(len(c)) if cnt[i] < 0]
        assert bad, "injected host errors must reach some greads"
        assert all(cnt[i] == -5 for i in bad)
        for i in range(len(c)):
            if cnt[i] >= 0:
                assert cnt[i] == c[i] and sm[i] == s[i] and hs[i] == h[i]
        st = ctx.stats()
        assert st["timeouts"] == 0 and st["host_errors"] > 0
        ctx.set_faults()
        ctx.reset_cache()
        cnt, sm, hs = ctx.scan_host(fid, MiB, blocks=8)
        assert cnt.tolist() == c and sm.tolist() == s and hs.tolist() == h


@pytest.mark.parametrize("map_pinned", [0, 1])
def test_mapped_file_is_mapped_and_exact(torch_cuda, gfs, datadir, map_pinned):
    """GFS_XFER_MAPPED on a tmpfs file: the GPU reads the page cache directly, through the
    host page tables (read-only, nothing pinned) where the device can, or through a pinned
    registration (map_pinned=1, and on devices that cannot)."""
    if not datadir.startswith("/dev/shm"):
        pytest.skip("no tmpfs for a mappable file")
    size = 96 * MiB + 333
    path = _file(datadir, 8, size)
    with gfs.Context(cache_bytes=16 * MiB, page_size=512 * KiB, xfer=2, max_rpc_pages=16, debug_counts=1,
                     map_pinned=map_pinned) as ctx:
        fid = ctx.open(path)
        mapped = ctx.fstat(fid).mapped
        assert mapped == 1 if map_pinned else mapped in (1, 2)
        for _ in range(2):
            out = ctx.scan(fid, MiB, blocks=48, threads=256)
            torch_cuda.cuda.synchronize()
            _check_scan(gfs, path, MiB, *out)
            st = ctx.stats()
            assert st["host_preads"] == 0 and st["timeouts"] == 0
            ctx.reset_cache()
        ctx.close(fid)


def test_mapped_through_host_page_tables_any_file_system(torch_cuda, gfs, tmp_path, datadir):
    """Where the GPU reads pageable host memory through the host page tables, a warm file
    on a disk file system (whose pages cannot be pinned) is mapped read-only too, and so is
    a file opened on the device (gopen: no CUDA call is needed to map it)."""
    path = str(tmp_path / "disk.bin")
    size = 40 * MiB + 99
    inputs.write_file(path, 17, size)
    with open(path, "rb") as f:  # warm: every page in the host page cache
        while f.read(1 << 24):
            pass
    with gfs.Context(cache_bytes=16 * MiB, page_size=512 * KiB, max_rpc_pages=16) as ctx:
        fid = ctx.open(path)
        if ctx.fstat(fid).mapped != 2:
            pytest.skip("the device does not read pageable memory through the host page tables")
        out = ctx.scan(fid, MiB, blocks=32, threads=256)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, MiB, *out)
        st = ctx.stats()
        assert st["host_preads"] == 0 and st["timeouts"] == 0
        ctx.close(fid)
        dev_path = _file(datadir, 18, 24 * MiB + 5)
        ctx.reset_cache()
        out = ctx.scan_path(dev_path, MiB, blocks=16)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, dev_path, MiB, *out)
        st = ctx.stats()
        assert st["host_controls"] > 0 and st["host_preads"] == 0 and st["timeouts"] == 0


def test_mapped_transfer_skips_files_not_in_the_host_page_cache(torch_cuda, gfs, datadir):
    """A file whose pages are not all resident is not mapped (its pages would be read from
    storage inside gfs_open); its requests are served by pread into staging instead.  A
    sparse tmpfs file has pages that were never written, so it is not fully resident."""
    if not datadir.startswith("/dev/shm"):
        pytest.skip("no tmpfs")
    path = os.path.join(datadir, "sparse.bin")
    size = 8 * MiB + 5
    with open(path, "wb") as f:
        f.write(b"\x5a" * 4096)
        f.truncate(size)
    with gfs.Context(cache_bytes=16 * MiB, page_size=256 * KiB, xfer=2, max_rpc_pages=16) as ctx:
        fid = ctx.open(path)
        assert ctx.fstat(fid).mapped == 0
        out = ctx.scan(fid, MiB, blocks=8)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, MiB, *out)
        assert ctx.stats()["host_preads"] > 0
    full = _file(datadir, 8, 4 * MiB)
    with gfs.Context(cache_bytes=16 * MiB, page_size=256 * KiB, max_rpc_pages=16) as ctx:  # the default transfer
        assert ctx.cfg.xfer == gfs.XFER_MAPPED
        assert ctx.fstat(ctx.open(full)).mapped in (1, 2)


@pytest.mark.parametrize("xfer", XFERS)
def test_direct_io_reads_from_storage_exact(torch_cuda, gfs, tmp_path, xfer):
    """GFS_DIRECT: the host I/O threads read with O_DIRECT (cold reads from storage, as the
    paper's runs after flushing the page cache); the file is never mapped, ragged ends
    (sizes and reads not multiples of 4 KiB) are exact."""
    path = str(tmp_path / "direct.bin")
    size = 24 * MiB + 4321
    inputs.write_file(path, 15, size)
    fd = os.open(path, os.O_RDONLY)
    os.fsync(fd)
    os.close(fd)
    with gfs.Context(cache_bytes=8 * MiB, page_size=256 * KiB, xfer=xfer, max_rpc_pages=16) as ctx:
        try:
            fid = ctx.open(path, gfs.RDONLY | gfs.DIRECT)
        except gfs.GfsError as e:
            pytest.skip("no O_DIRECT on this file system (%s)" % e)
        assert ctx.fstat(fid).mapped == 0
        for stride in (MiB, 300 * KiB + 7):
            ctx.reset_cache()
            out = ctx.scan(fid, stride, blocks=16, threads=256)
            torch_cuda.cuda.synchronize()
            _check_scan(gfs, path, stride, *out)
            st = ctx.stats()
            assert st["host_preads"] > 0 and st["timeouts"] == 0 and st["eio"] == 0


@pytest.mark.parametrize("xfer", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_merged_host_reads_exact(torch_cuda, gfs, datadir, xfer, mode):
    """Host threads that pread (dma, pull) claim the requests waiting at the head of the
    ring and serve each run of them whose pages continue one another with one read.  With
    64 KiB strides of 64 KiB pages neighbouring blocks ask for neighbouring pages at once,
    and two host threads let requests back up, so merging happens; every stride stays
    exact, and each page is still fetched once while the file fits."""
    size = 48 * MiB + 777
    path = _file(datadir, 16, size)
    page = 64 * KiB
    npages = (size + page - 1) // page
    for merge in (0, 1):
        with gfs.Context(cache_bytes=64 * MiB, page_size=page, xfer=xfer, mode=mode, host_threads=2,
                         max_rpc_pages=16, rpc_slots=256, host_merge_pages=merge, debug_counts=1) as ctx:
            fid = ctx.open(path)
            for stride in (page, MiB):
                ctx.reset_cache()
                out = ctx.scan(fid, stride, blocks=128, threads=256)
                torch_cuda.cuda.synchronize()
                _check_scan(gfs, path, stride, *out)
                st = ctx.stats()
                assert st["timeouts"] == 0 and st["eio"] == 0
                assert (ctx.fetch_counts(npages) == 1).all()
                if merge == 1:
                    assert st["host_merged"] == 0
                elif stride == page:
                    assert st["host_merged"] > 0 and st["host_preads"] < st["host_requests"]


@pytest.mark.parametrize("page", [4 * KiB, 512 * KiB])
def test_requests_for_mapped_files_served_by_the_gpu(torch_cuda, gfs, datadir, page):
    """With the mapped transfer a request for a mapped file is served by the block that
    makes it (it copies the pages from the mapping): no host request at all, every
    stride exact, every page fetched once while the file fits, and the serialized request
    and eviction logs still equal the oracle's (the policy does not change)."""
    if not datadir.startswith("/dev/shm"):
        pytest.skip("no tmpfs for a mappable file")
    size = 24 * MiB + 12345
    path = _file(datadir, 19, size)
    npages = (size + page - 1) // page
    with gfs.Context(cache_bytes=32 * MiB, page_size=page, xfer=2, max_rpc_pages=64, ra_cap_pages=15,
                     debug_counts=1) as ctx:
        fid = ctx.open(path)
        assert ctx.fstat(fid).mapped in (1, 2)
        for fused in (False, True):
            ctx.reset_cache()
            out = ctx.scan(fid, MiB, blocks=48, threads=256, fused=fused)
            torch_cuda.cuda.synchronize()
            _check_scan(gfs, path, MiB, *out)
            st = ctx.stats()
            assert st["rpcs"] > 0 and st["host_requests"] == 0 and st["timeouts"] == 0
            assert (ctx.fetch_counts(npages) == 1).all()
    frames, blocks, stride = 40, 4, 3 * page + 7
    path2 = _file(datadir, 20, 96 * page + 3)
    reserve = policy.default_reserve(blocks, stride, page)
    with gfs.Context(cache_bytes=frames * page, page_size=page, xfer=2, trace_capacity=1 << 16,
                     reserve_frames=reserve, max_rpc_pages=16) as ctx:
        fid = ctx.open(path2)
        out = ctx.scan(fid, stride, blocks=blocks, threads=256, serialize=True)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path2, stride, *out)
        rpc, ev, nr, ne = ctx.trace()
        assert ctx.stats()["host_requests"] == 0
    sim, res = policy.run_scan(path2, page, frames, stride, blocks, reserve=reserve, max_rpc_pages=16)
    assert rpc == sim.rpc_log and ev == sim.evict_log


def _golden(name):
    params, rows = {}, []
    for line in open(os.path.join(os.path.dirname(__file__), "golden", name)):
        parts = line.split()
        if not parts or parts[0].startswith("#"):
            continue
        if parts[0] == "params":
            params.update(kv.split("=") for kv in parts[1:])
        else:
            rows.append(parts)
    return params, rows


@pytest.mark.parametrize("xfer", XFERS)
def test_golden_demand_run_awaited_page_only_on_gpu(torch_cuda, gfs, datadir, xfer):
    """The hand-derived trace of tests/golden/policy_demand_run_awaited_only.txt replayed by
    one threadblock (greads one at a time): a later page of a demand run ends the request
    instead of evicting an unconsumed page; the logs equal the derivation."""
    torch = torch_cuda
    params, rows = _golden("policy_demand_run_awaited_only.txt")
    page, npg = int(params["page_size"]), int(params["file_pages"])
    path = _file(datadir, int(params["seed"]), npg * page)
    greads = [(int(r[2]), int(r[3])) for r in rows if r[0] == "gread"]
    kinds = {"DEMAND": 0, "SYNC_RA": 1, "ASYNC_RA": 2}
    with gfs.Context(cache_bytes=int(params["frames"]) * page, page_size=page, mode=0,
                     ra_cap_pages=int(params["ra_cap"]), async_ra=int(params["async_ra"]),
                     reserve_frames=int(params["reserve"]), trace_capacity=256, max_rpc_pages=16, xfer=xfer) as ctx:
        fid = ctx.open(path)
        d_off = torch.tensor([o for o, _ in greads], dtype=torch.int64, device="cuda")
        d_len = torch.tensor([n for _, n in greads], dtype=torch.int64, device="cuda")
        dst, pos = [], 0
        for _, n in greads:
            dst.append(pos)
            pos += (n + 255) // 256 * 256
        d_dst = torch.tensor(dst, dtype=torch.int64, device="cuda")
        buf = torch.zeros(pos, dtype=torch.uint8, device="cuda")
        ret = torch.zeros(len(greads), dtype=torch.int64, device="cuda")
        ctx.read_many(fid, d_off, d_len, d_dst, buf, ret, blocks=1, threads=256)
        torch.cuda.synchronize()
        rpc, ev, nr, ne = ctx.trace()
        st = ctx.stats()
    ref = np.fromfile(path, dtype=np.uint8)
    got = buf.cpu().numpy()
    for (o, n), d in zip(greads, dst):
        assert np.array_equal(got[d:d + n], ref[o:o + n])
    assert ret.cpu().tolist() == [n for _, n in greads]
    assert rpc == [(0, int(r[1]), int(r[2]), kinds[r[3]]) for r in rows if r[0] == "rpc"]
    assert ev == [(int(r[1]), (0, int(r[2])), (0, int(r[3]))) for r in rows if r[0] == "evict"]
    assert st["unconsumed_evictions"] == int([r for r in rows if r[0] == "unconsumed_evictions"][0][1])


@pytest.mark.parametrize("xfer", [1, 2])
def test_scan_graph_steady_loop_exact(torch_cuda, gfs, datadir, xfer):
    path = _file(datadir, 1, 64 * MiB)
    with gfs.Context(cache_bytes=128 * MiB, page_size=256 * KiB, xfer=xfer, max_rpc_pages=16) as ctx:
        fid = ctx.open(path)
        for reps in (1, 3, 3):
            out = ctx.scan_graph(fid, MiB, reps, blocks=64)
            torch_cuda.cuda.synchronize()
            _check_scan(gfs, path, MiB, *out)
            st = ctx.stats()
            assert st["pages_fetched"] == 256 and st["timeouts"] == 0  # last repetition, from an empty cache


@pytest.mark.parametrize("xfer", [1, 2])
@pytest.mark.parametrize("mode", [0, 2])  # readahead, the paper's prefetcher; both with per-block LRA
def test_scan_graph_repetitions_start_from_empty_lra_queues(torch_cuda, gfs, datadir, xfer, mode):
    """Every repetition of the captured loop starts from an empty cache, empty per-block
    LRA queues and (paper mode) empty private buffers: the last repetition's serialized
    logs equal a fresh oracle run."""
    size, page, frames, blocks, stride, ra = 24 * MiB + 999, 256 * KiB, 24, 6, 512 * KiB, 2
    path = _file(datadir, 12, size)
    with gfs.Context(cache_bytes=frames * page, page_size=page, mode=mode, replacement=1, ra_cap_pages=ra,
                     trace_capacity=1 << 16, max_rpc_pages=16, xfer=xfer, reserve_frames=1,
                     timeout_ns=2 * 10**9) as ctx:
        fid = ctx.open(path)
        out = ctx.scan_graph(fid, stride, 3, blocks=blocks, serialize=True)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, stride, *out)
        rpc, ev, nr, ne = ctx.trace()
    sim, res = policy.run_scan(path, page, frames, stride, blocks, mode=("paper" if mode == 2 else "readahead"),
                               ra_cap=ra, reserve=1, max_rpc_pages=16, replacement="tb_lra")
    assert rpc == sim.rpc_log
    assert ev == sim.evict_log


def test_scan_graph_refuses_dma(torch_cuda, gfs, datadir):
    path = _file(datadir, 1, 64 * MiB)
    with gfs.Context(cache_bytes=128 * MiB, page_size=256 * KiB, xfer=0) as ctx:
        fid = ctx.open(path)
        with pytest.raises(gfs.GfsError):
            ctx.scan_graph(fid, MiB, 2)


def test_tuner_measures_and_persists(torch_cuda, datadir, tmp_path):
    from paper_2109_05366_gb300 import tune
    path = _file(datadir, 3, 64 * MiB)
    space = {"page_size": [256 * KiB, 1 * MiB], "ra_cap_pages": [1, 8], "rpc_slots": [128], "blocks": [64]}
    start = {"page_size": 256 * KiB, "ra_cap_pages": 8, "rpc_slots": 128, "blocks": 64}
    best, allp = tune.tune(path, MiB, space, start, rounds=1, cache_bytes=32 * MiB, reps=1)
    assert len(allp) == 3 and best["gbps"] > 0 and all(p["short_strides"] == 0 for p in allp)
    f = str(tmp_path / "best.json")
    tune.save(best, f)
    assert tune.load(f) == best


def test_pull_partial_requests_are_helped(torch_cuda, gfs, datadir):
    # Large pages, small strides, few slots: a host thread's staging buffers
    # cycle inside one readahead request; the pages it already published must be
    # copied out by helpers even before the request is complete.
    size = 256 * MiB
    path = _file(datadir, 9, size)
    with gfs.Context(cache_bytes=512 * MiB, page_size=2 * MiB, xfer=1, rpc_slots=32, max_rpc_pages=16,
                     timeout_ns=3 * 10**9, max_streams=1024) as ctx:
        fid = ctx.open(path)
        out = ctx.scan(fid, 64 * KiB, blocks=592, threads=256)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, 64 * KiB, *out)
        assert ctx.stats()["timeouts"] == 0


# ------------------------------------------------ readahead with the per-block LRA of Section 5.1
@pytest.mark.parametrize("xfer", XFERS)
@pytest.mark.parametrize("replacement", ["fifo", "tb_lra"])
def test_serialized_logs_do_not_depend_on_the_queue(torch_cuda, gfs, datadir, xfer, replacement):
    """GPUfs's static slot partition carries the same requests as the shared ring: with
    one gread at a time the logs still equal the oracle's."""
    size, page, frames, blocks, stride, ra = 24 * MiB + 999, 256 * KiB, 24, 6, 512 * KiB, 2
    path = _file(datadir, 12, size)
    reserve = policy.default_reserve(blocks, stride, page)
    with gfs.Context(cache_bytes=frames * page, page_size=page, mode=0, ra_cap_pages=ra, queue=1, rpc_slots=4,
                     host_threads=2, replacement=(1 if replacement == "tb_lra" else 0), reserve_frames=reserve,
                     trace_capacity=1 << 16, max_rpc_pages=16, xfer=xfer, timeout_ns=2 * 10**9) as ctx:
        fid = ctx.open(path)
        out = ctx.scan(fid, stride, blocks=blocks, threads=256, serialize=True)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, stride, *out)
        rpc, ev, nr, ne = ctx.trace()
    sim, res = policy.run_scan(path, page, frames, stride, blocks, mode="readahead", ra_cap=ra, reserve=reserve,
                               max_rpc_pages=16, replacement=replacement)
    assert rpc == sim.rpc_log
    assert ev == sim.evict_log


@pytest.mark.parametrize("xfer", XFERS)
@pytest.mark.parametrize("size,page,frames,blocks,stride,ra_cap,async_ra", [
    (24 * MiB + 999, 256 * KiB, 24, 6, 512 * KiB, 2, 1),     # file 4x the cache, quota 4
    (16 * MiB + 7, 64 * KiB, 40, 4, 192 * KiB, 8, 0),        # sync readahead only, quota 10
    (8 * MiB, 128 * KiB, 64, 2, 128 * KiB, 8, 1),            # file as large as the cache, quota 32 each
    (4 * MiB + 5, 4 * KiB, 256, 4, 64 * KiB, 8, 1),          # small pages: runs of cached pages
])
def test_readahead_per_block_lra_serialized_logs_match_oracle(torch_cuda, gfs, datadir, xfer, size, page, frames,
                                                               blocks, stride, ra_cap, async_ra):
    path = _file(datadir, 12, size)
    with gfs.Context(cache_bytes=frames * page, page_size=page, mode=0, replacement=1, ra_cap_pages=ra_cap,
                     async_ra=async_ra, trace_capacity=1 << 16, max_rpc_pages=16, xfer=xfer,
                     timeout_ns=2 * 10**9) as ctx:
        fid = ctx.open(path)
        out = ctx.scan(fid, stride, blocks=blocks, threads=256, serialize=True)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, stride, *out)
        rpc, ev, nr, ne = ctx.trace()
    sim, res = policy.run_scan(path, page, frames, stride, blocks, mode="readahead", ra_cap=ra_cap, reserve=0,
                               async_ra=bool(async_ra), max_rpc_pages=16, replacement="tb_lra")
    assert rpc == sim.rpc_log
    assert ev == sim.evict_log


@pytest.mark.parametrize("xfer", XFERS)
@pytest.mark.parametrize("page,ra_cap", [(64 * KiB, 15), (4 * KiB, 63)])  # 4 KiB: 64-page runs from each queue
def test_readahead_per_block_lra_concurrent_exact(torch_cuda, gfs, datadir, xfer, page, ra_cap):
    size = 128 * MiB + 4096
    path = _file(datadir, 11, size)
    with gfs.Context(cache_bytes=32 * MiB, page_size=page, mode=0, replacement=1, ra_cap_pages=ra_cap,
                     max_rpc_pages=64, xfer=xfer, timeout_ns=5 * 10**9) as ctx:
        fid = ctx.open(path)
        for _ in range(2):
            out = ctx.scan(fid, MiB, blocks=96, threads=256)
            torch_cuda.cuda.synchronize()
            _check_scan(gfs, path, MiB, *out)
            st = ctx.stats()
            assert st["timeouts"] == 0 and st["enomem"] == 0 and st["evictions"] > 0
            ctx.reset_cache()


@pytest.mark.parametrize("xfer", [1, 2])
def test_per_block_lra_overlapping_greads_many_scans(torch_cuda, gfs, datadir, xfer):
    """Per-block LRA under overlapping greads (64 KiB every 16 KiB, four readers per page),
    twenty scans without a reset through a cache smaller than the file: frames that lose
    an install race stay in their block's queue and are reused from there, so lost races
    never pile up anywhere (every scan exact, no wait runs out)."""
    torch = torch_cuda
    size = 6 * MiB + 777
    path = _file(datadir, 37, size)
    with gfs.Context(cache_bytes=4 * MiB, page_size=4 * KiB, mode=0, replacement=1, ra_cap_pages=15,
                     max_rpc_pages=32, xfer=xfer, timeout_ns=2 * 10**9) as ctx:
        fid = ctx.open(path)
        for _ in range(20):
            out = ctx.scan(fid, 16 * KiB, read_len=64 * KiB, blocks=64, threads=256)
            torch.cuda.synchronize()
            _check_scan(gfs, path, 16 * KiB, *out, read_len=64 * KiB)
        st = ctx.stats()
        assert st["timeouts"] == 0 and st["enomem"] == 0 and st["eio"] == 0


# ------------------------------------------------ the paper's own design (Sections 4.1, 5.1)
@pytest.mark.parametrize("xfer", [1, 2])
@pytest.mark.parametrize("repl", [0, 1])
@pytest.mark.parametrize("size,page,frames,blocks,stride,prefetch", [
    (16 * MiB, 64 * KiB, 64, 4, 256 * KiB, 3),           # file fits
    (24 * MiB + 999, 256 * KiB, 16, 6, 512 * KiB, 2),    # file 6x the cache
])
def test_paper_mode_serialized_logs_match_oracle(torch_cuda, gfs, datadir, xfer, repl, size, page, frames, blocks,
                                                 stride, prefetch):
    path = _file(datadir, 10, size)
    with gfs.Context(cache_bytes=frames * page, page_size=page, mode=2, replacement=repl, ra_cap_pages=prefetch,
                     trace_capacity=1 << 16, max_rpc_pages=16, xfer=xfer, reserve_frames=1,
                     timeout_ns=2 * 10**9) as ctx:
        fid = ctx.open(path)
        out = ctx.scan(fid, stride, blocks=blocks, threads=256, serialize=True)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, stride, *out)
        rpc, ev, nr, ne = ctx.trace()
        st = ctx.stats()
    sim, res = policy.run_scan(path, page, frames, stride, blocks, mode="paper", ra_cap=prefetch, reserve=1,
                               max_rpc_pages=16, replacement=("tb_lra" if repl else "fifo"))
    assert rpc == sim.rpc_log
    assert ev == sim.evict_log
    assert st["buffer_hits"] == sim.stats.buffer_hits


@pytest.mark.parametrize("xfer", [1, 2])
@pytest.mark.parametrize("repl", [0, 1])
def test_paper_mode_concurrent_exact(torch_cuda, gfs, datadir, xfer, repl):
    size = 128 * MiB + 4096
    path = _file(datadir, 11, size)
    with gfs.Context(cache_bytes=32 * MiB, page_size=64 * KiB, mode=2, replacement=repl, ra_cap_pages=15,
                     max_rpc_pages=16, xfer=xfer, timeout_ns=2 * 10**9) as ctx:
        fid = ctx.open(path)
        out = ctx.scan(fid, MiB, blocks=96, threads=256)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, MiB, *out)
        st = ctx.stats()
        assert st["timeouts"] == 0 and st["buffer_hits"] > 0
