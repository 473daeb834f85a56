"""GPU tests of the device-side file API (Section 2.2: GPU threads open, read and
close files; Section 4.4: the access hint) and of closing files.

* gfs_close drops the file's cached pages: a file opened later under the same
  id reads its own bytes (checked against the oracle), not the old file's.
* gfs_scan_path: every threadblock gopens the path, greads its strides and
  gcloses; all blocks share one id (each page fetched once).
* A kernel compiled the way a library user compiles one (tests/devapi_user.cu)
  calls gopen / gfadvise / gfstat / gread / gclose through the handle that
  gfs_device_handle exports.
"""
import ctypes
import errno
import os

import numpy as np
import pytest

import inputs
from oracle import plain
from tests.devapi_build import build_user_kernel

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
    path = os.path.join(datadir, "d%d_%d.bin" % (seed, size))
    inputs.ensure_file(path, seed, size)
    return path


def _check_scan(gfs, path, stride, cnt, sm, hs):
    c, s, h = plain.scan_plain(path, stride)
    assert cnt.cpu().numpy()[:len(c)].tolist() == c
    assert np.array_equal(gfs.u64_view(sm)[:len(s)], np.array(s, dtype=np.uint64))
    assert np.array_equal(gfs.u64_view(hs)[:len(h)], np.array(h, dtype=np.uint64))


def _pages(path, page):
    return (os.path.getsize(path) + page - 1) // page


# ------------------------------------------------ close drops the file's pages
@pytest.mark.parametrize("mode,xfer", [(0, 0), (0, 2), (1, 1), (2, 2)])
def test_close_then_reuse_id_reads_new_file(torch_cuda, gfs, datadir, mode, xfer):
    a = _file(datadir, 21, 5 * MiB + 123)
    b = _file(datadir, 22, 5 * MiB + 4567)
    P = 256 * KiB
    with gfs.Context(cache_bytes=64 * MiB, page_size=P, mode=mode, xfer=xfer, max_files=1,
                     max_rpc_pages=16) as ctx:
        fa = ctx.open(a)
        out = ctx.scan(fa, MiB, blocks=8)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, a, MiB, *out)
        ctx.close(fa)
        fb = ctx.open(b)
        assert fb == fa                                  # one id: the same key space
        before = ctx.stats()["pages_fetched"]
        out = ctx.scan(fb, MiB, blocks=8)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, b, MiB, *out)
        st = ctx.stats()
        if mode != 2:  # the paper mode's private buffers may fetch a page more than once
            assert st["pages_fetched"] - before == _pages(b, P)  # every page of b came from b
        assert st["timeouts"] == 0 and st["eio"] == 0


def test_close_keeps_other_files_pages(torch_cuda, gfs, datadir):
    a = _file(datadir, 23, 3 * MiB)
    b = _file(datadir, 24, 3 * MiB + 77)
    P = 256 * KiB
    with gfs.Context(cache_bytes=64 * MiB, page_size=P, max_files=2) as ctx:
        fa, fb = ctx.open(a), ctx.open(b)
        ctx.scan(fa, MiB, blocks=4)
        ctx.scan(fb, MiB, blocks=4)
        torch_cuda.cuda.synchronize()
        ctx.close(fa)
        before = ctx.stats()["pages_fetched"]
        out = ctx.scan(fb, MiB, blocks=4)                 # still cached: no fetch
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, b, MiB, *out)
        assert ctx.stats()["pages_fetched"] == before
        fa2 = ctx.open(a)                                  # the dropped frames are reusable
        out = ctx.scan(fa2, MiB, blocks=4)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, a, MiB, *out)
        assert ctx.stats()["pages_fetched"] == before + _pages(a, P)


# ------------------------------------------------ gopen / gclose in the stride scan
@pytest.mark.parametrize("xfer", [0, 1, 2])
def test_scan_path_exact_and_shared_id(torch_cuda, gfs, datadir, xfer):
    path = _file(datadir, 25, 16 * MiB + 999)
    P = 256 * KiB
    blocks = 64
    with gfs.Context(cache_bytes=64 * MiB, page_size=P, xfer=xfer, max_rpc_pages=16) as ctx:
        out = ctx.scan_path(path, MiB, blocks=blocks)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, path, MiB, *out)
        st = ctx.stats()
        assert st["host_controls"] == 2 * blocks          # one gopen and one gclose per block
        assert st["pages_fetched"] == _pages(path, P)     # one shared id: each page once
        assert st["timeouts"] == 0 and st["eio"] == 0


@pytest.mark.parametrize("xfer", [0, 2])
def test_scan_path_with_static_queue_and_per_block_lra(torch_cuda, gfs, datadir, xfer):
    path = _file(datadir, 29, 40 * MiB + 77)
    with gfs.Context(cache_bytes=16 * MiB, page_size=256 * KiB, xfer=xfer, queue=1, replacement=1, rpc_slots=16,
                     host_threads=4, max_rpc_pages=16) as ctx:
        for _ in range(2):
            out = ctx.scan_path(path, MiB, blocks=32)
            torch_cuda.cuda.synchronize()
            _check_scan(gfs, path, MiB, *out)
            st = ctx.stats()
            assert st["host_controls"] == 64 and st["timeouts"] == 0 and st["evictions"] > 0
            ctx.reset_cache()


def test_scan_path_ids_retire_until_reset(torch_cuda, gfs, datadir):
    a = _file(datadir, 26, 2 * MiB + 5)
    b = _file(datadir, 27, 2 * MiB + 9)
    c = _file(datadir, 28, 2 * MiB + 11)
    with gfs.Context(cache_bytes=32 * MiB, page_size=256 * KiB, max_files=2) as ctx:
        for p in (a, b):                                  # each run leaves its id retired
            out = ctx.scan_path(p, MiB, blocks=4)
            torch_cuda.cuda.synchronize()
            _check_scan(gfs, p, MiB, *out)
        cnt, _, _ = ctx.scan_path(c, MiB, blocks=4)       # no id left for a third path
        torch_cuda.cuda.synchronize()
        assert (cnt.cpu().numpy()[:3] == -errno.EMFILE).all()
        for p in (a, b, a, b):                            # a retired path's id is opened again
            out = ctx.scan_path(p, MiB, blocks=8)         # (more blocks than strides: some close at once)
            torch_cuda.cuda.synchronize()
            _check_scan(gfs, p, MiB, *out)
        ctx.reset_cache()                                 # drops the retired ids' pages
        out = ctx.scan_path(b, MiB, blocks=4)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, b, MiB, *out)
        fid = ctx.open(a)                                 # reuses a retired id after dropping its pages
        out = ctx.scan(fid, MiB, blocks=4)
        torch_cuda.cuda.synchronize()
        _check_scan(gfs, a, MiB, *out)


def test_scan_path_errors(torch_cuda, gfs, datadir):
    path = _file(datadir, 25, 16 * MiB + 999)
    with gfs.Context(cache_bytes=32 * MiB, page_size=256 * KiB) as ctx:
        with pytest.raises(gfs.GfsError) as e:
            ctx.scan_path(os.path.join(datadir, "missing.bin"), MiB, blocks=4)
        assert e.value.errno == errno.ENOENT
        with pytest.raises(gfs.GfsError) as e:
            ctx.scan_path("/" + "a" * gfs.PATH_MAX, MiB, blocks=4)
        assert e.value.errno == errno.ENAMETOOLONG
    with gfs.Context(cache_bytes=32 * MiB, page_size=256 * KiB, mode=2, xfer=2) as ctx:
        with pytest.raises(gfs.GfsError) as e:
            ctx.scan_path(path, MiB, blocks=4)
        assert e.value.errno == errno.ENOTSUP


def test_device_handle_size(gfs):
    with gfs.Context(cache_bytes=16 * MiB, page_size=256 * KiB) as ctx:
        h = ctx.device_handle(8, MiB)
        assert len(h) > 256
        small = ctypes.create_string_buffer(16)
        assert gfs.load().gfs_device_handle(ctx.handle, 8, MiB, small, 16) == -errno.ENOSPC


# ------------------------------------------------ a user's own kernel
@pytest.fixture(scope="module")
def user_lib(tmp_path_factory):
    so = build_user_kernel(str(tmp_path_factory.mktemp("devapi")))
    lib = ctypes.CDLL(so)
    lib.user_scan.restype = ctypes.c_int
    lib.user_scan.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_char_p, ctypes.c_int, ctypes.c_uint64,
                              ctypes.c_uint64, ctypes.c_uint32] + [ctypes.c_void_p] * 5
    lib.user_replay.restype = ctypes.c_int
    lib.user_replay.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_uint32] + [ctypes.c_void_p] * 7
    return lib


def _golden(name):
    params, rows = {}, []
    for line in open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if parts[0] == "params":
            params.update(kv.split("=") for kv in parts[1:])
        else:
            rows.append(parts)
    return params, rows


@pytest.mark.parametrize("xfer", [0, 1, 2])
@pytest.mark.parametrize("name", ["policy_sequential_by_last_end.txt", "policy_reread_not_sequential.txt",
                                  "policy_gread_keeps_own_frames.txt"])
def test_user_kernel_replays_hand_derived_traces(torch_cuda, gfs, datadir, user_lib, name, xfer):
    """The hand-derived traces over two readers and tiny caches (tests/golden/<name>),
    replayed one gread at a time by a user kernel with gread_as: return values, the
    delivered bytes of every successful gread, and the request and eviction logs
    equal the derivation (R3's test on the reader's previous end, where a reader's
    gread ends, and the class-3 rule that a gread never evicts its own frames, which
    ends the too-wide gread with -ENOMEM at the device deadline)."""
    torch = torch_cuda
    params, rows = _golden(name)
    page, npg = int(params["page_size"]), int(params["file_pages"])
    path = _file(datadir, int(params["seed"]), npg * page)
    greads = [(int(r[1]), int(r[2]), int(r[3])) for r in rows if r[0] == "gread"]
    rets = [int(r[1]) for r in rows if r[0] == "ret"]
    kinds = {"DEMAND": 0, "SYNC_RA": 1, "ASYNC_RA": 2}
    dst, pos = [], 0
    for _, _, n in greads:
        dst.append(pos)
        pos += (n + 255) // 256 * 256
    with gfs.Context(cache_bytes=int(params["frames"]) * page, page_size=page, mode=0,
                     ra_cap_pages=int(params["ra_cap"]), async_ra=int(params["async_ra"]),
                     reserve_frames=int(params["reserve"]), trace_capacity=256, max_rpc_pages=16, xfer=xfer,
                     timeout_ns=300 * 10**6) as ctx:
        fid = ctx.open(path)
        h = ctx.device_handle(1, page)
        d_rd = torch.tensor([s for s, _, _ in greads], dtype=torch.int32, device="cuda")
        d_off = torch.tensor([o for _, o, _ in greads], dtype=torch.int64, device="cuda")
        d_len = torch.tensor([n for _, _, n in greads], dtype=torch.int64, device="cuda")
        d_dst = torch.tensor(dst, dtype=torch.int64, device="cuda")
        buf = torch.zeros(pos, dtype=torch.uint8, device="cuda")
        ret = torch.zeros(len(greads), dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        rc = user_lib.user_replay(h, len(h), fid, len(greads), d_rd.data_ptr(), d_off.data_ptr(), d_len.data_ptr(),
                                  d_dst.data_ptr(), buf.data_ptr(), ret.data_ptr(), None)
        assert rc == 0
        torch.cuda.synchronize()
        rpc, ev, nr, ne = ctx.trace()
        st = ctx.stats()
    assert ret.cpu().tolist() == rets
    ref = np.fromfile(path, dtype=np.uint8)
    got = buf.cpu().numpy()
    for (_, o, n), d, r in zip(greads, dst, rets):
        if r >= 0:
            assert np.array_equal(got[d:d + r], ref[o:o + r])
    assert rpc == [(0, int(r[1]), int(r[2]), kinds[r[3]]) for r in rows if r[0] == "rpc"]
    assert ev == [(int(r[1]), (0, int(r[2])), (0, int(r[3]))) for r in rows if r[0] == "evict"]
    assert st["unconsumed_evictions"] == int([r for r in rows if r[0] == "unconsumed_evictions"][0][1])


@pytest.mark.parametrize("advice", [-1, 2])  # none, GFS_ADV_RANDOM
@pytest.mark.parametrize("xfer", [0, 2])
def test_user_kernel_device_api(torch_cuda, gfs, datadir, user_lib, advice, xfer):
    torch = torch_cuda
    path = _file(datadir, 28, 8 * MiB + 321)
    P, S, blocks = 256 * KiB, 512 * KiB, 16
    size = os.path.getsize(path)
    ns = (size + S - 1) // S
    with gfs.Context(cache_bytes=64 * MiB, page_size=P, xfer=xfer, max_rpc_pages=16) as ctx:
        h = ctx.device_handle(blocks, S)
        bufs = torch.empty(blocks * S, dtype=torch.uint8, device="cuda")
        cnt = torch.empty(ns, dtype=torch.int64, device="cuda")
        sm = torch.empty(ns, dtype=torch.int64, device="cuda")
        info = torch.zeros(8 * blocks, dtype=torch.int64, device="cuda")
        rc = user_lib.user_scan(h, len(h), path.encode(), advice, S, ns, blocks, bufs.data_ptr(), cnt.data_ptr(),
                                sm.data_ptr(), info.data_ptr(), None)
        assert rc == 0
        torch.cuda.synchronize()
        c, s, _ = plain.scan_plain(path, S)
        assert cnt.cpu().numpy().tolist() == c
        assert np.array_equal(gfs.u64_view(sm), np.array(s, dtype=np.uint64))
        inf = info.cpu().numpy().reshape(blocks, 8)
        assert (inf[:, 0] == inf[0, 0]).all() and inf[0, 0] >= 0   # one id for every block
        assert (inf[:, 1] == 0).all() and (inf[:, 2] == 0).all() and (inf[:, 7] == 0).all()
        assert (inf[:, 3] == size).all() and (inf[:, 4] == P).all() and (inf[:, 6] == 0).all()
        st = ctx.stats()
        assert st["pages_fetched"] == _pages(path, P)
        if advice == 2:                                   # RANDOM: no readahead, one page per request
            assert (inf[:, 5] == 2).all()
            assert st["ra_pages_sync"] == 0 and st["ra_pages_async"] == 0
            assert st["rpcs"] == st["pages_fetched"]
        else:  # whether concurrent blocks leave readahead any page depends on timing: not checked
            assert (inf[:, 5] == 0).all()
        assert st["host_controls"] == blocks * (3 if advice >= 0 else 2)


def test_user_kernel_gopen_of_missing_file_fails_cleanly(torch_cuda, gfs, datadir, user_lib):
    """gopen of a path the host cannot open returns the host's -errno to every block;
    no request of the kernel hangs and the context stays usable."""
    torch = torch_cuda
    P, S, blocks = 256 * KiB, 512 * KiB, 8
    missing = os.path.join(datadir, "no_such_file.bin")
    with gfs.Context(cache_bytes=16 * MiB, page_size=P, xfer=2, max_rpc_pages=16) as ctx:
        h = ctx.device_handle(blocks, S)
        bufs = torch.empty(blocks * S, dtype=torch.uint8, device="cuda")
        cnt = torch.zeros(16, dtype=torch.int64, device="cuda")
        sm = torch.zeros(16, dtype=torch.int64, device="cuda")
        info = torch.zeros(8 * blocks, dtype=torch.int64, device="cuda")
        assert user_lib.user_scan(h, len(h), missing.encode(), -1, S, 16, blocks, bufs.data_ptr(), cnt.data_ptr(),
                                  sm.data_ptr(), info.data_ptr(), None) == 0
        torch.cuda.synchronize()
        inf = info.cpu().numpy().reshape(blocks, 8)
        assert (inf[:, 0] == -errno.ENOENT).all()
        assert (cnt.cpu().numpy() == -errno.ENOENT).all()
        assert ctx.stats()["timeouts"] == 0
        path = _file(datadir, 28, 8 * MiB + 321)          # the context still serves
        out = ctx.scan_path(path, MiB, blocks=8)
        torch.cuda.synchronize()
        _check_scan(gfs, path, MiB, *out)
