"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: expected values come from the
generator's definition (bytes), brute-force loops, closed forms, hand-derived
traces in tests/golden (with their derivation), and invariants.
"""
import os
import random

import numpy as np
import pytest

import inputs
from oracle import plain, policy

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
P = 4096


def _file(tmp_path, name, seed, size):
    p = str(tmp_path / name)
    inputs.write_file(p, seed, size, 2)
    return p


# ---------------------------------------------------------------- plain definition
@pytest.mark.parametrize("size", [0, 1, P - 1, P, P + 1, 3 * P + 17])
def test_gread_plain_matches_generator(tmp_path, size):
    path = _file(tmp_path, "f", 21, size)
    ref = inputs.xorshift64_bytes(21, size)
    fd = os.open(path, os.O_RDONLY)
    try:
        offs = sorted({0, 1, P - 1, P, P + 1, size - 1, size, size + 1, 2 * P + 5})
        lens = [0, 1, 15, P, P + 1, 3 * P, 10 * P]
        for off in offs:
            if off < 0:
                continue
            for ln in lens:
                n, data = plain.gread_plain(fd, size, off, ln)
                want = ref[off:off + ln]
                assert n == len(want) == max(0, min(ln, size - off))
                assert data == want
    finally:
        os.close(fd)


def test_gread_plain_rejects_negative(tmp_path):
    path = _file(tmp_path, "f", 2, 100)
    fd = os.open(path, os.O_RDONLY)
    assert plain.gread_plain(fd, 100, -1, 4)[0] == -22
    assert plain.gread_plain(fd, 100, 0, -4)[0] == -22
    os.close(fd)


def _sum_loop(data):
    s = 0
    for b in data:
        s += b
    return s % (1 << 64)


def _hash_loop(data, off):
    h = 0
    for i, b in enumerate(data):
        h += b * (off + i + 1)
    return h % (1 << 64)


@pytest.mark.parametrize("off", [0, 1, 4096, (1 << 40) + 3])
def test_checksums_brute_force(off):
    rng = random.Random(off)
    data = bytes(rng.randrange(256) for _ in range(3001))
    assert plain.byte_sum(data) == _sum_loop(data)
    assert plain.pos_hash(data, off) == _hash_loop(data, off)


@pytest.mark.parametrize("c,n,off", [(1, 10, 0), (255, 4096, 0), (7, 1000, 123456), (200, 1 << 20, 1 << 33)])
def test_checksums_closed_form(c, n, off):
    data = bytes([c]) * n
    assert plain.byte_sum(data) == (c * n) % (1 << 64)
    # sum_{i<n} c*(off+i+1) = c*(n*off + n(n+1)/2)
    assert plain.pos_hash(data, off) == (c * (n * off + n * (n + 1) // 2)) % (1 << 64)


def test_hash_wraps_mod_2_64():
    off = (1 << 64) - 10
    data = bytes([255]) * 64
    assert plain.pos_hash(data, off) == _hash_loop(data, off)


def test_hash_detects_swapped_pages():
    # hash(a+b) - hash(b+a) = len(a) * (sum(b) - sum(a)) for equal lengths
    a, b = bytes([1]) * 4096, bytes([2]) * 4096
    assert plain.byte_sum(a + b) == plain.byte_sum(b + a)
    assert plain.pos_hash(a + b, 0) != plain.pos_hash(b + a, 0)


def test_scan_plain_strides(tmp_path):
    size = 5 * 8192 + 100
    path = _file(tmp_path, "s", 9, size)
    ref = inputs.xorshift64_bytes(9, size)
    counts, sums, hashes = plain.scan_plain(path, 8192)
    assert len(counts) == 6
    for s in range(6):
        chunk = ref[s * 8192:(s + 1) * 8192]
        assert counts[s] == len(chunk)
        assert sums[s] == _sum_loop(chunk)
        assert hashes[s] == _hash_loop(chunk, s * 8192)


def test_stride_owner():
    assert plain.stride_owner(0, 64) == (0, 0)
    assert plain.stride_owner(65, 64) == (1, 1)
    assert plain.stride_count(0, 10) == 0 and plain.stride_count(10, 10) == 1 and plain.stride_count(11, 10) == 2


# ---------------------------------------------------------------- policy: data
def _random_trace(rng, size, n, streams, max_len):
    out = []
    for _ in range(n):
        off = rng.randrange(size + 2 * P)
        ln = rng.randrange(max_len + 1)
        out.append((rng.randrange(streams), 0, off, ln))
    return out


@pytest.mark.parametrize("mode", ["readahead", "ondemand"])
@pytest.mark.parametrize("frames,ra_cap,reserve,async_ra,max_rpc", [
    (64, 8, 0, True, 64), (5, 8, 2, True, 64), (3, 1, 0, False, 64), (8, 64, 1, True, 3), (2, 4, 0, True, 64)])
def test_policy_delivers_plain_bytes(tmp_path, mode, frames, ra_cap, reserve, async_ra, max_rpc):
    size = 23 * P + 1234
    path = _file(tmp_path, "p", 31, size)
    ref = inputs.xorshift64_bytes(31, size)
    rng = random.Random(frames * 131 + ra_cap)
    sim = policy.PageCacheSim(P, frames, mode, ra_cap, reserve, async_ra, max_rpc_pages=max_rpc)
    sim.open(0, path)
    seq = [(0, 0, k * 3000, 3000) for k in range(size // 3000 + 2)]
    for stream, fid, off, ln in seq + _random_trace(rng, size, 300, 4, 2 * P + 5):
        n, data = sim.gread(stream, fid, off, ln)
        want = ref[off:off + ln] if off < size else b""
        assert n == len(want)
        assert data == want
    sim.close_all()


def test_policy_rejects_bad_fid_and_args(tmp_path):
    path = _file(tmp_path, "b", 1, 100)
    sim = policy.PageCacheSim(P, 4)
    sim.open(0, path)
    assert sim.gread(0, 3, 0, 10)[0] == -9
    assert sim.gread(0, 0, -1, 10)[0] == -22
    assert sim.gread(0, 0, 100, 10) == (0, b"")
    assert sim.gread(0, 0, 0, 0) == (0, b"")
    sim.close_all()


# ---------------------------------------------------------------- policy: readahead rule
def _parse(name):
    params, rows = {}, []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if parts[0] == "params":
            for kv in parts[1:]:
                k, v = kv.split("=")
                params[k] = v
        else:
            rows.append(parts)
    return params, rows


def test_worked_example_first_window(tmp_path):
    params, rows = _parse("readahead_worked_example.txt")
    page = int([r for r in rows if r[0] == "page_size"][0][1])
    off, ln = map(int, [r for r in rows if r[0] == "read"][0][1:])
    lo, n = map(int, [r for r in rows if r[0] == "expect_first_request"][0][1:])
    path = _file(tmp_path, "w", 5, 64 * page)
    sim = policy.PageCacheSim(page, 64, ra_cap=64, reserve=0)
    sim.open(0, path)
    sim.gread(0, 0, off, ln)
    assert sim.rpc_log[0][1:3] == (lo, n)          # 4 KB read -> 16 KB fetched
    assert sim.rpc_log[0][1] * page == 0 and sim.rpc_log[0][2] * page == 16384
    sim.close_all()


def _windows(tmp_path, ra_cap, async_ra, pages=400, max_rpc=256):
    path = _file(tmp_path, "r%d%d%d" % (ra_cap, async_ra, max_rpc), 6, pages * P)
    sim = policy.PageCacheSim(P, pages + 1, ra_cap=ra_cap, reserve=0, async_ra=async_ra,
                              max_rpc_pages=max_rpc)
    sim.open(0, path)
    for q in range(pages):
        sim.gread(0, 0, q * P, P)
    sim.close_all()
    return sim


def test_window_doubles_async(tmp_path):
    # initial 4x (Section 3.1), then asynchronous windows doubling to Wmax (Section 2.3)
    sim = _windows(tmp_path, 64, True)
    sizes = [n for (_, _, n, _) in sim.rpc_log]
    assert sizes[:8] == [4, 8, 16, 32, 64, 64, 64, 64]
    kinds = [k for (_, _, _, k) in sim.rpc_log]
    assert kinds[0] == policy.SYNC_RA and set(kinds[1:]) == {policy.ASYNC_RA}
    starts = [lo for (_, lo, _, _) in sim.rpc_log]
    assert starts[:6] == [0, 4, 12, 28, 60, 124]
    assert sum(sizes) == 400 and sim.stats.misses == 1


def test_window_cap_one(tmp_path):
    sim = _windows(tmp_path, 1, True, pages=20)
    assert [n for (_, _, n, _) in sim.rpc_log] == [2] + [1] * 18


def test_window_cap_eight(tmp_path):
    sim = _windows(tmp_path, 8, True, pages=60)
    assert [n for (_, _, n, _) in sim.rpc_log][:5] == [4, 8, 8, 8, 8]


def test_window_doubles_sync_only(tmp_path):
    # async off (Section 4.1 synchronous prefetcher): each miss doubles the
    # previous window up to d + Wmax = 65
    sim = _windows(tmp_path, 64, False)
    sizes = [n for (_, _, n, _) in sim.rpc_log]
    assert sizes[:8] == [4, 8, 16, 32, 64, 65, 65, 65]
    assert all(k == policy.SYNC_RA for (_, _, _, k) in sim.rpc_log[:8])
    # and a request never exceeds the slot's page capacity
    sim = _windows(tmp_path, 64, False, max_rpc=64)
    assert [n for (_, _, n, _) in sim.rpc_log][:7] == [4, 8, 16, 32, 64, 64, 64]


def test_not_sequential_fetches_demand_run_only(tmp_path):
    path = _file(tmp_path, "n", 8, 64 * P)
    sim = policy.PageCacheSim(P, 64, ra_cap=8, reserve=0)
    sim.open(0, path)
    sim.gread(0, 0, 10 * P + 5, 2 * P)          # pages 10..12, page 9 absent
    assert sim.rpc_log == [(0, 10, 3, policy.DEMAND)]
    sim.gread(0, 0, 13 * P, P)                  # previous gread of this stream ended at page 13
    assert sim.rpc_log[1] == (0, 13, min(1 + 8, max(4, 2 * 0)), policy.SYNC_RA)
    sim.close_all()


def test_present_predecessor_is_sequential(tmp_path):
    path = _file(tmp_path, "q", 8, 64 * P)
    sim = policy.PageCacheSim(P, 64, ra_cap=8, reserve=0, async_ra=False)
    sim.open(0, path)
    sim.gread(0, 0, 0, P)                       # [0,4) window 4
    sim.gread(1, 0, 4 * P, P)                   # other stream; page 3 present, Tprev 4 -> T = min(9, 8)
    assert sim.rpc_log[1] == (0, 4, 8, policy.SYNC_RA)
    sim.close_all()


def test_window_cut_at_eof_and_present_page(tmp_path):
    path = _file(tmp_path, "e", 8, 10 * P + 7)
    sim = policy.PageCacheSim(P, 64, ra_cap=64, reserve=0)
    sim.open(0, path)
    sim.gread(0, 0, 5 * P, P)                   # not sequential: [5,6)
    sim.gread(1, 0, 0, P)                       # p=0: T=4 but page 5 present: [0,4) ... cut at 5? no: 4 < 5
    sim.gread(2, 0, 4 * P, 1)                   # p=4 mark -> not a miss; hit
    assert sim.rpc_log[0] == (0, 5, 1, policy.DEMAND)
    assert sim.rpc_log[1] == (0, 0, 4, policy.SYNC_RA)
    # page 4 missing: sequential (3 present), Tprev 4 -> T 8, cut at present page 5
    assert sim.rpc_log[2] == (0, 4, 1, policy.DEMAND)
    sim.gread(3, 0, 6 * P, 5 * P)               # pages 6..10 (10 is the 7-byte tail), cut at EOF
    assert sim.rpc_log[3][1:3] == (6, 5)
    sim.close_all()


def test_max_rpc_pages_caps_requests(tmp_path):
    path = _file(tmp_path, "m", 8, 40 * P)
    sim = policy.PageCacheSim(P, 64, ra_cap=64, reserve=0, max_rpc_pages=3)
    sim.open(0, path)
    sim.gread(0, 0, 0, 10 * P)
    assert all(n <= 3 for (_, _, n, _) in sim.rpc_log)
    sim.close_all()


# ---------------------------------------------------------------- plain definition on many cores
def test_pool_scan_equals_the_single_process_scan(tmp_path):
    from oracle import pool
    size = 5 * P * 7 + 333
    path = _file(tmp_path, "pl", 31, size)
    want = plain.scan_plain(path, 3 * P + 5, 2 * P)
    got = pool.scan_plain_parallel(path, 3 * P + 5, 2 * P, procs=3, chunk_bytes=4 * P)
    assert got == want
    assert pool.scan_plain_parallel(path, 3 * P + 5, 2 * P, procs=1, chunk_bytes=4 * P) == want


def test_pool_range_checksums_brute_force(tmp_path):
    from oracle import pool
    size = 9 * P + 7
    path = _file(tmp_path, "pr", 32, size)
    ref = inputs.xorshift64_bytes(32, size)
    for off, ln in ((0, size), (5, 3 * P), (P - 1, 10 * P), (size - 3, 100), (size, 10)):
        data = ref[off:off + ln]
        s = sum(data) % (1 << 64)
        h = sum(b * (off + i + 1) for i, b in enumerate(data)) % (1 << 64)
        assert pool.range_checksums(path, off, ln, procs=2, piece=P + 3) == (len(data), s, h)
    ranges = [(path, 0, size), (path, 7, 2 * P), (path, size + 5, 9)]
    want = [pool.range_checksums(path, o, n, procs=1) for _, o, n in ranges]
    assert pool.many_range_checksums(ranges, procs=3, piece=P) == want


# ---------------------------------------------------------------- policy: hand-derived traces
def _kind(name):
    return {"DEMAND": policy.DEMAND, "SYNC_RA": policy.SYNC_RA, "ASYNC_RA": policy.ASYNC_RA}[name]


def test_golden_stream_small_cache(tmp_path):
    params, rows = _parse("policy_stream_small_cache.txt")
    page, npg = int(params["page_size"]), int(params["file_pages"])
    path = _file(tmp_path, "g1", int(params["seed"]), npg * page)
    sim = policy.PageCacheSim(page, int(params["frames"]), ra_cap=int(params["ra_cap"]),
                              reserve=int(params["reserve"]), async_ra=params["async_ra"] == "1")
    sim.open(0, path)
    reads = [int(x) for x in [r for r in rows if r[0] == "reads"][0][1:]]
    for q in reads:
        assert sim.gread(0, 0, q * page, page)[0] == page
    want_rpc = [(0, int(r[1]), int(r[2]), _kind(r[3])) for r in rows if r[0] == "rpc"]
    want_ev = [(int(r[1]), (0, int(r[2])), (0, int(r[3]))) for r in rows if r[0] == "evict"]
    assert sim.rpc_log == want_rpc
    assert sim.evict_log == want_ev
    assert all(v == 1 for v in sim.stats.fetch_count.values()) and len(sim.stats.fetch_count) == npg
    sim.close_all()


def test_golden_ondemand_fallback(tmp_path):
    params, rows = _parse("policy_ondemand_fallback.txt")
    page, npg = int(params["page_size"]), int(params["file_pages"])
    path = _file(tmp_path, "g2", int(params["seed"]), npg * page)
    sim = policy.PageCacheSim(page, int(params["frames"]), params["mode"], reserve=0)
    sim.open(0, path)
    ref = inputs.xorshift64_bytes(int(params["seed"]), npg * page)
    for r in rows:
        if r[0] == "gread":
            s, off, ln = int(r[1]), int(r[2]), int(r[3])
            n, data = sim.gread(s, 0, off, ln)
            assert data == ref[off:off + ln]
    want_rpc = [(0, int(r[1]), int(r[2]), _kind(r[3])) for r in rows if r[0] == "rpc"]
    want_ev = [(int(r[1]), (0, int(r[2])), (0, int(r[3]))) for r in rows if r[0] == "evict"]
    assert sim.rpc_log == want_rpc
    assert sim.evict_log == want_ev
    unc = int([r for r in rows if r[0] == "unconsumed_evictions"][0][1])
    assert sim.stats.unconsumed_evictions == unc
    sim.close_all()


def test_golden_demand_run_awaited_page_only(tmp_path):
    """Only the page a gread waits for may evict an unconsumed frame; a later page of
    its demand run ends the request (tests/golden/policy_demand_run_awaited_only.txt)."""
    params, rows = _parse("policy_demand_run_awaited_only.txt")
    page, npg = int(params["page_size"]), int(params["file_pages"])
    path = _file(tmp_path, "g3", int(params["seed"]), npg * page)
    sim = policy.PageCacheSim(page, int(params["frames"]), "readahead", ra_cap=int(params["ra_cap"]),
                              reserve=int(params["reserve"]), async_ra=params["async_ra"] == "1")
    sim.open(0, path)
    ref = inputs.xorshift64_bytes(int(params["seed"]), npg * page)
    for r in rows:
        if r[0] == "gread":
            s, off, ln = int(r[1]), int(r[2]), int(r[3])
            n, data = sim.gread(s, 0, off, ln)
            assert n == ln and data == ref[off:off + ln]
    want_rpc = [(0, int(r[1]), int(r[2]), _kind(r[3])) for r in rows if r[0] == "rpc"]
    want_ev = [(int(r[1]), (0, int(r[2])), (0, int(r[3]))) for r in rows if r[0] == "evict"]
    assert sim.rpc_log == want_rpc
    assert sim.evict_log == want_ev
    unc = int([r for r in rows if r[0] == "unconsumed_evictions"][0][1])
    assert sim.stats.unconsumed_evictions == unc
    sim.close_all()


@pytest.mark.parametrize("name", [
    "policy_sequential_by_last_end.txt",   # R3: sequential when the stream's last gread ended at p
    "policy_reread_not_sequential.txt",    # R3: a stream's gread ends at the page after its last
    "policy_gread_keeps_own_frames.txt",   # class 3 never takes a frame the same gread allocated
])
def test_golden_two_streams_and_own_frames(tmp_path, name):
    """Hand-derived traces over two streams and tiny caches: returns, delivered bytes,
    request and eviction logs (tests/golden/<name>)."""
    params, rows = _parse(name)
    page, npg = int(params["page_size"]), int(params["file_pages"])
    path = _file(tmp_path, name[:-4], int(params["seed"]), npg * page)
    sim = policy.PageCacheSim(page, int(params["frames"]), "readahead", ra_cap=int(params["ra_cap"]),
                              reserve=int(params["reserve"]), async_ra=params["async_ra"] == "1")
    sim.open(0, path)
    ref = inputs.xorshift64_bytes(int(params["seed"]), npg * page)
    greads = [(int(r[1]), int(r[2]), int(r[3])) for r in rows if r[0] == "gread"]
    rets = [r for r in rows if r[0] == "ret"]
    assert len(rets) == len(greads)
    for (s, off, ln), r in zip(greads, rets):
        n, data = sim.gread(s, 0, off, ln)
        delivered = int(r[2]) if len(r) > 2 else int(r[1])
        assert n == int(r[1])
        assert data == ref[off:off + delivered]
    want_rpc = [(0, int(r[1]), int(r[2]), _kind(r[3])) for r in rows if r[0] == "rpc"]
    want_ev = [(int(r[1]), (0, int(r[2])), (0, int(r[3]))) for r in rows if r[0] == "evict"]
    assert sim.rpc_log == want_rpc
    assert sim.evict_log == want_ev
    unc = int([r for r in rows if r[0] == "unconsumed_evictions"][0][1])
    assert sim.stats.unconsumed_evictions == unc
    sim.close_all()


# ---------------------------------------------------------------- policy: invariants
def test_fits_each_page_fetched_once(tmp_path):
    # config-1 shape scaled down: file fits the cache -> no eviction, no refetch
    size = 64 * P
    path = _file(tmp_path, "c1", 1, size)
    sim, res = policy.run_scan(path, P, 128, 4 * P, 4, ra_cap=8)
    assert sim.stats.evictions == 0
    assert sorted(sim.stats.fetch_count) == [(0, q) for q in range(64)]
    assert set(sim.stats.fetch_count.values()) == {1}
    c, s, h = plain.scan_plain(path, 4 * P)
    assert [r[0] for r in res] == c and [r[1] for r in res] == s and [r[2] for r in res] == h


def test_ondemand_one_page_per_request(tmp_path):
    size = 50 * P + 3
    path = _file(tmp_path, "od", 2, size)
    sim, res = policy.run_scan(path, P, 128, 3 * P, 5, mode="ondemand")
    assert all(n == 1 and k == policy.DEMAND for (_, _, n, k) in sim.rpc_log)
    assert sim.stats.rpcs == 51


def test_big_file_streams_without_refetch(tmp_path):
    # config-2 shape scaled down: file 8x the cache, disjoint strides per stream
    size = 256 * P
    path = _file(tmp_path, "c2", 2, size)
    blocks, stride = 4, 2 * P
    sim, res = policy.run_scan(path, P, 32, stride, blocks, ra_cap=8)
    assert set(sim.stats.fetch_count.values()) == {1} and len(sim.stats.fetch_count) == 256
    assert sim.stats.unconsumed_evictions == 0
    assert sim.stats.evictions == 256 - 32
    c, s, h = plain.scan_plain(path, stride)
    assert [r[1] for r in res] == s and [r[2] for r in res] == h


def test_random_and_rdwr_disable_readahead(tmp_path):
    path = _file(tmp_path, "rr", 3, 32 * P)
    for kwargs in ({"advice": policy.ADV_RANDOM}, {"readonly": False}):
        sim = policy.PageCacheSim(P, 64, ra_cap=8, reserve=0)
        sim.open(0, path, **kwargs)
        for q in range(8):
            sim.gread(0, 0, q * P, P)
        assert sim.rpc_log == [(0, q, 1, policy.DEMAND) for q in range(8)]
        sim.close_all()


def test_short_host_read_gives_eio(tmp_path):
    path = _file(tmp_path, "sh", 3, 16 * P)

    def short_read(fd, off, n):
        return os.pread(fd, n // 2, off)

    sim = policy.PageCacheSim(P, 16, ra_cap=3, reserve=0, read_fn=short_read)
    sim.open(0, path)
    n, _ = sim.gread(0, 0, 0, P)       # [0,4) requested; only pages 0,1 arrive
    assert n == P
    assert sim.gread(0, 0, 2 * P, P)[0] == -policy.EIO
    sim.close_all()


def test_eviction_never_takes_unconsumed_while_fifo_nonempty(tmp_path):
    # random multi-stream trace on a tiny cache: every unconsumed eviction
    # happens when no free frame and no consumed frame existed
    size = 40 * P
    path = _file(tmp_path, "iv", 4, size)
    rng = random.Random(4)
    sim = policy.PageCacheSim(P, 6, ra_cap=4, reserve=1)
    sim.open(0, path)
    orig = sim._evict

    def checked(f, new_key):
        fr = sim.frames[f]
        if fr.key is not None and fr.consumed < fr.valid:
            assert sim.next_unused == sim.F and not sim.fifo
        orig(f, new_key)

    sim._evict = checked
    for stream, fid, off, ln in _random_trace(rng, size, 400, 3, 3 * P):
        sim.gread(stream, fid, off, ln)
    sim.close_all()


def _streaming_trace(rng, npages, streams, steps):
    """Interleaved sequential readers that start at different places and skip ahead."""
    pos = [rng.randrange(npages) for _ in range(streams)]
    out = []
    for _ in range(steps):
        s = rng.randrange(streams)
        if rng.random() < 0.05:
            pos[s] = rng.randrange(npages)
        out.append((s, 0, pos[s] * P, P))
        pos[s] = (pos[s] + 1) % npages
    return out


def test_readahead_never_refetches(tmp_path):
    # R8 (Section 5.1: data read sequentially is used once): asynchronous
    # readahead only requests pages not fetched since the last reset
    size = 64 * P
    path = _file(tmp_path, "r8", 9, size)
    rng = random.Random(8)
    sim = policy.PageCacheSim(P, 8, ra_cap=8, reserve=1)
    sim.open(0, path)
    for t in _streaming_trace(rng, 64, 3, 600):
        sim.gread(*t)
    seen = set()
    asyncs = 0
    for fid, lo, n, kind in sim.rpc_log:
        pages = {(fid, q) for q in range(lo, lo + n)}
        if kind == policy.ASYNC_RA:
            asyncs += 1
            assert not (pages & seen), "asynchronous readahead refetched a page"
        seen |= pages
    assert asyncs > 0 and sim.stats.evictions > 0
    sim.close_all()


# ---------------------------------------------------------------- application consumers
def test_rowdot_matches_fsum_and_closed_forms(tmp_path):
    import math

    from oracle import apps
    rows, cols = 6, 40
    path = str(tmp_path / "m.f32")
    inputs.write_f32(path, 7, rows * cols)
    a = np.fromfile(path, dtype=np.float32).reshape(rows, cols)
    v = inputs.f32_values(8, cols)
    dot, ab = apps.rowdot(path, rows, cols, v)
    for r in range(rows):
        exact = math.fsum(float(x) * float(y) for x, y in zip(a[r], v))
        assert abs(dot[r] - exact) <= 1e-12 * ab[r]
        assert ab[r] == pytest.approx(math.fsum(abs(float(x) * float(y)) for x, y in zip(a[r], v)), rel=1e-12)
    ones = np.ones(cols, dtype=np.float32)
    dot1, _ = apps.rowdot(path, rows, cols, ones)
    assert np.allclose(dot1, a.astype(np.float64).sum(axis=1), rtol=0, atol=1e-12)   # v = 1: row sums
    dot2, _ = apps.rowdot(path, rows, cols, ones, row_lo=2, row_hi=4)
    assert np.array_equal(dot2, dot1[2:4])
    assert apps.gamma(32768) == pytest.approx(32768 * 2.0 ** -24 / (1 - 32768 * 2.0 ** -24))


def test_histogram_brute_force(tmp_path):
    from collections import Counter

    from oracle import apps
    path = str(tmp_path / "z.i32")
    inputs.write_zipf(path, 8, 5000, 1 << 10, 1.1)
    x = np.fromfile(path, dtype=np.int32)
    counts, out = apps.histogram(path, 1 << 10)
    c = Counter(x.tolist())
    assert out == 0 and int(counts.sum()) == 5000
    assert all(int(counts[k]) == c.get(k, 0) for k in range(1 << 10))
    counts, out = apps.histogram(path, 4)       # values >= 4 are counted as outside
    assert out == sum(v for k, v in c.items() if k >= 4)
    counts, out = apps.histogram(path, 4, piece_values=333)  # read in pieces: same counts
    assert out == sum(v for k, v in c.items() if k >= 4)
    assert all(int(counts[k]) == c.get(k, 0) for k in range(4))


# ---------------------------------------------------------------- paper mode (Sections 4.1, 5.1)
def test_golden_paper_private_buffer(tmp_path):
    params, rows = _parse("policy_paper_private_buffer.txt")
    page, npg = int(params["page_size"]), int(params["file_pages"])
    path = _file(tmp_path, "pp", int(params["seed"]), npg * page)
    sim = policy.PageCacheSim(page, int(params["frames"]), "paper", ra_cap=int(params["prefetch"]), reserve=0,
                              replacement="tb_lra", streams=1)
    sim.open(0, path)
    ref = inputs.xorshift64_bytes(int(params["seed"]), npg * page)
    for q in range(npg):
        n, data = sim.gread(0, 0, q * page, page)
        assert data == ref[q * page:(q + 1) * page]
    assert [(lo, n) for (_, lo, n, _) in sim.rpc_log] == [(int(r[1]), int(r[2])) for r in rows if r[0] == "rpc"]
    assert sim.evict_log == [(int(r[1]), (0, int(r[2])), (0, int(r[3]))) for r in rows if r[0] == "evict"]
    assert sim.stats.buffer_hits == int([r for r in rows if r[0] == "buffer_hits"][0][1])
    sim.close_all()


def test_golden_readahead_with_per_block_lra(tmp_path):
    params, rows = _parse("policy_readahead_tb_lra.txt")
    page, npg = int(params["page_size"]), int(params["file_pages"])
    path = _file(tmp_path, "rl", int(params["seed"]), npg * page)
    sim = policy.PageCacheSim(page, int(params["frames"]), "readahead", ra_cap=int(params["wmax"]), reserve=0,
                              async_ra=False, replacement="tb_lra", streams=int(params["streams"]))
    sim.open(0, path)
    ref = inputs.xorshift64_bytes(int(params["seed"]), npg * page)
    for stream, fid, off, ln in policy.canonical_scan_trace(npg * page, page, int(params["streams"])):
        n, data = sim.gread(stream, fid, off, ln)
        assert n == ln and data == ref[off:off + ln]
    assert [(lo, n) for (_, lo, n, _) in sim.rpc_log] == [(int(r[1]), int(r[2])) for r in rows if r[0] == "rpc"]
    assert all(k == policy.SYNC_RA for (_, _, _, k) in sim.rpc_log)
    assert sim.evict_log == [(int(r[1]), (0, int(r[2])), (0, int(r[3]))) for r in rows if r[0] == "evict"]
    assert sim.next_unused == 2
    sim.close_all()


@pytest.mark.parametrize("mode", ["readahead", "ondemand"])
def test_per_block_lra_with_readahead_keeps_streams_apart(tmp_path, mode):
    # 3 streams, 12 frames: quota 4; every frame a stream takes (demand or
    # readahead) is one it allocated, and it never holds more than its quota
    path = _file(tmp_path, "rq", 6, 90 * P + 17)
    sim = policy.PageCacheSim(P, 12, mode, ra_cap=3, reserve=0, replacement="tb_lra", streams=3)
    sim.open(0, path)
    ref = open(path, "rb").read()
    owner = {}
    for stream, fid, off, ln in policy.canonical_scan_trace(len(ref), 2 * P, 3):
        n, data = sim.gread(stream, fid, off, ln)
        assert data == ref[off:off + ln]
        for s_, dq in sim.lra.items():
            assert len(dq) <= sim.quota == 4
            for f in dq:
                assert owner.setdefault(f, s_) == s_
    assert sim.stats.evictions > 0 and sim.next_unused <= 12
    sim.close_all()


def test_paper_lra_quota_isolates_streams(tmp_path):
    # 2 streams, 4 frames: quota 2; a stream only ever reuses frames it allocated
    path = _file(tmp_path, "pq", 4, 40 * P)
    sim = policy.PageCacheSim(P, 4, "paper", ra_cap=0, reserve=0, replacement="tb_lra", streams=2)
    sim.open(0, path)
    owner = {}
    for step in range(10):
        for s in range(2):
            q = s * 20 + step
            sim.gread(s, 0, q * P, P)
    for s, dq in sim.lra.items():
        assert len(dq) <= sim.quota == 2
        for f in dq:
            assert owner.setdefault(f, s) == s
    for f, old, new in sim.evict_log:
        assert (old[1] < 20) == (new[1] < 20)       # stream 0 pages stay in stream 0 frames
    sim.close_all()


def test_paper_mode_prefetches_duplicates_and_delivers_plain_bytes(tmp_path):
    # no coordination between streams (Section 4.3): neighbouring streams may
    # prefetch the same pages, but every delivered byte is the file's
    size = 37 * P + 11
    path = _file(tmp_path, "pd", 5, size)
    sim, res = policy.run_scan(path, P, 16, 2 * P, 3, mode="paper", ra_cap=3, replacement="tb_lra", keep_data=True)
    c, s, h = plain.scan_plain(path, 2 * P)
    assert [r[0] for r in res] == c and [r[1] for r in res] == s and [r[2] for r in res] == h
    assert max(sim.stats.fetch_count.values()) > 1        # duplicates happen
    assert sim.stats.buffer_hits > 0


@pytest.mark.parametrize("mode,replacement", [("readahead", "fifo"), ("readahead", "tb_lra"), ("ondemand", "fifo"),
                                              ("ondemand", "tb_lra"), ("paper", "fifo"), ("paper", "tb_lra")])
def test_random_configurations_deliver_the_file_and_keep_the_invariants(tmp_path, mode, replacement):
    """Seeded random page sizes, cache sizes, streams, strides and read lengths: every
    gread delivers exactly the file's bytes, every request stays inside the file and the
    request cap, frames never exceed the cache, and a page is never mapped twice."""
    import random
    rng = random.Random(hash((mode, replacement)) & 0xffff)
    for trial in range(6):
        P = rng.choice([4096, 8192, 65536])
        npages = rng.randint(5, 60)
        size = npages * P - rng.randint(0, P - 1)
        path = _file(tmp_path, "rc%d" % trial, 40 + trial, size)
        ref = open(path, "rb").read()
        blocks = rng.randint(1, 5)
        frames = rng.randint(max(blocks * 2, 3), 3 * npages)
        stride = P * rng.randint(1, 4) + rng.choice([0, 0, 17])
        read_len = max(1, stride - rng.choice([0, 1, 100]))
        cap = rng.choice([4, 16])
        sim = policy.PageCacheSim(P, frames, mode, ra_cap=rng.choice([1, 3, 8]), reserve=blocks + 1,
                                  async_ra=rng.random() < 0.5, max_rpc_pages=cap, replacement=replacement,
                                  streams=blocks)
        sim.open(0, path)
        for stream, fid, off, ln in policy.canonical_scan_trace(size, stride, blocks, read_len):
            n, data = sim.gread(stream, fid, off, ln)
            assert n == len(data) == min(ln, max(0, size - off))
            assert data == ref[off:off + n]
            assert len(sim.table) <= frames and len(set(sim.table.values())) == len(sim.table)
        for fid, lo, n, kind in sim.rpc_log:
            assert 0 <= lo and lo + n <= npages and 1 <= n <= cap
        sim.close_all()
