"""Failures made on the host (never a device fault): slow, short and failing host
reads, a tiny request ring, and a device wait that runs out.  Every kernel must
return, report the failure as a status, and leave the context usable."""
import os

import numpy as np
import pytest

import inputs
from oracle import plain

pytestmark = pytest.mark.gpu

KiB, MiB = 1 << 10, 1 << 20


def _file(datadir, seed, size):
    path = os.path.join(datadir, "f%d_%d.bin" % (seed, size))
    inputs.ensure_file(path, seed, size)
    return path


def _exact(path, stride, cnt, sm, hs):
    c, s, h = plain.scan_plain(path, stride)
    assert list(cnt) == c and list(sm) == s and list(hs) == h


@pytest.mark.parametrize("xfer", [0, 1])
def test_slow_host_reads_still_exact(datadir, xfer):
    from paper_2109_05366_gb300 import gfs
    path = _file(datadir, 21, 24 * MiB + 5)
    with gfs.Context(cache_bytes=8 * MiB, page_size=256 * KiB, xfer=xfer, max_rpc_pages=16, host_threads=4) as ctx:
        fid = ctx.open(path)
        ctx.set_faults(delay_us=3000)
        _exact(path, MiB, *ctx.scan_host(fid, MiB, blocks=8))
        assert ctx.stats()["timeouts"] == 0


@pytest.mark.parametrize("xfer", [0, 1])
def test_short_host_reads_give_eio_then_recover(datadir, xfer):
    from paper_2109_05366_gb300 import gfs
    path = _file(datadir, 22, 16 * MiB)
    with gfs.Context(cache_bytes=32 * MiB, page_size=256 * KiB, xfer=xfer, max_rpc_pages=16) as ctx:
        fid = ctx.open(path)
        ctx.set_faults(short_every=3)
        cnt, sm, hs = ctx.scan_host(fid, MiB, blocks=8)
        c, s, h = plain.scan_plain(path, MiB)
        assert any(x == -5 for x in cnt)
        for i in range(len(c)):
            assert cnt[i] in (c[i], -5)
            if cnt[i] >= 0:
                assert (sm[i], hs[i]) == (s[i], h[i])
        ctx.set_faults()
        ctx.reset_cache()
        _exact(path, MiB, *ctx.scan_host(fid, MiB, blocks=8))


@pytest.mark.parametrize("xfer", [0, 1, 2])
def test_two_slot_ring_backpressure(datadir, xfer):
    from paper_2109_05366_gb300 import gfs
    path = _file(datadir, 23, 20 * MiB + 77)
    with pytest.raises(gfs.GfsError):
        gfs.Context(rpc_slots=1)               # a ring needs two slots (sequence rule)
    # self_serve=0: mapped files' requests go through the two-slot ring too
    with gfs.Context(cache_bytes=16 * MiB, page_size=128 * KiB, xfer=xfer, rpc_slots=2, max_rpc_pages=16,
                     self_serve=0) as ctx:
        fid = ctx.open(path)
        _exact(path, 512 * KiB, *ctx.scan_host(fid, 512 * KiB, blocks=32, threads=128))
        assert ctx.stats()["timeouts"] == 0


@pytest.mark.parametrize("xfer", [0, 1])
def test_device_wait_runs_out_and_context_survives(datadir, xfer):
    # the host is made to stall longer than the device deadline: the gread
    # returns -ETIMEDOUT instead of hanging, and the context keeps working
    from paper_2109_05366_gb300 import gfs
    path = _file(datadir, 24, 2 * MiB)
    with gfs.Context(cache_bytes=8 * MiB, page_size=256 * KiB, xfer=xfer, max_rpc_pages=16, host_threads=2,
                     timeout_ns=300 * 10**6) as ctx:
        fid = ctx.open(path)
        ctx.set_faults(delay_us=1500000)
        cnt, sm, hs = ctx.scan_host(fid, 2 * MiB, blocks=1)
        assert list(cnt) == [-110]
        assert ctx.stats()["timeouts"] >= 1
        ctx.set_faults()
        ctx.reset_cache()                    # waits for the stalled request, then clears
        _exact(path, MiB, *ctx.scan_host(fid, MiB, blocks=2))


@pytest.mark.parametrize("queue", [0, 1])
@pytest.mark.parametrize("xfer", [0, 1])
def test_ring_wait_runs_out_and_the_ticket_is_skipped(datadir, xfer, queue):
    """Two ring slots, one slow host thread and a short device deadline: producers
    give up waiting for a slot after taking their ticket.  Each posts the ticket's
    cancellation and the host skips it, so the ring keeps moving: the reset
    succeeds and the next scan is exact."""
    from paper_2109_05366_gb300 import gfs
    path = _file(datadir, 25, 8 * MiB)
    with gfs.Context(cache_bytes=16 * MiB, page_size=256 * KiB, xfer=xfer, queue=queue, rpc_slots=2,
                     host_threads=1, max_rpc_pages=4, timeout_ns=300 * 10**6) as ctx:
        fid = ctx.open(path)
        ctx.set_faults(delay_us=250000)
        cnt, _, _ = ctx.scan_host(fid, MiB, blocks=8)
        assert (cnt == -110).any()                   # some greads ran out of time
        assert ctx.stats()["timeouts"] >= 1
        ctx.set_faults()
        ctx.reset_cache()                            # every ticket served or skipped
        _exact(path, MiB, *ctx.scan_host(fid, MiB, blocks=8))
        assert ctx.stats()["timeouts"] == 0
