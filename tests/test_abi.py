"""C-ABI library: builds, loads, exports what include/gfs.h and include/gfs_device.h
declare; host logic without a GPU."""
import os
import re

import pytest

import inputs
from paper_2109_05366_gb300 import gfs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gfs.h")
DEVICE_HEADER = os.path.join(ROOT, "include", "gfs_device.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gfs_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = gfs.load()
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(gfs.SIGNATURES), "binding and header disagree"


def _device_declared():
    text = open(DEVICE_HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"__device__\s+[a-z ]+?\s+(g[a-z_]+)\s*\(", text)))


def test_device_library_resolves_every_declared_device_call(tmp_path):
    """A kernel that calls every function include/gfs_device.h declares device-links
    against libgfs_device.a (nvlink fails on an unresolved device symbol); nothing runs."""
    import shutil
    import subprocess
    from paper_2109_05366_gb300 import build
    build.build()
    names = _device_declared()
    assert names == ["gclose", "gfadvise", "gfstat", "gopen", "gread", "gread_as"]
    src = tmp_path / "probe.cu"
    src.write_text("\n".join([
        '#include "gfs_device.h"',
        "__global__ void probe(const __grid_constant__ gfs_dev h, const char* p, char* buf, long long* out) {",
        "  gfs_stat st;",
        "  int fid = gopen(&h, p, GFS_RDONLY);",
        "  long long a = gread(&h, fid, 0, 4096, buf);",
        "  long long b = gread_as(&h, 3, fid, 4096, 4096, buf);",
        "  int c = gfstat(&h, fid, &st) + gfadvise(&h, fid, GFS_ADV_RANDOM) + gclose(&h, fid);",
        "  if (threadIdx.x == 0) out[blockIdx.x] = a + b + c + (long long)st.size;",
        "}",
        'extern "C" int probe_launch(const gfs_dev* h, const char* p, char* buf, long long* out) {',
        "  probe<<<1, 128>>>(*h, p, buf, out);",
        "  return (int)cudaGetLastError();",
        "}"]))
    nvcc = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = str(tmp_path / "probe.so")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-rdc=true", "-shared",
                           "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), str(src), build.DEVLIB,
                           "-o", out])
    assert os.path.getsize(out) > 0


def test_device_handle_fits_the_public_handle_type(tmp_path):
    import subprocess
    c = tmp_path / "h.c"
    c.write_text('#include <stdio.h>\n#include "%s"\nint main(void){printf("%%zu %%zu\\n", sizeof(gfs_dev), '
                 '_Alignof(gfs_dev));return 0;}' % DEVICE_HEADER)
    exe = str(tmp_path / "h")
    subprocess.check_call(["gcc", "-std=c11", "-o", exe, str(c)])
    size, align = [int(x) for x in subprocess.check_output([exe]).split()]
    assert size == 1024 and align == 8


def test_abi_version_and_errors():
    lib = gfs.load()
    assert lib.gfs_abi_version() == 3
    assert lib.gfs_strerror(-22) == b"invalid argument"
    assert lib.gfs_strerror(-110) == b"device wait timed out"


def test_config_defaults():
    c = gfs.default_config()
    assert c.cache_bytes == 1 << 30 and c.page_size == 512 << 10
    assert c.mode == gfs.MODE_READAHEAD and c.ra_cap_pages == 8 and c.async_ra == 1
    assert c.rpc_slots == 128 and c.max_rpc_pages == 64 and c.host_threads == 16


def test_struct_layouts_match_header(tmp_path):
    # compile a C program against include/gfs.h and compare sizes/offsets with ctypes
    import ctypes
    import subprocess
    checks = [("gfs_config", gfs.Config, ["cache_bytes", "page_size", "device", "latency_capacity", "replacement",
                                          "queue", "host_merge_pages", "map_pinned", "self_serve", "reserved"]),
              ("gfs_thread_stat", gfs.ThreadStat, ["requests", "first_request_ns", "bytes"]),
              ("gfs_io_rec", gfs.IoRec, ["offset", "bytes", "fid", "thread", "t_ns"]),
              ("gfs_stat", gfs.Stat, ["size", "advice", "mapped"]),
              ("gfs_stats", gfs.Stats, ["greads", "host_errors", "trace_evict_count", "host_ns_idle", "buffer_hits", "host_controls", "host_merged", "run_cuts", "reserved"]),
              ("gfs_rpc_rec", gfs.RpcRec, ["npages", "page_lo"]),
              ("gfs_evict_rec", gfs.EvictRec, ["new_fid", "new_page"]),
              ("gfs_scan_args", gfs.ScanArgs, ["read_len", "fused", "reserved"])]
    src = ['#include <stdio.h>', '#include <stddef.h>', '#include "%s"' % HEADER, "int main(void){"]
    for cname, _, fields in checks:
        src.append('printf("%%zu\\n", sizeof(%s));' % cname)
        for f in fields:
            src.append('printf("%%zu\\n", offsetof(%s, %s));' % (cname, f))
    src.append("return 0;}")
    c = tmp_path / "l.c"
    c.write_text("\n".join(src))
    exe = str(tmp_path / "l")
    subprocess.check_call(["gcc", "-o", exe, str(c)])
    got = [int(x) for x in subprocess.check_output([exe]).split()]
    want = []
    for _, st, fields in checks:
        want.append(ctypes.sizeof(st))
        want.extend(getattr(st, f).offset for f in fields)
    assert got == want


def test_init_rejects_bad_config_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("host has a GPU")
    with pytest.raises(gfs.GfsError) as e:
        gfs.Context()
    assert e.value.errno == 19  # ENODEV: no device, no crash
    with pytest.raises(gfs.GfsError) as e:
        gfs.Context(page_size=3000)
    assert e.value.errno == 22


@pytest.mark.parametrize("kw,err", [
    # limits a configuration may reach: accepted, so the call goes on to find no device
    (dict(page_size=4096, cache_bytes=((1 << 24) - 1) * 4096), 19),   # the most frames a key can name
    (dict(max_rpc_pages=256, ra_cap_pages=255), 19),                   # the largest request
    (dict(rpc_slots=2), 19),
    (dict(page_size=64 << 20, cache_bytes=64 << 20), 19),              # the largest page, one frame
    (dict(host_threads=256), 19),
    # one step past them: refused before any device call
    (dict(page_size=4096, cache_bytes=(1 << 24) * 4096), 22),
    (dict(max_rpc_pages=257), 22),
    (dict(max_rpc_pages=0), 22),
    (dict(rpc_slots=1), 22),
    (dict(page_size=128 << 20, cache_bytes=128 << 20), 22),
    (dict(page_size=2048), 22),
    (dict(page_size=1 << 20, cache_bytes=(1 << 20) - 1), 22),         # no whole frame
    (dict(host_threads=0), 22),
    (dict(host_threads=257), 22),
    (dict(max_files=0), 22),
    (dict(timeout_ns=0), 22),
    (dict(mode=2, xfer=0), 95),                                        # the paper mode copies its own pages
])
def test_init_limits_without_gpu(kw, err):
    import torch
    if torch.cuda.is_available():
        pytest.skip("host has a GPU")
    with pytest.raises(gfs.GfsError) as e:
        gfs.Context(**kw)
    assert e.value.errno == err


@pytest.mark.parametrize("page,frames,requests,max_pages,threads,slots,size", [
    (4096, 512, 2000, 16, 4, 32, (3 << 20) + 12345),
    (65536, 64, 400, 8, 8, 4, (5 << 20) + 1),
    (4096, 64, 500, 1, 2, 2, 4096 * 10),
    (16384, 256, 300, 64, 16, 128, 7 * 16384 - 5),
])
def test_ring_and_service_selftest(tmp_path, page, frames, requests, max_pages, threads, slots, size):
    path = str(tmp_path / "f.bin")
    inputs.write_file(path, 3, size)
    served = gfs.selftest_ring(path, page, frames, requests, max_pages, threads, slots, seed=7)
    assert served == requests


@pytest.mark.parametrize("threads,max_pages,merge", [(1, 4, 16), (2, 1, 8), (4, 8, 64), (1, 16, 4)])
def test_merged_host_reads_deliver_every_page(tmp_path, threads, max_pages, merge):
    """Section 4.1 has the CPU deliver several pages from one pread; here a host thread
    also takes the requests already waiting behind its own that continue the same file
    range and reads them all at once.  Every page still matches pread, every request is
    served once, and with a backlog some requests are merged."""
    path = str(tmp_path / "f.bin")
    inputs.write_file(path, 9, (2 << 20) + 333)
    served, merged = gfs.selftest_ring(path, 4096, 512, 3000, max_pages, threads, 64, seed=11, merge_pages=merge,
                                       merged=True)
    assert served == 3000
    assert merged > 0
    served, merged = gfs.selftest_ring(path, 4096, 512, 3000, max_pages, threads, 64, seed=11, merge_pages=1,
                                       merged=True)
    assert served == 3000 and merged == 0


@pytest.mark.parametrize("threads,slots,blocks", [(4, 64, 16), (4, 64, 48), (8, 16, 40), (3, 10, 7)])
def test_static_queue_selftest_leaves_unowned_threads_idle(tmp_path, threads, slots, blocks):
    """Section 3.2: with slot = block index and each host thread polling a fixed
    contiguous share of the slots, only the threads whose share holds a client
    block's slot ever serve; every request is still served exactly."""
    path = str(tmp_path / "f.bin")
    inputs.write_file(path, 3, (2 << 20) + 77)
    served, per = gfs.selftest_ring(path, 4096, 512, 1500, 8, threads, slots, seed=5, queue=gfs.QUEUE_STATIC,
                                    client_blocks=blocks, per_thread=True)
    assert served == 1500 and sum(per) == 1500
    used = {b % slots for b in range(blocks)}
    for k in range(threads):
        lo, hi = k * slots // threads, (k + 1) * slots // threads
        owns = any(lo <= s < hi for s in used)
        assert (per[k] > 0) == owns, (k, per)
    served, per = gfs.selftest_ring(path, 4096, 512, 1500, 8, threads, slots, seed=5, per_thread=True)
    assert served == 1500 and sum(per) == 1500


def test_replay_reads_the_recorded_ranges(tmp_path):
    path = str(tmp_path / "f.bin")
    size = (3 << 20) + 5
    inputs.write_file(path, 4, size)
    recs = [(0, 1 << 20), (1 << 20, 1 << 20), (3 << 20, 5), (size - 100, 100), (4096, 0)]
    secs, nbytes = gfs.replay_io(path, recs, 3)
    assert nbytes == sum(b for _, b in recs) and secs >= 0
    secs, nbytes = gfs.replay_io(path, [(size, 4096)], 2)  # past EOF: nothing read, no error
    assert nbytes == 0


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # the product path has no fallback: a missing library is an error
    monkeypatch.setattr(gfs, "_lib", None)
    monkeypatch.setattr(gfs._build, "LIB", str(tmp_path / "nope.so"))
    with pytest.raises(gfs.GfsError):
        gfs.load(build_if_missing=False)


def test_ring_needs_two_slots(tmp_path):
    path = str(tmp_path / "f.bin")
    inputs.write_file(path, 3, 4096 * 4)
    with pytest.raises(gfs.GfsError):
        gfs.selftest_ring(path, 4096, 16, 10, 1, 1, 1)


def test_user_kernel_builds_against_device_api(tmp_path):
    """A user's kernel that includes only include/gfs_device.h and calls gopen / gfadvise /
    gfstat / gread / gclose compiles for sm_103a, links libgfs_device.a and exports its
    launcher."""
    import subprocess

    from tests.devapi_build import build_user_kernel
    so = build_user_kernel(str(tmp_path))
    syms = subprocess.run(["nm", "-D", "--defined-only", so], capture_output=True, text=True, check=True).stdout
    assert " user_scan" in syms
