"""Benchmark of the GPU file-read path (one JSON line on stdout, rank 0).

Workload (default): the file-larger-than-cache stride scan -- an 8 GiB seeded
xorshift64 file, 1 GiB GPU page cache, 512 KiB pages, 296 threadblocks (2 per
SM of a 148-SM part; the GB300 has 152), each streaming 1 MiB strides
round-robin and computing a uint64 byte sum + position hash per stride; warm
host page cache.  A step is one whole scan of the file from an empty GPU page
cache.  The file (8 GiB) is far larger than L2, so no L2 flush is needed
between steps.

Reported beside the readahead path, in the same run: the on-demand path (one
page per request, the same steps), the CPU-I/O baseline (host pread threads +
cudaMemcpyAsync + the same checksum kernel), the host-link probes that bound
the path (pinned H2D copy, multi-thread pread, GPU reads of mapped host
memory), the mapped transfer's registration cost, readahead against on-demand
where requests cost something (4 KiB pages; 64 KiB pages with pread staging),
merged against one-request-per-read host service, cold reads (page cache
dropped, O_DIRECT), and the serving loop (Poisson and saturating arrivals).
Last, after every GPU measurement, the CPU-baseline leg: the CPU oracle timed
on a bounded sample, and parity -- every stride of the last timed step and
every serving completion compared with the oracle's plain definition.  These
side measurements run at N = 1; with N > 1 (one replica per rank, each its own
file) the line reports the replicas' rate, the link probes and the roofline.

`--impl reference` times the CPU oracle itself (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

KiB, MiB, GiB = 1 << 10, 1 << 20, 1 << 30

WORKLOADS = {
    # name: (file bytes, seed, page, cache, blocks, stride)
    "cfg2_8GiB_file_1GiB_cache": (8 * GiB, 2, 512 * KiB, 1 * GiB, 296, MiB),
    "cfg1_64MiB_file_128MiB_cache": (64 * MiB, 1, 256 * KiB, 128 * MiB, 64, MiB),
    # same shape as the 8 GiB workload at a quarter of the size (profiling captures)
    "cfg2s_2GiB_file_256MiB_cache": (2 * GiB, 2, 512 * KiB, 256 * MiB, 296, MiB),
    # the same with 4 KiB pages (profiling the per-page cost of small pages)
    "cfg2s4k_2GiB_file_256MiB_cache_4KiB_pages": (2 * GiB, 2, 4 * KiB, 256 * MiB, 296, MiB),
}
DEFAULT_WORKLOAD = "cfg2_8GiB_file_1GiB_cache"
METRIC = "sequential gread GB/s (readahead vs on-demand vs CPU-I/O) + % link roofline; p50/p99 latency"


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi's start-up and first query happen before the steps it watches
            t0 = time.time()
            while not self.lines and self.proc.poll() is None and time.time() - t0 < 5.0:
                time.sleep(0.02)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """Largest value of x over the ranks of the default process group (x itself alone)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(bytes_per_rank_step: int, steps: int, world: int, slowest_total_s: float) -> float:
    """Whole-job GB/s: every rank moves its own bytes; the job takes as long as its slowest rank."""
    return world * steps * bytes_per_rank_step / slowest_total_s / 1e9


def rank_seed(seed: int, rank: int) -> int:
    """Weak scaling by file: rank r scans its own file, generated with seed + r."""
    return seed + rank


def ensure_input(path, seed, size):
    import inputs
    t0 = time.time()
    inputs.ensure_file(path, seed, size)
    # warm host page cache: read it once
    with open(path, "rb", buffering=0) as f:
        while f.read(64 * MiB):
            pass
    return time.time() - t0


def data_dir():
    for d in (os.environ.get("GFS_BENCH_DIR"), "/dev/shm", tempfile.gettempdir()):
        if d and os.path.isdir(d) and os.access(d, os.W_OK):
            return d
    return tempfile.gettempdir()


# DRAM bytes per scanned file byte of k_scan, from an ncu capture of the 2 GiB
# quarter-scale case (traffic grows with the bytes scanned), valid only while the
# kernel's sources are those it was taken on.
NCU_DRAM = {"kernel_digest": "b5b802a1dc751caa76be05a61de6d9d6978dee8bd505b4581b3d22543a8f2275",
            "bytes_per_file_byte": (2.979424e9 + 4.263238e9) / (2 * GiB),
            "source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, 2 GiB case scaled by bytes scanned"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------- reference arm (CPU oracle)
def oracle_sample(path, page, frames, blocks, stride, budget_s, mode="readahead"):
    """Run the oracle over the canonical trace until budget_s; returns (bytes, seconds, strides)."""
    from oracle import plain, policy
    reserve = policy.default_reserve(blocks, stride, page)
    sim = policy.PageCacheSim(page, frames, mode, 8, reserve, True)
    sim.open(0, path)
    size = sim.files[0].size
    done = nbytes = 0
    t0 = time.perf_counter()
    for stream, fid, off, ln in policy.canonical_scan_trace(size, stride, blocks, stride):
        n, data = sim.gread(stream, fid, off, ln)
        plain.byte_sum(data)
        plain.pos_hash(data, off)
        nbytes += max(n, 0)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    sim.close_all()
    return nbytes, dt, done


def serving_files():
    """The serving workload's files: 64 sizes 2^(24+8u) bytes (log-uniform 16 MiB - 4 GiB), seeds 1000+i."""
    import inputs
    from paper_2109_05366_gb300 import serving
    sizes = serving.log_uniform_sizes(64, 24, 32, seed=5)
    paths = []
    for i, sz in enumerate(sizes):
        p = os.path.join(data_dir(), "gfs_serve_%d_%d.bin" % (i, sz))
        inputs.ensure_file(p, 1000 + i, sz)
        paths.append(p)
    return paths, sizes


def peak_admitted(results) -> int:
    """Largest number of requests admitted and not yet complete at one time (device timestamps)."""
    ev = []
    for r in results:
        ev.append((r["t_admit_ns"], 1))
        ev.append((r["t_done_ns"], -1))
    ev.sort(key=lambda e: (e[0], e[1]))  # a completion at the same instant goes first
    cur = best = 0
    for _, d in ev:
        cur += d
        best = max(best, cur)
    return best


def serving_bench(args, xfer, mode, rate_per_s):
    """Config 5: 64 scans over the serving files, Poisson arrivals at rate_per_s (None: all at
    once, saturating), 6 GiB cache.  Returns (summary, per-request results)."""
    import numpy as np
    import torch

    from paper_2109_05366_gb300 import gfs, serving
    paths, sizes = serving_files()
    arrivals = serving.poisson_arrivals(64, rate_per_s, seed=5) if rate_per_s else [0.0] * 64
    with gfs.Context(cache_bytes=6 * GiB, page_size=512 * KiB, mode=mode, xfer=xfer, max_rpc_pages=16,
                     rpc_slots=512, latency_capacity=1 << 20, max_files=80, max_streams=1024) as ctx:
        fids = [ctx.open(p) for p in paths]
        reqs = [(fid, 0, sz) for fid, sz in zip(fids, sizes)]
        stream = torch.cuda.Stream()
        ctx.serve_start(ctas=296, threads=256, unit_bytes=MiB, max_requests=64, queue_slots=128, stream=stream)
        try:
            res, t0 = serving.run(ctx, reqs, arrivals, timeout_s=300)
        finally:
            ctx.serve_stop()
        out = serving.summarize(res, t0)
        out["peak_admitted"] = peak_admitted(res)
        lat = ctx.latencies()
        if len(lat):
            out["gread_p50_us"] = round(float(np.percentile(lat, 50)) / 1e3, 1)
            out["gread_p99_us"] = round(float(np.percentile(lat, 99)) / 1e3, 1)
        out["total_file_bytes"] = int(sum(sizes))
        st = ctx.stats()
        out["timeouts"] = st["timeouts"]
    return out, res


def run_cfg3(args):
    """Config 3: autotuned sweep over a 16 GiB file (one JSON line per result)."""
    import torch

    from paper_2109_05366_gb300 import gfs, tune
    size = 16 * GiB
    path = os.path.join(data_dir(), "gfs_bench_s3_%d.bin" % size)
    ensure_input(path, 3, size)
    results = {"workload": "cfg3_16GiB_sweep", "cache_bytes": 2 * GiB, "strides": {}}
    for stride in (64 * KiB, MiB, 16 * MiB):
        best, allp = tune.tune(path, stride, xfer=gfs.XFER_MAPPED, reps=2)
        print(json.dumps({"stride": stride, "tuning_points": allp}), flush=True)
        cmp = {}
        for label, xf, mode, page in (("mapped_readahead", gfs.XFER_MAPPED, 0, best["page_size"]),
                                      ("mapped_ondemand", gfs.XFER_MAPPED, 1, best["page_size"]),
                                      ("pull_readahead", gfs.XFER_PULL, 0, best["page_size"]),
                                      ("pull_ondemand", gfs.XFER_PULL, 1, best["page_size"]),
                                      ("pull_readahead_64K", gfs.XFER_PULL, 0, 64 * KiB),
                                      ("pull_ondemand_64K", gfs.XFER_PULL, 1, 64 * KiB)):
            pt = dict(best)
            pt.pop("gbps"), pt.pop("ms"), pt.pop("rpcs"), pt.pop("timeouts"), pt.pop("short_strides"), pt.pop("stride")
            pt["page_size"] = page
            cmp[label] = tune.measure(path, stride, pt, xfer=xf, mode=mode, reps=2)["gbps"]
        # the captured steady loop: 4 scans in one graph
        with gfs.Context(cache_bytes=2 * GiB, page_size=best["page_size"], ra_cap_pages=best["ra_cap_pages"],
                         rpc_slots=best["rpc_slots"], xfer=gfs.XFER_MAPPED,
                         max_rpc_pages=min(256, max(16, best["ra_cap_pages"] + stride // best["page_size"] + 1)),
                         max_streams=4096) as ctx:
            fid = ctx.open(path)
            st = torch.cuda.Stream()
            ns = (size + stride - 1) // stride
            out = tuple(torch.empty(ns, dtype=torch.int64, device="cuda") for _ in range(3))
            ctx.scan_graph(fid, stride, 4, blocks=best["blocks"], out=out, stream=st)
            st.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            ctx.scan_graph(fid, stride, 4, blocks=best["blocks"], out=out, stream=st)
            e1.record(st)
            e1.synchronize()
            cmp["graph_loop_4_scans"] = round(4 * size / (e0.elapsed_time(e1) / 1e3) / 1e9, 2)
        d_file = torch.empty(size, dtype=torch.uint8, device="cuda")
        out = tuple(torch.empty((size + stride - 1) // stride, dtype=torch.int64, device="cuda") for _ in range(3))
        t = min(gfs.cpuio_scan(path, stride, stride, 16, 8 * MiB, d_file, out) for _ in range(2))
        cmp["cpuio_16thr"] = round(size / t / 1e9, 2)
        del d_file
        results["strides"][str(stride)] = {"best": best, "compare_gbps": cmp}
        print(json.dumps({"stride": stride, "best": best, "compare_gbps": cmp}), flush=True)
    print(json.dumps(results), flush=True)
    return 0


def run_cfg4(args):
    """Config 4: float32 32768x32768 row dots by 128-row stripes; 8 GiB Zipf int32 histogram.

    Rates only (with the kernels' status and the histogram's total count); every row and
    every bin is checked against the oracle at this size in tests/test_gpu_fullsize.py."""
    import numpy as np
    import torch

    import inputs
    from paper_2109_05366_gb300 import gfs
    rows = cols = 32768
    mpath = os.path.join(data_dir(), "gfs_cfg4_mat_%d.f32" % rows)
    vpath = os.path.join(data_dir(), "gfs_cfg4_vec_%d.f32" % cols)
    zpath = os.path.join(data_dir(), "gfs_cfg4_zipf.i32")
    nz = 1 << 31
    t0 = time.time()
    inputs.ensure_typed(mpath, "f32", 7, rows * cols)
    inputs.ensure_typed(vpath, "f32", 8, cols)
    inputs.ensure_typed(zpath, "zipf", 9, nz, nbins=1 << 20, s=1.1)
    gen_s = time.time() - t0
    vec = np.fromfile(vpath, dtype=np.float32)
    res = {"workload": "cfg4 application streams", "input_gen_s": round(gen_s, 1)}
    stream = torch.cuda.Stream()
    for xname, xf in (("mapped", gfs.XFER_MAPPED), ("pull", gfs.XFER_PULL)):
        with gfs.Context(cache_bytes=GiB, page_size=512 * KiB, xfer=xf, max_rpc_pages=16, rpc_slots=512) as ctx:
            fid = ctx.open(mpath)
            d_vec = torch.from_numpy(vec).cuda()
            ts = []
            for r in range(3):
                ctx.reset_cache(stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                out, ssum, shash, status = ctx.rowdot(fid, rows, cols, d_vec, 128, MiB, blocks=296, stream=stream)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1) / 1e3)
            finite = bool(torch.isfinite(out).all().item())
            res["rowdot_" + xname] = {"gbps": round(rows * cols * 4 / min(ts[1:]) / 1e9, 1), "status": int(status.item()),
                                      "all_finite": finite}
            fz = ctx.open(zpath)
            ts = []
            for r in range(3):
                ctx.reset_cache(stream)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                hist, sums, status = ctx.histogram(fz, 1 << 20, MiB, blocks=296, stream=stream)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1) / 1e3)
            h = hist.cpu().numpy().view(np.uint32).astype(np.uint64)
            res["histogram_" + xname] = {"gbps": round(nz * 4 / min(ts[1:]) / 1e9, 1), "status": int(status.item()),
                                         "total_count": int(h.sum()), "expected": nz,
                                         "outside": int(gfs.u64_view(sums)[1]), "top_bin_frac": round(float(h[0]) / nz, 4)}
    print(json.dumps(res), flush=True)
    return 0


def _resident_fraction(path):
    """Fraction of the file's pages in the host page cache (mincore on a read-only mapping)."""
    import ctypes
    import mmap
    size = os.path.getsize(path)
    if size == 0:
        return 0.0
    libc = ctypes.CDLL(None, use_errno=True)
    libc.mmap.restype = ctypes.c_void_p
    libc.mmap.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_long]
    libc.munmap.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
    libc.mincore.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    fd = os.open(path, os.O_RDONLY)
    try:
        addr = libc.mmap(None, size, mmap.PROT_READ, mmap.MAP_SHARED, fd, 0)
        if addr in (None, ctypes.c_void_p(-1).value):
            return -1.0
        pg = mmap.PAGESIZE
        n = (size + pg - 1) // pg
        vec = (ctypes.c_ubyte * n)()
        rc = libc.mincore(ctypes.c_void_p(addr), size, vec)
        libc.munmap(ctypes.c_void_p(addr), size)
    finally:
        os.close(fd)
    if rc != 0:
        return -1.0
    return sum(v & 1 for v in vec) / n


def run_cold(args):
    """Config 2 cold: the 8 GiB file on the box's disk, host page cache dropped before every scan."""
    import torch

    import inputs
    from paper_2109_05366_gb300 import gfs
    size, seed, page, cache, blocks, stride = WORKLOADS[DEFAULT_WORKLOAD]
    d = os.environ.get("GFS_COLD_DIR", tempfile.gettempdir())
    path = os.path.join(d, "gfs_cold_s%d_%d.bin" % (seed, size))
    inputs.ensure_file(path, seed, size)
    fd = os.open(path, os.O_RDONLY)
    os.fsync(fd)  # written pages must be clean before the cache can drop them
    os.close(fd)
    stream = torch.cuda.Stream()
    res = {"workload": "cfg2 cold: 8 GiB file on disk (%s), page cache dropped (posix_fadvise DONTNEED) "
                       "before each scan" % d}
    out = tuple(torch.empty(size // stride, dtype=torch.int64, device="cuda") for _ in range(3))
    for label, xf, mode in (("pull_readahead", gfs.XFER_PULL, 0), ("pull_ondemand", gfs.XFER_PULL, 1),
                            ("dma_readahead", gfs.XFER_DMA, 0)):
        with gfs.Context(cache_bytes=cache, page_size=page, xfer=xf, mode=mode, max_rpc_pages=16,
                         rpc_slots=512) as ctx:
            fid = ctx.open(path)
            ts, resident = [], []
            for r in range(2):
                ctx.reset_cache(stream)
                f = os.open(path, os.O_RDONLY)
                os.posix_fadvise(f, 0, 0, os.POSIX_FADV_DONTNEED)
                os.close(f)
                resident.append(round(_resident_fraction(path), 4))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ctx.scan(fid, stride, blocks=blocks, out=out, stream=stream)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1) / 1e3)
            ok = bool((out[0][:-1] == stride).all().item())
        res[label] = {"gbps": round(size / min(ts) / 1e9, 2), "resident_before": resident, "counts_ok": ok}
    # the same host read without the GPU: 16 pread threads after dropping the cache
    f = os.open(path, os.O_RDONLY)
    os.posix_fadvise(f, 0, 0, os.POSIX_FADV_DONTNEED)
    os.close(f)
    res["pread_16thr_cold_gbps"] = round(gfs.probe_pread(path, 16, 4 * MiB, 1), 2)
    f = os.open(path, os.O_RDONLY)
    os.posix_fadvise(f, 0, 0, os.POSIX_FADV_DONTNEED)
    os.close(f)
    d_file = torch.empty(size, dtype=torch.uint8, device="cuda")
    res["cpuio_16thr_cold_gbps"] = round(size / gfs.cpuio_scan(path, stride, stride, 16, 8 * MiB, d_file, out) / 1e9, 2)
    print(json.dumps(res), flush=True)
    return 0


def run_paper(args):
    """The paper's microbenchmarks on GB300 (Section 6.1), pread staging (pull) like its CPU threads.

    E9: 120 blocks x 512 threads read 1 GiB of a 10 GiB file, each block its own strides;
        original GPUfs (one page per request) at 4 KiB .. 1 MiB pages vs 4 KiB pages with
        the paper's prefetcher and with this library's readahead.
    E10: the same reading 4 GiB of the file through a 2 GiB cache: original vs
        prefetcher only vs prefetcher + per-block LRA replacement vs this library.
    """
    import torch

    from paper_2109_05366_gb300 import gfs
    size = 10 * GiB
    path = os.path.join(data_dir(), "gfs_paper_s4_%d.bin" % size)
    ensure_input(path, 4, size)
    stream = torch.cuda.Stream()
    res = {"workload": "paper microbenchmarks: 120 blocks x 512 threads, per-block strides, pull transfer"}

    def run(label, read_bytes, cache, page, mode, ra=8, repl=0, reps=2, stride=8 * MiB):
        cfg = dict(cache_bytes=cache, page_size=page, mode=mode, ra_cap_pages=ra, replacement=repl,
                   xfer=gfs.XFER_PULL, max_rpc_pages=min(256, ra + stride // page + 1), rpc_slots=512,
                   max_streams=4096, timeout_ns=5 * 10**9)
        try:
            with gfs.Context(**cfg) as ctx:
                fid = ctx.open(path)
                # read the first read_bytes of the file: strides of `stride` bytes, block b takes b, b+120, ...
                ns = read_bytes // stride
                offs = torch.arange(ns, dtype=torch.int64, device="cuda") * stride
                lens = torch.full((ns,), stride, dtype=torch.int64, device="cuda")
                dsts = (torch.arange(ns, dtype=torch.int64, device="cuda") % 120) * stride
                buf = torch.empty(120 * stride, dtype=torch.uint8, device="cuda")
                ret = torch.empty(ns, dtype=torch.int64, device="cuda")
                ts = []
                for r in range(reps + 1):
                    ctx.reset_cache(stream)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ctx.read_many(fid, offs, lens, dsts, buf, ret, blocks=120, threads=512, stream=stream)
                    e1.record(stream)
                    e1.synchronize()
                    if r:
                        ts.append(e0.elapsed_time(e1) / 1e3)
                st = ctx.stats(stream)
                ok = bool((ret == stride).all().item())
            res[label] = {"gbps": round(read_bytes / min(ts) / 1e9, 2), "rpcs": st["rpcs"],
                          "pages_fetched": st["pages_fetched"], "buffer_hits": st["buffer_hits"],
                          "evictions": st["evictions"], "ok": ok}
        except Exception as e:  # report and go on
            res[label] = {"error": str(e)}
        print(json.dumps({label: res[label]}), flush=True)

    # E9 (files fit: 2 GiB cache, read 1 GiB)
    for page in (4 * KiB, 64 * KiB, MiB):
        run("E9_original_page%dK" % (page // KiB), GiB, 2 * GiB, page, gfs.MODE_ONDEMAND)
    for pf in (15, 255):
        run("E9_paper_prefetcher_4K_prefetch%dK" % ((pf + 1) * 4), GiB, 2 * GiB, 4 * KiB, gfs.MODE_PAPER, ra=pf)
        run("E9_readahead_4K_cap%dK" % ((pf + 1) * 4), GiB, 2 * GiB, 4 * KiB, gfs.MODE_READAHEAD, ra=pf)
    # E10 (4 GiB through a 2 GiB cache)
    for page in (4 * KiB, 64 * KiB):
        k = page // KiB
        run("E10_original_page%dK" % k, 4 * GiB, 2 * GiB, page, gfs.MODE_ONDEMAND)
        run("E10_prefetcher_only_page%dK" % k, 4 * GiB, 2 * GiB, page, gfs.MODE_PAPER, ra=15)
        run("E10_prefetcher_tb_lra_page%dK" % k, 4 * GiB, 2 * GiB, page, gfs.MODE_PAPER, ra=15, repl=1)
        run("E10_readahead_page%dK" % k, 4 * GiB, 2 * GiB, page, gfs.MODE_READAHEAD, ra=15)
        run("E10_readahead_tb_lra_page%dK" % k, 4 * GiB, 2 * GiB, page, gfs.MODE_READAHEAD, ra=15, repl=1)
    print(json.dumps(res), flush=True)
    return 0


def run_random(args):
    """Random small reads and a mixed workload (Section 3.1's Mosaic case, synthetic stand-in).

    The paper's collage application reads 4 KB tiles at data-dependent places of a large
    database while it reads its base picture sequentially; 64 KB pages made it 45 % slower
    than 4 KB pages.  Here: 2^18 reads of 4 KiB at seeded uniform 4 KiB-aligned offsets of
    the 8 GiB bench file, alone and concurrently (second stream) with a sequential scan of a
    1 GiB file, at 4 KiB and 64 KiB pages, with readahead (NORMAL or RANDOM hint on the
    random file) and on-demand.  Mapped transfer, 1 GiB cache.
    """
    import numpy as np
    import torch

    from paper_2109_05366_gb300 import gfs
    db_size, db_seed = WORKLOADS[DEFAULT_WORKLOAD][0], WORKLOADS[DEFAULT_WORKLOAD][1]
    db = os.path.join(data_dir(), "gfs_bench_s%d_%d.bin" % (db_seed, db_size))
    base = os.path.join(data_dir(), "gfs_base_s5_%d.bin" % GiB)
    ensure_input(db, db_seed, db_size)
    ensure_input(base, 5, GiB)
    n, R = 1 << 18, 4 * KiB
    rng = np.random.default_rng(12345)
    offs_h = rng.integers(0, db_size // R, size=n, dtype=np.int64) * R
    offs = torch.from_numpy(offs_h).cuda()
    lens = torch.full((n,), R, dtype=torch.int64, device="cuda")
    dsts = torch.arange(n, dtype=torch.int64, device="cuda") * R
    buf = torch.empty(n * R, dtype=torch.uint8, device="cuda")
    ret = torch.empty(n, dtype=torch.int64, device="cuda")
    dbmap = np.memmap(db, dtype=np.uint8, mode="r")
    sample = rng.choice(n, size=256, replace=False)
    torch.cuda.synchronize()  # inputs written on the current stream before other streams read them
    s_rand, s_seq = torch.cuda.Stream(), torch.cuda.Stream()
    res = {"workload": "random 4 KiB reads (2^18 over 8 GiB) alone and beside a 1 GiB sequential scan; "
                       "mapped transfer, 1 GiB cache, warm host page cache"}

    def check_random():
        if not bool((ret == R).all().item()):
            return False
        got = buf.view(n, R)[torch.from_numpy(sample).cuda()].cpu().numpy()
        return all(np.array_equal(got[i], dbmap[offs_h[j]:offs_h[j] + R]) for i, j in enumerate(sample))

    def ctx_cfg(page, mode):
        ra = max(1, MiB // page - 1) if page < MiB else 8
        return dict(cache_bytes=GiB, page_size=page, mode=mode, ra_cap_pages=min(ra, 255), xfer=gfs.XFER_MAPPED,
                    max_rpc_pages=min(256, MiB // page + 1), rpc_slots=512, host_threads=16,
                    timeout_ns=20 * 10**9)

    def ev_time(fn, stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        return e0, e1

    # Reads alone: 1216 blocks of 128 threads (eight resident per SM: a 4 KiB read costs
    # a block mostly control-path latency, so the reads in flight set the rate), and
    # one row at 296 blocks of 256 threads (two per SM) for comparison.
    rows = [(page, label, mode, hint, 1216, 128) for page in (4 * KiB, 64 * KiB)
            for label, mode, hint in (("readahead", gfs.MODE_READAHEAD, None),
                                      ("readahead_hint_random", gfs.MODE_READAHEAD, gfs.ADV_RANDOM),
                                      ("ondemand", gfs.MODE_ONDEMAND, None))]
    rows.append((4 * KiB, "ondemand_296blocks_256threads", gfs.MODE_ONDEMAND, None, 296, 256))
    res["grid"] = "1216 blocks x 128 threads unless the row says otherwise"
    for page, label, mode, hint, blocks, threads in rows:
        k = page // KiB
        name = "random_page%dK_%s" % (k, label)
        try:
            with gfs.Context(**ctx_cfg(page, mode)) as ctx:
                fid = ctx.open(db)
                if hint is not None:
                    ctx.fadvise(fid, hint)
                ts = []
                for r in range(3):
                    ctx.reset_cache(s_rand)
                    e0, e1 = ev_time(lambda: ctx.read_many(fid, offs, lens, dsts, buf, ret, blocks=blocks,
                                                           threads=threads, stream=s_rand), s_rand)
                    e1.synchronize()
                    if r:
                        ts.append(e0.elapsed_time(e1) / 1e3)
                st = ctx.stats(s_rand)
                ok = check_random()
            t = min(ts)
            res[name] = {"reads_per_s": round(n / t), "useful_gbps": round(n * R / t / 1e9, 2),
                         "fetched_per_useful": round(st["bytes_fetched"] / (n * R), 2), "rpcs": st["rpcs"],
                         "ra_pages": st["ra_pages_sync"] + st["ra_pages_async"], "ok": ok}
        except Exception as e:
            res[name] = {"error": str(e)}
        print(json.dumps({name: res[name]}), flush=True)

    # mixed: sequential base-picture scan (148 blocks, 1 MiB strides) beside the random tiles (148 blocks)
    for page in (4 * KiB, 64 * KiB):
        k = page // KiB
        for label, mode in (("readahead", gfs.MODE_READAHEAD), ("ondemand", gfs.MODE_ONDEMAND)):
            name = "mixed_page%dK_%s" % (k, label)
            try:
                with gfs.Context(**ctx_cfg(page, mode)) as ctx:
                    fdb, fb = ctx.open(db), ctx.open(base)
                    ctx.fadvise(fdb, gfs.ADV_RANDOM)
                    out = None
                    best = None
                    for r in range(3):
                        ctx.reset_cache()
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        a0, a1 = ev_time(lambda: ctx.read_many(fdb, offs, lens, dsts, buf, ret, blocks=148,
                                                               threads=256, stream=s_rand), s_rand)
                        b0, b1 = ev_time(lambda: ctx.scan(fb, MiB, blocks=148, threads=256, fused=True,
                                                          stream=s_seq), s_seq)
                        a1.synchronize()
                        b1.synchronize()
                        wall = time.perf_counter() - t0
                        out = (a0.elapsed_time(a1) / 1e3, b0.elapsed_time(b1) / 1e3, wall)
                        if r and (best is None or out[2] < best[2]):
                            best = out
                    ok = check_random()
                    cnt = ctx.scan(fb, MiB, blocks=148, fused=True)[0]
                    torch.cuda.synchronize()
                    ok = ok and bool((cnt == MiB).all().item())
                res[name] = {"random_reads_per_s": round(n / best[0]), "seq_gbps": round(GiB / best[1] / 1e9, 2),
                             "wall_s": round(best[2], 4), "ok": ok}
            except Exception as e:
                res[name] = {"error": str(e)}
            print(json.dumps({name: res[name]}), flush=True)
    print(json.dumps(res), flush=True)
    return 0


def run_queue(args):
    """Section 3.2 on GB300: the GPUfs static queue (slot = block index, each host thread
    polls a fixed contiguous share of the slots) against the shared ring, and the host
    I/O trace replayed by CPU threads alone.

    The paper's case: 128 slots, 4 host threads of 32 slots, 120 blocks of which only 60
    are resident, so two threads wait for requests while the others work.  Here: the
    8 GiB bench file, 1 MiB strides, 1024 slots, 16 host threads of 64 slots, and more
    blocks (512 threads) than the GPU holds at once; pull transfer (the host threads
    pread, as GPUfs's do) and mapped transfer.
    """
    import torch

    from paper_2109_05366_gb300 import gfs
    size, seed = WORKLOADS[DEFAULT_WORKLOAD][0], WORKLOADS[DEFAULT_WORKLOAD][1]
    path = os.path.join(data_dir(), "gfs_bench_s%d_%d.bin" % (seed, size))
    ensure_input(path, seed, size)
    props = torch.cuda.get_device_properties(0)
    blocks = 2 * props.multi_processor_count * (props.max_threads_per_multi_processor // 512)
    res = {"workload": "8 GiB file, 1 MiB strides, %d blocks x 512 threads (more than fit at once), 1024 slots, "
                       "16 host threads, 1 GiB cache, warm host page cache" % blocks}
    stream = torch.cuda.Stream()
    for xfer_name, xfer in (("pull", gfs.XFER_PULL), ("mapped", gfs.XFER_MAPPED)):
        for page in (64 * KiB, 256 * KiB):
            for qname, queue in (("shared", gfs.QUEUE_SHARED), ("static", gfs.QUEUE_STATIC)):
                name = "%s_page%dK_%s" % (xfer_name, page // KiB, qname)
                try:
                    cfg = dict(cache_bytes=GiB, page_size=page, xfer=xfer, queue=queue, rpc_slots=1024,
                               host_threads=16, max_rpc_pages=min(256, MiB // page * 2), ra_cap_pages=MiB // page,
                               trace_capacity=(1 << 20) if queue == gfs.QUEUE_SHARED else 0,
                               timeout_ns=30 * 10**9, self_serve=0)  # the study is of host service
                    with gfs.Context(**cfg) as ctx:
                        fid = ctx.open(path)
                        best = None
                        for r in range(3):
                            ctx.reset_cache(stream)
                            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                            e0.record(stream)
                            out = ctx.scan(fid, MiB, blocks=blocks, threads=512, fused=True, stream=stream)
                            e1.record(stream)
                            e1.synchronize()
                            t = e0.elapsed_time(e1) / 1e3
                            if r and (best is None or t < best):
                                best = t
                                ts = ctx.thread_stats()
                                recs = ctx.io_trace() if queue == gfs.QUEUE_SHARED else []
                        ok = bool((out[0] == MiB).all().item())
                    req = [t_["requests"] for t_ in ts]
                    entry = {"gbps": round(size / best / 1e9, 2), "ok": ok,
                             "requests_per_thread": req,
                             "first_request_ms": [round(t_["first_request_ns"] / 1e6, 3) for t_ in ts],
                             "polls_before_first": [t_["polls_before_first"] for t_ in ts],
                             "idle_threads": sum(1 for q in req if q == 0)}
                    if recs:  # the same file ranges, pread by 16 CPU threads without the GPU
                        secs, nbytes = gfs.replay_io(path, recs, 16)
                        entry["replay_cpu_gbps"] = round(nbytes / secs / 1e9, 2)
                        entry["replay_ranges"] = len(recs)
                    res[name] = entry
                except Exception as e:
                    res[name] = {"error": str(e)}
                print(json.dumps({name: res[name]}), flush=True)
    print(json.dumps(res), flush=True)
    return 0


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    size, seed, page, cache, blocks, stride = WORKLOADS[args.workload]
    path = os.path.join(data_dir(), "gfs_bench_s%d_%d.bin" % (seed, size))
    ensure_input(path, seed, size)
    budget = args.ref_step_seconds
    for _ in range(args.warmup):
        oracle_sample(path, page, cache // page, blocks, stride, budget / 4)
    tot_b = tot_t = 0.0
    strides = 0
    for _ in range(args.steps):
        b, t, n = oracle_sample(path, page, cache // page, blocks, stride, budget)
        tot_b += b
        tot_t += t
        strides += n
    gbps = tot_b / tot_t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": round(gbps, 4), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * tot_t / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": args.workload, "file_bytes": size, "page_bytes": page, "cache_bytes": cache,
                   "blocks": blocks, "stride_bytes": stride, "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": round(gbps, 4), "unit": "GB/s", "cores": 1, "host_cores": os.cpu_count(),
                         "kind": "oracle", "sample": "first %d strides of the canonical trace per step (%.0f s budget)" % (
                             strides // max(args.steps, 1), budget)},
        "e2e": {"value": round(gbps, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- the GPU path
def xfer_code(name):
    from paper_2109_05366_gb300 import gfs
    return {"pull": gfs.XFER_PULL, "dma": gfs.XFER_DMA, "mapped": gfs.XFER_MAPPED}[name]


def scan_leg(path, stride, blocks, steps, warmup, stream, threads=256, fused=False, open_flags=0, before=None,
             **cfg):
    """Time `steps` scans of `path` (after `warmup` untimed ones), each from an empty GPU page
    cache, in a context of its own; every scan's counts are checked.  `before(i)` runs before
    scan i outside the timed region (e.g. dropping the host page cache).  Returns a dict."""
    import torch

    from paper_2109_05366_gb300 import gfs
    size = os.path.getsize(path)
    ns = (size + stride - 1) // stride
    out = tuple(torch.empty(ns, dtype=torch.int64, device="cuda") for _ in range(3))
    ts, ok = [], True
    with gfs.Context(**cfg) as ctx:
        fid = ctx.open(path, open_flags)
        mapped = int(ctx.fstat(fid).mapped)
        for i in range(warmup + steps):
            ctx.reset_cache(stream)
            if before:
                before(i)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.scan(fid, stride, blocks=blocks, threads=threads, fused=fused, out=out, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if i >= warmup:
                ts.append(e0.elapsed_time(e1) / 1e3)
            cnt = out[0].cpu().numpy()
            ok = ok and bool((cnt[:-1] == stride).all()) and int(cnt[-1]) == size - (ns - 1) * stride
        st = ctx.stats(stream)
    t = sum(ts) / len(ts)
    return {"gbps": round(size / t / 1e9, 2), "ms": round(1e3 * t, 3), "steps": steps, "counts_ok": ok,
            "rpcs": st["rpcs"], "host_preads": st["host_preads"], "host_merged": st["host_merged"],
            "timeouts": st["timeouts"], "mapped": mapped}


def ra_vs_od_legs(args, stream):
    """Readahead against on-demand, the same steps each, where a request costs something:
    4 KiB pages (the paper's page size, Section 6.1) with the mapped transfer, and 64 KiB
    pages with host pread staging (pull), as GPUfs's host threads read."""
    from paper_2109_05366_gb300 import gfs
    res = {}
    steps, warmup = max(1, min(args.steps, 5)), 1
    small = os.path.join(data_dir(), "gfs_bench_s2_%d.bin" % (2 * GiB))
    ensure_input(small, 2, 2 * GiB)
    big = os.path.join(data_dir(), "gfs_bench_s2_%d.bin" % (8 * GiB))
    ensure_input(big, 2, 8 * GiB)
    for name, path, page, cache, xf, ra, mx in (
            ("page4KiB_mapped_2GiB_file_256MiB_cache", small, 4 * KiB, 256 * MiB, gfs.XFER_MAPPED, 63, 64),
            ("page64KiB_pull_8GiB_file_1GiB_cache", big, 64 * KiB, GiB, gfs.XFER_PULL, 15, 32)):
        entry = {}
        for label, mode in (("readahead", gfs.MODE_READAHEAD), ("ondemand", gfs.MODE_ONDEMAND)):
            entry[label] = scan_leg(path, MiB, 296, steps, warmup, stream, cache_bytes=cache, page_size=page, mode=mode,
                                    xfer=xf, ra_cap_pages=ra, max_rpc_pages=mx, rpc_slots=512)
        entry["readahead_over_ondemand"] = round(entry["readahead"]["gbps"] / entry["ondemand"]["gbps"], 2)
        res[name] = entry
    return res


def merge_legs(args, path, stream):
    """Host reads merged across requests against one request per read, for the transfers whose
    host threads pread (pull, dma), on the 8 GiB file: the bench's shape (512 KiB pages,
    readahead, 1 MiB strides), and 64 KiB pages on demand with 64 KiB strides, where
    neighbouring threadblocks ask for neighbouring pages at once (one page per request)."""
    from paper_2109_05366_gb300 import gfs
    size = os.path.getsize(path)
    res = {}
    for xname in ("pull", "dma"):
        for page, stride, mode, mname in ((512 * KiB, MiB, gfs.MODE_READAHEAD, "readahead"),
                                          (64 * KiB, 64 * KiB, gfs.MODE_ONDEMAND, "ondemand")):
            key = "%s_page%dKiB_stride%dKiB_%s" % (xname, page // KiB, stride // KiB, mname)
            entry = {}
            for label, merge in (("one_request_per_read", 1), ("merged", 0)):
                r = scan_leg(path, stride, 296, 2, 1, stream, cache_bytes=GiB, page_size=page, mode=mode,
                             xfer=xfer_code(xname), ra_cap_pages=8, max_rpc_pages=16, rpc_slots=512,
                             host_merge_pages=merge)
                r["host_preads_per_GiB"] = round(r["host_preads"] / (size / GiB), 1)
                entry[label] = r
            entry["merged_over_one_per_read"] = round(entry["merged"]["gbps"] / entry["one_request_per_read"]["gbps"], 3)
            res[key] = entry
    return res


def mapped_open_close(path):
    """Cost of mapping a file for the GPU in gfs_open and unmapping it in gfs_close: through
    the host page tables (read-only, nothing pinned) and by registration (pins every page)."""
    from paper_2109_05366_gb300 import gfs
    out = {}
    for label, pinned in (("host_page_tables", 0), ("pinned", 1)):
        with gfs.Context(cache_bytes=GiB, page_size=512 * KiB, map_pinned=pinned) as ctx:
            t0 = time.perf_counter()
            fid = ctx.open(path)
            t1 = time.perf_counter()
            mapped = int(ctx.fstat(fid).mapped)
            ctx.close(fid)
            t2 = time.perf_counter()
        out[label] = {"open_s": round(t1 - t0, 4), "close_s": round(t2 - t1, 4), "mapped": mapped}
    return out


def _drop_host_cache(path):
    fd = os.open(path, os.O_RDONLY)
    try:
        os.posix_fadvise(fd, 0, 0, os.POSIX_FADV_DONTNEED)
    finally:
        os.close(fd)


def cold_legs(args, stream):
    """Cold reads of a 2 GiB file on the box's disk: the host page cache dropped before every
    scan (posix_fadvise DONTNEED, checked with mincore), and O_DIRECT reads (GFS_DIRECT)."""
    import torch

    import inputs
    from paper_2109_05366_gb300 import gfs
    d = os.environ.get("GFS_COLD_DIR", tempfile.gettempdir())
    size = 2 * GiB
    path = os.path.join(d, "gfs_cold_s6_%d.bin" % size)
    probe = os.path.join(d, "gfs_cold_probe")
    try:
        with open(probe, "wb") as f:
            f.write(b"\0" * 4096)
        fd = os.open(probe, os.O_RDONLY | os.O_DIRECT)
        os.close(fd)
    except OSError as e:
        return {"unavailable": "no O_DIRECT under %s (%s): no disk-backed file system to read cold from" % (d, e)}
    finally:
        if os.path.exists(probe):
            os.unlink(probe)
    t0 = time.time()
    inputs.ensure_file(path, 6, size)
    fd = os.open(path, os.O_RDONLY)
    os.fsync(fd)  # written pages must be clean before the cache can drop them
    os.close(fd)
    res = {"file": "2 GiB seeded file under %s (not tmpfs)" % d, "input_s": round(time.time() - t0, 1)}
    resident = []

    def drop(i):
        _drop_host_cache(path)
        resident.append(round(_resident_fraction(path), 4))

    for label, xf, mode, flags in (("pull_readahead", gfs.XFER_PULL, 0, 0), ("pull_ondemand", gfs.XFER_PULL, 1, 0),
                                   ("pull_readahead_direct", gfs.XFER_PULL, 0, gfs.DIRECT),
                                   ("dma_readahead_direct", gfs.XFER_DMA, 0, gfs.DIRECT),
                                   ("mapped_default_readahead", gfs.XFER_MAPPED, 0, 0)):
        resident.clear()
        _drop_host_cache(path)  # before the open too: a resident file would be mapped (and pinned)
        try:
            r = scan_leg(path, MiB, 296, 2, 0, stream, open_flags=flags, before=None if flags else drop,
                         cache_bytes=256 * MiB, page_size=512 * KiB, mode=mode, xfer=xf, max_rpc_pages=16,
                         rpc_slots=512)
            if not flags:
                r["resident_before_each_scan"] = list(resident)
            res[label] = r
        except Exception as e:  # report and go on
            res[label] = {"error": str(e)}
    _drop_host_cache(path)
    res["pread_16thr_cold_gbps"] = round(gfs.probe_pread(path, 16, 4 * MiB, 1), 2)
    _drop_host_cache(path)
    d_file = torch.empty(size, dtype=torch.uint8, device="cuda")
    out = tuple(torch.empty(size // MiB, dtype=torch.int64, device="cuda") for _ in range(3))
    res["cpuio_16thr_cold_gbps"] = round(size / gfs.cpuio_scan(path, MiB, MiB, 16, 8 * MiB, d_file, out) / 1e9, 2)
    return res


def oracle_checks(path, stride, last, serving_results, cpu_seconds, workload):
    """The CPU-baseline leg, after every GPU measurement: (1) the oracle as it stands timed on one
    host core on a bounded sample of the workload; (2) parity: every stride of the last timed
    step, and every serving completion, against the oracle's plain definition computed on all
    host cores (worker processes started by spawn)."""
    from oracle import pool
    size_, seed_, page_, cache_, blocks_, stride_ = WORKLOADS[workload]
    b, t, n = oracle_sample(path, page_, cache_ // page_, blocks_, stride_, cpu_seconds)
    cpu = {"value": round(b / t / 1e9, 4), "unit": "GB/s", "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
           "sample": "first %d strides (%d MiB) of the canonical trace, %.1f s" % (n, b // MiB, t)}
    t0 = time.perf_counter()
    c, s, h = pool.scan_plain_parallel(path, stride)
    import numpy as np
    cnt, sm, hs = last
    bad = int(np.count_nonzero(cnt[:len(c)] != np.array(c, dtype=np.int64)) +
              np.count_nonzero(sm[:len(s)].view(np.uint64) != np.array(s, dtype=np.uint64)) +
              np.count_nonzero(hs[:len(h)].view(np.uint64) != np.array(h, dtype=np.uint64)))
    parity = {"timed_step": {"strides": len(c), "fields_checked": 3 * len(c), "mismatches": bad,
                             "exact": bad == 0 and len(cnt) >= len(c),
                             "against": "oracle/plain.py per stride (count, byte sum, position hash)",
                             "oracle_s": round(time.perf_counter() - t0, 1), "oracle_procs": pool.workers()}}
    if serving_results:
        paths, sizes = serving_files()
        t0 = time.perf_counter()
        want = pool.many_range_checksums([(p, 0, sz) for p, sz in zip(paths, sizes)])
        for label, res in serving_results.items():
            wrong = sum(1 for i, r in enumerate(res)
                        if r["status"] != 0 or (r["bytes"], r["sum"], r["hash"]) != want[i])
            parity["serving_" + label] = {"completions": len(res), "mismatches": wrong, "exact": wrong == 0}
        parity["serving_oracle_s"] = round(time.perf_counter() - t0, 1)
    return cpu, parity


def run_gfs(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import inputs

    from paper_2109_05366_gb300 import gfs

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    size, seed, page, cache, blocks, stride = WORKLOADS[args.workload]
    if args.blocks:
        blocks = args.blocks
    # weak scaling: every rank scans its own file (seed + rank), no data-path collective
    path = os.path.join(data_dir(), "gfs_bench_s%d_%d.bin" % (rank_seed(seed, rank), size))
    gen_s = ensure_input(path, rank_seed(seed, rank), size)
    resident = round(_resident_fraction(path), 4)  # warm run: the file sits in the host page cache (mincore)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    nstr = (size + stride - 1) // stride
    out = tuple(torch.empty(nstr, dtype=torch.int64, device=dev) for _ in range(3))
    peaks = measured_peaks()

    def timed_scans(ctx, fid, steps, warmup, fused=False):
        ev = []
        for i in range(warmup + steps):
            ctx.reset_cache(stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize(dev)
            e0.record(stream)
            ctx.scan(fid, stride, blocks=blocks, threads=args.threads, fused=fused, out=out, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if i >= warmup:
                ev.append(e0.elapsed_time(e1) / 1e3)
        return ev

    cfg = dict(cache_bytes=cache, page_size=page, host_threads=args.host_threads, ra_cap_pages=args.ra_cap,
               latency_capacity=1 << 16,
               rpc_slots=args.rpc_slots, staging_bytes=args.staging_mib * MiB, max_rpc_pages=args.max_rpc_pages,
               xfer=xfer_code(args.xfer))
    with gfs.Context(mode=gfs.MODE_READAHEAD, **cfg) as ctx:
        fid = ctx.open(path)
        with ClockSampler(local) as clk:
            if world > 1:
                dist.barrier()
            times = timed_scans(ctx, fid, args.steps, args.warmup, fused=args.fused)
        st = ctx.stats(stream)
        lat = ctx.latencies(stream)
        # the last timed step's results, checked stride for stride against the oracle below
        last = tuple(t.cpu().numpy().copy() for t in out)
        cnt = last[0]
        assert (cnt[:-1] == stride).all() and cnt[-1] == size - (nstr - 1) * stride, "scan returned short counts"
        mapped = int(ctx.fstat(fid).mapped)
        # e2e: the C-ABI call with host result buffers, wall clock, cache reset outside
        e2e_t = []
        for _ in range(max(1, min(args.steps, 3))):
            ctx.reset_cache(stream)
            t0 = time.perf_counter()
            ctx.scan_host(fid, stride, blocks=blocks, threads=args.threads, fused=args.fused, stream=stream)
            e2e_t.append(time.perf_counter() - t0)
    total = max_over_ranks(sum(times), dist if world > 1 else None, dev)
    value = job_rate(size, args.steps, world, total)

    extra = {}
    binding, binding_src = None, None
    # the side measurements (baselines, other legs, serving, the CPU oracle) run at
    # N = 1 only: with N > 1 the line carries the replicas' rate, the link probes and
    # the roofline, and no rank's GPU is held while rank 0 measures more
    side = world == 1
    if rank == 0 and not args.quick and not side:
        extra["side_measurements"] = "at N=1 only"
    if rank == 0 and not args.quick:
        if side:
            with gfs.Context(mode=gfs.MODE_ONDEMAND, **cfg) as ctx:
                fid = ctx.open(path)
                od = timed_scans(ctx, fid, args.steps, args.warmup)
            extra["ondemand_gbps"] = round(size / (sum(od) / len(od)) / 1e9, 2)
            extra["ondemand_steps"] = len(od)
            d_file = torch.empty(size, dtype=torch.uint8, device=dev)
            cpu_t = []
            for i in range(3):
                cpu_t.append(gfs.cpuio_scan(path, stride, stride, args.host_threads, 8 * MiB, d_file, out, stream))
            extra["cpuio_gbps"] = round(size / min(cpu_t[1:]) / 1e9, 2)
            extra["cpuio_threads"] = args.host_threads
            one = gfs.cpuio_scan(path, stride, stride, 1, size, d_file, out, stream)
            extra["cpuio_naive_1thread_gbps"] = round(size / one / 1e9, 2)
            # context: the same checksums on the host alone, every core (pread + sums, no GPU)
            ncpu = os.cpu_count() or 1
            cs = min(gfs.cpu_scan(path, stride, stride, ncpu)[3] for _ in range(2))
            extra["cpu_scan"] = {"gbps": round(size / cs / 1e9, 2), "threads": ncpu,
                                 "kind": "host threads pread each stride and checksum it, no GPU (gfs_cpu_scan)"}
            t0 = time.perf_counter()
            extra["input_digest"] = {"file_bytes": size, "sha256_of_64MiB_piece_sha256s": inputs.file_digest(path),
                                     "s": round(time.perf_counter() - t0, 2)}
            del d_file
        h2d = gfs.probe_h2d(GiB, 16 * MiB, 3)
        h2d_page = gfs.probe_h2d(GiB, page, 3)
        prd = gfs.probe_pread(path, 16, 4 * MiB, 2)
        # the same preads into 64 MiB buffers per thread (1 GiB in all, larger than the
        # CPU's caches): what a pread costs when its destination lives in host DRAM
        prd_dram = gfs.probe_pread(path, 16, 64 * MiB, 2)
        pull = gfs.probe_pull(GiB, 3)
        extra["link_probe"] = {"h2d_pinned_16MiB_gbps": round(h2d, 1), "h2d_pinned_page_gbps": round(h2d_page, 1),
                               "pread_16thr_gbps": round(prd, 1), "pread_16thr_64MiB_buffers_gbps": round(prd_dram, 1),
                               "gpu_read_host_gbps": round(pull, 1)}
        # the link the chosen transfer moves data over: mapped = GPU reads of host
        # memory; pull = host pread + GPU reads; dma = host pread + copy engine
        if args.xfer == "mapped" and mapped:
            binding, binding_src = pull, "GPU threads reading mapped host memory"
        elif args.xfer in ("mapped", "pull"):
            binding, binding_src = min(pull, prd), "min(GPU reads of host memory, 16-thread pread)"
        else:
            binding, binding_src = min(h2d, prd), "min(pinned H2D copy, 16-thread pread)"
        if side and args.xfer == "mapped":
            oc = mapped_open_close(path)
            e2e_mean = sum(e2e_t) / len(e2e_t)
            for v in oc.values():  # one open, one scan through the C ABI, one close
                v["e2e_open_scan_close_gbps"] = round(size / (v["open_s"] + e2e_mean + v["close_s"]) / 1e9, 2)
            extra["mapped_open_close"] = oc
        if side and not args.no_extras:
            for key, fn in (("readahead_vs_ondemand", lambda: ra_vs_od_legs(args, stream)),
                            ("host_merge", lambda: merge_legs(args, path, stream)),
                            ("cold", lambda: cold_legs(args, stream))):
                try:
                    extra[key] = fn()
                except Exception as e:  # a side measurement must not cost the bench line
                    extra[key] = {"error": "%s: %s" % (type(e).__name__, e)}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0
    clocks = clk.summary()
    nbytes_hbm = 4 * size  # frame write (DMA) + frame read + user write + user read
    kt = sum(times) / len(times)
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": "GB/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(1e3 * kt, 3),
        "median_ms_per_step": round(1e3 * statistics.median(times), 3), "step_ms": [round(1e3 * t, 2) for t in times],
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic (seeded xorshift64 file, warm host page cache)",
        "config": {"workload": args.workload, "file_bytes": size, "page_bytes": page, "cache_bytes": cache,
                   "blocks": blocks, "threads": args.threads, "stride_bytes": stride, "ra_cap_pages": args.ra_cap,
                   "host_threads": args.host_threads, "rpc_slots": args.rpc_slots, "fused": bool(args.fused),
                   "xfer": args.xfer, "mapped": mapped, "max_rpc_pages": args.max_rpc_pages,
                   "l2": "inputs larger than L2 (%d MiB file); no flush" % (size // MiB),
                   "host_page_cache_resident": resident,
                   "parallelism": "replicas" if world > 1 else "1gpu"},
        "clocks": clocks,
        "e2e": {"value": round(size / (sum(e2e_t) / len(e2e_t)) / 1e9, 3), "unit": "GB/s",
                "h2d_bytes_per_step": size, "d2h_bytes_per_step": nstr * 24},
        "gpu_launches": args.steps,
        "stats_last_step": {k: st[k] for k in ("rpcs", "pages_fetched", "hits", "misses", "coalesced_waits",
                                               "ra_pages_sync", "ra_pages_async", "evictions",
                                               "unconsumed_evictions", "timeouts", "eio", "host_merged")},
        "input_gen_s": round(gen_s, 1),
    }
    if len(lat):
        line["gread_latency_us"] = {"p50": round(float(np.percentile(lat, 50)) / 1e3, 1),
                                    "p99": round(float(np.percentile(lat, 99)) / 1e3, 1),
                                    "greads": int(len(lat)), "read_len": stride}
    if binding:
        from paper_2109_05366_gb300 import build as _b
        traffic = None
        if (_b.kernel_digest() == NCU_DRAM["kernel_digest"] and args.xfer == "mapped" and mapped and not args.fused
                and args.workload == DEFAULT_WORKLOAD):
            traffic = int(NCU_DRAM["bytes_per_file_byte"] * size)  # DRAM bytes per launch
        line["roofline"] = {"bound": "link", "achieved": round(value / world, 2), "peak": round(binding, 1),
                            "unit": "GB/s", "frac": round(value / world / binding, 3), "traffic": traffic,
                            "traffic_source": NCU_DRAM["source"] if traffic else None,
                            "peak_source": "measured in this run: " + binding_src}
        hbm = peaks.get("hbm_gbs", 6800.0)
        line["hbm_roofline"] = {"bound": "hbm", "achieved": round(nbytes_hbm / kt / 1e9, 1), "peak": hbm,
                                "unit": "GB/s", "frac": round(nbytes_hbm / kt / 1e9 / hbm, 4),
                                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if "hbm_gbs" in peaks else "fallback"}
    line.update(extra)
    serving_results = {}
    if rank == 0 and not args.quick and not args.no_serving and side:
        xf = xfer_code(args.xfer)
        serv = {"workload": "64 scans, files 2^(24+8u) B (log-uniform 16 MiB-4 GiB), 6 GiB cache, 296 CTAs, "
                            "1 MiB units; Poisson 20/s and 200/s, and all 64 at once (saturating)"}
        for label, mode, rate in (("readahead_poisson20", gfs.MODE_READAHEAD, 20.0),
                                  ("ondemand_poisson20", gfs.MODE_ONDEMAND, 20.0),
                                  ("readahead_poisson200", gfs.MODE_READAHEAD, 200.0),
                                  ("readahead_saturating", gfs.MODE_READAHEAD, None),
                                  ("ondemand_saturating", gfs.MODE_ONDEMAND, None)):
            serv[label], serving_results[label] = serving_bench(args, xf, mode, rate)
        line["serving"] = serv
    if not args.quick and not args.no_cpu_baseline and side:
        line["cpu_baseline"], line["parity"] = oracle_checks(path, stride, last, serving_results, args.cpu_seconds,
                                                             args.workload)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gfs", "reference"], default="gfs")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--blocks", type=int, default=0)
    ap.add_argument("--threads", type=int, default=256)
    ap.add_argument("--host-threads", type=int, default=16)
    ap.add_argument("--ra-cap", type=int, default=8)
    ap.add_argument("--rpc-slots", type=int, default=512)
    ap.add_argument("--staging-mib", type=int, default=4)
    ap.add_argument("--fused", action="store_true")
    ap.add_argument("--xfer", choices=["mapped", "pull", "dma"], default="mapped")
    ap.add_argument("--max-rpc-pages", type=int, default=16)
    ap.add_argument("--quick", action="store_true", help="skip the side measurements")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the readahead-vs-on-demand, host-merge and cold legs")
    ap.add_argument("--sweep", choices=["cfg3", "cfg4", "cold", "paper", "random", "queue"], default=None,
                    help="run a sweep instead of the bench line")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-step-seconds", type=float, default=10.0)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.sweep == "cfg3":
        return run_cfg3(args)
    if args.sweep == "cfg4":
        return run_cfg4(args)
    if args.sweep == "cold":
        return run_cold(args)
    if args.sweep == "paper":
        return run_paper(args)
    if args.sweep == "random":
        return run_random(args)
    if args.sweep == "queue":
        return run_queue(args)
    return run_gfs(args)


if __name__ == "__main__":
    sys.exit(main())
