"""Python binding of the C ABI in include/gfs.h (ctypes; argument marshalling only).

Every step of the read path runs in libgfs.so (CUDA kernels + host I/O threads).
PyTorch only supplies device memory and streams.  There is no fallback: if the
library cannot be built or loaded, or there is no GPU, calls raise.
"""
from __future__ import annotations

import ctypes
import errno
import os
import threading

import numpy as np

from . import build as _build

RDONLY, RDWR, DIRECT = 0, 2, 0x100
MODE_READAHEAD, MODE_ONDEMAND, MODE_PAPER = 0, 1, 2
REPL_FIFO, REPL_TB_LRA = 0, 1
ADV_NORMAL, ADV_SEQUENTIAL, ADV_RANDOM = 0, 1, 2
XFER_DMA, XFER_PULL, XFER_MAPPED = 0, 1, 2
QUEUE_SHARED, QUEUE_STATIC = 0, 1
KIND_DEMAND, KIND_SYNC_RA, KIND_ASYNC_RA = 0, 1, 2
PATH_MAX = 1024

u32, u64, i32, i64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64
vp = ctypes.c_void_p


class Config(ctypes.Structure):
    _fields_ = [("cache_bytes", u64), ("timeout_ns", u64), ("page_size", u32), ("mode", u32),
                ("ra_cap_pages", u32), ("async_ra", u32), ("reserve_frames", u32), ("rpc_slots", u32),
                ("max_rpc_pages", u32), ("host_threads", u32), ("staging_bytes", u32), ("max_streams", u32),
                ("max_files", u32), ("trace_capacity", u32), ("xfer", u32), ("debug_counts", u32),
                ("device", i32), ("latency_capacity", u32), ("replacement", u32), ("queue", u32),
                ("host_merge_pages", u32), ("map_pinned", u32), ("self_serve", u32), ("reserved", u32 * 1)]


class Stat(ctypes.Structure):
    _fields_ = [("size", u64), ("page_size", u32), ("flags", u32), ("advice", u32), ("mapped", u32)]


STATS_FIELDS = ["greads", "hits", "misses", "coalesced_waits", "rpcs", "pages_fetched", "bytes_fetched",
                "ra_pages_sync", "ra_pages_async", "evictions", "unconsumed_evictions", "retries", "timeouts",
                "eio", "enomem", "host_requests", "host_preads", "host_bytes", "host_copies", "host_errors",
                "trace_rpc_count", "trace_evict_count", "host_ns_pread", "host_ns_wait_buf", "host_ns_idle",
                "buffer_hits", "host_controls", "host_merged", "run_cuts"]


class Stats(ctypes.Structure):
    _fields_ = [(n, u64) for n in STATS_FIELDS] + [("reserved", u64 * 1)]


class ThreadStat(ctypes.Structure):
    _fields_ = [("requests", u64), ("polls_before_first", u64), ("first_request_ns", u64), ("idle_ns", u64),
                ("pread_ns", u64), ("bytes", u64)]


class IoRec(ctypes.Structure):
    _fields_ = [("offset", u64), ("bytes", u64), ("fid", u32), ("thread", u32), ("t_ns", u64)]


class RpcRec(ctypes.Structure):
    _fields_ = [("fid", u32), ("kind", u32), ("npages", u32), ("reserved", u32), ("page_lo", u64)]


class EvictRec(ctypes.Structure):
    _fields_ = [("frame", u32), ("old_fid", u32), ("new_fid", u32), ("reserved", u32), ("old_page", u64),
                ("new_page", u64)]


class ScanArgs(ctypes.Structure):
    _fields_ = [("stride", u64), ("read_len", u64), ("blocks", u32), ("threads", u32), ("serialize", u32),
                ("fused", u32), ("reserved", u32 * 4)]


class ServeConfig(ctypes.Structure):
    _fields_ = [("ctas", u32), ("threads", u32), ("unit_bytes", u64), ("max_requests", u32), ("queue_slots", u32),
                ("units_in_flight", u32), ("frame_budget", u32), ("idle_exit_ms", u32), ("reserved", u32 * 5)]


class Completion(ctypes.Structure):
    _fields_ = [("tag", u64), ("status", i64), ("sum", u64), ("hash", u64), ("bytes", u64), ("t_admit_ns", u64),
                ("t_done_ns", u64)]


# name -> (restype, argtypes); every symbol include/gfs.h declares.
SIGNATURES = {
    "gfs_config_default": (ctypes.c_int, [ctypes.POINTER(Config)]),
    "gfs_init": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(vp)]),
    "gfs_shutdown": (ctypes.c_int, [vp]),
    "gfs_open": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "gfs_close": (ctypes.c_int, [vp, ctypes.c_int]),
    "gfs_fadvise": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_int]),
    "gfs_fstat": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(Stat)]),
    "gfs_set_faults": (ctypes.c_int, [vp, u32, u32, u32]),
    "gfs_reset_cache": (ctypes.c_int, [vp, vp]),
    "gfs_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(Stats), vp]),
    "gfs_get_trace": (ctypes.c_int, [vp, ctypes.POINTER(RpcRec), ctypes.POINTER(EvictRec), u32,
                                     ctypes.POINTER(u64), ctypes.POINTER(u64), vp]),
    "gfs_get_fetch_counts": (ctypes.c_int, [vp, vp, u64, vp]),
    "gfs_get_thread_stats": (ctypes.c_int, [vp, ctypes.POINTER(ThreadStat), u32]),
    "gfs_get_io_trace": (ctypes.c_int, [vp, ctypes.POINTER(IoRec), u64, ctypes.POINTER(u64)]),
    "gfs_replay_io": (ctypes.c_int, [ctypes.c_char_p, ctypes.POINTER(IoRec), u64, u32,
                                     ctypes.POINTER(ctypes.c_double), ctypes.POINTER(u64)]),
    "gfs_get_latencies": (ctypes.c_int, [vp, vp, u64, ctypes.POINTER(u64), vp]),
    "gfs_scan": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ScanArgs), vp, vp, vp, vp]),
    "gfs_scan_host": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ScanArgs), vp, vp, vp, vp]),
    "gfs_scan_static": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ScanArgs), vp, vp, vp, vp]),
    "gfs_scan_path": (ctypes.c_int, [vp, ctypes.c_char_p, ctypes.POINTER(ScanArgs), vp, vp, vp, vp]),
    "gfs_device_handle": (ctypes.c_int, [vp, u32, u64, vp, u64]),
    "gfs_read_many": (ctypes.c_int, [vp, ctypes.c_int, u32, vp, vp, vp, vp, vp, u32, u32, vp]),
    "gfs_scan_graph": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(ScanArgs), u32, vp, vp, vp, vp]),
    "gfs_cpuio_scan": (ctypes.c_int, [ctypes.c_char_p, u64, u64, u32, u64, vp, vp, vp, vp, vp,
                                      ctypes.POINTER(ctypes.c_double)]),
    "gfs_cpu_scan": (ctypes.c_int, [ctypes.c_char_p, u64, u64, u32, vp, vp, vp, ctypes.POINTER(ctypes.c_double)]),
    "gfs_probe_h2d": (ctypes.c_int, [u64, u64, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "gfs_probe_pread": (ctypes.c_int, [ctypes.c_char_p, u32, u64, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "gfs_probe_pull": (ctypes.c_int, [u64, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "gfs_selftest_ring": (ctypes.c_int, [ctypes.c_char_p, u32, u32, u32, u32, u32, u32, u32, u32, u64, u32,
                                         ctypes.POINTER(u64), vp, ctypes.POINTER(u64)]),
    "gfs_rowdot": (ctypes.c_int, [vp, ctypes.c_int, u32, u32, vp, vp, u32, u64, u32, vp, vp, vp, vp]),
    "gfs_histogram": (ctypes.c_int, [vp, ctypes.c_int, u32, vp, u64, u32, vp, vp, vp]),
    "gfs_serve_start": (ctypes.c_int, [vp, ctypes.POINTER(ServeConfig), vp]),
    "gfs_submit_scan": (ctypes.c_int, [vp, ctypes.c_int, u64, u64, u64]),
    "gfs_poll": (ctypes.c_int, [vp, ctypes.POINTER(Completion), ctypes.c_int]),
    "gfs_serve_stop": (ctypes.c_int, [vp]),
    "gfs_abi_version": (ctypes.c_int, []),
    "gfs_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}

_lib = None
_lock = threading.Lock()


class GfsError(OSError):
    pass


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libgfs.so (building it first when needed).  Raises if that fails."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise GfsError(errno.ENOENT, "libgfs.so is missing; run paper_2109_05366_gb300.build.build()")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(rc: int, what: str) -> int:
    if rc < 0:
        msg = load().gfs_strerror(rc).decode()
        raise GfsError(-rc, "%s: %s" % (what, msg))
    return rc


def _ptr(t) -> int | None:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return int(t)


def _stream(s) -> int | None:
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream
    return int(s)


def default_config(**overrides) -> Config:
    c = Config()
    _check(load().gfs_config_default(ctypes.byref(c)), "gfs_config_default")
    for k, v in overrides.items():
        if not hasattr(c, k):
            raise TypeError("unknown config field %r" % k)
        setattr(c, k, v)
    return c


class Context:
    """A gfs_ctx: GPU page cache + request ring + host I/O threads."""

    def __init__(self, **cfg):
        self.cfg = default_config(**cfg)
        h = vp()
        _check(load().gfs_init(ctypes.byref(self.cfg), ctypes.byref(h)), "gfs_init")
        self._h = h

    @property
    def handle(self):
        if self._h is None:
            raise GfsError(errno.EBADF, "context is shut down")
        return self._h

    def shutdown(self):
        if getattr(self, "_h", None) is not None:
            load().gfs_shutdown(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.shutdown()

    def __del__(self):
        try:
            self.shutdown()
        except Exception:
            pass

    def open(self, path: str, flags: int = RDONLY) -> int:
        fid = ctypes.c_int(-1)
        _check(load().gfs_open(self.handle, path.encode(), flags, ctypes.byref(fid)), "gfs_open(%s)" % path)
        return fid.value

    def close(self, fid: int):
        _check(load().gfs_close(self.handle, fid), "gfs_close")

    def fadvise(self, fid: int, advice: int):
        _check(load().gfs_fadvise(self.handle, fid, advice), "gfs_fadvise")

    def fstat(self, fid: int) -> Stat:
        st = Stat()
        _check(load().gfs_fstat(self.handle, fid, ctypes.byref(st)), "gfs_fstat")
        return st

    def set_faults(self, eio_every: int = 0, short_every: int = 0, delay_us: int = 0):
        _check(load().gfs_set_faults(self.handle, eio_every, short_every, delay_us), "gfs_set_faults")

    def reset_cache(self, stream=None):
        _check(load().gfs_reset_cache(self.handle, _stream(stream)), "gfs_reset_cache")

    def stats(self, stream=None) -> dict:
        st = Stats()
        _check(load().gfs_get_stats(self.handle, ctypes.byref(st), _stream(stream)), "gfs_get_stats")
        return {n: int(getattr(st, n)) for n in STATS_FIELDS}

    def trace(self, cap: int = 1 << 16, stream=None):
        """(rpc list of (fid, page_lo, npages, kind), evict list of (frame, (fid, page), (fid, page)))."""
        rpc = (RpcRec * cap)()
        ev = (EvictRec * cap)()
        nr, ne = u64(), u64()
        _check(load().gfs_get_trace(self.handle, rpc, ev, cap, ctypes.byref(nr), ctypes.byref(ne),
                                    _stream(stream)), "gfs_get_trace")
        kr, ke = min(nr.value, cap, self.cfg.trace_capacity), min(ne.value, cap, self.cfg.trace_capacity)
        rl = [(r.fid, r.page_lo, r.npages, r.kind) for r in rpc[:kr]]
        el = [(e.frame, (e.old_fid, e.old_page), (e.new_fid, e.new_page)) for e in ev[:ke]]
        return rl, el, nr.value, ne.value

    def latencies(self, stream=None) -> np.ndarray:
        """gread latencies (ns) recorded since the last reset."""
        cap = int(self.cfg.latency_capacity)
        out = np.zeros(max(cap, 1), dtype=np.uint64)
        n = u64()
        _check(load().gfs_get_latencies(self.handle, out.ctypes.data, cap, ctypes.byref(n), _stream(stream)),
               "gfs_get_latencies")
        return out[:min(cap, n.value)]

    def thread_stats(self) -> list[dict]:
        """Per host I/O thread counters since the last reset."""
        arr = (ThreadStat * 256)()
        n = _check(load().gfs_get_thread_stats(self.handle, arr, 256), "gfs_get_thread_stats")
        return [{f: int(getattr(arr[i], f)) for f, _ in ThreadStat._fields_} for i in range(min(n, 256))]

    def io_trace(self) -> list:
        """Host I/O trace (IoRec records) since the last reset."""
        cap = int(self.cfg.trace_capacity)
        arr = (IoRec * max(cap, 1))()
        n = u64()
        _check(load().gfs_get_io_trace(self.handle, arr, cap, ctypes.byref(n)), "gfs_get_io_trace")
        return list(arr[:min(cap, n.value)])

    def fetch_counts(self, n: int, stream=None) -> np.ndarray:
        out = np.zeros(n, dtype=np.uint32)
        _check(load().gfs_get_fetch_counts(self.handle, out.ctypes.data, n, _stream(stream)),
               "gfs_get_fetch_counts")
        return out

    @staticmethod
    def _args(stride, read_len, blocks, threads, serialize, fused) -> ScanArgs:
        a = ScanArgs()
        a.stride = stride
        a.read_len = stride if read_len is None else read_len
        a.blocks = blocks
        a.threads = threads
        a.serialize = 1 if serialize else 0
        a.fused = 1 if fused else 0
        return a

    def scan(self, fid: int, stride: int, read_len: int | None = None, blocks: int = 64, threads: int = 256,
             serialize: bool = False, fused: bool = False, out=None, stream=None):
        """Launch the stride scan; returns device tensors (count, sum, hash) (int64; sum/hash hold u64 bits)."""
        import torch
        size = self.fstat(fid).size
        ns = (size + stride - 1) // stride if size else 0
        if out is None:
            out = tuple(torch.empty(max(ns, 1), dtype=torch.int64, device="cuda") for _ in range(3))
        a = self._args(stride, read_len, blocks, threads, serialize, fused)
        _check(load().gfs_scan(self.handle, fid, ctypes.byref(a), _ptr(out[0]), _ptr(out[1]), _ptr(out[2]),
                               _stream(stream)), "gfs_scan")
        return out

    def scan_path(self, path: str, stride: int, read_len: int | None = None, blocks: int = 64, threads: int = 256,
                  out=None, stream=None):
        """Stride scan whose threadblocks open `path` on the device (gopen / gclose); device tensors as scan()."""
        import torch
        try:
            size = os.path.getsize(path)
        except OSError:  # the library reports the error
            size = 0
        ns = (size + stride - 1) // stride if size else 0
        if out is None:
            out = tuple(torch.empty(max(ns, 1), dtype=torch.int64, device="cuda") for _ in range(3))
        a = self._args(stride, read_len, blocks, threads, False, True)
        _check(load().gfs_scan_path(self.handle, path.encode(), ctypes.byref(a), _ptr(out[0]), _ptr(out[1]),
                                    _ptr(out[2]), _stream(stream)), "gfs_scan_path(%s)" % path)
        return out

    def device_handle(self, blocks: int, read_len: int) -> bytes:
        """The plain-data device handle that kernels calling the device API take by value."""
        buf = ctypes.create_string_buffer(4096)
        n = load().gfs_device_handle(self.handle, blocks, read_len, buf, len(buf))
        _check(n if n < 0 else 0, "gfs_device_handle")
        return buf.raw[:n]

    def scan_graph(self, fid: int, stride: int, reps: int, read_len: int | None = None, blocks: int = 64,
                   threads: int = 256, serialize: bool = False, fused: bool = False, out=None, stream=None):
        """reps x (drain, reset, scan) as one captured CUDA graph; returns the last scan's outputs."""
        import torch
        size = self.fstat(fid).size
        ns = (size + stride - 1) // stride if size else 0
        if out is None:
            out = tuple(torch.empty(max(ns, 1), dtype=torch.int64, device="cuda") for _ in range(3))
        a = self._args(stride, read_len, blocks, threads, serialize, fused)
        _check(load().gfs_scan_graph(self.handle, fid, ctypes.byref(a), reps, _ptr(out[0]), _ptr(out[1]),
                                     _ptr(out[2]), _stream(stream)), "gfs_scan_graph")
        return out

    def scan_host(self, fid: int, stride: int, read_len: int | None = None, blocks: int = 64, threads: int = 256,
                  serialize: bool = False, fused: bool = False, stream=None):
        """Stride scan with host result arrays (count int64, sum uint64, hash uint64)."""
        size = self.fstat(fid).size
        ns = (size + stride - 1) // stride if size else 0
        cnt = np.zeros(max(ns, 1), dtype=np.int64)
        sm = np.zeros(max(ns, 1), dtype=np.uint64)
        hs = np.zeros(max(ns, 1), dtype=np.uint64)
        a = self._args(stride, read_len, blocks, threads, serialize, fused)
        _check(load().gfs_scan_host(self.handle, fid, ctypes.byref(a), cnt.ctypes.data, sm.ctypes.data,
                                    hs.ctypes.data, _stream(stream)), "gfs_scan_host")
        return cnt[:ns], sm[:ns], hs[:ns]

    # ---- application streams
    def rowdot(self, fid: int, rows: int, cols: int, d_vec, stripe_rows: int = 128, read_len: int = 1 << 20,
               blocks: int = 296, stream=None):
        """Per-row float32 dot products of a row-major matrix file with d_vec.

        Returns device tensors (out float32[rows], stripe_sum int64, stripe_hash int64, status int64[1])."""
        import torch
        ns = (rows + stripe_rows - 1) // stripe_rows
        out = torch.empty(rows, dtype=torch.float32, device="cuda")
        ssum = torch.empty(ns, dtype=torch.int64, device="cuda")
        shash = torch.empty(ns, dtype=torch.int64, device="cuda")
        status = torch.zeros(1, dtype=torch.int64, device="cuda")
        _check(load().gfs_rowdot(self.handle, fid, rows, cols, _ptr(d_vec), _ptr(out), stripe_rows, read_len,
                                 blocks, _ptr(ssum), _ptr(shash), _ptr(status), _stream(stream)), "gfs_rowdot")
        return out, ssum, shash, status

    def histogram(self, fid: int, nbins: int = 1 << 20, read_len: int = 1 << 20, blocks: int = 296, stream=None):
        """Histogram of an int32 file.  Returns device tensors (hist int32[nbins], sums int64[2], status int64[1])."""
        import torch
        hist = torch.empty(nbins, dtype=torch.int32, device="cuda")
        sums = torch.empty(2, dtype=torch.int64, device="cuda")
        status = torch.zeros(1, dtype=torch.int64, device="cuda")
        _check(load().gfs_histogram(self.handle, fid, nbins, _ptr(hist), read_len, blocks, _ptr(sums), _ptr(status),
                                    _stream(stream)), "gfs_histogram")
        return hist, sums, status

    # ---- serving
    def serve_start(self, ctas: int = 152, threads: int = 256, unit_bytes: int = 1 << 20, max_requests: int = 64,
                    queue_slots: int = 256, units_in_flight: int = 16, frame_budget: int = 0, idle_exit_ms: int = 0,
                    stream=None):
        c = ServeConfig()
        c.ctas, c.threads, c.unit_bytes, c.max_requests = ctas, threads, unit_bytes, max_requests
        c.queue_slots, c.units_in_flight, c.frame_budget, c.idle_exit_ms = queue_slots, units_in_flight, frame_budget, idle_exit_ms
        _check(load().gfs_serve_start(self.handle, ctypes.byref(c), _stream(stream)), "gfs_serve_start")

    def submit_scan(self, fid: int, off: int, length: int, tag: int) -> bool:
        """Queue a scan; False when the submission ring is full (try again)."""
        rc = load().gfs_submit_scan(self.handle, fid, off, length, tag)
        if rc == -errno.EAGAIN:
            return False
        _check(rc, "gfs_submit_scan")
        return True

    def poll(self, max_n: int = 64) -> list:
        buf = (Completion * max_n)()
        n = _check(load().gfs_poll(self.handle, buf, max_n), "gfs_poll")
        return [{"tag": c.tag, "status": c.status, "sum": c.sum, "hash": c.hash, "bytes": c.bytes,
                 "t_admit_ns": c.t_admit_ns, "t_done_ns": c.t_done_ns} for c in buf[:n]]

    def serve_stop(self):
        _check(load().gfs_serve_stop(self.handle), "gfs_serve_stop")

    def read_many(self, fid: int, d_off, d_len, d_dst, d_buf, d_ret, blocks: int = 32, threads: int = 256,
                  stream=None):
        n = int(d_off.numel())
        _check(load().gfs_read_many(self.handle, fid, n, _ptr(d_off), _ptr(d_len), _ptr(d_dst), _ptr(d_buf),
                                    _ptr(d_ret), blocks, threads, _stream(stream)), "gfs_read_many")


def cpuio_scan(path: str, stride: int, read_len: int | None, threads: int, chunk: int, d_file, out,
               stream=None) -> float:
    secs = ctypes.c_double(0.0)
    read_len = stride if read_len is None else read_len
    _check(load().gfs_cpuio_scan(path.encode(), stride, read_len, threads, chunk, _ptr(d_file), _ptr(out[0]),
                                 _ptr(out[1]), _ptr(out[2]), _stream(stream), ctypes.byref(secs)),
           "gfs_cpuio_scan")
    return secs.value


def cpu_scan(path: str, stride: int, read_len: int | None = None, threads: int = 0):
    """CPU-only stride scan on `threads` host threads (0: every host core): (count, sum,
    hash) numpy arrays of the per-stride checksums, and the seconds it took."""
    read_len = stride if read_len is None else read_len
    threads = threads or os.cpu_count() or 1
    size = os.path.getsize(path)
    ns = (size + stride - 1) // stride if size else 0
    cnt = np.zeros(max(ns, 1), dtype=np.int64)
    sm = np.zeros(max(ns, 1), dtype=np.uint64)
    hs = np.zeros(max(ns, 1), dtype=np.uint64)
    secs = ctypes.c_double(0.0)
    _check(load().gfs_cpu_scan(path.encode(), stride, read_len, threads, cnt.ctypes.data, sm.ctypes.data,
                               hs.ctypes.data, ctypes.byref(secs)), "gfs_cpu_scan")
    return cnt[:ns], sm[:ns], hs[:ns], secs.value


def probe_h2d(nbytes: int, chunk: int, reps: int = 3) -> float:
    g = ctypes.c_double(0.0)
    _check(load().gfs_probe_h2d(nbytes, chunk, reps, ctypes.byref(g)), "gfs_probe_h2d")
    return g.value


def probe_pull(nbytes: int, reps: int = 3) -> float:
    g = ctypes.c_double(0.0)
    _check(load().gfs_probe_pull(nbytes, reps, ctypes.byref(g)), "gfs_probe_pull")
    return g.value


def probe_pread(path: str, threads: int, chunk: int, reps: int = 2) -> float:
    g = ctypes.c_double(0.0)
    _check(load().gfs_probe_pread(path.encode(), threads, chunk, reps, ctypes.byref(g)), "gfs_probe_pread")
    return g.value


def selftest_ring(path: str, page_size: int = 4096, frames: int = 256, requests: int = 500, max_pages: int = 8,
                  threads: int = 4, slots: int = 16, seed: int = 1, queue: int = QUEUE_SHARED,
                  client_blocks: int = 0, per_thread: bool = False, merge_pages: int = 1, merged: bool = False):
    """Requests served (and, with per_thread, each host thread's request count; with merged,
    the number of requests served merged with the one before)."""
    served, nmerged = u64(), u64()
    counts = np.zeros(threads, dtype=np.uint64)
    _check(load().gfs_selftest_ring(path.encode(), page_size, frames, requests, max_pages, threads, slots, queue,
                                    client_blocks, seed, merge_pages, ctypes.byref(served), counts.ctypes.data,
                                    ctypes.byref(nmerged)),
           "gfs_selftest_ring")
    out = [served.value]
    if per_thread:
        out.append(counts.tolist())
    if merged:
        out.append(nmerged.value)
    return out[0] if len(out) == 1 else tuple(out)


def replay_io(path: str, recs, threads: int):
    """CPU replay of a host I/O trace (list of IoRec or (offset, bytes) pairs): (seconds, bytes)."""
    arr = (IoRec * max(len(recs), 1))()
    for i, r in enumerate(recs):
        if isinstance(r, IoRec):
            arr[i] = r
        else:
            arr[i].offset, arr[i].bytes = r
    secs, nbytes = ctypes.c_double(), u64()
    _check(load().gfs_replay_io(path.encode(), arr, len(recs), threads, ctypes.byref(secs), ctypes.byref(nbytes)),
           "gfs_replay_io")
    return secs.value, nbytes.value


def u64_view(t) -> np.ndarray:
    """Host numpy uint64 view of an int64 tensor holding u64 bits."""
    return t.detach().cpu().numpy().view(np.uint64)
