"""Serving driver: submit scans at seeded arrival times, collect completions.

Host-side orchestration only (timing and bookkeeping); the scans run in the
persistent serving kernel of libgfs.so (gfs_serve_start / gfs_submit_scan /
gfs_poll).
"""
from __future__ import annotations

import random
import time

import numpy as np


def poisson_arrivals(n: int, rate_per_s: float, seed: int) -> list[float]:
    """n arrival times (s from start) with seeded exponential gaps of mean 1/rate."""
    rng = random.Random(seed)
    t, out = 0.0, []
    for _ in range(n):
        out.append(t)
        t += rng.expovariate(rate_per_s)
    return out


def log_uniform_sizes(n: int, lo_log2: int, hi_log2: int, seed: int) -> list[int]:
    """Sizes floor(2^(lo + (hi-lo) u)) bytes, u uniform in [0, 1) (seeded)."""
    rng = random.Random(seed)
    return [int(2.0 ** (lo_log2 + (hi_log2 - lo_log2) * rng.random())) for _ in range(n)]


def run(ctx, requests, arrivals=None, timeout_s: float = 120.0):
    """Submit requests [(fid, off, len)] (at arrival times if given) and wait for all.

    Returns per-request dicts with the completion fields plus host-side
    'submit_s' and 'done_s' (time.perf_counter) and 'latency_s'.
    """
    n = len(requests)
    arrivals = arrivals or [0.0] * n
    order = sorted(range(n), key=lambda i: arrivals[i])
    t0 = time.perf_counter()
    submit_t = [None] * n
    done = {}
    k = 0
    while len(done) < n:
        now = time.perf_counter() - t0
        while k < n and arrivals[order[k]] <= now:
            i = order[k]
            fid, off, ln = requests[i]
            if not ctx.submit_scan(fid, off, ln, i):
                break  # ring full: try again after polling
            submit_t[i] = time.perf_counter()
            k += 1
        for c in ctx.poll(256):
            c["done_s"] = time.perf_counter()
            done[c["tag"]] = c
        if time.perf_counter() - t0 > timeout_s:
            raise TimeoutError("serving: %d of %d requests done" % (len(done), n))
        if k < n and not done:
            nxt = arrivals[order[k]] - (time.perf_counter() - t0)
            if nxt > 0.0005:
                time.sleep(min(nxt, 0.0005))
    out = []
    for i in range(n):
        c = dict(done[i])
        c["submit_s"] = submit_t[i]
        c["latency_s"] = c["done_s"] - submit_t[i]
        out.append(c)
    return out, t0


def summarize(results, t0) -> dict:
    lat = np.array([r["latency_s"] for r in results])
    dev_lat = np.array([(r["t_done_ns"] - r["t_admit_ns"]) * 1e-9 for r in results])
    total = sum(r["bytes"] for r in results)
    span = max(r["done_s"] for r in results) - min(r["submit_s"] for r in results)
    return {"requests": len(results), "bytes": int(total), "span_s": round(span, 4),
            "gbps": round(total / span / 1e9, 2) if span > 0 else None,
            "scan_latency_p50_ms": round(1e3 * float(np.percentile(lat, 50)), 3),
            "scan_latency_p99_ms": round(1e3 * float(np.percentile(lat, 99)), 3),
            "device_scan_p50_ms": round(1e3 * float(np.percentile(dev_lat, 50)), 3),
            "device_scan_p99_ms": round(1e3 * float(np.percentile(dev_lat, 99)), 3),
            "errors": int(sum(1 for r in results if r["status"] != 0))}
