"""Autotuner for the stride scan: picks page size, readahead cap, request-ring
slots and threadblocks for a file and stride, by measurement.

Coordinate descent: start from a point, sweep one knob at a time over its
values holding the others, keep the best, and repeat until a full round finds
nothing better (or `rounds` is reached).  Every measured point is kept, and the
best point can be saved as JSON and loaded later.  Each point is timed with
CUDA events around gfs_scan (median of `reps` scans, each from an empty cache).
"""
from __future__ import annotations

import json
import os
import statistics

KiB, MiB, GiB = 1 << 10, 1 << 20, 1 << 30

SPACE = {
    "page_size": [64 * KiB, 256 * KiB, 1 * MiB, 2 * MiB],
    "ra_cap_pages": [1, 8, 64],
    "rpc_slots": [32, 128, 512],
    "blocks": [148, 296, 592],
}
START = {"page_size": 512 * KiB, "ra_cap_pages": 8, "rpc_slots": 128, "blocks": 296}


def measure(path: str, stride: int, point: dict, cache_bytes: int = 2 * GiB, xfer: int = 2, mode: int = 0,
            reps: int = 2, threads: int = 256) -> dict:
    """GB/s of the stride scan of `path` at one configuration point."""
    import torch

    from . import gfs
    size = os.path.getsize(path)
    page = point["page_size"]
    need = point["ra_cap_pages"] + (stride + page - 1) // page + 1
    stream = torch.cuda.Stream()
    with gfs.Context(cache_bytes=cache_bytes, page_size=page, ra_cap_pages=point["ra_cap_pages"],
                     rpc_slots=point["rpc_slots"], max_rpc_pages=min(256, max(16, need)), xfer=xfer,
                     mode=mode, max_streams=max(4096, point["blocks"])) as ctx:
        fid = ctx.open(path)
        ns = (size + stride - 1) // stride
        out = tuple(torch.empty(ns, dtype=torch.int64, device="cuda") for _ in range(3))
        times = []
        for r in range(reps + 1):
            ctx.reset_cache(stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ctx.scan(fid, stride, blocks=point["blocks"], threads=threads, out=out, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if r:
                times.append(e0.elapsed_time(e1) / 1e3)
        st = ctx.stats(stream)
        bad = int((out[0][:-1] != stride).sum().item())
    t = statistics.median(times)
    return {**point, "stride": stride, "gbps": round(size / t / 1e9, 2), "ms": round(1e3 * t, 3),
            "rpcs": st["rpcs"], "timeouts": st["timeouts"], "short_strides": bad}


def tune(path: str, stride: int, space: dict = SPACE, start: dict = START, rounds: int = 2, **kw):
    """Coordinate descent; returns (best point, every measured point)."""
    seen = {}

    def key(p):
        return tuple(sorted(p.items()))

    def get(p):
        k = key(p)
        if k not in seen:
            try:
                r = measure(path, stride, p, **kw)
            except OSError as e:  # a point the library refuses or that fails is never the best
                r = {**p, "stride": stride, "gbps": 0.0, "error": str(e), "timeouts": -1, "short_strides": -1}
            seen[k] = r
        return seen[k]

    best = dict(start)
    best_r = get(best)
    for _ in range(rounds):
        improved = False
        for knob, values in space.items():
            for v in values:
                cand = dict(best, **{knob: v})
                r = get(cand)
                if r["gbps"] > best_r["gbps"] and r["timeouts"] == 0 and r["short_strides"] == 0:
                    best, best_r, improved = cand, r, True
        if not improved:
            break
    return best_r, list(seen.values())


def save(best: dict, path: str):
    with open(path, "w") as f:
        json.dump(best, f, indent=1, sort_keys=True)


def load(path: str) -> dict:
    with open(path) as f:
        return json.load(f)
