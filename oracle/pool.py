"""The plain definition run over many host cores.  TEST INFRASTRUCTURE ONLY.

Full-size parity (files of 8-16 GiB and more) with the single-threaded
`plain.scan_plain` takes minutes on one core.  This module only splits the
stride indices into contiguous ranges, runs `plain.scan_plain` on each range in
its own worker process, and concatenates the results in stride order: no
arithmetic of its own.  `range_checksums` adds per-range values of the plain
definition into the checksums of a longer range, which is what the definition
itself says (both checksums are sums over the bytes, mod 2^64, with absolute
file offsets in the hash).

Worker processes are started with the "spawn" method: a process forked from a
parent that has already used the GPU can hang.
"""
from __future__ import annotations

import multiprocessing as mp
import os
from concurrent.futures import ProcessPoolExecutor

from . import plain

U64_MASK = (1 << 64) - 1


def _scan_range(args):
    path, stride, read_len, lo, hi = args
    return plain.scan_plain(path, stride, read_len, strides=list(range(lo, hi)))


def workers(n: int | None = None) -> int:
    return max(1, min(n or os.cpu_count() or 1, 64))


def scan_plain_parallel(path: str, stride: int, read_len: int | None = None, procs: int | None = None,
                        chunk_bytes: int = 256 << 20):
    """plain.scan_plain(path, stride, read_len) for every stride, computed on `procs` processes."""
    read_len = stride if read_len is None else read_len
    size = os.path.getsize(path)
    ns = plain.stride_count(size, stride)
    if ns == 0:
        return [], [], []
    per = max(1, chunk_bytes // max(stride, 1))
    jobs = [(path, stride, read_len, lo, min(ns, lo + per)) for lo in range(0, ns, per)]
    counts, sums, hashes = [], [], []
    n = workers(procs)
    if n == 1 or len(jobs) == 1:
        parts = map(_scan_range, jobs)
        for c, s, h in parts:
            counts += c
            sums += s
            hashes += h
        return counts, sums, hashes
    with ProcessPoolExecutor(max_workers=min(n, len(jobs)), mp_context=mp.get_context("spawn")) as ex:
        for c, s, h in ex.map(_scan_range, jobs):
            counts += c
            sums += s
            hashes += h
    return counts, sums, hashes


def range_checksums(path: str, off: int, length: int, procs: int | None = None, piece: int = 64 << 20):
    """(count, sum, hash) of the plain gread of [off, off + length): the per-piece values of
    the plain definition added mod 2^64 (pieces of `piece` bytes starting at off)."""
    return many_range_checksums([(path, off, length)], procs, piece)[0]


def many_range_checksums(ranges, procs: int | None = None, piece: int = 64 << 20):
    """range_checksums for every (path, off, length) of `ranges`, on one pool of processes."""
    jobs, owner = [], []
    for k, (path, off, length) in enumerate(ranges):
        size = os.path.getsize(path)
        end = min(off + length, size) if length > 0 else off
        p = off
        while p < end:
            q = min(end, p + piece)
            jobs.append((path, p, q - p))
            owner.append(k)
            p = q
    n = workers(procs)
    if n == 1 or len(jobs) <= 1:
        res = list(map(_piece, jobs))
    else:
        with ProcessPoolExecutor(max_workers=min(n, len(jobs)), mp_context=mp.get_context("spawn")) as ex:
            res = list(ex.map(_piece, jobs, chunksize=1))
    out = [[0, 0, 0] for _ in ranges]
    for k, (c, s, h) in zip(owner, res):
        out[k][0] += c
        out[k][1] = (out[k][1] + s) & U64_MASK
        out[k][2] = (out[k][2] + h) & U64_MASK
    return [tuple(o) for o in out]


def _piece(args):
    path, off, length = args
    size = os.path.getsize(path)
    fd = os.open(path, os.O_RDONLY)
    try:
        n, data = plain.gread_plain(fd, size, off, length)
    finally:
        os.close(fd)
    return n, plain.byte_sum(data), plain.pos_hash(data, off)
