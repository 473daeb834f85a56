"""Plain definition of what a gread delivers and of the benchmark checksums.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Section 2.2 (GPUfs): a threadblock's read request returns the file's data for
the requested range; the page cache only changes where the bytes come from.
So gread(fid, off, len) delivers file[off : min(off+len, size)], exactly what
POSIX pread(fd, buf, len, off) returns, with count max(0, min(len, size-off)).

Section 6.1 (microbenchmark): every threadblock reads its own strides of the
file in a data-parallel way.  Block b of B reads strides b, b+B, b+2B, ... in
that order; stride s covers [s*S, s*S + L).  Per stride the benchmark keeps
  sum  = sum of the delivered bytes                         (mod 2^64)
  hash = sum over delivered bytes of byte * (file offset + 1) (mod 2^64)
The hash is position sensitive, so a page delivered to the wrong place changes
it even when the byte sum does not.
"""
from __future__ import annotations

import os

import numpy as np

U64 = np.uint64


def pread_exact(fd: int, off: int, n: int) -> bytes:
    """Read n bytes at off, looping over short reads; stops early only at EOF."""
    parts = []
    got = 0
    while got < n:
        chunk = os.pread(fd, min(n - got, 1 << 30), off + got)
        if not chunk:
            break
        parts.append(chunk)
        got += len(chunk)
    return b"".join(parts)


def gread_plain(fd: int, size: int, off: int, length: int) -> tuple[int, bytes]:
    """(count, bytes) a gread of [off, off+length) must deliver for a file of `size` bytes."""
    if off < 0 or length < 0:
        return -22, b""  # -EINVAL
    if off >= size or length == 0:
        return 0, b""
    n = min(length, size - off)
    data = pread_exact(fd, off, n)
    return len(data), data


def byte_sum(data: bytes) -> int:
    """Sum of the bytes, mod 2^64."""
    if not data:
        return 0
    return int(np.frombuffer(data, dtype=np.uint8).sum(dtype=U64))


def pos_hash(data: bytes, off: int) -> int:
    """Sum of byte_i * (off + i + 1) over the bytes, mod 2^64 (uint64 wraps)."""
    if not data:
        return 0
    b = np.frombuffer(data, dtype=np.uint8).astype(U64)
    w = np.arange(off + 1, off + 1 + len(data), dtype=U64)
    with np.errstate(over="ignore"):
        return int((b * w).sum(dtype=U64))


def stride_count(size: int, stride: int) -> int:
    """Number of strides that start before EOF."""
    return (size + stride - 1) // stride if size > 0 else 0


def stride_owner(s: int, blocks: int) -> tuple[int, int]:
    """Block that reads stride s, and the step k at which it does (s = k*B + b)."""
    return s % blocks, s // blocks


def scan_plain(path: str, stride: int, read_len: int | None = None,
               strides: list[int] | None = None):
    """Per-stride (count, sum, hash) of the stride-scan benchmark, by the plain definition.

    `strides` selects a sample of stride indices (default: all of them).
    """
    read_len = stride if read_len is None else read_len
    size = os.path.getsize(path)
    ns = stride_count(size, stride)
    sel = range(ns) if strides is None else strides
    counts, sums, hashes = [], [], []
    fd = os.open(path, os.O_RDONLY)
    try:
        for s in sel:
            off = s * stride
            n, data = gread_plain(fd, size, off, read_len)
            counts.append(n)
            sums.append(byte_sum(data))
            hashes.append(pos_hash(data, off))
    finally:
        os.close(fd)
    return counts, sums, hashes
