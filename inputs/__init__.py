"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This package holds none of the method's arithmetic: it only makes the files that
both sides read.  The byte stream is xorshift64 (Marsaglia 2003, shifts 13/7/17),
state = seed, each step emitting the new state as 8 little-endian bytes; a file of
`size` bytes is the first `size` bytes of that stream.  The fast writer is
`xorshift_gen.c` (multi-threaded, GF(2) jump-ahead); `xorshift64_bytes` is the
plain Python definition used to pin it on small sizes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xorshift_gen.c")
_LIB = os.path.join(_HERE, "_xorshift_gen.so")
_MASK = (1 << 64) - 1
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the generator with gcc into inputs/_xorshift_gen.so (host code only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.xs_state_after.restype = ctypes.c_uint64
            lib.xs_state_after.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.xs_fill.restype = ctypes.c_int
            lib.xs_fill.argtypes = [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
            lib.xs_write_file.restype = ctypes.c_int
            lib.xs_write_file.argtypes = [ctypes.c_char_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]
            lib.xs_write_f32.restype = ctypes.c_int
            lib.xs_write_f32.argtypes = [ctypes.c_char_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]
            lib.xs_write_zipf.restype = ctypes.c_int
            lib.xs_write_zipf.argtypes = [ctypes.c_char_p, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32,
                                          ctypes.c_double, ctypes.c_int]
            lib.xs_zipf_cdf.restype = ctypes.c_int
            lib.xs_zipf_cdf.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_double]
            _lib = lib
    return _lib


def xorshift64_step(x: int) -> int:
    """One step of Marsaglia's xorshift64 with triple (13, 7, 17)."""
    x ^= (x << 13) & _MASK
    x ^= x >> 7
    x ^= (x << 17) & _MASK
    return x


def xorshift64_words(seed: int, n: int, start_word: int = 0) -> list[int]:
    """Output words start_word .. start_word+n-1 (word j = state after j+1 steps). Slow."""
    if seed == 0:
        raise ValueError("xorshift64 seed must be non-zero")
    x = seed
    for _ in range(start_word):
        x = xorshift64_step(x)
    out = []
    for _ in range(n):
        x = xorshift64_step(x)
        out.append(x)
    return out


def xorshift64_bytes(seed: int, size: int) -> bytes:
    """The first `size` bytes of the stream, by the plain definition (small sizes only)."""
    words = xorshift64_words(seed, (size + 7) // 8)
    return b"".join(w.to_bytes(8, "little") for w in words)[:size]


def state_after(seed: int, k: int) -> int:
    """xorshift64 state after k steps, by the C jump-ahead."""
    return int(_load().xs_state_after(seed, k))


def fill(seed: int, byte_off: int, n: int) -> bytes:
    """Stream bytes [byte_off, byte_off+n) via the C generator."""
    buf = ctypes.create_string_buffer(max(n, 1))
    rc = _load().xs_fill(buf, seed, byte_off, n)
    if rc != 0:
        raise OSError(-rc, os.strerror(-rc))
    return buf.raw[:n]


def write_file(path: str, seed: int, size: int, threads: int | None = None) -> str:
    """Write `size` stream bytes for `seed` to `path` (multi-threaded)."""
    threads = threads or min(32, os.cpu_count() or 1)
    rc = _load().xs_write_file(path.encode(), seed, size, threads)
    if rc != 0:
        raise OSError(-rc, "xs_write_file(%s): %s" % (path, os.strerror(-rc)))
    return path


def ensure_file(path: str, seed: int, size: int, threads: int | None = None) -> str:
    """Write the file unless one of the right size with a matching head and tail exists."""
    if os.path.exists(path) and os.path.getsize(path) == size:
        k = min(size, 4096)
        with open(path, "rb") as f:
            head = f.read(k)
            f.seek(size - k)
            tail = f.read(k)
        if head == fill(seed, 0, k) and tail == fill(seed, size - k, k):
            return path
    return write_file(path, seed, size, threads)


# ---------------------------------------------------------------- typed streams
def f32_of_word(x: int) -> float:
    """Uniform [-1, 1) value of one output word: ((x >> 40) * 2^-24) * 2 - 1 (exact in float32)."""
    return ((x >> 40) * 2.0 ** -24) * 2.0 - 1.0


def f32_values(seed: int, n: int):
    """Plain definition of the first n float32 elements (small n)."""
    import numpy as np
    return np.array([f32_of_word(x) for x in xorshift64_words(seed, n)], dtype=np.float32)


def zipf_cdf(nbins: int, s: float):
    import numpy as np
    w = (np.arange(1, nbins + 1, dtype=np.float64)) ** (-s)
    c = np.cumsum(w)
    c /= c[-1]
    c[-1] = 1.0
    return c


def zipf_values(seed: int, n: int, nbins: int, s: float):
    """Plain definition of the first n Zipf(s) values over [0, nbins) (small n)."""
    import bisect

    import numpy as np
    cdf = list(zipf_cdf(nbins, s))
    out = []
    for x in xorshift64_words(seed, n):
        u = (x >> 11) * 2.0 ** -53
        out.append(bisect.bisect_right(cdf, u))  # first k with cdf[k] > u
    return np.array(out, dtype=np.int32)


def write_f32(path: str, seed: int, n: int, threads: int | None = None) -> str:
    threads = threads or min(32, os.cpu_count() or 1)
    rc = _load().xs_write_f32(path.encode(), seed, n, threads)
    if rc != 0:
        raise OSError(-rc, "xs_write_f32(%s)" % path)
    return path


def write_zipf(path: str, seed: int, n: int, nbins: int = 1 << 20, s: float = 1.1,
               threads: int | None = None) -> str:
    threads = threads or min(32, os.cpu_count() or 1)
    rc = _load().xs_write_zipf(path.encode(), seed, n, nbins, s, threads)
    if rc != 0:
        raise OSError(-rc, "xs_write_zipf(%s)" % path)
    return path


def ensure_typed(path: str, kind: str, seed: int, n: int, **kw) -> str:
    """Write the f32 or zipf file unless one of the right size with the right head exists."""
    import numpy as np
    k = min(n, 64)
    if os.path.exists(path) and os.path.getsize(path) == 4 * n:
        head = np.fromfile(path, dtype=np.float32 if kind == "f32" else np.int32, count=k)
        ref = f32_values(seed, k) if kind == "f32" else zipf_values(seed, k, kw.get("nbins", 1 << 20),
                                                                      kw.get("s", 1.1))
        if np.array_equal(head, ref):
            return path
    return write_f32(path, seed, n) if kind == "f32" else write_zipf(path, seed, n, **kw)


def file_digest(path: str, piece: int = 64 << 20, threads: int | None = None) -> str:
    """A record of a generated file's bytes: SHA-256 over the concatenated SHA-256
    digests of its consecutive `piece`-byte pieces (the last one shorter), the pieces
    hashed in parallel threads.  Hex string; an empty file digests zero pieces."""
    import hashlib
    from concurrent.futures import ThreadPoolExecutor
    size = os.path.getsize(path)
    offs = list(range(0, size, piece))
    fd = os.open(path, os.O_RDONLY)
    try:
        def one(off):
            h = hashlib.sha256()
            end = min(off + piece, size)
            while off < end:
                b = os.pread(fd, min(end - off, 8 << 20), off)
                if not b:
                    raise OSError("short read of %s at %d" % (path, off))
                h.update(b)
                off += len(b)
            return h.digest()
        with ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 1) as ex:
            parts = list(ex.map(one, offs))
    finally:
        os.close(fd)
    return hashlib.sha256(b"".join(parts)).hexdigest()
