"""Application-shaped consumers (Section 6.2 evaluates GPU applications that read
their input through GPUfs): per-row dot products of a float32 matrix with a
vector, and a histogram of int32 values.  TEST INFRASTRUCTURE ONLY.

Row dot products are computed in float64 from the exact float32 inputs (each
product of two float32 values is exact in float64); the float32 result of any
summation order then lies within gamma_n * sum_i |a_i b_i| of it, with
gamma_n = n u / (1 - n u), u = 2^-24 (standard forward error bound of recursive
or pairwise summation of n terms), n = number of columns.
"""
from __future__ import annotations

import numpy as np

U32 = 2.0 ** -24


def gamma(n: int, u: float = U32) -> float:
    return n * u / (1.0 - n * u)


def rowdot(path: str, rows: int, cols: int, vec: np.ndarray, row_lo: int = 0, row_hi: int | None = None):
    """(dot, abs) per row in float64: sum_c A[r][c] v[c] and sum_c |A[r][c] v[c]|."""
    row_hi = rows if row_hi is None else row_hi
    a = np.memmap(path, dtype=np.float32, mode="r", shape=(rows, cols))
    v = vec.astype(np.float64)
    dots, abss = [], []
    for r0 in range(row_lo, row_hi, 256):
        blk = np.asarray(a[r0:min(r0 + 256, row_hi)], dtype=np.float64)
        dots.append(blk @ v)
        abss.append(np.abs(blk) @ np.abs(v))
    del a
    return np.concatenate(dots), np.concatenate(abss)


def histogram(path: str, nbins: int, piece_values: int = 1 << 26) -> tuple[np.ndarray, int]:
    """(counts of each value < nbins, number of values outside [0, nbins)).

    The file is counted `piece_values` values at a time (exact integer counts add up,
    so the pieces only bound the memory a multi-GiB file needs)."""
    counts = np.zeros(nbins, dtype=np.uint64)
    outside = 0
    with open(path, "rb") as f:
        while True:
            x = np.fromfile(f, dtype=np.int32, count=piece_values)
            if x.size == 0:
                break
            inside = (x >= 0) & (x < nbins)
            counts += np.bincount(x[inside], minlength=nbins).astype(np.uint64)
            outside += int((~inside).sum())
    return counts, outside
