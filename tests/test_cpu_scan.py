"""The CPU-only scan of the C ABI (gfs_cpu_scan, a context figure beside the GPU
path): its per-stride counts and checksums equal the oracle's plain definition
(Section 6.1's stride scan), with ragged tails, reads longer and shorter than the
stride, one and several threads.  Runs without a GPU."""
import errno
import os

import numpy as np
import pytest

import inputs
from oracle import plain

KiB, MiB = 1 << 10, 1 << 20


@pytest.fixture(scope="module")
def gfs():
    from paper_2109_05366_gb300 import gfs as g
    g.load()
    return g


@pytest.mark.parametrize("size,stride,read_len,threads", [
    (37 * MiB + 5, MiB, MiB, 7),              # ragged last stride
    (37 * MiB + 5, MiB + 3, 700 * KiB + 1, 3),  # unaligned strides, reads shorter than the stride
    (9 * MiB + 4095, 3 * MiB, 5 * MiB, 4),    # reads overlap the next stride, clipped at EOF
    (6 * MiB, 6 * MiB + 1, 6 * MiB + 1, 1),   # one stride covering the whole file
    (1, 4096, 4096, 2),                       # one byte
])
def test_cpu_scan_equals_plain_definition(tmp_path, gfs, size, stride, read_len, threads):
    path = str(tmp_path / "c.bin")
    inputs.ensure_file(path, 41, size)
    cnt, sm, hs, secs = gfs.cpu_scan(path, stride, read_len, threads)
    c, s, h = plain.scan_plain(path, stride, read_len)
    assert cnt.tolist() == c
    assert np.array_equal(sm, np.array(s, dtype=np.uint64))
    assert np.array_equal(hs, np.array(h, dtype=np.uint64))
    assert secs >= 0


def test_cpu_scan_errors(tmp_path, gfs):
    path = str(tmp_path / "e.bin")
    inputs.ensure_file(path, 42, 4096)
    with pytest.raises(OSError) as e:
        gfs.cpu_scan(str(tmp_path / "missing.bin"), 4096)
    assert e.value.errno == errno.ENOENT
    with pytest.raises(gfs.GfsError) as e:
        gfs.cpu_scan(path, 4096, 0)
    assert e.value.errno == errno.EINVAL
    empty = str(tmp_path / "z.bin")
    open(empty, "wb").close()
    cnt, sm, hs, _ = gfs.cpu_scan(empty, 4096)
    assert cnt.size == 0 and sm.size == 0 and hs.size == 0
