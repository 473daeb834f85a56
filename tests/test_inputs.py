"""Seeded input generator: pinned to Marsaglia's definition, independent of the method."""
import os

import pytest

import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden", "xorshift64_seed1.txt")


def _golden():
    vals = {}
    for line in open(GOLD):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = v
    return vals


def test_first_word_by_hand():
    g = _golden()
    assert inputs.xorshift64_words(1, 1)[0] == int(g["word0"], 16)
    assert inputs.xorshift64_bytes(1, 8).hex() == g["bytes0_7"]
    assert inputs.fill(1, 0, 8).hex() == g["bytes0_7"]


@pytest.mark.parametrize("seed", [1, 2, 0x9E3779B97F4A7C15])
@pytest.mark.parametrize("k", [0, 1, 2, 63, 64, 1000, 4097])
def test_jump_ahead_matches_stepping(seed, k):
    x = seed
    for _ in range(k):
        x = inputs.xorshift64_step(x)
    assert inputs.state_after(seed, k) == x


def test_jump_ahead_is_linear():
    # xorshift is linear over GF(2): M^k (a ^ b) = M^k a ^ M^k b
    a, b, k = 0x1234567, 0xABCDEF0123, 12345
    assert inputs.state_after(a ^ b, k) == inputs.state_after(a, k) ^ inputs.state_after(b, k)


@pytest.mark.parametrize("off,n", [(0, 1), (0, 17), (3, 29), (8, 8), (1001, 513)])
def test_fill_matches_definition(off, n):
    assert inputs.fill(5, off, n) == inputs.xorshift64_bytes(5, off + n)[off:]


@pytest.mark.parametrize("size", [0, 1, 7, 8, 9, 4095, 4096, 4097, (3 << 20) + 17])
@pytest.mark.parametrize("threads", [1, 3])
def test_write_file(tmp_path, size, threads):
    p = str(tmp_path / "f.bin")
    inputs.write_file(p, 11, size, threads)
    data = open(p, "rb").read()
    assert len(data) == size
    head = min(size, 256)
    assert data[:head] == inputs.xorshift64_bytes(11, head)
    if size > 300:
        assert data[-100:] == inputs.fill(11, size - 100, 100)


def test_thread_count_independent(tmp_path):
    a, b = str(tmp_path / "a"), str(tmp_path / "b")
    inputs.write_file(a, 3, (5 << 20) + 3, 1)
    inputs.write_file(b, 3, (5 << 20) + 3, 7)
    assert open(a, "rb").read() == open(b, "rb").read()


def test_seed_zero_rejected(tmp_path):
    with pytest.raises(OSError):
        inputs.write_file(str(tmp_path / "z"), 0, 10)


def test_f32_stream_definition(tmp_path):
    import numpy as np
    p = str(tmp_path / "a.f32")
    inputs.write_f32(p, 7, 3000, threads=3)
    a = np.fromfile(p, dtype=np.float32)
    assert np.array_equal(a, inputs.f32_values(7, 3000))
    x0 = inputs.xorshift64_words(7, 1)[0]
    assert a[0] == np.float32(((x0 >> 40) * 2.0 ** -24) * 2 - 1)
    assert a.min() >= -1.0 and a.max() < 1.0


def test_zipf_stream_definition(tmp_path):
    import numpy as np
    p = str(tmp_path / "z.i32")
    inputs.write_zipf(p, 8, 4000, 1 << 20, 1.1, threads=2)
    z = np.fromfile(p, dtype=np.int32)
    assert np.array_equal(z, inputs.zipf_values(8, 4000, 1 << 20, 1.1))
    # P(0) = 1 / H(2^20, 1.1); H(2^20, 1.1) is about 7.9, so the top bin holds ~12.6 %
    assert 0.09 < (z == 0).mean() < 0.16 and z.min() >= 0 and z.max() < (1 << 20)


@pytest.mark.parametrize("size,threads", [((48 << 20) + 3, 16), ((48 << 20) + 3, 8), ((6 << 20) + 5, 3),
                                          ((16 << 20) + 1, 16)])
def test_every_byte_written_whatever_the_split(tmp_path, size, threads):
    """The writer splits the file among threads in whole-MiB ranges; the ranges must
    cover every byte even when size / threads is a whole number of MiB with a remainder
    (a file whose last bytes were never written is a hole of zeros, not the stream)."""
    path = str(tmp_path / "f.bin")
    inputs.write_file(path, 7, size, threads)
    assert os.path.getsize(path) == size
    k = 4096
    with open(path, "rb") as f:
        f.seek(size - k)
        tail = f.read(k)
    assert tail == inputs.fill(7, size - k, k)
    per = size // threads
    with open(path, "rb") as f:  # the edges of every thread's range
        for t in range(1, threads):
            off = min(size - 16, t * per)
            f.seek(off)
            assert f.read(16) == inputs.fill(7, off, 16)


def test_every_zipf_value_written_whatever_the_split(tmp_path):
    """The same for the Zipf writer: value i comes from stream word i, so the last values
    can be recomputed from the words after a jump ahead."""
    import bisect

    import numpy as np
    path = str(tmp_path / "z.i32")
    n = (3 << 20) + 3
    inputs.write_zipf(path, 9, n, 1 << 10, 1.1, 3)
    x = np.fromfile(path, dtype=np.int32)
    assert len(x) == n
    cdf = list(inputs.zipf_cdf(1 << 10, 1.1))
    st = inputs.state_after(9, n - 8)
    want = []
    for _ in range(8):
        st = inputs.xorshift64_step(st)
        want.append(bisect.bisect_right(cdf, (st >> 11) * 2.0 ** -53))
    assert list(x[-8:]) == want


def test_file_digest_definition(tmp_path):
    # SHA-256 over the pieces' SHA-256 digests, pieces in file order, the last one short
    import hashlib
    size, piece = 3 * 4096 + 17, 4096
    path = str(tmp_path / "d.bin")
    inputs.write_file(path, 5, size)
    data = inputs.xorshift64_bytes(5, size)
    want = hashlib.sha256(b"".join(hashlib.sha256(data[o:o + piece]).digest()
                                   for o in range(0, size, piece))).hexdigest()
    assert inputs.file_digest(path, piece=piece, threads=3) == want
    assert inputs.file_digest(path, piece=piece, threads=1) == want
    empty = str(tmp_path / "e.bin")
    open(empty, "wb").close()
    assert inputs.file_digest(empty) == hashlib.sha256(b"").hexdigest()
