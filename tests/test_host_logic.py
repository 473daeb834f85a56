"""CPU tests of host-side logic around the GPU path: the autotuner's coordinate
descent, the serving driver's arrival and size generators and its submit/poll
loop (against a fake context), and the kernel-code digest that keeps profile
figures tied to the kernel they were measured on."""
import math
import os
import shutil

from paper_2109_05366_gb300 import build, serving, tune


def test_tuner_descends_to_the_best_point_and_skips_failures(monkeypatch):
    # a separable score: best at page 1 MiB, Wmax 8, 512 slots, 592 blocks; one point fails
    pref = {"page_size": {64 << 10: 0, 256 << 10: 1, 512 << 10: 0, 1 << 20: 3, 2 << 20: 2},
            "ra_cap_pages": {1: 0, 8: 2, 64: 1}, "rpc_slots": {32: 0, 128: 1, 512: 2},
            "blocks": {148: 0, 296: 1, 592: 2}}
    calls = []

    def fake_measure(path, stride, point, **kw):
        calls.append(dict(point))
        if point["page_size"] == 2 << 20 and point["blocks"] == 296:
            raise OSError(110, "device wait timed out")
        score = sum(pref[k][v] for k, v in point.items())
        return {**point, "stride": stride, "gbps": float(score), "timeouts": 0, "short_strides": 0}

    monkeypatch.setattr(tune, "measure", fake_measure)
    best, points = tune.tune("unused", 1 << 20)
    assert (best["page_size"], best["ra_cap_pages"], best["rpc_slots"], best["blocks"]) == (1 << 20, 8, 512, 592)
    failed = [p for p in points if "error" in p]
    assert failed and all(p["gbps"] == 0.0 for p in failed)
    assert len({tuple(sorted(c.items())) for c in calls}) == len(calls)  # each point measured once


def test_tuner_rejects_points_with_timeouts(monkeypatch):
    def fake_measure(path, stride, point, **kw):
        fast = point["blocks"] == 592
        return {**point, "stride": stride, "gbps": 300.0 if fast else 100.0, "timeouts": 3 if fast else 0,
                "short_strides": 0}

    monkeypatch.setattr(tune, "measure", fake_measure)
    best, _ = tune.tune("unused", 1 << 20)
    assert best["blocks"] != 592 and best["timeouts"] == 0


def test_tuned_points_round_trip(tmp_path):
    p = tmp_path / "t.json"
    tune.save({"page_size": 1 << 20, "blocks": 296}, str(p))
    assert tune.load(str(p)) == {"page_size": 1 << 20, "blocks": 296}


def test_poisson_arrivals_are_seeded_and_have_the_rate():
    a = serving.poisson_arrivals(20000, 20.0, seed=3)
    assert a == serving.poisson_arrivals(20000, 20.0, seed=3) and a[0] == 0.0
    gaps = [y - x for x, y in zip(a, a[1:])]
    assert all(g >= 0 for g in gaps)
    assert abs(sum(gaps) / len(gaps) - 1 / 20.0) < 0.05 / 20.0  # mean gap 1/rate within 5 %


def test_log_uniform_sizes_span_the_range():
    s = serving.log_uniform_sizes(5000, 24, 32, seed=1)
    assert all(2 ** 24 <= x < 2 ** 32 for x in s)
    logs = [math.log2(x) for x in s]
    assert abs(sum(logs) / len(logs) - 28.0) < 0.2  # uniform in log2 over [24, 32)


class _FakeServer:
    """Completes each submitted scan two polls later; the ring holds `slots` at once."""

    def __init__(self, slots=3):
        self.slots, self.pending, self.polls = slots, [], 0

    def submit_scan(self, fid, off, ln, tag):
        if len(self.pending) >= self.slots:
            return False
        self.pending.append((tag, self.polls + 2, ln))
        return True

    def poll(self, n):
        self.polls += 1
        out = [p for p in self.pending if p[1] <= self.polls][:n]
        self.pending = [p for p in self.pending if p not in out]
        return [{"tag": t, "status": 0, "sum": 0, "hash": 0, "bytes": ln, "t_admit_ns": 0, "t_done_ns": 1000}
                for t, _, ln in out]


def test_serving_driver_submits_everything_through_a_small_ring():
    reqs = [(0, i << 20, (i + 1) << 10) for i in range(10)]
    res, t0 = serving.run(_FakeServer(slots=3), reqs, arrivals=[0.0] * 10, timeout_s=10.0)
    assert [r["tag"] for r in res] == list(range(10))
    assert all(r["bytes"] == (i + 1) << 10 for i, r in enumerate(res))
    assert all(r["done_s"] >= r["submit_s"] >= t0 for r in res)
    summ = serving.summarize(res, t0)
    assert summ["requests"] == 10 and summ["errors"] == 0
    assert summ["bytes"] == sum((i + 1) << 10 for i in range(10))


def test_kernel_digest_ignores_comments_but_not_code(tmp_path, monkeypatch):
    csrc = tmp_path / "csrc"
    inc = tmp_path / "include"
    shutil.copytree(build.CSRC, csrc, ignore=shutil.ignore_patterns("*.o", "*.so"))
    shutil.copytree(os.path.join(build.ROOT, "include"), inc)
    monkeypatch.setattr(build, "CSRC", str(csrc))
    monkeypatch.setattr(build, "ROOT", str(tmp_path))
    d0 = build.kernel_digest()
    dev = csrc / "gfs_device.cuh"
    text = dev.read_text()
    dev.write_text(text.replace("#pragma once", "#pragma once\n// a new comment line\n/* and a block */", 1))
    assert build.kernel_digest() == d0
    dev.write_text(text.replace("kLraWindow = 1024", "kLraWindow = 2048", 1))
    assert build.kernel_digest() != d0
