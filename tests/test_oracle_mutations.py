"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a copy of oracle/ (a dropped term, a wrong bound, a
wrong index, a rule left out), runs tests/test_oracle.py against the copy, and
requires it to fail.  The mistakes cover the plain definition (Section 2.2's read,
Section 6.1's checksums) and every rule of the policy simulation (R2-R8, victim
classes 1-3, the per-block LRA of Section 5.1, the paper's private buffer of
Section 4.1), so a pin that stops pinning shows up here.

Three mistakes are not listed because no trace can tell them from the oracle
(equivalent mutants): letting the demand run R2 reach max_rpc_pages + 1 pages (the
request is capped at max_rpc_pages afterwards), dropping R4's check that the mark
page was fetched since the last reset (R8 then ends the request at its first page),
and dropping the consumed FIFO's skip of the frame being delivered (with one gread
at a time that frame is never in the FIFO when its mark fires).
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = {
    # plain definition
    "gread_drops_last_byte": ("plain.py", "n = min(length, size - off)", "n = min(length, size - off - 1)"),
    "hash_weight_from_zero": ("plain.py", "w = np.arange(off + 1, off + 1 + len(data), dtype=U64)",
                              "w = np.arange(off, off + len(data), dtype=U64)"),
    "stride_count_floor": ("plain.py", "return (size + stride - 1) // stride if size > 0 else 0",
                           "return size // stride if size > 0 else 0"),
    # R3: the three sequential-access tests and where a gread ends
    "r3_no_previous_end": ("policy.py", "               or self.last_end.get((stream, fid)) == p)", "               )"),
    "r3_no_previous_page": ("policy.py", "seq = (p == 0 or (fid, p - 1) in self.table", "seq = (p == 0"),
    "gread_ends_at_last_page": ("policy.py", "self.last_end[(stream, fid)] = p1 + 1", "self.last_end[(stream, fid)] = p1"),
    # window growth (sync and async) and the recorded window
    "sync_first_window_2x": ("policy.py", "max(4 * d, 2 * t_prev)", "max(2 * d, 2 * t_prev)"),
    "sync_cap_off_by_one": ("policy.py", "T = min(d + self.Wmax,", "T = min(d + self.Wmax + 1,"),
    "async_no_doubling": ("policy.py", "min(self.Wmax, 2 * t)", "min(self.Wmax, t)"),
    "window_records_demand": ("policy.py", "        for f in taken:\n            self.frames[f].window = n\n        if n > d:",
                              "        for f in taken:\n            self.frames[f].window = d\n        if n > d:"),
    # R4 mark placement, R5 consumption, R7 hint, R8 refetch
    "mark_on_first_page": ("policy.py", "self.frames[taken[d]].ra_end = p + n", "self.frames[taken[0]].ra_end = p + n"),
    "fifo_push_every_read": ("policy.py", "if before < fr.valid <= fr.consumed:", "if fr.valid <= fr.consumed:"),
    "readahead_ignores_hint": ("policy.py", "if self.mode != \"readahead\" or not fi.readahead:",
                               "if self.mode != \"readahead\":"),
    "no_r8": ("policy.py", "            if q - p >= demand and (fid, q) in self.fetched:      # R8\n                break\n", ""),
    # victims: reserve, class 3
    "reserve_off_by_one": ("policy.py", "self._avail() <= self.reserve", "self._avail() < self.reserve"),
    "class3_own_frames": ("policy.py", "or fr.alloc_seq >= gread_seq0)", "or fr.alloc_seq > gread_seq0)"),
    "class3_newest": ("policy.py", "if best is None or fr.alloc_seq < self.frames[best].alloc_seq:",
                      "if best is None or fr.alloc_seq > self.frames[best].alloc_seq:"),
    "class3_any_demand_page": ("policy.py", "fallback=q == p)", "fallback=True)"),
    # Section 5.1 per-block LRA, Section 4.1 private buffer
    "lra_over_quota": ("policy.py", "if len(q) < self.quota and self.next_unused < self.F:",
                       "if len(q) <= self.quota and self.next_unused < self.F:"),
    "lra_quota_divisor": ("policy.py", "self.quota = max(1, n_frames // max(1, streams))",
                          "self.quota = max(1, n_frames // max(1, streams + 1))"),
    "lra_reuses_busy": ("policy.py", "            if f == self._pinned or f in self._busy:\n                continue\n",
                        "            if f == self._pinned:\n                continue\n"),
    "paper_request_size": ("policy.py", "n = min(1 + self.Wmax, fi.npages - p, self.max_rpc)",
                           "n = min(self.Wmax, fi.npages - p, self.max_rpc)"),
    "paper_no_buffer_hits": ("policy.py", "        if buf is not None and buf[0] == fid and p in buf[1]:", "        if False:"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_the_pins(tmp_path, name):
    fn, old, new = MUTANTS[name]
    for d in ("oracle", "inputs"):
        shutil.copytree(os.path.join(ROOT, d), str(tmp_path / d),
                        ignore=shutil.ignore_patterns("__pycache__", "_build", "*.so", "*.o"))
    os.makedirs(str(tmp_path / "tests"))
    for f in ("conftest.py", "test_oracle.py", "__init__.py"):
        if os.path.exists(os.path.join(ROOT, "tests", f)):
            shutil.copy(os.path.join(ROOT, "tests", f), str(tmp_path / "tests" / f))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), str(tmp_path / "tests" / "golden"))
    target = tmp_path / "oracle" / fn
    src = target.read_text()
    assert src.count(old) == 1, "the mutation site moved: " + name
    target.write_text(src.replace(old, new))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "tests/test_oracle.py"],
                       cwd=str(tmp_path), capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, "planted mistake %s passed every pin:\n%s" % (name, r.stdout[-2000:])
