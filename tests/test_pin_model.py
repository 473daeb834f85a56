"""Exhaustive interleavings of a model of the frame pin / claim handshake (CPU only).

A reader pins a frame before it reads it (`frame_pin`, and `run_begin` for runs of
pages, in csrc/gfs_device.cuh): add 1 to the pin count, fence, then check that the
frame still holds its page (state not RECLAIM or EMPTY, key unchanged).  An evictor
claims it (`frame_claim`): compare-and-swap the state to RECLAIM, fence, then check that
the pin count is 0, else put the state back.  Each side writes its own word and then
reads the other's, with a fence between (the fences make these accesses sequentially
consistent), so at least one of them sees the other.

The model restates both sides one shared access per step and explores every
interleaving of readers and evictors on one frame: a reader never holds the frame while
an evictor goes on to remap it, some schedule always finishes, and at the end the pin
count is 0 and the frame either still holds its page or was remapped exactly once.
"""
import pytest

READY, RECLAIM, FILLING = "READY", "RECLAIM", "FILLING"
PAGE, NEW = "page", "new"


def step(sh, th):
    """Successors of one step of thread `th` on the shared frame (state, key, pins, remaps)."""
    state, key, pins, remaps = sh
    kind, pc, seen = th
    if kind == "reader":
        if pc == "pin":
            return [((state, key, pins + 1, remaps), ("reader", "state", None))]
        if pc == "state":  # after the fence
            return [(sh, ("reader", "key", state))]
        if pc == "key":
            ok = seen not in (RECLAIM, "EMPTY") and key == PAGE
            return [(sh, ("reader", "hold" if ok else "unpin_miss", None))]
        if pc == "hold":  # reads the frame's bytes, then releases it
            return [(sh, ("reader", "unpin_hit", None))]
        if pc in ("unpin_hit", "unpin_miss"):
            return [((state, key, pins - 1, remaps), ("reader", "done_" + pc[6:], None))]
        return []
    if kind == "evictor":
        if pc == "state":
            if state != READY:
                return [(sh, ("evictor", "done_none", None))]
            return [(sh, ("evictor", "cas", state))]
        if pc == "cas":
            if state != seen:
                return [(sh, ("evictor", "done_none", None))]
            return [((RECLAIM, key, pins, remaps), ("evictor", "pins", seen))]
        if pc == "pins":  # after the fence
            return [(sh, ("evictor", "restore" if pins else "remap", seen))]
        if pc == "restore":
            return [((seen, key, pins, remaps), ("evictor", "done_busy", None))]
        if pc == "remap":  # old page out of the table, new page installed
            return [((FILLING, NEW, pins, remaps + 1), ("evictor", "done_claimed", None))]
        return []
    raise AssertionError(kind)


def _explore(threads0, stepper=step):
    start = ((READY, PAGE, 0, 0), tuple(threads0))
    seen, edges, finals, stack = {start}, {}, [], [start]
    while stack:
        st = stack.pop()
        sh, threads = st
        succ = []
        for i, th in enumerate(threads):
            for sh2, th2 in stepper(sh, th):
                nt = list(threads)
                nt[i] = th2
                succ.append((sh2, tuple(nt)))
        for s2 in succ:
            if s2 not in seen:
                seen.add(s2)
                stack.append(s2)
        edges[st] = succ
        if all(t[1].startswith("done") for t in threads):
            finals.append(st)
    return seen, edges, finals


def _unsafe(st):
    """A reader holds the frame for its page while it no longer holds that page."""
    (state, key, pins, remaps), threads = st
    return any(t[1] in ("hold", "unpin_hit") for t in threads) and (remaps > 0 or key != PAGE)


def _can_finish(seen, edges, finals):
    rev = {s: [] for s in seen}
    for s, succ in edges.items():
        for s2 in succ:
            rev[s2].append(s)
    good, stack = set(finals), list(finals)
    while stack:
        s = stack.pop()
        for p in rev[s]:
            if p not in good:
                good.add(p)
                stack.append(p)
    return good


@pytest.mark.parametrize("readers,evictors", [(1, 1), (2, 1), (1, 2), (2, 2)])
def test_pinned_frames_are_never_remapped(readers, evictors):
    threads = [("reader", "pin", None)] * readers + [("evictor", "state", None)] * evictors
    seen, edges, finals = _explore(threads)
    assert not [s for s in seen if _unsafe(s)]
    assert len(_can_finish(seen, edges, finals)) == len(seen)
    outcomes = set()
    for (state, key, pins, remaps), threads_f in finals:
        assert pins == 0 and remaps <= 1
        assert (state, key) == ((READY, PAGE) if remaps == 0 else (FILLING, NEW))
        hits = sum(t[1] == "done_hit" for t in threads_f)
        outcomes.add((remaps, hits))
    assert (0, readers) in outcomes and (1, 0) in outcomes  # both races are won in some run


def test_a_claim_that_reads_the_pins_before_its_cas_is_caught():
    """The same model with the evictor's two accesses swapped (pins read, then the CAS):
    a reader can then hold a frame that is being remapped."""
    def bad(sh, th):
        state, key, pins, remaps = sh
        kind, pc, seen = th
        if kind == "evictor" and pc == "state":
            return [] if state != READY else [(sh, ("evictor", "pins_first", state))]
        if kind == "evictor" and pc == "pins_first":
            return [(sh, ("evictor", "done_busy" if pins else "cas_late", seen))]
        if kind == "evictor" and pc == "cas_late":
            if state != seen:
                return [(sh, ("evictor", "done_none", None))]
            return [((RECLAIM, key, pins, remaps), ("evictor", "remap", seen))]
        return step(sh, th)

    seen, edges, finals = _explore([("reader", "pin", None), ("evictor", "state", None)], bad)
    assert any(_unsafe(s) for s in seen)
