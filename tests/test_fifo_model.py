"""Exhaustive interleavings of a model of the consumed-FIFO protocol (CPU only).

The device code (`fifo_put`, `fifo_take`, `fifo_pop` in csrc/gfs_device.cuh) keeps the
consumed frames (Section 5.1's queue of pages read once) in a bounded MPMC queue whose
two ends take tickets by fetch-and-add; a pop whose ticket ran past the tail gives it up
by moving its cell to the next lap, and a push that finds its cell past its ticket draws
another.  This test restates that protocol step by step — one shared-memory access per
step, the same branch conditions — and explores every interleaving of small scenarios:

* liveness: from every reachable state some schedule finishes every thread (no
  deadlock, no state in which waiting threads can only wait for each other);
* conservation: at every final state the frames the pops returned plus the frames a
  sequential drain then finds are exactly the frames that were in the queue or pushed,
  each once, and the queue works afterwards (a push and a pop round-trip);
* order: pushes that completed before the pops began come out in push order.
"""
import itertools

import pytest

EMPTY = -1  # frame field of a free cell


def _cell_init(cap):
    return tuple((i, EMPTY) for i in range(cap))


class Model:
    """Shared state: cells (seq, frame), head, tail.  A thread is a tuple
    (kind, pc, a, b, v): kind 'push' carries (ticket, frame), kind 'pop' (ticket,
    result); v is the cell value last read.  Every pc performs exactly one access to
    shared state, as the device code does; a spin re-reads (a cycle in the graph)."""

    def __init__(self, cap):
        self.cap = cap

    def step(self, shared, th):
        """The successor (shared, thread) of one step of `th`; [] once it is done."""
        cells, head, tail = shared
        kind, pc, a, b, v = th
        cap = self.cap

        def put(i, val):
            c = list(cells)
            c[i] = val
            return tuple(c)

        if kind == "push":  # a = ticket, b = frame
            if pc == "draw":  # fetch-and-add on the tail
                return [((cells, head, tail + 1), ("push", "read", tail, b, None))]
            if pc == "read":
                cv = cells[a % cap]
                s = cv[0]
                nxt = "cas" if s == a else ("draw" if s > a else "read")  # s > a: given up by a pop
                return [(shared, ("push", nxt, a, b, cv))]
            if pc == "cas":  # compare-and-swap (t + 1, frame) over the value read
                if cells[a % cap] == v:
                    return [((put(a % cap, (a + 1, b)), head, tail), ("push", "done", a, b, None))]
                return [(shared, ("push", "read", a, b, None))]
            return []
        if kind == "pop":  # a = ticket, b = result
            if pc == "h":  # pre-check: head, then tail
                return [(shared, ("pop", "t", head, None, None))]
            if pc == "t":
                if a >= tail:
                    return [(shared, ("pop", "done", None, -1, None))]
                return [(shared, ("pop", "draw", None, None, None))]
            if pc == "draw":  # fetch-and-add on the head
                return [((cells, head + 1, tail), ("pop", "read", head, None, None))]
            if pc == "read":
                cv = cells[a % cap]
                s = cv[0]
                nxt = "take" if s == a + 1 else ("tail" if s == a else "read")
                return [(shared, ("pop", nxt, a, None, cv))]
            if pc == "take":
                return [((put(a % cap, (a + cap, EMPTY)), head, tail), ("pop", "done", a, v[1], None))]
            if pc == "tail":  # no push holds the ticket: give it up; else wait for the push
                return [(shared, ("pop", "cas" if tail <= a else "read", a, None, v))]
            if pc == "cas":
                if cells[a % cap] == v:
                    return [((put(a % cap, (a + cap, EMPTY)), head, tail), ("pop", "done", a, -1, None))]
                return [(shared, ("pop", "read", a, None, None))]
            return []
        raise AssertionError(kind)


def _done(th):
    return th[1] == "done"


def _explore(model, shared0, threads0):
    """State graph of all interleavings: returns (states, edges, finals)."""
    start = (shared0, tuple(threads0))
    seen = {start}
    edges = {}
    stack = [start]
    finals = []
    while stack:
        st = stack.pop()
        shared, threads = st
        succ = []
        for i, th in enumerate(threads):
            for sh2, th2 in model.step(shared, th):
                nt = list(threads)
                nt[i] = th2
                s2 = (sh2, tuple(nt))
                succ.append(s2)
                if s2 not in seen:
                    seen.add(s2)
                    stack.append(s2)
        edges[st] = succ
        if all(_done(t) for t in threads):
            finals.append(st)
    return seen, edges, finals


def _can_finish(seen, edges, finals):
    """States from which some schedule reaches a final state."""
    rev = {s: [] for s in seen}
    for s, succ in edges.items():
        for s2 in succ:
            rev[s2].append(s)
    good = set(finals)
    stack = list(finals)
    while stack:
        s = stack.pop()
        for p in rev[s]:
            if p not in good:
                good.add(p)
                stack.append(p)
    return good


def _run_alone(model, shared, th, max_steps=1000):
    """Run one thread with nobody else scheduled; a thread that cannot finish alone
    (it waits for another) fails the test instead of spinning."""
    for _ in range(max_steps):
        if _done(th):
            return shared, th
        (shared, th), = model.step(shared, th)
    raise AssertionError("a lone thread did not finish: %r" % (th,))


def _drain(model, shared):
    """Sequential pops until one returns -1; the frames in order and the final state."""
    out = []
    for _ in range(64):
        shared, th = _run_alone(model, shared, ("pop", "h", None, None, None))
        if th[3] == -1:
            return out, shared
        out.append(th[3])
    raise AssertionError("drain did not end")


def _round_trip(model, shared, frame=99):
    shared, _ = _run_alone(model, shared, ("push", "draw", None, frame, None))
    got, shared = _drain(model, shared)
    return got == [frame]


def _preload(model, frames):
    shared = (_cell_init(model.cap), 0, 0)
    for f in frames:
        shared, _ = _run_alone(model, shared, ("push", "draw", None, f, None))
    return shared


def _pushers_with_reserved_tickets(shared, frames):
    """A run's release: one fetch-and-add reserved len(frames) tickets; each lane then
    stores its frame into its own ticket's cell (page order = ticket order)."""
    cells, head, tail = shared
    ths = [("push", "read", tail + i, f, None) for i, f in enumerate(frames)]
    return (cells, head, tail + len(frames)), ths


SCENARIOS = {
    # name: (cap, frames already in the queue, pushes, pops, reserved-ticket pushes)
    "two_pushes_two_pops_empty": (2, [], [1, 2], 2, []),
    "pops_race_one_item": (2, [7], [3], 2, []),
    "pop_first_then_pushes": (3, [], [1, 2], 3, []),
    "wraps_the_ring": (2, [5, 6], [1], 2, []),
    "run_release_beside_pops": (3, [4], [], 2, [1, 2]),
    "run_release_and_push": (2, [], [9], 2, [1, 2]),
}


@pytest.mark.parametrize("name", sorted(SCENARIOS))
def test_ticket_fifo_every_interleaving(name):
    cap, pre, pushes, pops, reserved = SCENARIOS[name]
    m = Model(cap)
    shared = _preload(m, pre)
    shared, threads = _pushers_with_reserved_tickets(shared, reserved)
    threads += [("push", "draw", None, f, None) for f in pushes]
    threads += [("pop", "h", None, None, None) for _ in range(pops)]
    seen, edges, finals = _explore(m, shared, threads)
    assert finals
    good = _can_finish(seen, edges, finals)
    stuck = [s for s in seen if s not in good]
    assert not stuck, "states from which no schedule finishes: %d" % len(stuck)
    expected = sorted(pre + pushes + reserved)
    for sh, ths in finals:
        popped = [t[3] for t in ths if t[0] == "pop" and t[3] != -1]
        rest, sh2 = _drain(m, sh)
        assert sorted(popped + rest) == expected, (popped, rest)
        assert _round_trip(m, sh2)


def test_pushes_before_pops_come_out_in_order():
    m = Model(4)
    for n in range(1, 5):
        for perm in itertools.permutations(range(10, 10 + n)):
            shared = _preload(m, list(perm))
            got, shared = _drain(m, shared)
            assert got == list(perm)
            assert _round_trip(m, shared)


def test_a_pop_on_an_empty_queue_takes_no_ticket():
    """The pre-check keeps a sequential pop on an empty queue from drawing (and then
    giving up) a ticket, so serialized runs never give tickets up."""
    m = Model(2)
    shared, th = _run_alone(m, _preload(m, []), ("pop", "h", None, None, None))
    assert th[3] == -1 and shared[1] == 0 and shared[2] == 0
