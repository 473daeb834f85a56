"""Exhaustive interleavings of a model of the request ring's cancellation protocol (CPU).

Producers (GPU warps, `ring_acquire` / `rpc_submit` in csrc/gfs_device.cuh) draw
tickets by fetch-and-add and wait until their slot is free for their ticket
(seq == t); a producer whose wait runs out posts `cancel[t % n] = t + 1` and leaves.
Host threads (`IoService::run_shared` / `skip_cancelled` in csrc/gfs_service.cpp) draw
tickets in the same order and wait for the request (seq == t + 1); a host thread that
finds its ticket cancelled and its slot free for it clears the cancellation and frees
the slot for the next lap.  A served request's slot is freed later by whoever copies
its pages (the GPU in the pull and mapped transfers), modelled as a separate actor.

A host thread that has a request may also take the ticket at the head of the ring (the
next one no host thread has drawn) when its request is already published
(`IoService::gather`: it reads the head, then the slot's sequence word, then claims the
ticket by compare-and-swap on the head), and serve both with one host read; the model
explores that step too, one claimed ticket at a time.

Every step below is one access to shared state, as in the code; a producer may run out
of time at any wait.  For every interleaving of small scenarios the test checks that
some schedule always finishes every thread (a host thread is never stuck behind an
abandoned ticket), that every ticket ends either served once or skipped once — served
exactly when its producer published it — and that the ring is left free for the next
lap with no cancellation left behind.
"""
import pytest


class Ring:
    def __init__(self, slots, cancel_n, tickets, merge=None):
        # merge: None (one request at a time), "cas" (the claim is one compare-and-swap, as
        # in the code) or "racy" (a planted mistake: the claim is a load and a later store)
        self.R, self.n, self.P, self.merge = slots, cancel_n, tickets, merge

    def initial(self):
        # seq, cancel, head (host tickets), tail (producer tickets), pending copies, served, skipped,
        # and whether some ticket was served twice
        return (tuple(range(self.R)), (0,) * self.n, 0, 0, frozenset(), frozenset(), frozenset(), False)

    def step(self, sh, th):
        seq, cancel, head, tail, pending, served, skipped, dup = sh
        R, n = self.R, self.n
        kind, pc, t = th

        def with_seq(i, v):
            s = list(seq)
            s[i] = v
            return tuple(s)

        def with_cancel(i, v):
            c = list(cancel)
            c[i] = v
            return tuple(c)

        if kind == "prod":
            if pc == "draw":
                return [((seq, cancel, head, tail + 1, pending, served, skipped, dup), ("prod", "check", tail))]
            if pc == "check":
                if seq[t % R] == t:
                    return [(sh, ("prod", "write", t))]
                return [(sh, ("prod", "late", t))]  # not free: wait again, or run out of time
            if pc == "late":
                return [(sh, ("prod", "check", t)), (sh, ("prod", "cancel", t))]
            if pc == "write":  # publish the request
                return [((with_seq(t % R, t + 1), cancel, head, tail, pending, served, skipped, dup), ("prod", "wrote", t))]
            if pc == "cancel":
                return [((seq, with_cancel(t % n, t + 1), head, tail, pending, served, skipped, dup),
                         ("prod", "cancelled", t))]
            return []
        if kind == "host":
            if pc == "draw":
                if head >= self.P:  # every ticket of the scenario is taken: the thread stops
                    return [(sh, ("host", "stopped", None))]
                return [((seq, cancel, head + 1, tail, pending, served, skipped, dup), ("host", "wait", head))]
            if pc == "wait":
                if seq[t % R] == t + 1:
                    return [(sh, ("host", "serve", t))]
                return [(sh, ("host", "skip_c", t))]
            if pc == "serve":  # publish the pages; their copier frees the slot later
                nxt = ("host", "mcheck", t) if self.merge else ("host", "draw", None)
                return [((seq, cancel, head, tail, pending | {t}, served | {t}, skipped, dup or t in served), nxt)]
            if pc == "mcheck":  # read the head: the first ticket no host thread has drawn
                return [(sh, ("host", "mseq", head))]
            if pc == "mseq":  # is that ticket's request already published?
                return [(sh, ("host", "mclaim" if t < self.P and seq[t % R] == t + 1 else "draw", t))]
            if pc == "mclaim":
                if self.merge == "cas":  # head: t -> t + 1 only if no host thread drew t meanwhile
                    if head != t:
                        return [(sh, ("host", "draw", None))]
                    return [((seq, cancel, t + 1, tail, pending, served, skipped, dup), ("host", "serve", t))]
                return [(sh, ("host", "mstore" if head == t else "draw", t))]
            if pc == "mstore":  # the planted mistake: store after a separate load
                return [((seq, cancel, t + 1, tail, pending, served, skipped, dup), ("host", "serve", t))]
            if pc == "skip_c":
                return [(sh, ("host", "skip_s" if cancel[t % n] == t + 1 else "wait", t))]
            if pc == "skip_s":
                return [(sh, ("host", "clear" if seq[t % R] == t else "wait", t))]
            if pc == "clear":
                return [((seq, with_cancel(t % n, 0), head, tail, pending, served, skipped, dup), ("host", "free", t))]
            if pc == "free":
                return [((with_seq(t % R, t + R), cancel, head, tail, pending, served, skipped | {t}, dup),
                         ("host", "draw", None))]
            return []
        raise AssertionError(kind)

    def copier(self, sh):
        """The GPU copies a served request's pages and frees its slot."""
        seq, cancel, head, tail, pending, served, skipped, dup = sh
        out = []
        for t in pending:
            s = list(seq)
            s[t % self.R] = t + self.R
            out.append((tuple(s), cancel, head, tail, pending - {t}, served, skipped, dup))
        return out


def _finished(th):
    return th[1] in ("wrote", "cancelled", "stopped")


def _explore(ring, threads0):
    start = (ring.initial(), tuple(threads0))
    seen, edges, finals, stack = {start}, {}, [], [start]
    while stack:
        st = stack.pop()
        sh, threads = st
        succ = []
        for i, th in enumerate(threads):
            for sh2, th2 in ring.step(sh, th):
                nt = list(threads)
                nt[i] = th2
                succ.append((sh2, tuple(nt)))
        for sh2 in ring.copier(sh):
            succ.append((sh2, threads))
        for s2 in succ:
            if s2 not in seen:
                seen.add(s2)
                stack.append(s2)
        edges[st] = succ
        if all(_finished(t) for t in threads) and not sh[4]:
            finals.append(st)
    return seen, edges, finals


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


@pytest.mark.parametrize("merge", [None, "cas"])
@pytest.mark.parametrize("slots,producers,hosts", [(2, 3, 1), (2, 3, 2), (2, 2, 1), (3, 4, 1), (2, 4, 2)])
def test_cancelled_tickets_are_skipped_and_nothing_sticks(slots, producers, hosts, merge):
    ring = Ring(slots, cancel_n=slots + producers, tickets=producers, merge=merge)
    threads = [("prod", "draw", None)] * producers + [("host", "draw", None)] * hosts
    seen, edges, finals = _explore(ring, threads)
    assert finals
    good = _can_finish(seen, edges, finals)
    assert len(good) == len(seen), "states from which no schedule finishes: %d" % (len(seen) - len(good))
    outcomes = set()
    assert not any(sh[7] for sh, _ in seen), "a ticket was served twice"
    for sh, ths in finals:
        seq, cancel, head, tail, pending, served, skipped, dup = sh
        wrote = {t for k, pc, t in ths if pc == "wrote"}
        gave_up = {t for k, pc, t in ths if pc == "cancelled"}
        assert served == wrote and skipped == gave_up
        assert served | skipped == set(range(producers)) and not served & skipped
        # every slot is free for the first ticket of its next lap; no cancellation is left
        assert all(seq[i] == min(t for t in range(producers, producers + slots) if t % slots == i)
                   for i in range(slots))
        assert not any(cancel)
        outcomes.add((frozenset(served), frozenset(skipped)))
    # every ticket is served in some run; every ticket that can find its slot busy (one of
    # a later lap) is skipped in another
    for t in range(producers):
        assert any(t in s for s, _ in outcomes)
        assert (t >= slots) == any(t in k for _, k in outcomes)


def test_one_slot_is_not_enough():
    """With one slot, "published for ticket t" (seq = t + 1) and "free for ticket t + 1"
    (seq = t + R) are the same value, so a producer can overwrite a request that was
    never served and leave its host thread waiting forever: the library rejects
    rpc_slots < 2 (gfs_init, gfs_selftest_ring)."""
    ring = Ring(1, cancel_n=3, tickets=2)
    threads = [("prod", "draw", None)] * 2 + [("host", "draw", None)]
    seen, edges, finals = _explore(ring, threads)
    assert len(_can_finish(seen, edges, finals)) < len(seen)


def test_merge_claim_must_be_one_compare_and_swap():
    """Planted mistake: a host thread that claims the next ticket with a load of the head
    and a later store lets another host thread draw the same ticket in between, and the
    request is served twice."""
    ring = Ring(2, cancel_n=5, tickets=3, merge="racy")
    threads = [("prod", "draw", None)] * 3 + [("host", "draw", None)] * 2
    seen, edges, finals = _explore(ring, threads)
    assert any(sh[7] for sh, _ in seen)
    ring = Ring(2, cancel_n=5, tickets=3, merge="cas")
    seen, edges, finals = _explore(ring, threads)
    assert not any(sh[7] for sh, _ in seen)


def test_merging_happens_in_some_schedule():
    """With a host thread behind published requests no other thread has drawn, the thread
    serves the one at the head merged with its own (the head moves past it by the claim,
    not by a draw)."""
    ring = Ring(3, cancel_n=5, tickets=3, merge="cas")
    threads = [("prod", "draw", None)] * 3 + [("host", "draw", None)] * 2
    seen, edges, finals = _explore(ring, threads)
    merged = any(th[1] == "mclaim" and sh[0][th[2] % 3] == th[2] + 1 and sh[2] == th[2]
                 for sh, ths in seen for th in ths if th[0] == "host")
    assert merged
