"""Page cache + readahead prefetcher + replacement, stepped over a serialized gread trace.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

What the paper fixes, and the reading taken where it does not (each reading is
listed with its reason in the design notes of the repository):

* Section 2.2 (GPUfs): a read is split into pages of the GPU page cache; a page
  found in the cache is copied to the user buffer; a missing page is requested
  from the CPU over the request queue, the CPU reads the file with pread and
  sends the data to the GPU page cache, and the page is then copied to the user
  buffer.  Original GPUfs fetches one page per request (rule R1 below).
* Section 2.3 (Linux readahead): a per-descriptor state decides whether the
  access is sequential; if so a larger read than requested is issued, the size
  doubling on each sequential access up to a maximum; several streams per
  descriptor; asynchronous readahead.  Section 3.1 gives the worked example: a
  4 KB read at offset 0 makes the prefetcher fetch 16 KB (initial window = 4x
  the request).
* Section 4.1 (GPU prefetcher): on a miss the GPU requests PAGE_SIZE +
  PREFETCH_SIZE bytes in one request and the CPU uses the returned size to set
  up every page it delivers.  Readahead only for read-only files and not when
  the user hints random access (fadvise).
* Section 5.1 (replacement): data read sequentially is used once; pages are
  evicted in least-recently-allocated order and remapped in the page table
  rather than freed and reallocated.

Rules (R1-R7) as implemented below:
  R1 on-demand: each missing page is one request of exactly one page.
  R2 demand run: a miss at page p takes d = number of consecutive non-present
     pages from p up to the last page p1 of the gread.
  R3 sync readahead: the access is sequential iff p == 0, or page p-1 of the
     file is present, or the stream's previous gread of this file ended at page
     p.  Not sequential: fetch [p, p+d) and record window 0.  Sequential:
     T = min(d + Wmax, max(4d, 2*Tprev)), Tprev = window recorded on the frame
     of page p-1 (0 if absent).  [p, p+T) is cut at EOF, at the first present
     page and at the readahead allowance (R6); n = pages actually requested;
     every frame of the request records window n; if n > d the page p+d gets
     the readahead mark with end = p+n.
  R4 async readahead: the first reader of a marked page clears the mark; if
     page `end` is not present it requests [end, end + min(Wmax, 2*T)) (T = the
     window recorded on the marked frame), cut as in R3; the first page of that
     request gets the mark with the new end.  Disabled by async_ra=False.
  R5 consumption: each delivered slice adds its length to the frame's consumed
     count; when it first reaches the page's valid bytes the frame is appended
     to the consumed FIFO.
  R6 victims: (1) never-used frames, lowest index first; (2) the consumed FIFO,
     oldest first; (3) only for the page the gread waits for (the first page of
     a demand run), when (1) and (2) are empty: the oldest-allocated frame not
     allocated during the current gread; later pages of the run end the request
     instead of evicting unconsumed pages.  Readahead
     pages take victims only from (1)/(2) and only while
     free + consumed > reserve.  Frames of the request being built and the
     frame of the page being delivered are never victims (a FIFO entry for the
     latter goes back to the tail).  An evicted frame is removed from the page
     table before reuse.
  A request never spans more than max_rpc_pages pages (the request-queue slot
  size); the window and the demand run are cut to it.
  R7 readahead is enabled only for read-only opens without the RANDOM hint;
     otherwise R1 applies.
  R8 data read sequentially is used once (Section 5.1): a readahead window is
     also cut at the first page already fetched since the last cache reset
     (it was read and evicted, or is being read); demand misses always fetch.
Paper mode (mode="paper"; Sections 4.1 and 5.1 as the paper designs them):
  P1 every stream (threadblock) has a private buffer; on a miss at page p the
     stream allocates a frame for p and looks in its buffer: if p is there the
     page is copied from it (no request); otherwise one request of
     1 + W pages (PAGE_SIZE + PREFETCH_SIZE, W = ra_cap, static) is sent, page p
     goes to the frame and pages p+1 .. p+W replace the buffer's contents.
     No window growth, no asynchronous readahead, no coordination between
     streams (two streams may prefetch the same pages).
  P2 replacement "tb_lra": each stream keeps the frames it allocated in
     allocation order, at most quota = max(1, F // streams) of them; below the
     quota it takes a never-used frame, at the quota it evicts its own least
     recently allocated frame and reuses it (remapping it in the page table);
     a frame of the request being built or the page being delivered is passed
     over (it moves to the newest end).  replacement "fifo" uses rule R6 instead.
     P2 also combines with modes "readahead" and "ondemand": every frame a
     request takes, demand or readahead, then comes from the requesting
     stream's queue, and the quota takes the place of the readahead reserve
     (readahead just stops when the stream has no frame to pass).
A demand page that finds no victim at all (every frame belongs to the current
gread) makes the gread return -ENOMEM; later pages of a demand run just end the
request early.
A page is READY only when the host read returned all of its bytes (its valid
size is P, or size - page*P for the last page); otherwise it is in state ERROR,
a gread reaching it returns -EIO, and the frame stays mapped until it is
evicted under (3).
"""
from __future__ import annotations

import os
from collections import deque
from dataclasses import dataclass, field

EMPTY, READY, ERROR = 0, 2, 3
DEMAND, SYNC_RA, ASYNC_RA = 0, 1, 2
KIND_NAMES = {DEMAND: "DEMAND", SYNC_RA: "SYNC_RA", ASYNC_RA: "ASYNC_RA"}

ADV_NORMAL, ADV_SEQUENTIAL, ADV_RANDOM = 0, 1, 2
EIO = 5
ENOMEM = 12


class NoFrame(RuntimeError):
    """No victim frame exists for a demand page (every frame belongs to the current gread)."""


@dataclass
class Frame:
    key: tuple | None = None      # (fid, page)
    state: int = EMPTY
    valid: int = 0                # bytes of the page that hold file data
    consumed: int = 0             # bytes delivered from this frame so far
    window: int = 0               # readahead window recorded on this frame
    ra_end: int = -1              # readahead mark: page after the window, -1 = none
    alloc_seq: int = -1           # allocation order
    data: bytes = b""


@dataclass
class FileInfo:
    fd: int
    size: int
    npages: int
    readonly: bool = True
    advice: int = ADV_NORMAL

    @property
    def readahead(self) -> bool:
        return self.readonly and self.advice != ADV_RANDOM


@dataclass
class Stats:
    greads: int = 0
    hits: int = 0
    misses: int = 0
    rpcs: int = 0
    pages_fetched: int = 0
    bytes_fetched: int = 0
    evictions: int = 0
    unconsumed_evictions: int = 0
    fetch_count: dict = field(default_factory=dict)  # (fid, page) -> times fetched
    buffer_hits: int = 0                              # paper mode: misses served from the private buffer


class PageCacheSim:
    """Single-threaded page cache over real files; one gread at a time."""

    def __init__(self, page_size: int, n_frames: int, mode: str = "readahead",
                 ra_cap: int = 8, reserve: int = 0, async_ra: bool = True,
                 read_fn=None, max_rpc_pages: int = 64, replacement: str = "fifo", streams: int = 1):
        if page_size <= 0 or n_frames <= 0:
            raise ValueError("page_size and n_frames must be positive")
        if mode not in ("readahead", "ondemand", "paper"):
            raise ValueError("mode must be 'readahead', 'ondemand' or 'paper'")
        self.P = page_size
        self.F = n_frames
        self.mode = mode
        self.Wmax = ra_cap
        self.reserve = reserve
        self.async_ra = async_ra
        self.max_rpc = max_rpc_pages
        if replacement not in ("fifo", "tb_lra"):
            raise ValueError("replacement must be 'fifo' or 'tb_lra'")
        self.replacement = replacement
        self.quota = max(1, n_frames // max(1, streams))
        self.lra: dict[int, deque] = {}          # P2: frames each stream allocated, oldest first
        self.privbuf: dict[int, tuple] = {}      # P1: stream -> (fid, {page: data})
        self.read_fn = read_fn or (lambda fd, off, n: os.pread(fd, n, off))
        self.frames = [Frame() for _ in range(n_frames)]
        self.table: dict[tuple, int] = {}
        self.next_unused = 0
        self.fifo: deque[int] = deque()
        self.alloc_counter = 0
        self.last_end: dict[tuple, int] = {}
        self.files: dict[int, FileInfo] = {}
        self.rpc_log: list[tuple] = []     # (fid, page_lo, npages, kind)
        self.evict_log: list[tuple] = []   # (frame, old_key, new_key)
        self.stats = Stats()
        self.fetched: set[tuple] = set()     # pages fetched since the last reset (R8)
        self._busy: set[int] = set()        # frames of the request being built
        self._pinned: int | None = None      # frame of the page being delivered

    # ---- files -----------------------------------------------------------
    def open(self, fid: int, path: str, readonly: bool = True, advice: int = ADV_NORMAL):
        fd = os.open(path, os.O_RDONLY)
        size = os.fstat(fd).st_size
        self.files[fid] = FileInfo(fd, size, (size + self.P - 1) // self.P, readonly, advice)

    def close_all(self):
        for fi in self.files.values():
            os.close(fi.fd)
        self.files.clear()

    def reset_cache(self):
        self.frames = [Frame() for _ in range(self.F)]
        self.table.clear()
        self.next_unused = 0
        self.fifo.clear()
        self.alloc_counter = 0
        self.last_end.clear()
        self.fetched.clear()
        self.lra.clear()
        self.privbuf.clear()

    def present(self, fid: int, page: int) -> bool:
        return (fid, page) in self.table

    # ---- R6: victims -------------------------------------------------------
    def _avail(self) -> int:
        return (self.F - self.next_unused) + len(self.fifo)

    def _evict(self, f: int, new_key):
        fr = self.frames[f]
        if fr.key is not None:
            del self.table[fr.key]
            self.evict_log.append((f, fr.key, new_key))
            self.stats.evictions += 1
            if fr.consumed < fr.valid or fr.state == ERROR:
                self.stats.unconsumed_evictions += 1

    def _take(self, for_readahead: bool, gread_seq0: int, new_key, fallback: bool = True) -> int | None:
        if for_readahead and self._avail() <= self.reserve:
            return None
        if self.next_unused < self.F:                      # (1)
            f = self.next_unused
            self.next_unused += 1
            return f
        for _ in range(len(self.fifo)):                     # (2)
            f = self.fifo.popleft()
            if f == self._pinned:
                self.fifo.append(f)
                continue
            self._evict(f, new_key)
            return f
        if for_readahead or not fallback:
            return None
        best = None                                         # (3)
        for f, fr in enumerate(self.frames):
            if (f in self._busy or f == self._pinned or fr.key is None
                    or fr.alloc_seq >= gread_seq0):
                continue
            if best is None or fr.alloc_seq < self.frames[best].alloc_seq:
                best = f
        if best is None:
            raise NoFrame("no victim frame for a demand page")
        self._evict(best, new_key)
        return best

    def _install(self, f: int, key: tuple):
        self.frames[f] = Frame(key=key, state=EMPTY, alloc_seq=self.alloc_counter)
        self.alloc_counter += 1
        self.table[key] = f
        self._busy.add(f)

    # ---- the host side of one request (Section 4.1, CPU modifications) ----
    def _fetch(self, fi: FileInfo, fid: int, page_lo: int, fr_list: list[int], kind: int):
        n = len(fr_list)
        self.rpc_log.append((fid, page_lo, n, kind))
        self.stats.rpcs += 1
        want = min(n * self.P, fi.size - page_lo * self.P)
        try:
            data = self.read_fn(fi.fd, page_lo * self.P, want)
        except OSError:
            data = b""
        for i, f in enumerate(fr_list):
            fr = self.frames[f]
            page = page_lo + i
            expect = min(self.P, fi.size - page * self.P)
            chunk = data[i * self.P:i * self.P + expect]
            full = len(chunk) == expect
            fr.data = chunk if full else b""
            fr.valid = expect if full else 0
            fr.state = READY if full else ERROR
            key = (fid, page)
            self.stats.pages_fetched += 1
            self.stats.bytes_fetched += len(chunk) if full else 0
            self.stats.fetch_count[key] = self.stats.fetch_count.get(key, 0) + 1
        self._busy.clear()

    def _request(self, stream: int, fi: FileInfo, fid: int, p: int, want: int, demand: int,
                 gread_seq0: int) -> list[int]:
        """Allocate frames for [p, p+want), cut at EOF / present page / allowance."""
        want = min(want, self.max_rpc)
        taken = []
        for q in range(p, p + want):
            if q >= fi.npages or (fid, q) in self.table:
                break
            if q - p >= demand and (fid, q) in self.fetched:      # R8
                break
            try:
                if self.replacement == "tb_lra":                   # P2
                    f = self._take_lra(stream, q - p >= demand, (fid, q))
                else:  # only the page the gread waits for may take an unconsumed victim (3)
                    f = self._take(q - p >= demand, gread_seq0, (fid, q), fallback=q == p)
            except NoFrame:
                if q == p:
                    raise
                f = None
            if f is None:
                break
            self._install(f, (fid, q))
            self.fetched.add((fid, q))
            taken.append(f)
        return taken

    # ---- paper mode (P1, P2) -----------------------------------------------------
    def _take_lra(self, stream: int, for_readahead: bool, new_key) -> int | None:
        """P2: the stream's own least recently allocated frame (None: readahead stops)."""
        q = self.lra.setdefault(stream, deque())
        if len(q) < self.quota and self.next_unused < self.F:
            f = self.next_unused
            self.next_unused += 1
            q.append(f)
            return f
        for _ in range(len(q)):
            f = q.popleft()
            q.append(f)
            if f == self._pinned or f in self._busy:
                continue
            self._evict(f, new_key)
            return f
        if for_readahead:
            return None
        raise NoFrame("stream has no frame to reuse")

    def _take_paper(self, stream: int, gread_seq0: int, new_key) -> int:
        if self.replacement == "fifo":
            return self._take(False, gread_seq0, new_key)
        return self._take_lra(stream, False, new_key)

    def _miss_paper(self, stream: int, fi: FileInfo, fid: int, p: int, gread_seq0: int):
        self.stats.misses += 1
        f = self._take_paper(stream, gread_seq0, (fid, p))
        self._install(f, (fid, p))
        self.fetched.add((fid, p))
        buf = self.privbuf.get(stream)
        if buf is not None and buf[0] == fid and p in buf[1]:          # P1: buffer hit
            fr = self.frames[f]
            fr.data = buf[1][p]
            fr.valid = len(fr.data)
            fr.state = READY
            self.stats.buffer_hits += 1
            self._busy.clear()
            return
        n = min(1 + self.Wmax, fi.npages - p, self.max_rpc)
        kind = SYNC_RA if n > 1 else DEMAND
        self.rpc_log.append((fid, p, n, kind))
        self.stats.rpcs += 1
        want = min(n * self.P, fi.size - p * self.P)
        try:
            data = self.read_fn(fi.fd, p * self.P, want)
        except OSError:
            data = b""
        pages = {}
        for i in range(n):
            q = p + i
            expect = min(self.P, fi.size - q * self.P)
            chunk = data[i * self.P:i * self.P + expect]
            if len(chunk) == expect:
                pages[q] = chunk
            self.stats.pages_fetched += 1
            self.stats.fetch_count[(fid, q)] = self.stats.fetch_count.get((fid, q), 0) + 1
        fr = self.frames[f]
        ok = p in pages
        fr.data = pages.get(p, b"")
        fr.valid = len(fr.data) if ok else 0
        fr.state = READY if ok else ERROR
        self.stats.bytes_fetched += fr.valid
        self.privbuf[stream] = (fid, {q: d for q, d in pages.items() if q != p})
        self._busy.clear()

    # ---- R1-R3: a miss ----------------------------------------------------------
    def _miss(self, stream: int, fi: FileInfo, fid: int, p: int, p1: int, gread_seq0: int):
        self.stats.misses += 1
        if self.mode != "readahead" or not fi.readahead:            # R1 / R7
            taken = self._request(stream, fi, fid, p, 1, 1, gread_seq0)
            self._fetch(fi, fid, p, taken, DEMAND)
            return
        d = 0                                                         # R2
        while p + d <= p1 and d < self.max_rpc and (fid, p + d) not in self.table:
            d += 1
        seq = (p == 0 or (fid, p - 1) in self.table
               or self.last_end.get((stream, fid)) == p)              # R3
        if not seq:
            taken = self._request(stream, fi, fid, p, d, d, gread_seq0)
            self._fetch(fi, fid, p, taken, DEMAND)
            for f in taken:
                self.frames[f].window = 0
            return
        prev = self.table.get((fid, p - 1)) if p > 0 else None
        t_prev = self.frames[prev].window if prev is not None else 0
        T = min(d + self.Wmax, max(4 * d, 2 * t_prev), self.max_rpc)
        taken = self._request(stream, fi, fid, p, T, d, gread_seq0)
        n = len(taken)
        self._fetch(fi, fid, p, taken, SYNC_RA if n > d else DEMAND)
        for f in taken:
            self.frames[f].window = n
        if n > d:
            self.frames[taken[d]].ra_end = p + n

    # ---- R4: a readahead mark ---------------------------------------------------
    def _async(self, stream: int, fi: FileInfo, fid: int, end: int, t: int, gread_seq0: int):
        if end >= fi.npages or (fid, end) in self.table or (fid, end) in self.fetched:
            return
        taken = self._request(stream, fi, fid, end, min(self.Wmax, 2 * t), 0, gread_seq0)
        if not taken:
            return
        n = len(taken)
        self._fetch(fi, fid, end, taken, ASYNC_RA)
        for f in taken:
            self.frames[f].window = n
        self.frames[taken[0]].ra_end = end + n

    # ---- the gread -----------------------------------------------------------------
    def gread(self, stream: int, fid: int, off: int, length: int) -> tuple[int, bytes]:
        """One threadblock-collective read; returns (count or -errno, bytes delivered)."""
        fi = self.files.get(fid)
        if fi is None:
            return -9, b""                                            # -EBADF
        if off < 0 or length < 0:
            return -22, b""                                           # -EINVAL
        self.stats.greads += 1
        if off >= fi.size or length == 0:
            return 0, b""
        end = min(off + length, fi.size)
        p0, p1 = off // self.P, (end - 1) // self.P
        seq0 = self.alloc_counter
        out = []
        ret = None
        for p in range(p0, p1 + 1):
            key = (fid, p)
            if key in self.table:
                self.stats.hits += 1
            else:
                try:
                    if self.mode == "paper" and fi.readahead:
                        self._miss_paper(stream, fi, fid, p, seq0)
                    else:
                        self._miss(stream, fi, fid, p, p1, seq0)
                except NoFrame:
                    ret = -ENOMEM
                    break
            f = self.table[key]
            fr = self.frames[f]
            if fr.state == ERROR:
                ret = -EIO
                break
            if fr.ra_end >= 0:                                        # R4
                mark, fr.ra_end = fr.ra_end, -1
                if self.async_ra and self.mode == "readahead" and fi.readahead:
                    self._pinned = f
                    self._async(stream, fi, fid, mark, fr.window, seq0)
                    self._pinned = None
            base = p * self.P
            lo = max(off, base) - base
            hi = min(end, base + self.P) - base
            piece = fr.data[lo:hi]
            out.append(piece)
            before = fr.consumed                                      # R5
            fr.consumed += len(piece)
            if before < fr.valid <= fr.consumed:
                self.fifo.append(f)
        self.last_end[(stream, fid)] = p1 + 1
        data = b"".join(out)
        return (ret if ret is not None else len(data)), data


def canonical_scan_trace(size: int, stride: int, blocks: int, read_len: int | None = None,
                         fid: int = 0):
    """Serialized order of the stride scan: step k, then block b (stride s = k*B + b)."""
    read_len = stride if read_len is None else read_len
    ns = (size + stride - 1) // stride if size > 0 else 0
    for s in range(ns):
        yield (s % blocks, fid, s * stride, read_len)


def default_reserve(blocks: int, read_len: int, page_size: int) -> int:
    """Demand reserve: one gread's pages per concurrent stream, plus one."""
    return blocks * ((read_len + page_size - 1) // page_size) + 1


def run_scan(path: str, page_size: int, n_frames: int, stride: int, blocks: int,
             mode: str = "readahead", ra_cap: int = 8, reserve: int | None = None,
             async_ra: bool = True, read_len: int | None = None, keep_data: bool = False,
             max_rpc_pages: int = 64, replacement: str = "fifo"):
    """Run the stride scan through the simulator in canonical order.

    Returns (sim, results) with results[s] = (count, sum, hash, data-or-None) per
    stride s, the checksums as defined in oracle.plain.
    """
    from .plain import byte_sum, pos_hash
    read_len = stride if read_len is None else read_len
    if reserve is None:
        reserve = default_reserve(blocks, read_len, page_size)
    sim = PageCacheSim(page_size, n_frames, mode, ra_cap, reserve, async_ra,
                       max_rpc_pages=max_rpc_pages, replacement=replacement, streams=blocks)
    sim.open(0, path)
    results = []
    try:
        for stream, fid, off, ln in canonical_scan_trace(sim.files[0].size, stride, blocks, read_len):
            n, data = sim.gread(stream, fid, off, ln)
            results.append((n, byte_sum(data), pos_hash(data, off), data if keep_data else None))
    finally:
        sim.close_all()
    return sim, results
