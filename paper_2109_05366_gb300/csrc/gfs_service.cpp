// Host I/O service of the GPU file-read path.  Plain C++ (no CUDA calls here:
// the sink decides how served bytes reach the frames).
#include "gfs_service.h"

#include <errno.h>
#include <sys/prctl.h>
#include <time.h>
#include <unistd.h>

#include <algorithm>
#include <chrono>
#include <cstring>

namespace gfs {

static inline uint64_t mono_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

IoService::IoService(const ServiceConfig& cfg, SinkFactory make_sink, FileLookup files, Control control)
    : cfg_(cfg), make_sink_(std::move(make_sink)), files_(std::move(files)), control_(std::move(control)) {
  tstats_.reset(new ThreadCounters[cfg_.threads ? cfg_.threads : 1]);
  io_trace_.resize(cfg_.io_trace_cap);
  t0_ns_.store(mono_ns());
}

IoService::~IoService() { stop(); }

int IoService::start() {
  stop_.store(false);
  for (uint32_t i = 0; i < cfg_.threads; ++i) {
    Sink* s = make_sink_((int)i);
    if (!s) {
      stop();
      return -ENOMEM;
    }
    sinks_.push_back(s);
  }
  try {
    for (uint32_t i = 0; i < cfg_.threads; ++i) threads_.emplace_back(&IoService::run, this, (int)i);
  } catch (...) {
    stop();
    return -EAGAIN;
  }
  return 0;
}

void IoService::stop() {
  stop_.store(true);
  for (auto& t : threads_)
    if (t.joinable()) t.join();
  threads_.clear();
  for (Sink* s : sinks_) {
    s->drain();
    delete s;
  }
  sinks_.clear();
}

void IoService::drain_sinks() {
  for (Sink* s : sinks_) s->drain();
}

void IoService::set_faults(uint32_t eio_every, uint32_t short_every, uint32_t delay_us) {
  eio_every_.store(eio_every);
  short_every_.store(short_every);
  delay_us_.store(delay_us);
}

void IoService::clear_stats() {
  stats.clear();
  for (uint32_t i = 0; i < cfg_.threads; ++i) {
    ThreadCounters& c = tstats_[i];
    c.got_first.store(false, std::memory_order_relaxed);
    c.requests = 0;
    c.polls_before_first = 0;
    c.first_ns = 0;
    c.idle_ns = 0;
    c.pread_ns = 0;
    c.bytes = 0;
  }
  io_n_.store(0, std::memory_order_release);
  t0_ns_.store(mono_ns(), std::memory_order_release);
}

void IoService::polled_empty(int idx, uint64_t idle_ns) {
  ThreadCounters& c = tstats_[idx];
  if (!c.got_first.load(std::memory_order_relaxed)) c.polls_before_first.fetch_add(1, std::memory_order_relaxed);
  if (idle_ns) c.idle_ns.fetch_add(idle_ns, std::memory_order_relaxed);
}

void IoService::took_request(int idx) {
  ThreadCounters& c = tstats_[idx];
  c.requests.fetch_add(1, std::memory_order_relaxed);
  if (!c.got_first.load(std::memory_order_relaxed)) {
    const uint64_t t0 = t0_ns_.load(std::memory_order_relaxed), now = mono_ns();
    c.first_ns.store(now > t0 ? now - t0 : 1, std::memory_order_relaxed);
    c.got_first.store(true, std::memory_order_relaxed);
  }
}

void IoService::record_io(int idx, uint32_t fid, uint64_t off, uint64_t bytes, uint64_t t_ns) {
  if (io_trace_.empty()) return;
  const uint64_t i = io_n_.fetch_add(1, std::memory_order_relaxed);
  if (i >= io_trace_.size()) return;
  gfs_io_rec& r = io_trace_[i];
  r.offset = off;
  r.bytes = bytes;
  r.fid = fid;
  r.thread = (uint32_t)idx;
  r.t_ns = t_ns;
}

// Read n bytes at off into buf (looping over short reads; stops at EOF).  With
// O_DIRECT the length is rounded up to whole 4 KiB blocks (offsets and staging
// buffers are page aligned already; a read past EOF just returns less).
ssize_t IoService::do_pread(int idx, const FileView& fv, uint8_t* buf, size_t n, uint64_t off) {
  const int fd = fv.fd;
  const uint64_t k = pread_count_.fetch_add(1, std::memory_order_relaxed);
  const uint32_t eio = eio_every_.load(std::memory_order_relaxed);
  const uint32_t sh = short_every_.load(std::memory_order_relaxed);
  const uint32_t delay = delay_us_.load(std::memory_order_relaxed);
  if (delay) usleep(delay);
  if (eio && k % eio == eio - 1) return -EIO;
  if (sh && k % sh == sh - 1) n /= 2;
  const uint64_t t0 = mono_ns();
  struct Acc {
    std::atomic<uint64_t>& a;
    std::atomic<uint64_t>& b;
    uint64_t t0;
    ~Acc() {
      const uint64_t d = mono_ns() - t0;
      a.fetch_add(d, std::memory_order_relaxed);
      b.fetch_add(d, std::memory_order_relaxed);
    }
  } acc{stats.ns_pread, tstats_[idx].pread_ns, t0};
  const size_t want = n;
  if (fv.direct) n = (n + 4095) & ~(size_t)4095;
  size_t got = 0;
  while (got < n) {
    ssize_t r = ::pread(fd, buf + got, n - got, (off_t)(off + got));
    if (r < 0) {
      if (errno == EINTR) continue;
      return got ? (ssize_t)std::min(got, want) : -errno;
    }
    if (r == 0) break;  // EOF
    got += (size_t)r;
  }
  return (ssize_t)std::min(got, want);
}

void IoService::serve(Worker& w, uint32_t fid, uint64_t page_lo, uint32_t npages, const uint32_t* frames) {
  Sink* sink = w.sink;
  int& cur = w.cur;
  FileView fv{-1, 0, 0, false};
  const bool have = files_(fid, &fv);
  const uint64_t P = cfg_.page_size;
  const uint64_t off0 = page_lo << cfg_.page_shift;
  if (have && off0 < fv.size)
    record_io(w.idx, fid, off0, std::min<uint64_t>((uint64_t)npages * P, fv.size - off0), mono_ns());
  if (w.full.size() < cfg_.staging_pages) w.full.resize(cfg_.staging_pages);
  uint8_t* full = w.full.data();
  for (uint32_t c0 = 0; c0 < npages; c0 += cfg_.staging_pages) {
    const uint32_t cn = std::min(cfg_.staging_pages, npages - c0);
    const uint64_t coff = off0 + (uint64_t)c0 * P;
    const int k = cur;
    sink->wait_staging(k);
    uint8_t* buf = sink->staging(k);
    size_t want = 0;
    if (have && coff < fv.size) want = (size_t)std::min<uint64_t>((uint64_t)cn * P, fv.size - coff);
    ssize_t got = 0;
    if (want) {
      got = do_pread(w.idx, fv, buf, want, coff);
      stats.preads.fetch_add(1, std::memory_order_relaxed);
      if (got < 0) {
        stats.errors.fetch_add(1, std::memory_order_relaxed);
        got = 0;
      } else {
        stats.bytes.fetch_add((uint64_t)got, std::memory_order_relaxed);
        tstats_[w.idx].bytes.fetch_add((uint64_t)got, std::memory_order_relaxed);
      }
    }
    // Section 4.1: the returned size decides which pages are delivered.
    for (uint32_t i = 0; i < cn; ++i) {
      const uint64_t base = coff + (uint64_t)i * P;
      const uint64_t expect = (have && base < fv.size) ? std::min<uint64_t>(P, fv.size - base) : 0;
      full[i] = expect > 0 && (uint64_t)got >= (uint64_t)i * P + expect ? 1 : 0;
    }
    for (uint32_t i = 0; i < cn;) {
      if (!full[i]) {
        ++i;
        continue;
      }
      uint32_t j = i + 1;
      while (j < cn && full[j] && frames[c0 + j] == frames[c0 + j - 1] + 1) ++j;
      const uint64_t last_base = coff + (uint64_t)(j - 1) * P;
      const uint64_t bytes = (uint64_t)(j - 1 - i) * P + std::min<uint64_t>(P, fv.size - last_base);
      if (sink->copy(frames[c0 + i], buf + (size_t)i * P, (size_t)bytes) != 0) {
        stats.errors.fetch_add(1, std::memory_order_relaxed);
        for (uint32_t q = i; q < j; ++q) full[q] = 0;
      } else {
        stats.copies.fetch_add(1, std::memory_order_relaxed);
      }
      i = j;
    }
    for (uint32_t i = 0; i < cn; ++i) sink->set_state(frames[c0 + i], full[i] ? FR_READY : FR_ERROR);
    sink->end_chunk(k);
    cur ^= 1;
  }
}

void IoService::serve_pull(Worker& w, uint32_t fid, const Req* group, int ng) {
  const int idx = w.idx;
  uint32_t& cur = w.pull_cur;
  FileView fv{-1, 0, 0, false};
  const bool have = files_(fid, &fv);
  const uint64_t P = cfg_.page_size;
  const uint64_t off0 = group[0].page_lo << cfg_.page_shift;
  uint64_t npages = 0;
  for (int k = 0; k < ng; ++k) npages += group[k].npages;
  if (have && off0 < fv.size) record_io(idx, fid, off0, std::min<uint64_t>(npages * P, fv.size - off0), mono_ns());
  auto publish_done = [&](const Req& r, long long result) {
    PullDone* d = cfg_.pull_done + r.slot;
    __atomic_store_n(&d->result, result, __ATOMIC_RELAXED);
    __atomic_store_n(&d->done, r.ticket + 1, __ATOMIC_RELEASE);
  };
  if (have && fv.dev_map) {  // mapped file: the pages are already in host memory the GPU can read
    for (int k = 0; k < ng; ++k) {
      const Req& r = group[k];
      // injected host read errors apply here too (the request fails as a whole)
      const uint64_t c = pread_count_.fetch_add(1, std::memory_order_relaxed);
      const uint32_t eio = eio_every_.load(std::memory_order_relaxed);
      const bool fail = eio && c % eio == eio - 1;
      long long total = 0;
      if (fail) {
        stats.errors.fetch_add(1, std::memory_order_relaxed);
        total = -EIO;
      }
      const uint64_t roff = r.page_lo << cfg_.page_shift;
      for (uint32_t i = 0; i < r.npages; ++i) {
        const uint64_t base = roff + (uint64_t)i * P;
        PullPage* pp = cfg_.pull_pages + (size_t)r.slot * cfg_.max_pages + i;
        pp->src = fv.dev_map + base;
        pp->buf = BUF_MAPPED;
        pp->ok = (!fail && base < fv.size) ? 1u : 0u;
        if (!fail && base < fv.size) total += (long long)std::min<uint64_t>(P, fv.size - base);
        __atomic_store_n(&pp->tag, r.ticket + 1, __ATOMIC_RELEASE);
      }
      if (total > 0) {
        stats.bytes.fetch_add((uint64_t)total, std::memory_order_relaxed);
        tstats_[idx].bytes.fetch_add((uint64_t)total, std::memory_order_relaxed);
      }
      publish_done(r, total);
    }
    return;
  }
  // The group's pages in file order, one pread per staging buffer: request k's
  // page i goes to its own slot's descriptor, and request k's completion record is
  // published after its last page.
  const uint32_t cpages = (uint32_t)(cfg_.chunk_bytes >> cfg_.page_shift);
  long long result[kMaxGroup];
  for (int k = 0; k < ng; ++k) result[k] = have ? 0 : -EBADF;
  int k = 0;
  uint32_t i = 0;
  for (uint64_t g0 = 0; g0 < npages; g0 += cpages) {
    const uint32_t cn = (uint32_t)std::min<uint64_t>(cpages, npages - g0);
    const uint32_t id = (uint32_t)idx * cfg_.bufs_per_thread + cur;
    cur = (cur + 1) % cfg_.bufs_per_thread;
    uint8_t* buf = cfg_.pull_arena + (size_t)id * cfg_.chunk_bytes;
    uint64_t spins = 0;
    if (__atomic_load_n(&cfg_.pull_bcount[id], __ATOMIC_ACQUIRE) != 0) {
      const uint64_t w0 = mono_ns();
      while (__atomic_load_n(&cfg_.pull_bcount[id], __ATOMIC_ACQUIRE) != 0) {  // GPU still copying out of it
        if (stop_.load(std::memory_order_relaxed)) return;
        if (++spins > 20000) {
          struct timespec ts = {0, 2000};
          nanosleep(&ts, nullptr);
        }
      }
      stats.ns_wait_buf.fetch_add(mono_ns() - w0, std::memory_order_relaxed);
    }
    const uint64_t coff = off0 + g0 * P;
    size_t want = 0;
    if (have && coff < fv.size) want = (size_t)std::min<uint64_t>((uint64_t)cn * P, fv.size - coff);
    ssize_t got = 0;
    long long err = 0;
    if (want) {
      got = do_pread(idx, fv, buf, want, coff);
      stats.preads.fetch_add(1, std::memory_order_relaxed);
      if (got < 0) {
        stats.errors.fetch_add(1, std::memory_order_relaxed);
        err = got;
        got = 0;
      } else {
        stats.bytes.fetch_add((uint64_t)got, std::memory_order_relaxed);
        tstats_[idx].bytes.fetch_add((uint64_t)got, std::memory_order_relaxed);
      }
    }
    __atomic_store_n(&cfg_.pull_bcount[id], cn, __ATOMIC_RELAXED);  // published by the page tags below
    for (uint32_t j = 0; j < cn; ++j) {
      const Req& r = group[k];
      const uint64_t base = coff + (uint64_t)j * P;
      const uint64_t expect = (have && base < fv.size) ? std::min<uint64_t>(P, fv.size - base) : 0;
      const bool ok = expect > 0 && (uint64_t)got >= (uint64_t)j * P + expect;
      PullPage* pp = cfg_.pull_pages + (size_t)r.slot * cfg_.max_pages + i;
      pp->src = (uint64_t)id * cfg_.chunk_bytes + (uint64_t)j * P;
      pp->buf = id;
      pp->ok = ok ? 1u : 0u;
      if (result[k] >= 0) result[k] = err ? err : result[k] + (long long)(ok ? expect : 0);
      __atomic_store_n(&pp->tag, r.ticket + 1, __ATOMIC_RELEASE);  // the GPU may copy this page now
      if (++i == r.npages) {
        publish_done(r, result[k]);
        ++k;
        i = 0;
      }
    }
  }
  for (; k < ng; ++k) publish_done(group[k], result[k]);  // requests with no page (none in practice)
}

// Answer a control request from the device in the slot's payload.  The slot
// stays taken: the requesting warp frees it once it has read the answer.
void IoService::control(RingSlot* s, uint32_t slot, uint32_t op, uint32_t fid) {
  CtlMsg* m = reinterpret_cast<CtlMsg*>(s->frames);
  CtlMsg ans{};
  ans.arg = ((volatile CtlMsg*)m)->arg;
  ans.status = -ENOTSUP;
  if (control_) {
    char path[GFS_PATH_MAX];
    path[0] = '\0';
    if (op == OP_OPEN && cfg_.paths) {
      memcpy(path, cfg_.paths + (size_t)slot * GFS_PATH_MAX, GFS_PATH_MAX);
      path[GFS_PATH_MAX - 1] = '\0';
    }
    control_(op, fid, ans.arg, path, &ans);
  }
  m->status = ans.status;
  m->last = ans.last;
  __atomic_store_n(&m->done, 1u, __ATOMIC_RELEASE);
}

void IoService::run(int idx) {
  Worker w{idx, sinks_[idx], 0, 0u, {}, {}};
  w.sink->thread_init();
  prctl(PR_SET_TIMERSLACK, 1000UL, 0, 0, 0);  // short sleeps while polling the ring
  if (cfg_.queue == GFS_QUEUE_STATIC) run_static(w);
  else run_shared(w);
}

bool IoService::skip_cancelled(uint64_t h, RingSlot* s) {
  if (!cfg_.cancel || !cfg_.cancel_n) return false;
  unsigned long long* c = &cfg_.cancel[h % cfg_.cancel_n];
  if (__atomic_load_n(c, __ATOMIC_ACQUIRE) != h + 1 || __atomic_load_n(&s->seq, __ATOMIC_ACQUIRE) != h) return false;
  __atomic_store_n(c, 0ull, __ATOMIC_RELAXED);
  __atomic_store_n(&s->seq, h + cfg_.slots, __ATOMIC_RELEASE);  // the slot is free for the next lap
  if (cfg_.skipped) __atomic_fetch_add(cfg_.skipped, 1ull, __ATOMIC_RELEASE);
  stats.skipped.fetch_add(1, std::memory_order_relaxed);
  served_.fetch_add(1, std::memory_order_release);
  return true;
}

// GFS_QUEUE_SHARED: take the next ticket and wait for its request (or its
// cancellation).
void IoService::run_shared(Worker& w) {
  while (!stop_.load(std::memory_order_relaxed)) {
    const uint64_t h = head_.fetch_add(1, std::memory_order_relaxed);
    RingSlot* s = (RingSlot*)(cfg_.ring + (size_t)(h % cfg_.slots) * cfg_.slot_stride);
    uint64_t spins = 0;
    const uint64_t i0 = mono_ns();
    bool skipped = false;
    while (__atomic_load_n(&s->seq, __ATOMIC_ACQUIRE) != h + 1) {
      if (stop_.load(std::memory_order_relaxed)) return;
      if ((spins & 63) == 0 && skip_cancelled(h, s)) {
        skipped = true;
        break;
      }
      ++spins;
      polled_empty(w.idx, 0);
      if (spins > 20000) {
        struct timespec ts = {0, spins > 2000000 ? 50000 : 2000};
        nanosleep(&ts, nullptr);
      }
    }
    const uint64_t idle = mono_ns() - i0;
    stats.ns_idle.fetch_add(idle, std::memory_order_relaxed);
    tstats_[w.idx].idle_ns.fetch_add(idle, std::memory_order_relaxed);
    if (!skipped) handle(w, h, s);
  }
}

// GFS_QUEUE_STATIC (Section 3.2): thread k owns slots [k R / T, (k+1) R / T)
// and sweeps them in turn; slot i's uses have tickets i, i + R, i + 2R, ...
void IoService::run_static(Worker& w) {
  const uint32_t T = cfg_.threads, R = cfg_.slots;
  const uint32_t lo = (uint32_t)((uint64_t)w.idx * R / T), hi = (uint32_t)((uint64_t)(w.idx + 1) * R / T);
  std::vector<uint64_t> lap(hi > lo ? hi - lo : 0, 0);
  uint64_t sweeps = 0;
  uint64_t i0 = mono_ns();
  while (!stop_.load(std::memory_order_relaxed)) {
    bool any = false;
    for (uint32_t si = lo; si < hi; ++si) {
      const uint64_t h = lap[si - lo] * R + si;
      RingSlot* s = (RingSlot*)(cfg_.ring + (size_t)si * cfg_.slot_stride);
      if (__atomic_load_n(&s->seq, __ATOMIC_ACQUIRE) != h + 1) {
        if (skip_cancelled(h, s)) ++lap[si - lo];
        continue;
      }
      const uint64_t idle = mono_ns() - i0;
      stats.ns_idle.fetch_add(idle, std::memory_order_relaxed);
      tstats_[w.idx].idle_ns.fetch_add(idle, std::memory_order_relaxed);
      ++lap[si - lo];
      any = true;
      handle(w, h, s);
      i0 = mono_ns();
    }
    if (any) {
      sweeps = 0;
      continue;
    }
    polled_empty(w.idx, 0);
    if (++sweeps > 20000) {
      struct timespec ts = {0, sweeps > 2000000 ? 50000 : 2000};
      nanosleep(&ts, nullptr);
    }
  }
}

int IoService::gather(Worker& w, uint32_t fid, Req* group, uint32_t max_pages_each) {
  if (cfg_.queue != GFS_QUEUE_SHARED || cfg_.merge_pages <= 1) return 1;
  // The requests waiting at the head of the ring: published, not drawn by any
  // thread (idle threads draw tickets before they are published, so a waiting
  // request means every thread is busy), reads of the same file.
  const uint64_t u = head_.load(std::memory_order_acquire);
  uint64_t pages = group[0].npages;
  int k = 0;
  while (1 + k < kMaxGroup) {
    const uint64_t t = u + (uint64_t)k;
    RingSlot* st = (RingSlot*)(cfg_.ring + (size_t)(t % cfg_.slots) * cfg_.slot_stride);
    if (__atomic_load_n(&st->seq, __ATOMIC_ACQUIRE) != t + 1) break;  // not published (yet)
    // Read before claiming: while no thread has drawn ticket t its slot keeps its
    // request; if one has, the claim below fails and what was read is dropped.
    const volatile RingSlot* vt = st;
    const uint32_t op = vt->op, f2 = vt->fid, n2 = vt->npages;
    const uint64_t lo2 = vt->page_lo;
    if (op != OP_READ || f2 != fid || n2 == 0 || n2 > max_pages_each || pages + n2 > cfg_.merge_pages) break;
    group[1 + k] = Req{t, (uint32_t)(t % cfg_.slots), n2, lo2};
    pages += n2;
    ++k;
  }
  if (k == 0) return 1;
  uint64_t expect = u;
  if (!head_.compare_exchange_strong(expect, u + (uint64_t)k, std::memory_order_acq_rel)) return 1;  // drawn meanwhile
  for (int i = 0; i < k; ++i) {
    took_request(w.idx);
    stats.requests.fetch_add(1, std::memory_order_relaxed);
  }
  return 1 + k;
}

void IoService::handle(Worker& w, uint64_t h, RingSlot* s) {
  took_request(w.idx);
  const volatile RingSlot* vs = s;
  const uint32_t fid = vs->fid;
  const uint32_t npages = vs->npages;
  const uint64_t page_lo = vs->page_lo;
  const uint32_t op = vs->op;
  if (op == OP_OPEN || op == OP_CLOSE || op == OP_ADVISE) {
    control(s, (uint32_t)(h % cfg_.slots), op, fid);
    stats.controls.fetch_add(1, std::memory_order_relaxed);
    served_.fetch_add(1, std::memory_order_release);
    return;
  }
  stats.requests.fetch_add(1, std::memory_order_relaxed);
  const uint32_t max_each = cfg_.pull_arena ? cfg_.max_pages : MAX_RPC_PAGES;
  Req group[kMaxGroup];
  group[0] = Req{h, (uint32_t)(h % cfg_.slots), std::min(npages, max_each), page_lo};
  FileView fv{-1, 0, 0, false};
  // a mapped file has no host read to share: its requests are served one by one
  const bool mergeable = npages >= 1 && npages <= max_each && files_(fid, &fv) && !fv.dev_map;
  const int ng = mergeable ? gather(w, fid, group, max_each) : 1;
  // in file order; each maximal run of requests whose pages continue one another is
  // served with one host read per staging buffer
  std::sort(group, group + ng, [](const Req& a, const Req& b) {
    return a.page_lo != b.page_lo ? a.page_lo < b.page_lo : a.ticket < b.ticket;
  });
  auto for_runs = [&](auto&& serve_run) {
    for (int i = 0; i < ng;) {
      int j = i + 1;
      while (j < ng && group[j].npages && group[j - 1].npages &&
             group[j - 1].page_lo + group[j - 1].npages == group[j].page_lo)
        ++j;
      if (group[i].npages) {
        if (j - i > 1) stats.merged.fetch_add((uint64_t)(j - i - 1), std::memory_order_relaxed);
        serve_run(i, j);
      }
      i = j;
    }
  };
  if (cfg_.pull_arena) {  // the GPU frees the slots once it has copied the pages
    for_runs([&](int i, int j) { serve_pull(w, fid, group + i, j - i); });
    served_.fetch_add((uint64_t)ng, std::memory_order_release);
    return;
  }
  // copy-engine transfer: take the frame lists out and free the slots for their next lap
  uint64_t total = 0;
  for (int k = 0; k < ng; ++k) total += group[k].npages;
  if (w.frames.size() < total) w.frames.resize(total);
  uint32_t* frames = w.frames.data();
  uint64_t at[kMaxGroup];
  uint64_t pos = 0;
  for (int k = 0; k < ng; ++k) {
    RingSlot* sk = (RingSlot*)(cfg_.ring + (size_t)group[k].slot * cfg_.slot_stride);
    const volatile RingSlot* vk = sk;
    const uint32_t nk = group[k].npages;
    bool bad = nk == 0 || (group[k].ticket == h && (npages == 0 || npages > MAX_RPC_PAGES));
    for (uint32_t i = 0; i < nk; ++i) frames[pos + i] = vk->frames[i];
    __atomic_store_n(&sk->seq, group[k].ticket + cfg_.slots, __ATOMIC_RELEASE);  // slot free for the next lap
    for (uint32_t i = 0; i < nk && !bad; ++i) bad = frames[pos + i] >= cfg_.n_frames;
    if (bad) {
      stats.errors.fetch_add(1, std::memory_order_relaxed);
      group[k].npages = 0;  // not served: its pages stay FILLING until the device deadline
    }
    at[k] = pos;
    pos += nk;
  }
  for_runs([&](int i, int j) {
    // the run's frame lists, in page order (its requests are consecutive in `frames` only
    // when no bad request sits between them, which for_runs guarantees)
    uint32_t n = 0;
    for (int k = i; k < j; ++k) n += group[k].npages;
    if (j - i == 1) {
      serve(w, fid, group[i].page_lo, n, frames + at[i]);
      return;
    }
    if (w.run.size() < n) w.run.resize(n);
    uint32_t q = 0;
    for (int k = i; k < j; ++k)
      for (uint32_t x = 0; x < group[k].npages; ++x) w.run[q++] = frames[at[k] + x];
    serve(w, fid, group[i].page_lo, n, w.run.data());
  });
  served_.fetch_add((uint64_t)ng, std::memory_order_release);
}

}  // namespace gfs
