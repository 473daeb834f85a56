// Host I/O service: threads that serve the request ring (Section 2.2: host
// threads poll the shared queue, pread the file and send the data to the GPU;
// Section 4.1: one pread serves every page of a readahead request, and the
// returned size decides which pages are delivered).
//
// GFS_QUEUE_SHARED (default): every thread takes the next ticket of one shared
// ring.  GFS_QUEUE_STATIC is GPUfs as Section 3.2 describes it: each thread
// polls a fixed slice of the slots, which leaves threads idle when the running
// threadblocks map to other slices.
#pragma once

#include <atomic>
#include <cstdint>
#include <functional>
#include <memory>
#include <thread>
#include <vector>

#include "gfs_internal.h"

namespace gfs {

// Where served pages go.  One instance per I/O thread.
class Sink {
 public:
  virtual ~Sink() = default;
  // Called once on the I/O thread before it serves anything.
  virtual void thread_init() {}
  // Staging buffer k (0/1) of this thread; wait until the previous use is done.
  virtual uint8_t* staging(int k) = 0;
  virtual void wait_staging(int k) = 0;
  // Copy `bytes` from staging to the frame run starting at `frame` (contiguous frames).
  virtual int copy(uint32_t frame, const uint8_t* src, size_t bytes) = 0;
  // Set the state word of a frame after the copies issued so far.
  virtual int set_state(uint32_t frame, uint32_t state) = 0;
  // Flush state writes; mark staging k in use until the queued work completes.
  virtual int end_chunk(int k) = 0;
  // Wait for everything this sink queued.
  virtual void drain() = 0;
};

struct FileView {
  int fd;
  uint64_t size;
  uint64_t dev_map;  // device address of the file's registered mapping, 0 if not mapped
  bool direct;       // fd was opened with O_DIRECT: reads are whole 4 KiB blocks into aligned buffers
};

struct ServiceConfig {
  uint8_t* ring = nullptr;  // host view of the ring
  uint32_t slots = 0, slot_stride = 0;
  uint32_t page_size = 0, page_shift = 0;
  uint32_t staging_pages = 1;  // pages per staging buffer
  uint32_t threads = 1;
  uint32_t n_frames = 0xffffffffu;  // frame indices at or above this are rejected
  // GFS_XFER_PULL: every thread preads through its own ring of small staging
  // buffers (small enough to stay in the CPU caches), publishes per-page
  // descriptors and a per-request completion record; the GPU copies the pages,
  // releases the buffers and frees the slot.
  uint8_t* pull_arena = nullptr;
  PullDone* pull_done = nullptr;
  PullPage* pull_pages = nullptr;
  uint32_t* pull_bcount = nullptr;
  uint64_t chunk_bytes = 0;
  uint32_t bufs_per_thread = 0;
  uint32_t max_pages = 0;
  // device opens: per-slot path buffers (host view), GFS_PATH_MAX bytes each
  const char* paths = nullptr;
  uint32_t queue = GFS_QUEUE_SHARED;  // GFS_QUEUE_*: how a thread finds its requests
  // GFS_QUEUE_SHARED: a thread that takes a read also claims the requests waiting
  // at the head of the ring (published, drawn by no thread) that read the same
  // file, up to this many pages in all, and serves each run of them whose pages
  // continue one another with one read (<= 1: one request at a time)
  uint32_t merge_pages = 1;
  uint64_t io_trace_cap = 0;          // host I/O trace entries kept (0 = off)
  // at t % cancel_n: t + 1 for a ticket t its producer gave up (skipped once the slot
  // is free for it); count of skipped tickets.  Host views of mapped memory; may be null.
  unsigned long long* cancel = nullptr;
  uint32_t cancel_n = 0;
  unsigned long long* skipped = nullptr;
};

// Counters of one host thread (gfs_thread_stat).
struct ThreadCounters {
  std::atomic<uint64_t> requests{0}, polls_before_first{0}, first_ns{0}, idle_ns{0}, pread_ns{0}, bytes{0};
  std::atomic<bool> got_first{false};
};

struct ServiceStats {
  std::atomic<uint64_t> requests{0}, preads{0}, bytes{0}, copies{0}, errors{0};
  std::atomic<uint64_t> ns_pread{0}, ns_wait_buf{0}, ns_idle{0};
  std::atomic<uint64_t> controls{0};  // device opens and closes answered
  std::atomic<uint64_t> skipped{0};   // tickets skipped because their producer gave them up
  std::atomic<uint64_t> merged{0};    // requests served together with the request before them
  void clear() {
    requests = 0; preads = 0; bytes = 0; copies = 0; errors = 0;
    ns_pread = 0; ns_wait_buf = 0; ns_idle = 0; controls = 0; skipped = 0; merged = 0;
  }
};

class IoService {
 public:
  using SinkFactory = std::function<Sink*(int thread_index)>;
  using FileLookup = std::function<bool(uint32_t fid, FileView* out)>;
  // OP_OPEN / OP_CLOSE / OP_ADVISE from the device: fill msg->status (and
  // msg->last); the service then publishes the answer.
  using Control = std::function<void(uint32_t op, uint32_t fid, uint32_t arg, const char* path, CtlMsg* msg)>;

  IoService(const ServiceConfig& cfg, SinkFactory make_sink, FileLookup files, Control control = nullptr);
  ~IoService();
  int start();
  void stop();
  // Requests fully handed to the sinks so far (drain: compare with tickets issued).
  uint64_t served() const { return served_.load(std::memory_order_acquire); }
  // Wait for all sinks' queued work.
  void drain_sinks();
  void set_faults(uint32_t eio_every, uint32_t short_every, uint32_t delay_us);
  // Zero the service and per-thread counters and the I/O trace (a quiet point).
  void clear_stats();
  uint32_t threads() const { return cfg_.threads; }
  const ThreadCounters& thread_counters(uint32_t i) const { return tstats_[i]; }
  // I/O trace: ranges recorded so far (may exceed the capacity) and the records kept.
  uint64_t io_trace_count() const { return io_n_.load(std::memory_order_acquire); }
  const gfs_io_rec* io_trace() const { return io_trace_.data(); }
  ServiceStats stats;

 private:
  struct Worker {  // one host thread's serving state
    int idx;
    Sink* sink;
    int cur;
    uint32_t pull_cur;
    std::vector<uint32_t> frames;  // frame lists of a merged group (copy-engine transfer)
    std::vector<uint32_t> run;     // frame list of one run of it, in page order
    std::vector<uint8_t> full;     // per page of a staging chunk: delivered whole
  };
  // One read request of a merged group: ticket, slot, its first page and page count.
  // The pages of a group are contiguous in one file, in ticket order.
  struct Req {
    uint64_t ticket;
    uint32_t slot;
    uint32_t npages;
    uint64_t page_lo;
  };
  static constexpr int kMaxGroup = 64;  // requests one host read serves at most
  void run(int idx);
  void run_shared(Worker& w);
  void run_static(Worker& w);
  // Serve the published request with ticket h in slot s.
  void handle(Worker& w, uint64_t h, RingSlot* s);
  // Skip ticket h if its producer gave it up and the slot is free for it.
  bool skip_cancelled(uint64_t h, RingSlot* s);
  void control(RingSlot* s, uint32_t slot, uint32_t op, uint32_t fid);
  // Claim the requests waiting at the head of the ring for the same file as
  // group[0] (see merge_pages) into group[1 ..]; returns the group's request count.
  int gather(Worker& w, uint32_t fid, Req* group, uint32_t max_pages_each);
  void serve(Worker& w, uint32_t fid, uint64_t page_lo, uint32_t npages, const uint32_t* frames);
  void serve_pull(Worker& w, uint32_t fid, const Req* group, int ng);
  ssize_t do_pread(int idx, const FileView& fv, uint8_t* buf, size_t n, uint64_t off);
  void record_io(int idx, uint32_t fid, uint64_t off, uint64_t bytes, uint64_t t_ns);
  void polled_empty(int idx, uint64_t idle_ns);
  void took_request(int idx);

  ServiceConfig cfg_;
  SinkFactory make_sink_;
  FileLookup files_;
  Control control_;
  std::vector<std::thread> threads_;
  std::vector<Sink*> sinks_;
  std::atomic<bool> stop_{false};
  std::atomic<uint64_t> head_{0};
  std::atomic<uint64_t> served_{0};
  std::atomic<uint64_t> pread_count_{0};
  std::atomic<uint32_t> eio_every_{0}, short_every_{0}, delay_us_{0};
  std::unique_ptr<ThreadCounters[]> tstats_;
  std::atomic<uint64_t> t0_ns_{0};  // start of the current counting period
  std::vector<gfs_io_rec> io_trace_;
  std::atomic<uint64_t> io_n_{0};
};

}  // namespace gfs
