// Host I/O service: threads that serve the request ring (Section 2.2: host
// threads poll the shared queue, pread the file and send the data to the GPU;
// Section 4.1: one pread serves every page of a readahead request, and the
// returned size decides which pages are delivered).
//
// Unlike GPUfs, which gives each host thread a fixed slice of the queue and so
// leaves threads idle when the running threadblocks map to one slice
// (Section 3.2), every thread takes the next ticket of one shared ring.
#pragma once

#include <atomic>
#include <cstdint>
#include <functional>
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
};

struct ServiceStats {
  std::atomic<uint64_t> requests{0}, preads{0}, bytes{0}, copies{0}, errors{0};
  std::atomic<uint64_t> ns_pread{0}, ns_wait_buf{0}, ns_idle{0};
  std::atomic<uint64_t> controls{0};  // device opens and closes answered
  void clear() {
    requests = 0; preads = 0; bytes = 0; copies = 0; errors = 0;
    ns_pread = 0; ns_wait_buf = 0; ns_idle = 0; controls = 0;
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
  ServiceStats stats;

 private:
  void run(int idx);
  void control(RingSlot* s, uint32_t slot, uint32_t op, uint32_t fid);
  void serve(Sink* sink, int& cur, uint32_t fid, uint64_t page_lo, uint32_t npages, const uint32_t* frames);
  void serve_pull(int idx, uint32_t& cur, uint32_t slot, uint64_t ticket, uint32_t fid, uint64_t page_lo,
                  uint32_t npages);
  ssize_t do_pread(int fd, uint8_t* buf, size_t n, uint64_t off);

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
};

}  // namespace gfs
