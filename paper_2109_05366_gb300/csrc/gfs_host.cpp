// Host runtime and C ABI of the GPU file-read path (see include/gfs.h).
#include "gfs_host.h"

#include <cuda.h>
#include <errno.h>
#include <fcntl.h>
#include <sys/mman.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <new>

#include "gfs_serve.h"
#include "gfs_service.h"

using namespace gfs;

namespace {

int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return 0;
  if (e == cudaErrorMemoryAllocation) return -ENOMEM;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return -ENODEV;
  return -EINVAL;
}
#define CK(x)                           \
  do {                                  \
    int rc_ = cuda_err(x);              \
    if (rc_) return rc_;                \
  } while (0)

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

uint64_t next_pow2(uint64_t v) {
  uint64_t p = 1;
  while (p < v) p <<= 1;
  return p;
}
bool is_pow2(uint64_t v) { return v && !(v & (v - 1)); }
uint32_t log2u(uint64_t v) {
  uint32_t s = 0;
  while ((1ull << s) < v) ++s;
  return s;
}

// Stream memory operations from the driver (the frame state is written on the
// I/O thread's stream right after the copies of the frame).
typedef CUresult (*BatchMemOpFn)(CUstream, unsigned int, CUstreamBatchMemOpParams*, unsigned int);
typedef CUresult (*WriteValue32Fn)(CUstream, CUdeviceptr, cuuint32_t, unsigned int);
BatchMemOpFn g_batch = nullptr;
WriteValue32Fn g_write32 = nullptr;

int load_driver_fns() {
  if (g_batch || g_write32) return 0;
  cudaDriverEntryPointQueryResult q;
  void* fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuStreamBatchMemOp", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_batch = (BatchMemOpFn)fn;
  fn = nullptr;
  if (cudaGetDriverEntryPointByVersion("cuStreamWriteValue32", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
      q == cudaDriverEntryPointSuccess)
    g_write32 = (WriteValue32Fn)fn;
  return (g_batch || g_write32) ? 0 : -ENOSYS;
}

// GFS_XFER_DMA sink: copy engine into the frames, then a stream write of each
// frame state (the write is ordered after the copies on the same stream and
// carries a memory barrier, so a GPU reader that sees READY sees the data).
class DmaSink : public Sink {
 public:
  DmaSink(int device, uint8_t* d_frames, uint32_t* d_state, uint32_t page_shift, size_t staging_bytes)
      : device_(device), d_frames_(d_frames), d_state_(d_state), page_shift_(page_shift), bytes_(staging_bytes) {}
  int init() {
    CK(cudaSetDevice(device_));
    CK(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
      CK(cudaHostAlloc((void**)&stg_[k], bytes_, cudaHostAllocDefault));
      CK(cudaEventCreateWithFlags(&ev_[k], cudaEventDisableTiming));
    }
    ops_.reserve(MAX_RPC_PAGES);
    return 0;
  }
  ~DmaSink() override {
    cudaSetDevice(device_);
    if (stream_) cudaStreamSynchronize(stream_);
    for (int k = 0; k < 2; ++k) {
      if (stg_[k]) cudaFreeHost(stg_[k]);
      if (ev_[k]) cudaEventDestroy(ev_[k]);
    }
    if (stream_) cudaStreamDestroy(stream_);
  }
  void thread_init() override { cudaSetDevice(device_); }
  uint8_t* staging(int k) override { return stg_[k]; }
  void wait_staging(int k) override {
    if (pending_[k]) cudaEventSynchronize(ev_[k]);
    pending_[k] = false;
  }
  int copy(uint32_t frame, const uint8_t* src, size_t bytes) override {
    return cuda_err(cudaMemcpyAsync(d_frames_ + ((size_t)frame << page_shift_), src, bytes, cudaMemcpyHostToDevice,
                                    stream_));
  }
  int set_state(uint32_t frame, uint32_t state) override {
    CUstreamBatchMemOpParams p;
    memset(&p, 0, sizeof(p));
    p.writeValue.operation = CU_STREAM_MEM_OP_WRITE_VALUE_32;
    p.writeValue.address = (CUdeviceptr)(d_state_ + frame);
    p.writeValue.value = state;
    p.writeValue.flags = CU_STREAM_WRITE_VALUE_DEFAULT;
    ops_.push_back(p);
    return 0;
  }
  int end_chunk(int k) override {
    int rc = flush();
    cudaEventRecord(ev_[k], stream_);
    pending_[k] = true;
    // Submit now: the driver may hold queued work until the stream is touched
    // again, and a GPU reader may be waiting on exactly these state writes.
    cudaStreamQuery(stream_);
    return rc;
  }
  void drain() override {
    if (stream_) cudaStreamSynchronize(stream_);
    pending_[0] = pending_[1] = false;
  }

 private:
  int flush() {
    int rc = 0;
    if (ops_.empty()) return 0;
    if (g_batch) {
      for (size_t i = 0; i < ops_.size(); i += 128) {
        unsigned cnt = (unsigned)std::min<size_t>(128, ops_.size() - i);
        if (g_batch((CUstream)stream_, cnt, ops_.data() + i, 0) != CUDA_SUCCESS) rc = -EIO;
      }
    } else {
      for (auto& p : ops_)
        if (g_write32((CUstream)stream_, p.writeValue.address, p.writeValue.value, 0) != CUDA_SUCCESS) rc = -EIO;
    }
    ops_.clear();
    return rc;
  }
  int device_;
  uint8_t* d_frames_;
  uint32_t* d_state_;
  uint32_t page_shift_;
  size_t bytes_;
  cudaStream_t stream_ = nullptr;
  uint8_t* stg_[2] = {nullptr, nullptr};
  cudaEvent_t ev_[2] = {nullptr, nullptr};
  bool pending_[2] = {false, false};
  std::vector<CUstreamBatchMemOpParams> ops_;
};

// Host-memory sink for the CPU self-test of the ring and service.
class HostSink : public Sink {
 public:
  HostSink(uint8_t* frames, uint32_t* states, uint32_t page_shift, size_t staging_bytes)
      : frames_(frames), states_(states), shift_(page_shift) {
    buf_[0].resize(staging_bytes);
    buf_[1].resize(staging_bytes);
  }
  uint8_t* staging(int k) override { return buf_[k].data(); }
  void wait_staging(int) override {}
  int copy(uint32_t frame, const uint8_t* src, size_t bytes) override {
    memcpy(frames_ + ((size_t)frame << shift_), src, bytes);
    return 0;
  }
  int set_state(uint32_t frame, uint32_t state) override {
    __atomic_store_n(&states_[frame], state, __ATOMIC_RELEASE);
    return 0;
  }
  int end_chunk(int) override { return 0; }
  void drain() override {}

 private:
  uint8_t* frames_;
  uint32_t* states_;
  uint32_t shift_;
  std::vector<uint8_t> buf_[2];
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Whether every page of the mapping [m, m + len) is in the host page cache
// (mincore; touches no page).
bool fully_resident(void* m, size_t len) {
  const long pg = sysconf(_SC_PAGESIZE);
  if (pg <= 0) return false;
  const size_t n = (len + (size_t)pg - 1) / (size_t)pg;
  std::vector<unsigned char> v(n);
  if (mincore(m, len, v.data()) != 0) return false;
  for (unsigned char c : v)
    if (!(c & 1)) return false;
  return true;
}

bool file_lookup(gfs_ctx* ctx, uint32_t fid, FileView* out) {
  if (fid >= ctx->files.size()) return false;
  std::lock_guard<std::mutex> lk(ctx->files_mu);
  const HostFile& f = ctx->files[fid];
  if (!f.open) return false;
  out->fd = f.fd;
  out->size = f.size;
  out->dev_map = f.dev_map;
  out->direct = f.direct;
  return true;
}

// Give every page of the mapping [m, m + len) its page-table entry now, on the
// host.  A fresh mapping has none: the GPU's first touch of each page would take
// the I/O page-fault path, and hundreds of concurrent first touches there can
// wait out a scan's device deadline.  The pages are resident, so nothing is read
// from storage.
void populate(void* m, size_t len) {
#ifdef MADV_POPULATE_READ
  if (madvise(m, len, MADV_POPULATE_READ) == 0) return;
#endif
  const long pg = sysconf(_SC_PAGESIZE);
  const size_t step = pg > 0 ? (size_t)pg : 4096;
  const volatile unsigned char* p = (const volatile unsigned char*)m;
  unsigned char acc = 0;
  for (size_t off = 0; off < len; off += step) acc ^= p[off];
  (void)acc;
}

// GFS_XFER_MAPPED: map the file shared so the GPU can read its page-cache pages.
// Only a file whose pages are all in the host page cache is mapped: a page not
// yet read would be read from storage where no read is timed (inside the open
// when the mapping is pinned, on the GPU's first touch otherwise).  Two ways:
//   * host page tables (device attribute PageableMemoryAccessUsesHostPageTables):
//     a read-only mapping of the read-only descriptor, nothing pinned; the GPU
//     reads it at its host virtual address.  Any file system.
//   * registration: the mapping is registered with CUDA (pinned).  Read-only
//     registration is not available on every platform, so the mapping is
//     read-write (nothing ever writes through it); file systems whose pages
//     cannot be pinned refuse it (tmpfs accepts).
// Returns false (and leaves the file unmapped: its requests are then served by
// pread into staging) when the file is not fully resident or a step fails.
bool map_file(HostFile& hf, bool host_page_tables) {
  if (hf.size == 0) return false;
  const size_t len = (hf.size + 4095) & ~(size_t)4095;
  if (host_page_tables) {
    void* m = mmap(nullptr, len, PROT_READ, MAP_SHARED, hf.fd, 0);
    if (m == MAP_FAILED) return false;
    if (!fully_resident(m, len)) {
      munmap(m, len);
      return false;
    }
    populate(m, len);
    hf.map = m;
    hf.map_len = len;
    hf.dev_map = (uint64_t)(uintptr_t)m;
    hf.map_pinned = false;
    return true;
  }
  int rw = open(hf.path.c_str(), O_RDWR | O_CLOEXEC);
  if (rw < 0) return false;
  void* m = mmap(nullptr, len, PROT_READ | PROT_WRITE, MAP_SHARED, rw, 0);
  close(rw);
  if (m == MAP_FAILED) return false;
  if (!fully_resident(m, len)) {
    munmap(m, len);
    return false;
  }
  if (cudaHostRegister(m, len, cudaHostRegisterMapped) != cudaSuccess) {
    cudaGetLastError();
    munmap(m, len);
    return false;
  }
  void* dp = nullptr;
  if (cudaHostGetDevicePointer(&dp, m, 0) != cudaSuccess || !dp) {
    cudaGetLastError();
    cudaHostUnregister(m);
    munmap(m, len);
    return false;
  }
  hf.map = m;
  hf.map_len = len;
  hf.dev_map = (uint64_t)(uintptr_t)dp;
  hf.map_pinned = true;
  return true;
}

void unmap_file(HostFile& hf) {
  if (!hf.map) return;
  if (hf.map_pinned) cudaHostUnregister(hf.map);
  munmap(hf.map, hf.map_len);
  hf.map = nullptr;
  hf.map_len = 0;
  hf.dev_map = 0;
  hf.map_pinned = false;
}

FileDev make_filedev(gfs_ctx* ctx, const HostFile& hf) {
  FileDev fd{};
  fd.size = hf.size;
  fd.npages = (hf.size + ctx->cfg.page_size - 1) >> ctx->dev.page_shift;
  fd.open = hf.open ? 1u : 0u;
  fd.ra = (hf.open && (hf.flags & 3) == GFS_RDONLY && hf.advice != GFS_ADV_RANDOM) ? 1u : 0u;
  fd.fetched = hf.open ? hf.d_fetched : nullptr;
  fd.flags = (uint32_t)hf.flags;
  fd.advice = (uint32_t)hf.advice;
  fd.mapped = hf.open && hf.map ? (hf.map_pinned ? 1u : 2u) : 0u;
  fd.dev_map = hf.open && hf.map ? hf.dev_map : 0ull;
  return fd;
}

// Write a file's device state (host API calls: the device is not waiting).
int push_file(gfs_ctx* ctx, int fid) {
  const FileDev fd = make_filedev(ctx, ctx->files[fid]);
  CK(cudaMemcpy(ctx->dev.files + fid, &fd, sizeof(fd), cudaMemcpyHostToDevice));
  return 0;
}

// The same from a host I/O thread while kernels run: a copy on the control
// stream (non-blocking, so it waits for no kernel), finished before the caller
// answers the device.  Caller holds dev_open_mu (h_ctl_fd is one buffer).
int push_file_async(gfs_ctx* ctx, int fid) {
  FileDev fd;
  {
    std::lock_guard<std::mutex> lk(ctx->files_mu);
    fd = make_filedev(ctx, ctx->files[fid]);
  }
  cudaSetDevice(ctx->cfg.device);
  memcpy(ctx->h_ctl_fd, &fd, sizeof(fd));
  CK(cudaMemcpyAsync(ctx->dev.files + fid, ctx->h_ctl_fd, sizeof(fd), cudaMemcpyHostToDevice, ctx->ctl_stream));
  return cuda_err(cudaStreamSynchronize(ctx->ctl_stream));
}

// Free what a file id holds and make it reusable.  No kernel may use it.
void release_file(gfs_ctx* ctx, int fid) {
  HostFile& hf = ctx->files[fid];
  unmap_file(hf);
  if (hf.d_fetched) {
    if (hf.fetched_async) {
      cudaFreeAsync(hf.d_fetched, ctx->ctl_stream);
      cudaStreamSynchronize(ctx->ctl_stream);
    } else {
      cudaFree(hf.d_fetched);
    }
  }
  if (hf.fd >= 0) close(hf.fd);
  std::lock_guard<std::mutex> lk(ctx->files_mu);
  hf = HostFile();
}

// Wait until every request issued so far has been served (or skipped) and, in
// the GPU copy transfers, copied out of staging: the cache is quiet afterwards.
// The caller has synchronised the kernels that issue requests.  The drain kernel
// runs while the host catches up: a host thread of the pull transfer may be
// waiting for staging buffers that only GPU copies release.
int quiesce(gfs_ctx* ctx, cudaStream_t s) {
  unsigned long long tail = 0;
  CK(cudaMemcpy(&tail, &ctx->dev.ctrl->ring_tail.v, 8, cudaMemcpyDeviceToHost));
  const bool gpu_copies = ctx->cfg.xfer != GFS_XFER_DMA;
  const double t0 = now_s();
  for (;;) {
    bool dev_done = true;
    if (gpu_copies) {  // copy out what was served but never read
      int rc = launch_drain(ctx->dev, s);
      if (rc) return rc;
      CK(cudaStreamSynchronize(s));
      unsigned long long freed = 0;
      CK(cudaMemcpy(&freed, &ctx->dev.ctrl->freed.v, 8, cudaMemcpyDeviceToHost));
      dev_done = freed + __atomic_load_n(ctx->h_skipped, __ATOMIC_ACQUIRE) >= tail;
    }
    if (ctx->io->served() >= tail && dev_done) break;
    if (now_s() - t0 > (double)ctx->cfg.timeout_ns * 1e-9 + 5.0) return -ETIMEDOUT;
    if (!gpu_copies) usleep(50);
  }
  ctx->io->drain_sinks();
  return 0;
}

// Drop the cached pages of a file id (device and host quiet).  The paper mode's
// private buffers and the per-block LRA queues are not per file: with either
// the cache is cleared.
int purge_pages(gfs_ctx* ctx, int fid) {
  if (ctx->cfg.mode == GFS_MODE_PAPER || ctx->cfg.replacement == GFS_REPL_TB_LRA) return gfs_reset_cache(ctx, nullptr);
  int rc = launch_purge(ctx->dev, (uint32_t)fid, nullptr);
  if (rc) return rc;
  return cuda_err(cudaStreamSynchronize(nullptr));
}

// Open, close or hint requested by the device (a host I/O thread; Section
// 2.2).  Blocks holding a path open share one id; an id whose last device
// reference is gone is retired: its pages may still be cached, so it is not
// reused until they are dropped at a quiet point.  Every change reaches the
// file's device state before the answer.
void device_control(gfs_ctx* ctx, uint32_t op, uint32_t fid, uint32_t arg, const char* path, CtlMsg* m) {
  std::lock_guard<std::mutex> dl(ctx->dev_open_mu);
  m->last = 0;
  if (op == OP_CLOSE || op == OP_ADVISE) {
    {
      std::lock_guard<std::mutex> lk(ctx->files_mu);
      const bool ok = fid < ctx->files.size() && ctx->files[fid].open &&
                      (op == OP_ADVISE || (ctx->files[fid].by_device && ctx->files[fid].dev_refs > 0));
      if (!ok) {
        m->status = -EBADF;
        return;
      }
      if (op == OP_ADVISE && arg > GFS_ADV_RANDOM) {
        m->status = -EINVAL;
        return;
      }
      HostFile& hf = ctx->files[fid];
      if (op == OP_ADVISE) {
        hf.advice = (int)arg;
      } else if (--hf.dev_refs == 0) {
        hf.open = false;
        hf.retired = true;
        m->last = 1;
      }
    }
    m->status = (op == OP_ADVISE || m->last) ? push_file_async(ctx, (int)fid) : 0;
    return;
  }
  if (op != OP_OPEN) {
    m->status = -EINVAL;
    return;
  }
  const uint32_t mode = arg & 3u;
  if (arg != mode || (mode != GFS_RDONLY && mode != GFS_RDWR)) {
    m->status = -EINVAL;
    return;
  }
  const uint32_t P = ctx->cfg.page_size;
  int slot = -1;
  int revive = -1;
  {
    std::lock_guard<std::mutex> lk(ctx->files_mu);
    for (size_t i = 0; i < ctx->files.size(); ++i) {
      HostFile& hf = ctx->files[i];
      if (hf.open && hf.by_device && hf.path == path && (uint32_t)hf.flags == arg) {
        ++hf.dev_refs;
        m->status = (int32_t)i;
        return;
      }
    }
    // A block may close the path's last reference before another block's open of
    // it gets here: the retired id still holds the file (descriptor, mapping and
    // cached pages of the same read-only file), so it is opened again.
    for (size_t i = 0; i < ctx->files.size() && revive < 0; ++i) {
      HostFile& hf = ctx->files[i];
      if (hf.retired && hf.by_device && hf.path == path && (uint32_t)hf.flags == arg) {
        hf.retired = false;
        hf.open = true;
        hf.dev_refs = 1;
        revive = (int)i;
      }
    }
    for (size_t i = 0; i < ctx->files.size() && revive < 0; ++i) {
      HostFile& hf = ctx->files[i];
      if (!hf.open && !hf.retired && !hf.opening) {
        hf.opening = true;
        slot = (int)i;
        break;
      }
    }
  }
  if (revive >= 0) {
    const int rc = push_file_async(ctx, revive);
    if (rc) {  // the id stays retired: its device state is unknown
      std::lock_guard<std::mutex> lk(ctx->files_mu);
      ctx->files[revive].open = false;
      ctx->files[revive].retired = true;
      m->status = rc;
      return;
    }
    m->status = revive;
    return;
  }
  if (slot < 0) {
    m->status = -EMFILE;
    return;
  }
  auto give_back = [&](int err) {
    std::lock_guard<std::mutex> lk(ctx->files_mu);
    ctx->files[slot].opening = false;
    m->status = err;
  };
  const int fd = open(path, O_RDONLY | O_CLOEXEC);
  if (fd < 0) return give_back(-errno);
  struct stat st;
  if (fstat(fd, &st) != 0) {
    const int e = errno;
    close(fd);
    return give_back(-e);
  }
  const uint64_t size = (uint64_t)st.st_size;
  // mapped for the GPU only through the host page tables: registration (pinning)
  // is a CUDA call, which must not wait behind the kernels that wait for this answer
  HostFile mapping;
  if (ctx->cfg.xfer == GFS_XFER_MAPPED && ctx->host_page_tables && !ctx->cfg.map_pinned) {
    mapping.fd = fd;
    mapping.size = size;
    map_file(mapping, true);
  }
  const uint64_t np = (size + P - 1) >> ctx->dev.page_shift;
  const size_t fbytes = (size_t)((np + 31) / 32) * 4;
  uint32_t* bits = nullptr;
  if (fbytes) {  // stream-ordered on the control stream: nothing waits for the running kernels
    cudaSetDevice(ctx->cfg.device);
    if (cudaMallocAsync((void**)&bits, fbytes, ctx->ctl_stream) != cudaSuccess ||
        cudaMemsetAsync(bits, 0, fbytes, ctx->ctl_stream) != cudaSuccess ||
        cudaStreamSynchronize(ctx->ctl_stream) != cudaSuccess) {
      cudaGetLastError();
      if (bits) {
        cudaFreeAsync(bits, ctx->ctl_stream);
        cudaStreamSynchronize(ctx->ctl_stream);
      }
      unmap_file(mapping);
      close(fd);
      return give_back(-ENOMEM);
    }
  }
  {
    std::lock_guard<std::mutex> lk(ctx->files_mu);
    HostFile& hf = ctx->files[slot];
    hf.fd = fd;
    hf.size = size;
    hf.map = mapping.map;
    hf.map_len = mapping.map_len;
    hf.dev_map = mapping.dev_map;
    hf.map_pinned = mapping.map_pinned;
    hf.flags = (int)arg;
    hf.advice = GFS_ADV_NORMAL;
    hf.path = path;
    hf.d_fetched = bits;
    hf.fetched_bytes = fbytes;
    hf.fetched_async = true;
    hf.by_device = true;
    hf.dev_refs = 1;
    hf.opening = false;
    hf.open = true;
  }
  const int rc = push_file_async(ctx, slot);
  if (rc) {  // the id stays retired: its device state is unknown
    std::lock_guard<std::mutex> lk(ctx->files_mu);
    ctx->files[slot].open = false;
    ctx->files[slot].retired = true;
    m->status = rc;
    return;
  }
  m->status = slot;
}

// Drop the pages of every retired id and make the ids reusable (quiet point;
// `cleared`: the whole cache was just reset, nothing to drop).
int reclaim_retired(gfs_ctx* ctx, bool cleared) {
  for (size_t i = 0; i < ctx->files.size(); ++i) {
    if (!ctx->files[i].retired) continue;
    if (!cleared) {
      int rc = purge_pages(ctx, (int)i);
      if (rc) return rc;
    }
    release_file(ctx, (int)i);
    int rc = push_file(ctx, (int)i);
    if (rc) return rc;
  }
  return 0;
}

}  // namespace

extern "C" {

int gfs_abi_version(void) { return GFS_ABI_VERSION; }

const char* gfs_strerror(int err) {
  switch (-err) {
    case 0: return "success";
    case EINVAL: return "invalid argument";
    case EBADF: return "bad file id";
    case ENOMEM: return "out of memory (or no victim frame)";
    case EIO: return "host read failed";
    case ENODEV: return "no CUDA device";
    case ETIMEDOUT: return "device wait timed out";
    case ENOSYS: return "stream memory operations unavailable";
    case EMFILE: return "too many open files";
    case EAGAIN: return "resource temporarily unavailable";
    case ENOTSUP: return "not supported with this transfer or mode";
    case ENOSPC: return "does not fit the fixed-size buffer";
    case ENAMETOOLONG: return "path too long";
    default: return strerror(-err);
  }
}

int gfs_config_default(gfs_config* c) {
  if (!c) return -EINVAL;
  memset(c, 0, sizeof(*c));
  c->cache_bytes = 1ull << 30;
  c->timeout_ns = 10ull * 1000 * 1000 * 1000;
  c->page_size = 512u << 10;
  c->mode = GFS_MODE_READAHEAD;
  c->ra_cap_pages = 8;
  c->async_ra = 1;
  c->reserve_frames = 0;
  c->rpc_slots = 128;
  c->max_rpc_pages = 64;
  c->host_threads = 16;
  c->staging_bytes = 4u << 20;
  c->max_streams = 4096;
  c->max_files = 16;
  c->trace_capacity = 0;
  c->xfer = GFS_XFER_MAPPED;
  c->self_serve = 1;
  c->debug_counts = 0;
  c->device = 0;
  return 0;
}

int gfs_shutdown(gfs_ctx* ctx) {
  if (!ctx) return 0;
  cudaSetDevice(ctx->cfg.device);
  if (ctx->server) gfs_serve_stop(ctx);
  if (ctx->io) {
    ctx->io->stop();
    delete ctx->io;
    ctx->io = nullptr;
  }
  cudaDeviceSynchronize();
  for (size_t i = 0; i < ctx->files.size(); ++i) release_file(ctx, (int)i);
  if (ctx->ctl_stream) cudaStreamDestroy(ctx->ctl_stream);
  if (ctx->h_paths) cudaFreeHost(ctx->h_paths);
  if (ctx->h_ctl_fd) cudaFreeHost(ctx->h_ctl_fd);
  if (ctx->h_cancel) cudaFreeHost(ctx->h_cancel);
  if (ctx->d_arena) cudaFree(ctx->d_arena);
  if (ctx->d_frames) cudaFree(ctx->d_frames);
  if (ctx->d_scan_buf) cudaFree(ctx->d_scan_buf);
  if (ctx->d_paper) cudaFree(ctx->d_paper);
  if (ctx->d_out) cudaFree(ctx->d_out);
  if (ctx->h_out) cudaFreeHost(ctx->h_out);
  if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
  if (ctx->dev.fetch_count) cudaFree(ctx->dev.fetch_count);
  if (ctx->h_ring) cudaFreeHost(ctx->h_ring);
  if (ctx->h_staging) cudaFreeHost(ctx->h_staging);
  if (ctx->h_pullmeta) cudaFreeHost(ctx->h_pullmeta);
  delete ctx;
  return 0;
}

int gfs_init(const gfs_config* cfg_in, gfs_ctx** out) {
  if (!cfg_in || !out) return -EINVAL;
  const gfs_config c = *cfg_in;
  if (!is_pow2(c.page_size) || c.page_size < 4096 || c.page_size > (64u << 20)) return -EINVAL;
  if (c.cache_bytes < c.page_size) return -EINVAL;
  if (c.mode > GFS_MODE_PAPER || c.xfer > GFS_XFER_MAPPED || c.replacement > GFS_REPL_TB_LRA) return -EINVAL;
  if (c.mode == GFS_MODE_PAPER && c.xfer == GFS_XFER_DMA) return -ENOTSUP;  // the requesting block copies its pages
  if (c.queue > GFS_QUEUE_STATIC) return -EINVAL;
  // a Vyukov ring needs 2 slots at least: with one, "published for ticket t" and
  // "free for ticket t+1" are the same sequence value
  if (c.rpc_slots < 2 || c.max_rpc_pages < 1 || c.max_rpc_pages > MAX_RPC_PAGES) return -EINVAL;
  if (c.host_threads < 1 || c.host_threads > 256 || c.max_files < 1 || c.max_files > MAX_FILES) return -EINVAL;
  if (c.max_streams < 1 || c.timeout_ns == 0) return -EINVAL;
  const uint64_t F64 = c.cache_bytes / c.page_size;
  if (F64 > MAX_FRAMES) return -EINVAL;
  // pull staging: per host thread, a ring of small buffers of whole pages
  const uint64_t chunk_bytes = std::max<uint64_t>(c.page_size, 1ull << 20);
  const uint32_t bufs_per_thread = (uint32_t)std::max<uint64_t>(2, c.staging_bytes / chunk_bytes);
  const uint32_t nbufs = c.host_threads * bufs_per_thread;
  if (c.xfer != GFS_XFER_DMA && (uint64_t)nbufs * chunk_bytes > (16ull << 30)) return -EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return -ENODEV;
  if (c.device < 0 || c.device >= ndev) return -EINVAL;
  int rc = load_driver_fns();
  if (rc) return rc;
  CK(cudaSetDevice(c.device));

  gfs_ctx* ctx = new (std::nothrow) gfs_ctx();
  if (!ctx) return -ENOMEM;
  ctx->cfg = c;
  {  // can the GPU read pageable host memory through the host's page tables?
    int pageable = 0, hpt = 0;
    if (cudaDeviceGetAttribute(&pageable, cudaDevAttrPageableMemoryAccess, c.device) != cudaSuccess ||
        cudaDeviceGetAttribute(&hpt, cudaDevAttrPageableMemoryAccessUsesHostPageTables, c.device) != cudaSuccess) {
      cudaGetLastError();
      pageable = hpt = 0;
    }
    ctx->host_page_tables = pageable && hpt;
  }
  DevHandle& g = ctx->dev;
  const uint32_t F = (uint32_t)F64;
  g.timeout_ns = c.timeout_ns;
  g.cache_bytes = (uint64_t)F * c.page_size;
  g.page_size = c.page_size;
  g.page_shift = log2u(c.page_size);
  g.n_frames = F;
  g.mode = c.mode;
  g.ra_cap = c.ra_cap_pages;
  g.async_ra = c.async_ra ? 1 : 0;
  g.max_rpc_pages = c.max_rpc_pages;
  g.reserve = c.reserve_frames;
  g.nbuckets = (uint32_t)std::max<uint64_t>(4, next_pow2(((uint64_t)F * 4 + BUCKET - 1) / BUCKET));
  g.max_streams = c.max_streams;
  g.max_files = c.max_files;
  g.trace_cap = c.trace_capacity;
  g.rpc_slots = c.rpc_slots;
  g.slot_stride = slot_stride(c.max_rpc_pages);
  g.fifo_cap = std::max<uint32_t>(F, 2);  // same sequence rule as the ring
  g.xfer = c.xfer;
  g.self_serve = (c.xfer == GFS_XFER_MAPPED && c.self_serve) ? 1u : 0u;
  g.repl = c.replacement;
  g.paper_streams = 0;
  g.nbufs = nbufs;
  g.chunk_bytes = chunk_bytes;

  // device arena
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  const size_t o_fkey = take((size_t)F * 8), o_fstate = take((size_t)F * 4), o_fpins = take((size_t)F * 4),
               o_fcons = take((size_t)F * 4), o_fvalid = take((size_t)F * 4), o_fwin = take((size_t)F * 4),
               o_fmark = take((size_t)F * 4), o_faseq = take((size_t)F * 8),
               o_tab = take((size_t)g.nbuckets * BUCKET * 8), o_tlock = take((size_t)g.nbuckets * 4),
               o_tovf = take((size_t)g.nbuckets * 4), o_fifo = take((size_t)std::max<uint32_t>(F, 2) * 8),
               o_ret = take((size_t)std::max<uint32_t>(F, 2) * 8), o_ctrl = take(sizeof(Ctrl)),
               o_files = take((size_t)c.max_files * sizeof(FileDev)),
               o_last = take((size_t)c.max_streams * c.max_files * 8),
               o_trpc = take((size_t)std::max<uint32_t>(1, c.trace_capacity) * sizeof(gfs_rpc_rec)),
               o_tev = take((size_t)std::max<uint32_t>(1, c.trace_capacity) * sizeof(gfs_evict_rec)),
               o_dtick = take((size_t)c.rpc_slots * 8), o_dnp = take((size_t)c.rpc_slots * 4),
               o_dcop = take((size_t)c.rpc_slots * 4), o_dfr = take((size_t)c.rpc_slots * c.max_rpc_pages * 4),
               o_fsrc = take((size_t)F * 4), o_lat = take((size_t)std::max<uint32_t>(1, c.latency_capacity) * 8),
               o_lap = take((size_t)c.rpc_slots * 8), o_sfree = take((size_t)c.rpc_slots * 8);
  ctx->arena_bytes = off;
  rc = cuda_err(cudaMalloc(&ctx->d_arena, off));
  if (!rc) rc = cuda_err(cudaMemset(ctx->d_arena, 0, off));
  if (!rc) rc = cuda_err(cudaMalloc((void**)&ctx->d_frames, (size_t)F << g.page_shift));
  if (rc) {
    gfs_shutdown(ctx);
    return rc;
  }
  uint8_t* a = (uint8_t*)ctx->d_arena;
  g.frames = ctx->d_frames;
  g.fkey = (unsigned long long*)(a + o_fkey);
  g.fstate = (uint32_t*)(a + o_fstate);
  g.fpins = (uint32_t*)(a + o_fpins);
  g.fconsumed = (uint32_t*)(a + o_fcons);
  g.fvalid = (uint32_t*)(a + o_fvalid);
  g.fwindow = (uint32_t*)(a + o_fwin);
  g.fmark = (uint32_t*)(a + o_fmark);
  g.faseq = (unsigned long long*)(a + o_faseq);
  g.tab = (unsigned long long*)(a + o_tab);
  g.tlock = (uint32_t*)(a + o_tlock);
  g.tovf = (uint32_t*)(a + o_tovf);
  g.fifo = (unsigned long long*)(a + o_fifo);
  g.ret = (unsigned long long*)(a + o_ret);
  g.ctrl = (Ctrl*)(a + o_ctrl);
  g.files = (FileDev*)(a + o_files);
  g.last_end = (unsigned long long*)(a + o_last);
  g.trace_rpc = (gfs_rpc_rec*)(a + o_trpc);
  g.trace_evict = (gfs_evict_rec*)(a + o_tev);
  g.fetch_count = nullptr;
  g.debug_pages = 0;
  g.dticket = (unsigned long long*)(a + o_dtick);
  g.dnpages = (uint32_t*)(a + o_dnp);
  g.dcopied = (uint32_t*)(a + o_dcop);
  g.dframes = (uint32_t*)(a + o_dfr);
  g.fsrc = (uint32_t*)(a + o_fsrc);
  g.lat = (unsigned long long*)(a + o_lat);
  g.lat_cap = c.latency_capacity;
  g.queue = c.queue;
  g.slot_lap = (unsigned long long*)(a + o_lap);  // zero: every slot at lap 0, for the life of the context
  g.slot_free = (unsigned long long*)(a + o_sfree);
  {
    std::vector<unsigned long long> init(c.rpc_slots);
    for (uint32_t i = 0; i < c.rpc_slots; ++i) init[i] = i;  // slot i free for ticket i, like its seq
    rc = cuda_err(cudaMemcpy(g.slot_free, init.data(), init.size() * 8, cudaMemcpyHostToDevice));
    if (rc) {
      gfs_shutdown(ctx);
      return rc;
    }
  }
  g.staging = nullptr;
  g.done = nullptr;
  g.pages = nullptr;
  g.bcount = nullptr;
  if (c.xfer != GFS_XFER_DMA) {
    const size_t pages_bytes = sizeof(PullPage) * c.rpc_slots * c.max_rpc_pages;
    const size_t meta_bytes = align_up(sizeof(PullDone) * c.rpc_slots, 256) + align_up(pages_bytes, 256) +
                              align_up((size_t)nbufs * 4, 256);
    rc = cuda_err(cudaHostAlloc((void**)&ctx->h_staging, (size_t)nbufs * chunk_bytes,
                                cudaHostAllocMapped | cudaHostAllocPortable));
    if (!rc) rc = cuda_err(cudaHostAlloc((void**)&ctx->h_pullmeta, meta_bytes,
                                         cudaHostAllocMapped | cudaHostAllocPortable));
    void* dp = nullptr;
    void* dm = nullptr;
    if (!rc) rc = cuda_err(cudaHostGetDevicePointer(&dp, ctx->h_staging, 0));
    if (!rc) rc = cuda_err(cudaHostGetDevicePointer(&dm, ctx->h_pullmeta, 0));
    if (rc) {
      gfs_shutdown(ctx);
      return rc;
    }
    memset(ctx->h_pullmeta, 0, meta_bytes);
    const size_t o_pages = align_up(sizeof(PullDone) * c.rpc_slots, 256);
    const size_t o_bcount = o_pages + align_up(pages_bytes, 256);
    ctx->h_done = (PullDone*)ctx->h_pullmeta;
    ctx->h_pages = (PullPage*)(ctx->h_pullmeta + o_pages);
    ctx->h_bcount = (uint32_t*)(ctx->h_pullmeta + o_bcount);
    g.staging = (uint8_t*)dp;
    g.done = (PullDone*)dm;
    g.pages = (PullPage*)((uint8_t*)dm + o_pages);
    g.bcount = (uint32_t*)((uint8_t*)dm + o_bcount);
  }

  // request ring in mapped pinned memory
  const size_t ring_bytes = (size_t)c.rpc_slots * g.slot_stride;
  rc = cuda_err(cudaHostAlloc((void**)&ctx->h_ring, ring_bytes, cudaHostAllocMapped | cudaHostAllocPortable));
  if (rc) {
    gfs_shutdown(ctx);
    return rc;
  }
  memset(ctx->h_ring, 0, ring_bytes);
  for (uint32_t i = 0; i < c.rpc_slots; ++i) ((RingSlot*)(ctx->h_ring + (size_t)i * g.slot_stride))->seq = i;
  void* d_ring = nullptr;
  rc = cuda_err(cudaHostGetDevicePointer(&d_ring, ctx->h_ring, 0));
  if (rc) {
    gfs_shutdown(ctx);
    return rc;
  }
  g.ring = (uint8_t*)d_ring;
  // path buffers of device opens (one per slot) and the stream their allocations use
  rc = cuda_err(cudaHostAlloc((void**)&ctx->h_paths, (size_t)c.rpc_slots * GFS_PATH_MAX,
                              cudaHostAllocMapped | cudaHostAllocPortable));
  void* d_paths = nullptr;
  if (!rc) rc = cuda_err(cudaHostGetDevicePointer(&d_paths, ctx->h_paths, 0));
  if (!rc) rc = cuda_err(cudaStreamCreateWithFlags(&ctx->ctl_stream, cudaStreamNonBlocking));
  if (!rc) rc = cuda_err(cudaHostAlloc((void**)&ctx->h_ctl_fd, sizeof(FileDev), cudaHostAllocPortable));
  // per-slot ticket cancellations and the count of skipped tickets (its own line)
  const size_t cancel_n = (size_t)c.rpc_slots + CANCEL_SPAN;
  if (!rc) rc = cuda_err(cudaHostAlloc((void**)&ctx->h_cancel, cancel_n * 8 + 128,
                                       cudaHostAllocMapped | cudaHostAllocPortable));
  void* d_cancel = nullptr;
  if (!rc) rc = cuda_err(cudaHostGetDevicePointer(&d_cancel, ctx->h_cancel, 0));
  if (rc) {
    gfs_shutdown(ctx);
    return rc;
  }
  memset(ctx->h_paths, 0, (size_t)c.rpc_slots * GFS_PATH_MAX);
  g.paths = (char*)d_paths;
  memset(ctx->h_cancel, 0, cancel_n * 8 + 128);
  ctx->h_skipped = ctx->h_cancel + cancel_n + 8;  // 64 bytes past the last cancellation word
  g.cancel = (unsigned long long*)d_cancel;
  g.cancel_n = (uint32_t)cancel_n;
  g.skipped = (unsigned long long*)d_cancel + cancel_n + 8;

  ctx->files.resize(c.max_files);
  rc = launch_reset(g, 0);
  if (!rc) rc = cuda_err(cudaDeviceSynchronize());
  if (rc) {
    gfs_shutdown(ctx);
    return rc;
  }

  ServiceConfig sc;
  sc.ring = ctx->h_ring;
  sc.slots = c.rpc_slots;
  sc.slot_stride = g.slot_stride;
  sc.page_size = c.page_size;
  sc.page_shift = g.page_shift;
  sc.staging_pages = std::max<uint32_t>(1, c.staging_bytes / c.page_size);
  sc.threads = c.host_threads;
  sc.n_frames = F;
  sc.paths = ctx->h_paths;
  sc.cancel = ctx->h_cancel;
  sc.cancel_n = (uint32_t)cancel_n;
  sc.skipped = ctx->h_skipped;
  sc.queue = c.queue;
  sc.io_trace_cap = c.trace_capacity;
  // merged host reads: by default one staging buffer's worth of pages
  sc.merge_pages = c.host_merge_pages ? c.host_merge_pages
                                      : (c.xfer != GFS_XFER_DMA ? (uint32_t)(chunk_bytes / c.page_size)
                                                                : sc.staging_pages);
  if (c.xfer != GFS_XFER_DMA) {
    sc.pull_arena = ctx->h_staging;
    sc.pull_done = ctx->h_done;
    sc.pull_pages = ctx->h_pages;
    sc.pull_bcount = ctx->h_bcount;
    sc.chunk_bytes = chunk_bytes;
    sc.bufs_per_thread = bufs_per_thread;
    sc.max_pages = c.max_rpc_pages;
  }
  const size_t stg = (size_t)sc.staging_pages * c.page_size;
  ctx->io = new IoService(
      sc,
      [ctx, stg](int) -> Sink* {
        if (ctx->cfg.xfer != GFS_XFER_DMA) return new (std::nothrow) HostSink(nullptr, nullptr, 0, 0);
        DmaSink* s = new (std::nothrow) DmaSink(ctx->cfg.device, ctx->d_frames, ctx->dev.fstate, ctx->dev.page_shift, stg);
        if (s && s->init() != 0) {
          delete s;
          return nullptr;
        }
        return s;
      },
      [ctx](uint32_t fid, FileView* fv) { return file_lookup(ctx, fid, fv); },
      [ctx](uint32_t op, uint32_t fid, uint32_t arg, const char* path, CtlMsg* m) {
        device_control(ctx, op, fid, arg, path, m);
      });
  rc = ctx->io->start();
  if (rc) {
    gfs_shutdown(ctx);
    return rc;
  }
  *out = ctx;
  return 0;
}

int gfs_set_faults(gfs_ctx* ctx, uint32_t eio_every, uint32_t short_every, uint32_t delay_us) {
  if (!ctx || !ctx->io) return -EINVAL;
  ctx->io->set_faults(eio_every, short_every, delay_us);
  // injected host faults only reach requests the host serves: while any is set,
  // requests for mapped files go to the host too (from the next launch on)
  const bool faults = eio_every || short_every || delay_us;
  ctx->dev.self_serve = (!faults && ctx->cfg.self_serve) ? 1u : 0u;
  return 0;
}

int gfs_open(gfs_ctx* ctx, const char* path, int flags, int* fid) {
  if (!ctx || !path || !fid) return -EINVAL;
  if ((flags & 3) != GFS_RDONLY && (flags & 3) != GFS_RDWR) return -EINVAL;
  if (flags & ~(3 | GFS_DIRECT)) return -EINVAL;
  const bool direct = (flags & GFS_DIRECT) != 0;
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->cfg.device));
  auto pick = [ctx]() {
    std::lock_guard<std::mutex> fl(ctx->files_mu);
    for (size_t i = 0; i < ctx->files.size(); ++i) {
      HostFile& f = ctx->files[i];
      if (!f.open && !f.retired && !f.opening) {
        f.opening = true;
        return (int)i;
      }
    }
    return -1;
  };
  int slot = pick();
  if (slot < 0) {  // ids closed on the device: drop their pages now and reuse them
    bool any = false;
    for (auto& f : ctx->files) any = any || f.retired;
    if (!any) return -EMFILE;
    CK(cudaDeviceSynchronize());
    int rc = quiesce(ctx, nullptr);
    if (!rc) rc = reclaim_retired(ctx, false);
    if (rc) return rc;
    slot = pick();
    if (slot < 0) return -EMFILE;
  }
  int fd = open(path, O_RDONLY | O_CLOEXEC | (direct ? O_DIRECT : 0));
  if (fd < 0) {
    const int e = errno;
    std::lock_guard<std::mutex> fl(ctx->files_mu);
    ctx->files[slot].opening = false;
    return -e;
  }
  struct stat st;
  if (fstat(fd, &st) != 0) {
    int e = errno;
    close(fd);
    std::lock_guard<std::mutex> fl(ctx->files_mu);
    ctx->files[slot].opening = false;
    return -e;
  }
  HostFile& hf = ctx->files[slot];
  {
    std::lock_guard<std::mutex> fl(ctx->files_mu);
    hf.fd = fd;
    hf.size = (uint64_t)st.st_size;
    hf.flags = flags;
    hf.direct = direct;
    hf.advice = GFS_ADV_NORMAL;
    hf.path = path;
  }
  // falls back to pread staging when it fails; a direct file is read from storage every time
  if (ctx->cfg.xfer == GFS_XFER_MAPPED && !direct) map_file(hf, ctx->host_page_tables && !ctx->cfg.map_pinned);
  {
    const uint64_t np = (hf.size + ctx->cfg.page_size - 1) >> ctx->dev.page_shift;
    hf.fetched_bytes = (size_t)((np + 31) / 32) * 4;
    if (hf.fetched_bytes) {
      if (cudaMalloc((void**)&hf.d_fetched, hf.fetched_bytes) != cudaSuccess ||
          cudaMemset(hf.d_fetched, 0, hf.fetched_bytes) != cudaSuccess) {
        release_file(ctx, slot);
        return -ENOMEM;
      }
    }
  }
  if (slot == 0 && ctx->cfg.debug_counts) {
    const uint64_t np = (hf.size + ctx->cfg.page_size - 1) >> ctx->dev.page_shift;
    if (ctx->dev.fetch_count) cudaFree(ctx->dev.fetch_count);
    ctx->dev.fetch_count = nullptr;
    ctx->dev.debug_pages = 0;
    if (np) {
      CK(cudaMalloc((void**)&ctx->dev.fetch_count, np * 4));
      CK(cudaMemset(ctx->dev.fetch_count, 0, np * 4));
      ctx->dev.debug_pages = (uint32_t)std::min<uint64_t>(np, 0xffffffffull);
    }
  }
  {
    std::lock_guard<std::mutex> fl(ctx->files_mu);
    hf.opening = false;
    hf.open = true;
  }
  int rc = push_file(ctx, slot);
  if (rc) {
    release_file(ctx, slot);
    return rc;
  }
  *fid = slot;
  memset(ctx->graph_key, 0, sizeof(ctx->graph_key));  // a cached graph clears the files' bits: rebuild
  return 0;
}

int gfs_close(gfs_ctx* ctx, int fid) {
  if (!ctx || fid < 0 || (size_t)fid >= ctx->files.size() || !ctx->files[fid].open) return -EBADF;
  std::lock_guard<std::mutex> lk(ctx->mu);
  CK(cudaSetDevice(ctx->cfg.device));
  // nothing may still read the file: no kernel, no request in flight
  CK(cudaDeviceSynchronize());
  int rc = quiesce(ctx, nullptr);
  if (rc) return rc;
  {
    std::lock_guard<std::mutex> fl(ctx->files_mu);
    ctx->files[fid].open = false;
  }
  rc = push_file(ctx, fid);
  if (!rc) rc = purge_pages(ctx, fid);
  release_file(ctx, fid);
  return rc;
}

int gfs_fadvise(gfs_ctx* ctx, int fid, int advice) {
  if (!ctx || fid < 0 || (size_t)fid >= ctx->files.size() || !ctx->files[fid].open) return -EBADF;
  if (advice < GFS_ADV_NORMAL || advice > GFS_ADV_RANDOM) return -EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  {
    std::lock_guard<std::mutex> fl(ctx->files_mu);
    ctx->files[fid].advice = advice;
  }
  CK(cudaSetDevice(ctx->cfg.device));
  return push_file(ctx, fid);
}

int gfs_fstat(gfs_ctx* ctx, int fid, gfs_stat* st) {
  if (!ctx || !st) return -EINVAL;
  if (fid < 0 || (size_t)fid >= ctx->files.size() || !ctx->files[fid].open) return -EBADF;
  memset(st, 0, sizeof(*st));
  st->size = ctx->files[fid].size;
  st->page_size = ctx->cfg.page_size;
  st->flags = (uint32_t)ctx->files[fid].flags;
  st->advice = (uint32_t)ctx->files[fid].advice;
  st->mapped = ctx->files[fid].map ? (ctx->files[fid].map_pinned ? 1u : 2u) : 0u;
  return 0;
}

int gfs_reset_cache(gfs_ctx* ctx, void* stream) {
  if (!ctx) return -EINVAL;
  CK(cudaSetDevice(ctx->cfg.device));
  cudaStream_t s = (cudaStream_t)stream;
  CK(cudaStreamSynchronize(s));
  int qrc = quiesce(ctx, s);
  if (qrc) return qrc;
  ctx->io->clear_stats();
  if (ctx->dev.fetch_count) CK(cudaMemsetAsync(ctx->dev.fetch_count, 0, (size_t)ctx->dev.debug_pages * 4, s));
  for (auto& f : ctx->files)
    if (f.open && f.d_fetched) CK(cudaMemsetAsync(f.d_fetched, 0, f.fetched_bytes, s));
  if (ctx->dev.paper_streams) {  // private buffers and LRA queues start empty
    CK(cudaMemsetAsync(ctx->dev.pmeta, 0, (size_t)ctx->dev.paper_streams * sizeof(PrivBuf), s));
    CK(cudaMemsetAsync(ctx->dev.lra_head, 0, (size_t)ctx->dev.paper_streams * 4, s));
    CK(cudaMemsetAsync(ctx->dev.lra_len, 0, (size_t)ctx->dev.paper_streams * 4, s));
  }
  int rc = launch_reset(ctx->dev, s);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s));
  return reclaim_retired(ctx, true);  // ids closed on the device: their pages are gone now
}

int gfs_get_stats(gfs_ctx* ctx, gfs_stats* o, void* stream) {
  if (!ctx || !o) return -EINVAL;
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  unsigned long long st[ST_COUNT];
  unsigned long long tr[2];
  CK(cudaMemcpy(st, ctx->dev.ctrl->stat, sizeof(st), cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&tr[0], &ctx->dev.ctrl->trace_rpc_n.v, 8, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&tr[1], &ctx->dev.ctrl->trace_evict_n.v, 8, cudaMemcpyDeviceToHost));
  memset(o, 0, sizeof(*o));
  o->greads = st[ST_GREADS];
  o->hits = st[ST_HITS];
  o->misses = st[ST_MISSES];
  o->coalesced_waits = st[ST_COALESCED];
  o->rpcs = st[ST_RPCS];
  o->pages_fetched = st[ST_PAGES];
  o->bytes_fetched = st[ST_BYTES];
  o->ra_pages_sync = st[ST_RA_SYNC];
  o->ra_pages_async = st[ST_RA_ASYNC];
  o->evictions = st[ST_EVICT];
  o->unconsumed_evictions = st[ST_EVICT_UNCONSUMED];
  o->retries = st[ST_RETRIES];
  o->timeouts = st[ST_TIMEOUTS];
  o->eio = st[ST_EIO];
  o->enomem = st[ST_ENOMEM];
  o->host_requests = ctx->io->stats.requests.load();
  o->host_preads = ctx->io->stats.preads.load();
  o->host_bytes = ctx->io->stats.bytes.load();
  o->host_copies = ctx->io->stats.copies.load();
  o->host_errors = ctx->io->stats.errors.load();
  o->trace_rpc_count = tr[0];
  o->trace_evict_count = tr[1];
  o->host_ns_pread = ctx->io->stats.ns_pread.load();
  o->host_ns_wait_buf = ctx->io->stats.ns_wait_buf.load();
  o->host_ns_idle = ctx->io->stats.ns_idle.load();
  o->buffer_hits = st[ST_BUFHITS];
  o->host_controls = ctx->io->stats.controls.load();
  o->host_merged = ctx->io->stats.merged.load();
  o->run_cuts = st[ST_RUN_CUTS];
  return 0;
}

int gfs_get_trace(gfs_ctx* ctx, gfs_rpc_rec* h_rpc, gfs_evict_rec* h_evict, uint32_t cap, uint64_t* n_rpc,
                  uint64_t* n_evict, void* stream) {
  if (!ctx) return -EINVAL;
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  unsigned long long nr = 0, ne = 0;
  CK(cudaMemcpy(&nr, &ctx->dev.ctrl->trace_rpc_n.v, 8, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&ne, &ctx->dev.ctrl->trace_evict_n.v, 8, cudaMemcpyDeviceToHost));
  const uint64_t kr = std::min<uint64_t>({nr, (uint64_t)cap, (uint64_t)ctx->dev.trace_cap});
  const uint64_t ke = std::min<uint64_t>({ne, (uint64_t)cap, (uint64_t)ctx->dev.trace_cap});
  if (h_rpc && kr) CK(cudaMemcpy(h_rpc, ctx->dev.trace_rpc, kr * sizeof(gfs_rpc_rec), cudaMemcpyDeviceToHost));
  if (h_evict && ke) CK(cudaMemcpy(h_evict, ctx->dev.trace_evict, ke * sizeof(gfs_evict_rec), cudaMemcpyDeviceToHost));
  if (n_rpc) *n_rpc = nr;
  if (n_evict) *n_evict = ne;
  return 0;
}

int gfs_get_latencies(gfs_ctx* ctx, uint64_t* h_ns, uint64_t cap, uint64_t* n, void* stream) {
  if (!ctx) return -EINVAL;
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  unsigned long long k = 0;
  CK(cudaMemcpy(&k, &ctx->dev.ctrl->lat_n.v, 8, cudaMemcpyDeviceToHost));
  const uint64_t c = std::min<uint64_t>({k, cap, (uint64_t)ctx->dev.lat_cap});
  if (h_ns && c) CK(cudaMemcpy(h_ns, ctx->dev.lat, c * 8, cudaMemcpyDeviceToHost));
  if (n) *n = k;
  return 0;
}

int gfs_get_thread_stats(gfs_ctx* ctx, gfs_thread_stat* h_out, uint32_t cap) {
  if (!ctx || !ctx->io || (cap && !h_out)) return -EINVAL;
  const uint32_t T = ctx->io->threads();
  for (uint32_t i = 0; i < T && i < cap; ++i) {
    const ThreadCounters& c = ctx->io->thread_counters(i);
    gfs_thread_stat& o = h_out[i];
    o.requests = c.requests.load();
    o.polls_before_first = c.polls_before_first.load();
    o.first_request_ns = c.first_ns.load();
    o.idle_ns = c.idle_ns.load();
    o.pread_ns = c.pread_ns.load();
    o.bytes = c.bytes.load();
  }
  return (int)T;
}

int gfs_get_io_trace(gfs_ctx* ctx, gfs_io_rec* h_out, uint64_t cap, uint64_t* n) {
  if (!ctx || !ctx->io || (cap && !h_out)) return -EINVAL;
  const uint64_t k = ctx->io->io_trace_count();
  const uint64_t c = std::min<uint64_t>({k, cap, (uint64_t)ctx->cfg.trace_capacity});
  if (c) memcpy(h_out, ctx->io->io_trace(), c * sizeof(gfs_io_rec));
  if (n) *n = k;
  return 0;
}

int gfs_get_fetch_counts(gfs_ctx* ctx, uint32_t* h_counts, uint64_t cap, void* stream) {
  if (!ctx || !h_counts) return -EINVAL;
  if (!ctx->dev.fetch_count) return -EINVAL;
  CK(cudaSetDevice(ctx->cfg.device));
  CK(cudaStreamSynchronize((cudaStream_t)stream));
  const uint64_t n = std::min<uint64_t>(cap, ctx->dev.debug_pages);
  CK(cudaMemcpy(h_counts, ctx->dev.fetch_count, n * 4, cudaMemcpyDeviceToHost));
  return 0;
}

}  // extern "C"

int ensure_paper_state(gfs_ctx* ctx, uint32_t streams) {
  const bool paper = ctx->cfg.mode == GFS_MODE_PAPER;
  if ((!paper && ctx->cfg.replacement != GFS_REPL_TB_LRA) || streams <= ctx->dev.paper_streams) return 0;
  if (cudaSetDevice(ctx->cfg.device) != cudaSuccess) return -ENODEV;
  cudaDeviceSynchronize();  // no kernel may still use the old state
  if (ctx->d_paper) cudaFree(ctx->d_paper);
  ctx->d_paper = nullptr;
  ctx->dev.paper_streams = 0;
  const uint32_t quota = std::max<uint32_t>(1, ctx->dev.n_frames / streams);
  // private buffers only for the paper's prefetcher; the LRA queues for GFS_REPL_TB_LRA
  const size_t pbuf = paper ? std::max<size_t>(256, (size_t)streams * ctx->dev.ra_cap * ctx->cfg.page_size) : 256;
  const size_t o_meta = align_up(pbuf, 256);
  const size_t o_lra = o_meta + align_up((size_t)streams * sizeof(PrivBuf), 256);
  const size_t o_head = o_lra + align_up((size_t)streams * quota * 4, 256);
  const size_t o_len = o_head + align_up((size_t)streams * 4, 256);
  const size_t total = o_len + align_up((size_t)streams * 4, 256);
  CK(cudaMalloc((void**)&ctx->d_paper, total));
  CK(cudaMemset(ctx->d_paper + o_meta, 0, total - o_meta));
  ctx->dev.pbuf = ctx->d_paper;
  ctx->dev.pmeta = (PrivBuf*)(ctx->d_paper + o_meta);
  ctx->dev.lra = (uint32_t*)(ctx->d_paper + o_lra);
  ctx->dev.lra_head = (uint32_t*)(ctx->d_paper + o_head);
  ctx->dev.lra_len = (uint32_t*)(ctx->d_paper + o_len);
  ctx->dev.quota = quota;
  ctx->dev.paper_streams = streams;
  return 0;
}

int ensure_scan_buf(gfs_ctx* ctx, size_t need) {
  if (cudaSetDevice(ctx->cfg.device) != cudaSuccess) return -ENODEV;
  if (need <= ctx->scan_buf_bytes) return 0;
  if (ctx->d_scan_buf) cudaFree(ctx->d_scan_buf);
  ctx->d_scan_buf = nullptr;
  ctx->scan_buf_bytes = 0;
  CK(cudaMalloc((void**)&ctx->d_scan_buf, need));
  ctx->scan_buf_bytes = need;
  return 0;
}

extern "C" {

static int scan_prepare(gfs_ctx* ctx, int fid, const gfs_scan_args* a, uint64_t* nstrides, uint64_t* buf_stride,
                        DevHandle* g) {
  if (!ctx || !a) return -EINVAL;
  if (fid < 0 || (size_t)fid >= ctx->files.size() || !ctx->files[fid].open) return -EBADF;
  if (a->stride == 0 || a->read_len == 0 || a->blocks == 0) return -EINVAL;
  if (a->threads != 128 && a->threads != 256 && a->threads != 512) return -EINVAL;
  const uint64_t size = ctx->files[fid].size;
  *nstrides = size ? (size + a->stride - 1) / a->stride : 0;
  // a gread never delivers more than the file holds; the checks divide so that
  // no size wraps around
  const uint64_t per_block = std::min<uint64_t>(a->read_len, size);
  if (per_block > SIZE_MAX / 2) return -ENOMEM;
  *buf_stride = align_up(per_block, 256);
  if (*buf_stride && a->blocks > SIZE_MAX / *buf_stride) return -ENOMEM;
  CK(cudaSetDevice(ctx->cfg.device));
  const size_t need = (size_t)a->blocks * *buf_stride;
  if (need > ctx->scan_buf_bytes) {
    if (ctx->d_scan_buf) cudaFree(ctx->d_scan_buf);
    ctx->d_scan_buf = nullptr;
    ctx->scan_buf_bytes = 0;
    CK(cudaMalloc((void**)&ctx->d_scan_buf, need));
    ctx->scan_buf_bytes = need;
  }
  {
    int prc = ensure_paper_state(ctx, a->blocks);
    if (prc) return prc;
  }
  *g = ctx->dev;
  g->exact_lra = a->serialize ? 1u : 0u;
  const uint64_t pages_per_read = (a->read_len >> ctx->dev.page_shift) + ((a->read_len & (ctx->cfg.page_size - 1)) != 0);
  g->reserve = ctx->cfg.reserve_frames ? ctx->cfg.reserve_frames
                                       : (uint32_t)(pages_per_read >= 0xffffffffull / a->blocks ? 0xffffffffull
                                                                      : a->blocks * pages_per_read + 1);
  if (a->serialize) {
    int maxb = 0;
    int rc = scan_max_resident_blocks(a->threads, a->fused != 0, ctx->cfg.device, &maxb);
    if (rc) return rc;
    if ((int)a->blocks > maxb) return -EINVAL;  // every block must be resident to take its turn
  }
  return 0;
}

int gfs_scan(gfs_ctx* ctx, int fid, const gfs_scan_args* a, int64_t* d_count, uint64_t* d_sum, uint64_t* d_hash,
             void* stream) {
  uint64_t ns = 0, bs = 0;
  DevHandle g;
  int rc = scan_prepare(ctx, fid, a, &ns, &bs, &g);
  if (rc) return rc;
  if (ns == 0) return 0;
  if (!d_count || !d_sum || !d_hash) return -EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (a->serialize) CK(cudaMemsetAsync(&g.ctrl->ticket.v, 0, 8, s));
  return launch_scan(g, fid, *a, ns, ctx->d_scan_buf, bs, d_count, d_sum, d_hash, s);
}

int gfs_scan_path(gfs_ctx* ctx, const char* path, const gfs_scan_args* a, int64_t* d_count, uint64_t* d_sum,
                  uint64_t* d_hash, void* stream) {
  if (!ctx || !path || !a) return -EINVAL;
  const size_t len = strnlen(path, GFS_PATH_MAX);
  if (len == 0) return -EINVAL;
  if (len >= GFS_PATH_MAX) return -ENAMETOOLONG;
  if (ctx->cfg.mode == GFS_MODE_PAPER) return -ENOTSUP;
  if (a->stride == 0 || a->read_len == 0 || a->blocks == 0 || a->serialize) return -EINVAL;
  if (a->threads != 128 && a->threads != 256 && a->threads != 512) return -EINVAL;
  struct stat st;
  if (stat(path, &st) != 0) return -errno;
  const uint64_t size = (uint64_t)st.st_size;
  const uint64_t ns = size ? (size + a->stride - 1) / a->stride : 0;
  if (ns == 0) return 0;
  if (!d_count || !d_sum || !d_hash) return -EINVAL;
  CK(cudaSetDevice(ctx->cfg.device));
  const uint64_t per_block = std::min<uint64_t>(a->read_len, size);
  if (per_block > SIZE_MAX / 2) return -ENOMEM;
  const uint64_t bs = align_up(per_block, 256);
  if (bs && a->blocks > SIZE_MAX / bs) return -ENOMEM;
  int rc = ensure_scan_buf(ctx, (size_t)a->blocks * bs);
  if (!rc) rc = ensure_paper_state(ctx, a->blocks);
  if (rc) return rc;
  DevHandle g = ctx->dev;
  const uint64_t pages_per_read = (a->read_len >> ctx->dev.page_shift) + ((a->read_len & (ctx->cfg.page_size - 1)) != 0);
  g.reserve = ctx->cfg.reserve_frames ? ctx->cfg.reserve_frames
                                      : (uint32_t)(pages_per_read >= 0xffffffffull / a->blocks ? 0xffffffffull
                                                                      : a->blocks * pages_per_read + 1);
  PathArg pa;
  memset(pa.s, 0, sizeof(pa.s));
  memcpy(pa.s, path, len);
  return launch_scan_path(g, pa, *a, ns, ctx->d_scan_buf, bs, d_count, d_sum, d_hash, (cudaStream_t)stream);
}

int gfs_device_handle(gfs_ctx* ctx, uint32_t blocks, uint64_t read_len, void* out, uint64_t cap) {
  if (!ctx || !out || blocks == 0 || read_len == 0) return -EINVAL;
  if (cap < sizeof(DevHandle)) return -ENOSPC;
  DevHandle g = ctx->dev;
  const uint64_t pages_per_read = (read_len >> ctx->dev.page_shift) + ((read_len & (ctx->cfg.page_size - 1)) != 0);
  g.reserve = ctx->cfg.reserve_frames ? ctx->cfg.reserve_frames
                                      : (uint32_t)(pages_per_read >= 0xffffffffull / blocks ? 0xffffffffull
                                                                      : blocks * pages_per_read + 1);
  memcpy(out, &g, sizeof(g));
  return (int)sizeof(DevHandle);
}

int gfs_scan_host(gfs_ctx* ctx, int fid, const gfs_scan_args* a, int64_t* h_count, uint64_t* h_sum, uint64_t* h_hash,
                  void* stream) {
  uint64_t ns = 0, bs = 0;
  DevHandle g;
  int rc = scan_prepare(ctx, fid, a, &ns, &bs, &g);
  if (rc) return rc;
  if (ns == 0) return 0;
  if (!h_count || !h_sum || !h_hash) return -EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // Result buffers are allocated before the launch and the copy back goes to
  // pinned memory: a pageable device-to-host copy issued while the kernel runs
  // blocks in the driver, and so would the I/O threads' submissions the kernel
  // is waiting for.
  const size_t need = (size_t)ns * 24;
  if (need > ctx->out_bytes) {
    if (ctx->d_out) cudaFree(ctx->d_out);
    if (ctx->h_out) cudaFreeHost(ctx->h_out);
    ctx->d_out = ctx->h_out = nullptr;
    ctx->out_bytes = 0;
    CK(cudaMalloc((void**)&ctx->d_out, need));
    CK(cudaHostAlloc((void**)&ctx->h_out, need, cudaHostAllocDefault));
    ctx->out_bytes = need;
  }
  int64_t* dc = (int64_t*)ctx->d_out;
  uint64_t* dsum = (uint64_t*)(ctx->d_out + ns * 8);
  uint64_t* dh = (uint64_t*)(ctx->d_out + ns * 16);
  if (a->serialize) CK(cudaMemsetAsync(&g.ctrl->ticket.v, 0, 8, s));
  rc = launch_scan(g, fid, *a, ns, ctx->d_scan_buf, bs, dc, dsum, dh, s);
  if (!rc) rc = cuda_err(cudaMemcpyAsync(ctx->h_out, ctx->d_out, need, cudaMemcpyDeviceToHost, s));
  int rc2 = cuda_err(cudaStreamSynchronize(s));
  if (!rc && !rc2) {
    memcpy(h_count, ctx->h_out, ns * 8);
    memcpy(h_sum, ctx->h_out + ns * 8, ns * 8);
    memcpy(h_hash, ctx->h_out + ns * 16, ns * 8);
  }
  return rc ? rc : rc2;
}

int gfs_scan_graph(gfs_ctx* ctx, int fid, const gfs_scan_args* a, uint32_t reps, int64_t* d_count, uint64_t* d_sum,
                   uint64_t* d_hash, void* stream) {
  uint64_t ns = 0, bs = 0;
  DevHandle g;
  if (ctx && ctx->cfg.xfer == GFS_XFER_DMA) return -ENOTSUP;
  if (reps == 0) return -EINVAL;
  int rc = scan_prepare(ctx, fid, a, &ns, &bs, &g);  // allocates the scan buffers before capture
  if (rc) return rc;
  if (ns == 0) return 0;
  if (!d_count || !d_sum || !d_hash) return -EINVAL;
  const unsigned long long key[8] = {(unsigned long long)fid, a->stride, a->read_len,
                                     ((unsigned long long)a->blocks << 32) | a->threads,
                                     ((unsigned long long)a->serialize << 32) | a->fused, reps,
                                     (unsigned long long)(uintptr_t)d_count ^ ((unsigned long long)(uintptr_t)d_sum << 1),
                                     (unsigned long long)(uintptr_t)d_hash};
  if (!ctx->graph || memcmp(key, ctx->graph_key, sizeof(key)) != 0) {
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    ctx->graph = nullptr;
    cudaStream_t cs = nullptr;
    CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    rc = cuda_err(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    for (uint32_t r = 0; r < reps && !rc; ++r) {
      rc = launch_drain(ctx->dev, cs);
      if (!rc && ctx->dev.fetch_count)
        rc = cuda_err(cudaMemsetAsync(ctx->dev.fetch_count, 0, (size_t)ctx->dev.debug_pages * 4, cs));
      for (auto& f : ctx->files)
        if (!rc && f.open && f.d_fetched) rc = cuda_err(cudaMemsetAsync(f.d_fetched, 0, f.fetched_bytes, cs));
      if (!rc && ctx->dev.paper_streams) {  // private buffers and per-block LRA queues start empty too
        rc = cuda_err(cudaMemsetAsync(ctx->dev.pmeta, 0, (size_t)ctx->dev.paper_streams * sizeof(PrivBuf), cs));
        if (!rc) rc = cuda_err(cudaMemsetAsync(ctx->dev.lra_head, 0, (size_t)ctx->dev.paper_streams * 4, cs));
        if (!rc) rc = cuda_err(cudaMemsetAsync(ctx->dev.lra_len, 0, (size_t)ctx->dev.paper_streams * 4, cs));
      }
      if (!rc) rc = launch_reset(ctx->dev, cs);
      if (!rc && a->serialize) rc = cuda_err(cudaMemsetAsync(&g.ctrl->ticket.v, 0, 8, cs));
      if (!rc) rc = launch_scan(g, fid, *a, ns, ctx->d_scan_buf, bs, d_count, d_sum, d_hash, cs);
    }
    const int rc2 = cuda_err(cudaStreamEndCapture(cs, &graph));
    if (!rc) rc = rc2;
    if (!rc) rc = cuda_err(cudaGraphInstantiate(&ctx->graph, graph, 0));
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    if (rc) {
      ctx->graph = nullptr;
      return rc;
    }
    memcpy(ctx->graph_key, key, sizeof(key));
  }
  return cuda_err(cudaGraphLaunch(ctx->graph, (cudaStream_t)stream));
}

int gfs_read_many(gfs_ctx* ctx, int fid, uint32_t n, const uint64_t* d_off, const uint64_t* d_len, const uint64_t* d_dst,
                  uint8_t* d_buf, int64_t* d_ret, uint32_t blocks, uint32_t threads, void* stream) {
  if (!ctx) return -EINVAL;
  if (fid < 0 || (size_t)fid >= ctx->files.size() || !ctx->files[fid].open) return -EBADF;
  if (n == 0) return 0;
  if (!d_off || !d_len || !d_dst || !d_buf || !d_ret || blocks == 0) return -EINVAL;
  if (threads != 128 && threads != 256 && threads != 512) return -EINVAL;
  CK(cudaSetDevice(ctx->cfg.device));
  int prc = ensure_paper_state(ctx, blocks);
  if (prc) return prc;
  DevHandle g = ctx->dev;
  g.reserve = ctx->cfg.reserve_frames ? ctx->cfg.reserve_frames : blocks + 1;
  return launch_read_many(g, fid, n, d_off, d_len, d_dst, d_buf, d_ret, blocks, threads, (cudaStream_t)stream);
}

// ---------------------------------------------------------------- CPU-I/O baseline
int gfs_cpuio_scan(const char* path, uint64_t stride, uint64_t read_len, uint32_t threads, uint64_t chunk,
                   uint8_t* d_file, int64_t* d_count, uint64_t* d_sum, uint64_t* d_hash, void* stream,
                   double* seconds) {
  if (!path || !d_file || !d_count || !d_sum || !d_hash || stride == 0 || read_len == 0 || threads == 0 ||
      chunk == 0 || threads > 256)
    return -EINVAL;
  int fd = open(path, O_RDONLY | O_CLOEXEC);
  if (fd < 0) return -errno;
  struct stat st;
  if (fstat(fd, &st) != 0) {
    int e = errno;
    close(fd);
    return -e;
  }
  const uint64_t size = (uint64_t)st.st_size;
  chunk = std::min<uint64_t>(chunk, std::max<uint64_t>(size, 1));
  struct Worker {
    cudaStream_t s = nullptr;
    uint8_t* buf[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int err = 0;
  };
  std::vector<Worker> w(threads);
  int rc = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  for (auto& x : w) {
    if (!rc) rc = cuda_err(cudaStreamCreateWithFlags(&x.s, cudaStreamNonBlocking));
    for (int k = 0; k < 2 && !rc; ++k) {
      rc = cuda_err(cudaHostAlloc((void**)&x.buf[k], chunk, cudaHostAllocDefault));
      if (!rc) rc = cuda_err(cudaEventCreateWithFlags(&x.ev[k], cudaEventDisableTiming));
    }
  }
  double t0 = now_s(), t1 = t0;
  if (!rc) {
    std::atomic<uint64_t> next{0};
    std::vector<std::thread> th;
    for (uint32_t t = 0; t < threads; ++t)
      th.emplace_back([&, t] {
        cudaSetDevice(dev);
        Worker& x = w[t];
        bool pend[2] = {false, false};
        int k = 0;
        for (;;) {
          const uint64_t o = next.fetch_add(chunk);
          if (o >= size) break;
          const size_t nb = (size_t)std::min<uint64_t>(chunk, size - o);
          if (pend[k]) cudaEventSynchronize(x.ev[k]);
          size_t got = 0;
          while (got < nb) {
            ssize_t r = pread(fd, x.buf[k] + got, nb - got, (off_t)(o + got));
            if (r < 0 && errno == EINTR) continue;
            if (r <= 0) {
              x.err = -EIO;
              break;
            }
            got += (size_t)r;
          }
          if (x.err) break;
          if (cudaMemcpyAsync(d_file + o, x.buf[k], nb, cudaMemcpyHostToDevice, x.s) != cudaSuccess) {
            x.err = -EIO;
            break;
          }
          cudaEventRecord(x.ev[k], x.s);
          pend[k] = true;
          k ^= 1;
        }
        cudaStreamSynchronize(x.s);
      });
    for (auto& t : th) t.join();
    for (auto& x : w)
      if (x.err) rc = x.err;
    if (!rc) rc = launch_checksum(d_file, size, stride, read_len, d_count, d_sum, d_hash, (cudaStream_t)stream);
    if (!rc) rc = cuda_err(cudaStreamSynchronize((cudaStream_t)stream));
    t1 = now_s();
  }
  for (auto& x : w) {
    for (int k = 0; k < 2; ++k) {
      if (x.buf[k]) cudaFreeHost(x.buf[k]);
      if (x.ev[k]) cudaEventDestroy(x.ev[k]);
    }
    if (x.s) cudaStreamDestroy(x.s);
  }
  close(fd);
  if (seconds) *seconds = t1 - t0;
  return rc;
}

// ---------------------------------------------------------------- link probes
int gfs_probe_h2d(uint64_t bytes, uint64_t chunk, int reps, double* gbps) {
  if (!gbps || bytes == 0 || chunk == 0 || reps < 1) return -EINVAL;
  uint8_t* h = nullptr;
  uint8_t* d = nullptr;
  cudaStream_t s = nullptr;
  int rc = cuda_err(cudaHostAlloc((void**)&h, bytes, cudaHostAllocDefault));
  if (!rc) rc = cuda_err(cudaMalloc((void**)&d, bytes));
  if (!rc) rc = cuda_err(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  double best = 0;
  if (!rc) {
    memset(h, 1, bytes);
    for (int r = 0; r <= reps && !rc; ++r) {
      const double t0 = now_s();
      for (uint64_t o = 0; o < bytes; o += chunk)
        cudaMemcpyAsync(d + o, h + o, std::min<uint64_t>(chunk, bytes - o), cudaMemcpyHostToDevice, s);
      rc = cuda_err(cudaStreamSynchronize(s));
      const double bw = bytes / (now_s() - t0) / 1e9;
      if (r > 0 && bw > best) best = bw;  // r == 0 is a warm-up
    }
  }
  if (s) cudaStreamDestroy(s);
  if (d) cudaFree(d);
  if (h) cudaFreeHost(h);
  *gbps = best;
  return rc;
}

int gfs_probe_pull(uint64_t bytes, int reps, double* gbps) {
  if (!gbps || bytes < 16 || reps < 1) return -EINVAL;
  bytes &= ~(uint64_t)15;
  uint8_t* h = nullptr;
  uint8_t* dh = nullptr;
  uint8_t* d = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = cuda_err(cudaHostAlloc((void**)&h, bytes, cudaHostAllocMapped));
  if (!rc) rc = cuda_err(cudaHostGetDevicePointer((void**)&dh, h, 0));
  if (!rc) rc = cuda_err(cudaMalloc((void**)&d, bytes));
  if (!rc) rc = cuda_err(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  if (!rc) rc = cuda_err(cudaEventCreate(&e0));
  if (!rc) rc = cuda_err(cudaEventCreate(&e1));
  double best = 0;
  if (!rc) {
    memset(h, 1, bytes);
    for (int r = 0; r <= reps && !rc; ++r) {
      cudaEventRecord(e0, s);
      rc = launch_pull_probe(dh, d, bytes, s);
      cudaEventRecord(e1, s);
      if (!rc) rc = cuda_err(cudaEventSynchronize(e1));
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      const double bw = bytes / (ms * 1e-3) / 1e9;
      if (r > 0 && bw > best) best = bw;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) cudaStreamDestroy(s);
  if (d) cudaFree(d);
  if (h) cudaFreeHost(h);
  *gbps = best;
  return rc;
}

int gfs_probe_pread(const char* path, uint32_t threads, uint64_t chunk, int reps, double* gbps) {
  if (!path || !gbps || threads == 0 || threads > 256 || chunk == 0 || reps < 1) return -EINVAL;
  int fd = open(path, O_RDONLY | O_CLOEXEC);
  if (fd < 0) return -errno;
  struct stat st;
  fstat(fd, &st);
  const uint64_t size = (uint64_t)st.st_size;
  std::vector<uint8_t*> bufs(threads, nullptr);
  int rc = 0;
  for (auto& b : bufs)
    if (!rc) rc = cuda_err(cudaHostAlloc((void**)&b, chunk, cudaHostAllocDefault));
  double best = 0;
  for (int r = 0; r < reps && !rc; ++r) {
    std::atomic<uint64_t> next{0};
    const double t0 = now_s();
    std::vector<std::thread> th;
    for (uint32_t t = 0; t < threads; ++t)
      th.emplace_back([&, t] {
        for (;;) {
          const uint64_t o = next.fetch_add(chunk);
          if (o >= size) break;
          if (pread(fd, bufs[t], (size_t)std::min<uint64_t>(chunk, size - o), (off_t)o) < 0) break;
        }
      });
    for (auto& x : th) x.join();
    const double bw = size / (now_s() - t0) / 1e9;
    if (bw > best) best = bw;
  }
  for (auto& b : bufs)
    if (b) cudaFreeHost(b);
  close(fd);
  *gbps = best;
  return rc;
}

// ---------------------------------------------------------------- CPU-only scan
// Checksums of n bytes at p, file offset `off` of p[0]: sum of the bytes and sum
// of byte * (offset + 1), both mod 2^64.  Pieces of 2048 bytes keep the inner
// sums in 32 bits (2048 * 255 * 2047 < 2^32), so the loops vectorise; each piece
// adds (off + j0 + 1) * its byte sum + its sum of byte * local index.
static void cpu_checksums(const uint8_t* p, uint64_t n, uint64_t off, uint64_t* sum, uint64_t* hash) {
  uint64_t s = 0, h = 0;
  for (uint64_t j0 = 0; j0 < n; j0 += 2048) {
    const uint32_t m = (uint32_t)std::min<uint64_t>(2048, n - j0);
    uint32_t ps = 0, pw = 0;
    for (uint32_t j = 0; j < m; ++j) {
      ps += p[j0 + j];
      pw += (uint32_t)p[j0 + j] * j;
    }
    s += ps;
    h += (off + j0 + 1) * (uint64_t)ps + pw;
  }
  *sum += s;
  *hash += h;
}

int gfs_cpu_scan(const char* path, uint64_t stride, uint64_t read_len, uint32_t threads, int64_t* h_count,
                 uint64_t* h_sum, uint64_t* h_hash, double* seconds) {
  if (!path || stride == 0 || read_len == 0 || threads == 0 || threads > 1024 || !h_count || !h_sum || !h_hash ||
      !seconds)
    return -EINVAL;
  int fd = open(path, O_RDONLY | O_CLOEXEC);
  if (fd < 0) return -errno;
  struct stat st;
  if (fstat(fd, &st) != 0) {
    const int e = -errno;
    close(fd);
    return e;
  }
  const uint64_t size = (uint64_t)st.st_size;
  const uint64_t ns = size ? (size + stride - 1) / stride : 0;
  const uint64_t chunk = std::min<uint64_t>(read_len, 4ull << 20);
  std::atomic<uint64_t> next{0};
  std::atomic<int> fail{0};
  const double t0 = now_s();
  std::vector<std::thread> th;
  for (uint32_t t = 0; t < threads; ++t) try {
    th.emplace_back([&] {
      std::vector<uint8_t> buf;
      try {
        buf.resize((size_t)chunk);
      } catch (...) {
        fail.store(-ENOMEM);
        return;
      }
      for (;;) {
        const uint64_t s = next.fetch_add(1);
        if (s >= ns) break;
        const uint64_t off = s * stride;
        const uint64_t n = std::min<uint64_t>(read_len, size - off);
        uint64_t sum = 0, hash = 0, got = 0;
        int64_t cnt = 0;
        while (got < n) {
          const size_t want = (size_t)std::min<uint64_t>(chunk, n - got);
          const ssize_t r = pread(fd, buf.data(), want, (off_t)(off + got));
          if (r < 0 && errno == EINTR) continue;
          if (r <= 0) {
            cnt = r < 0 ? -errno : (int64_t)got;  // an error, or EOF (the file shrank)
            break;
          }
          cpu_checksums(buf.data(), (uint64_t)r, off + got, &sum, &hash);
          got += (uint64_t)r;
          cnt = (int64_t)got;
        }
        h_count[s] = cnt;
        h_sum[s] = sum;
        h_hash[s] = hash;
      }
    });
  } catch (...) {  // no more threads: the ones started serve every stride
    if (th.empty()) fail.store(-EAGAIN);
    break;
  }
  for (auto& x : th) x.join();
  *seconds = now_s() - t0;
  close(fd);
  return fail.load();
}

// ---------------------------------------------------------------- trace replay (Section 3.2)
int gfs_replay_io(const char* path, const gfs_io_rec* recs, uint64_t n, uint32_t threads, double* seconds,
                  uint64_t* bytes) {
  if (!path || (n && !recs) || threads == 0 || threads > 256 || !seconds) return -EINVAL;
  uint64_t maxb = 0;
  for (uint64_t i = 0; i < n; ++i) maxb = std::max<uint64_t>(maxb, recs[i].bytes);
  if (maxb > (1ull << 32)) return -EINVAL;
  int fd = open(path, O_RDONLY | O_CLOEXEC);
  if (fd < 0) return -errno;
  std::atomic<uint64_t> next{0}, total{0};
  std::atomic<int> err{0};
  const double t0 = now_s();
  std::vector<std::thread> th;
  for (uint32_t t = 0; t < threads; ++t)
    th.emplace_back([&] {
      std::vector<uint8_t> buf((size_t)std::max<uint64_t>(maxb, 1));
      for (;;) {
        const uint64_t i = next.fetch_add(1);
        if (i >= n) break;
        uint64_t got = 0;
        while (got < recs[i].bytes) {
          const ssize_t r = pread(fd, buf.data() + got, (size_t)(recs[i].bytes - got), (off_t)(recs[i].offset + got));
          if (r < 0 && errno == EINTR) continue;
          if (r < 0) {
            err.store(-errno);
            break;
          }
          if (r == 0) break;
          got += (uint64_t)r;
        }
        total.fetch_add(got);
      }
    });
  for (auto& x : th) x.join();
  *seconds = now_s() - t0;
  close(fd);
  if (bytes) *bytes = total.load();
  return err.load();
}

// ---------------------------------------------------------------- CPU self-test
int gfs_selftest_ring(const char* path, uint32_t page_size, uint32_t frames, uint32_t requests, uint32_t max_pages,
                      uint32_t threads, uint32_t slots, uint32_t queue, uint32_t client_blocks, uint64_t seed,
                      uint32_t merge_pages, uint64_t* h_served, uint64_t* h_thread_requests, uint64_t* h_merged) {
  if (!path || !is_pow2(page_size) || page_size < 16 || frames == 0 || max_pages == 0 ||
      max_pages > MAX_RPC_PAGES || threads == 0 || threads > 64 || slots < 2 || seed == 0 ||
      queue > GFS_QUEUE_STATIC || (queue == GFS_QUEUE_STATIC && client_blocks == 0))
    return -EINVAL;
  int fd = open(path, O_RDONLY | O_CLOEXEC);
  if (fd < 0) return -errno;
  struct stat st;
  fstat(fd, &st);
  const uint64_t size = (uint64_t)st.st_size;
  const uint64_t npages = (size + page_size - 1) / page_size;
  const uint32_t shift = log2u(page_size);
  const uint32_t stride = slot_stride(max_pages);
  std::vector<uint8_t> ring((size_t)slots * stride + 64);
  uint8_t* rb = (uint8_t*)(((uintptr_t)ring.data() + 63) & ~(uintptr_t)63);
  for (uint32_t i = 0; i < slots; ++i) ((RingSlot*)(rb + (size_t)i * stride))->seq = i;
  std::vector<uint8_t> fr((size_t)frames << shift);
  std::vector<uint32_t> state(frames, FR_EMPTY);
  ServiceConfig sc;
  sc.ring = rb;
  sc.slots = slots;
  sc.slot_stride = stride;
  sc.page_size = page_size;
  sc.page_shift = shift;
  sc.staging_pages = std::max<uint32_t>(1, (uint32_t)std::min<uint64_t>(4, max_pages));
  sc.threads = threads;
  sc.n_frames = frames;
  sc.queue = queue;
  sc.merge_pages = merge_pages;
  const size_t stg = (size_t)sc.staging_pages * page_size;
  IoService io(
      sc, [&](int) -> Sink* { return new HostSink(fr.data(), state.data(), shift, stg); },
      [&](uint32_t fid, FileView* fv) {
        if (fid != 0) return false;
        fv->fd = fd;
        fv->size = size;
        return true;
      });
  int rc = io.start();
  if (rc) {
    close(fd);
    return rc;
  }
  // Emulated device client: batches of requests over disjoint frame runs.
  uint64_t x = seed, ticket = 0, bad = 0;
  std::vector<uint8_t> want((size_t)max_pages << shift);
  auto rnd = [&]() {
    x ^= x << 13;
    x ^= x >> 7;
    x ^= x << 17;
    return x;
  };
  struct Pending {
    uint64_t page_lo;
    uint32_t n, frame0;
  };
  uint32_t done = 0, issued = 0;
  std::vector<uint64_t> lap(slots, 0);
  const uint32_t batch_max = std::max<uint32_t>(1, std::min<uint32_t>(slots, frames / max_pages));
  while (done < requests && !bad && npages) {
    std::vector<Pending> batch;
    uint32_t next_frame = 0;
    while (batch.size() < batch_max && done + batch.size() < requests) {
      Pending p;
      p.page_lo = rnd() % (npages + 1);  // one past the end exercises EOF
      // every other request continues the one before it (host threads may merge them)
      if (!batch.empty() && (rnd() & 1)) p.page_lo = batch.back().page_lo + batch.back().n;
      p.n = 1 + (uint32_t)(rnd() % max_pages);
      p.frame0 = next_frame;
      if (next_frame + p.n > frames) break;
      next_frame += p.n;
      for (uint32_t i = 0; i < p.n; ++i) __atomic_store_n(&state[p.frame0 + i], (uint32_t)FR_FILLING, __ATOMIC_RELAXED);
      if (queue == GFS_QUEUE_STATIC) {  // the client block's own slot, numbered by its uses
        const uint32_t si = (issued % client_blocks) % slots;
        ticket = lap[si]++ * slots + si;
      }
      ++issued;
      RingSlot* s = (RingSlot*)(rb + (size_t)(ticket % slots) * stride);
      const double t0 = now_s();
      while (__atomic_load_n(&s->seq, __ATOMIC_ACQUIRE) != ticket)
        if (now_s() - t0 > 10) {
          bad = 1;
          break;
        }
      if (bad) break;
      s->fid = 0;
      s->npages = p.n;
      s->page_lo = p.page_lo;
      s->kind = GFS_KIND_DEMAND;
      s->op = 1;
      for (uint32_t i = 0; i < p.n; ++i) s->frames[i] = p.frame0 + i;
      __atomic_store_n(&s->seq, ticket + 1, __ATOMIC_RELEASE);
      ++ticket;
      batch.push_back(p);
    }
    for (const Pending& p : batch) {
      for (uint32_t i = 0; i < p.n && !bad; ++i) {
        const double t0 = now_s();
        uint32_t sv;
        while ((sv = __atomic_load_n(&state[p.frame0 + i], __ATOMIC_ACQUIRE)) == FR_FILLING)
          if (now_s() - t0 > 10) {
            bad = 2;
            break;
          }
        if (bad) break;
        const uint64_t page = p.page_lo + i;
        const uint64_t base = page << shift;
        const bool expect_ok = page < npages;
        if ((sv == FR_READY) != expect_ok) {
          bad = 3;
          break;
        }
        if (expect_ok) {
          const size_t nb = (size_t)std::min<uint64_t>(page_size, size - base);
          if (pread(fd, want.data(), nb, (off_t)base) != (ssize_t)nb) {
            bad = 4;
            break;
          }
          if (memcmp(want.data(), fr.data() + ((size_t)(p.frame0 + i) << shift), nb) != 0) bad = 5;
        }
      }
    }
    done += (uint32_t)batch.size();
    if (batch.empty()) break;
  }
  io.stop();
  close(fd);
  if (h_served) *h_served = io.stats.requests.load();
  if (h_merged) *h_merged = io.stats.merged.load();
  if (h_thread_requests)
    for (uint32_t i = 0; i < threads; ++i) h_thread_requests[i] = io.thread_counters(i).requests.load();
  return bad ? -(int)(1000 + bad) : 0;
}

}  // extern "C"
