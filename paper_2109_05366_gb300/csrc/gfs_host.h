// Host-side context of the GPU file-read path (shared by gfs_host.cpp and gfs_kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "gfs_internal.h"

struct gfs_faults_cfg {
  uint32_t eio_every = 0;    // every Nth pread fails with EIO (0 = never)
  uint32_t short_every = 0;  // every Nth pread returns half of what was asked
  uint32_t delay_us = 0;     // sleep before every pread
};

namespace gfs {

struct HostFile {
  int fd = -1;
  uint64_t size = 0;
  void* map = nullptr;     // GFS_XFER_MAPPED: shared mapping of the file the GPU reads
  size_t map_len = 0;
  uint64_t dev_map = 0;    // its device address
  bool map_pinned = false; // registered with CUDA (pinned); else read through the host page tables
  uint32_t* d_fetched = nullptr;  // per-page fetched bits (device)
  size_t fetched_bytes = 0;
  int flags = 0;
  bool direct = false;     // GFS_DIRECT: fd was opened with O_DIRECT
  int advice = GFS_ADV_NORMAL;
  bool open = false;
  std::string path;
  // opened on the device (gopen): reference count of the blocks holding it
  bool by_device = false;
  uint32_t dev_refs = 0;
  bool opening = false;        // a device open is setting the id up
  bool fetched_async = false;  // d_fetched came from cudaMallocAsync on the control stream
  // closed on the device: the id keeps its cached pages (and its descriptor)
  // until they are dropped at a quiet point
  bool retired = false;
};

class IoService;

// Entry points of the device code, implemented in gfs_kernels.cu.
int launch_reset(const DevHandle& g, cudaStream_t s);
int launch_drain(const DevHandle& g, cudaStream_t s);
int launch_scan(const DevHandle& g, int fid, const gfs_scan_args& a, unsigned long long nstrides, uint8_t* bufs,
                uint64_t buf_stride, int64_t* d_count, uint64_t* d_sum, uint64_t* d_hash, cudaStream_t s);
// A path passed by value as a kernel parameter (readable through a pointer).
struct PathArg {
  char s[GFS_PATH_MAX];
};
int launch_scan_path(const DevHandle& g, const PathArg& path, const gfs_scan_args& a, unsigned long long nstrides,
                     uint8_t* bufs, uint64_t buf_stride, int64_t* d_count, uint64_t* d_sum, uint64_t* d_hash,
                     cudaStream_t s);
int launch_purge(const DevHandle& g, uint32_t fid, cudaStream_t s);
int launch_read_many(const DevHandle& g, int fid, uint32_t n, const uint64_t* d_off, const uint64_t* d_len,
                     const uint64_t* d_dst, uint8_t* d_buf, int64_t* d_ret, uint32_t blocks, uint32_t threads,
                     cudaStream_t s);
int launch_checksum(const uint8_t* d_file, uint64_t size, uint64_t stride, uint64_t read_len, int64_t* d_count,
                    uint64_t* d_sum, uint64_t* d_hash, cudaStream_t s);
int scan_max_resident_blocks(uint32_t threads, bool fused, int device, int* out);
int launch_pull_probe(const uint8_t* src, uint8_t* dst, uint64_t n, cudaStream_t s);
}  // namespace gfs
struct gfs_ctx;
// Grow the context's per-block gread buffers to at least `bytes` (before a launch).
int ensure_scan_buf(gfs_ctx* ctx, size_t bytes);
// GFS_MODE_PAPER: private buffers and LRA queues for `streams` streams (before a launch).
int ensure_paper_state(gfs_ctx* ctx, uint32_t streams);
namespace gfs {

}  // namespace gfs

struct gfs_server;

struct gfs_ctx {
  gfs_server* server = nullptr;  // running serving kernel, if any
  gfs_config cfg{};
  gfs::DevHandle dev{};
  void* d_arena = nullptr;
  uint8_t* d_frames = nullptr;
  size_t arena_bytes = 0;
  uint8_t* h_ring = nullptr;  // mapped pinned
  uint8_t* h_staging = nullptr;     // GFS_XFER_PULL: staging arena, mapped pinned
  uint8_t* h_pullmeta = nullptr;    // GFS_XFER_PULL: completion records + page descriptors + buffer counts
  gfs::PullDone* h_done = nullptr;
  gfs::PullPage* h_pages = nullptr;
  uint32_t* h_bcount = nullptr;
  std::vector<gfs::HostFile> files;
  gfs::IoService* io = nullptr;
  uint8_t* d_scan_buf = nullptr;  // per-block gread buffers of gfs_scan
  size_t scan_buf_bytes = 0;
  cudaGraphExec_t graph = nullptr;  // gfs_scan_graph: cached executable and its key
  unsigned long long graph_key[8] = {};
  uint8_t* d_paper = nullptr;       // GFS_MODE_PAPER state (private buffers, metadata, LRA queues)
  uint8_t* d_out = nullptr;        // gfs_scan_host results: device side
  uint8_t* h_out = nullptr;        // and a pinned host copy
  size_t out_bytes = 0;
  char* h_paths = nullptr;         // per-slot path buffers of device opens (mapped pinned)
  cudaStream_t ctl_stream = nullptr;  // device control requests: allocations and file-state copies
  void* h_ctl_fd = nullptr;           // pinned FileDev staging of those copies
  unsigned long long* h_cancel = nullptr;   // mapped pinned: per-slot ticket cancellations
  unsigned long long* h_skipped = nullptr;  // mapped pinned: tickets the host skipped
  bool host_page_tables = false;   // the GPU reads pageable host memory through the host page tables
  std::mutex mu;
  std::mutex files_mu;             // HostFile fields read by the host I/O threads
  std::mutex dev_open_mu;          // device opens and closes, one at a time
};
