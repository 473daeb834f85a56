// Kernels of the GPU file-read path: the scan with the file opened on the device,
// cache purge, drain and reset, the checksum kernel of the CPU-I/O baseline, the
// link probe, and the launches of the stride scan and of independent greads
// (whose instances are compiled in gfs_scan_wide.cu and gfs_scan_narrow.cu).
#include <cuda.h>
#include <cuda_runtime.h>
#include <errno.h>

#include <mutex>

#include "gfs_scan.cuh"

namespace gfs {

// The stride scan with the file opened on the device (Section 2.2: GPU threads
// open, read and close files through GPUfs calls): every block gopens `path`,
// reads its strides with the fused checksum, and gcloses.  A block whose gopen
// fails reports the error for each of its strides.
__global__ void __launch_bounds__(512, 1) k_scan_path(DevHandle g, const __grid_constant__ PathArg path,
                                                    unsigned long long stride,
                                                    unsigned long long read_len, unsigned long long nstrides,
                                                    uint8_t* bufs, unsigned long long buf_stride, long long* cnt,
                                                    unsigned long long* sum, unsigned long long* hash) {
  const uint32_t b = blockIdx.x, tid = threadIdx.x;
  uint8_t* buf = bufs + (size_t)b * buf_stride;
  const int fid = dev::gopen(g, path.s, GFS_RDONLY);
  const long long size = fid >= 0 ? dev::gfstat_size(g, fid) : (long long)fid;
  for (unsigned long long s = b; s < nstrides; s += gridDim.x) {
    Sums acc{0ull, 0ull};
    const long long r = size < 0 ? size : dev::gread_impl<true>(g, (int)b, fid, s * stride, read_len, buf, acc);
    dev::block_sum2(acc.sum, acc.hash);
    if (tid == 0) {
      cnt[s] = r;
      sum[s] = r > 0 ? acc.sum : 0ull;
      hash[s] = r > 0 ? acc.hash : 0ull;
    }
    __syncthreads();
  }
  if (fid >= 0) dev::gclose(g, fid);
  block_help_drain(g);
}

// Host close: drop the cached pages and the sequential contexts of `fid` (the
// device is otherwise idle).
__global__ void __launch_bounds__(256) k_purge(DevHandle g, uint32_t fid) {
  const uint32_t gt = blockIdx.x * blockDim.x + threadIdx.x, nt = gridDim.x * blockDim.x;
  dev::purge_fid(g, fid, gt >> 5, nt >> 5, dev::now_ns() + g.timeout_ns);
  for (uint32_t i = gt; i < g.max_streams; i += nt) g.last_end[(size_t)i * g.max_files + fid] = 0;
}

// GFS_XFER_PULL: copy out every request in flight (cache reset, end of use).
__global__ void __launch_bounds__(512) k_drain(DevHandle g) {
  if (g.xfer == GFS_XFER_DMA) return;
  __shared__ int s_more;
  const unsigned long long dl = dev::now_ns() + g.timeout_ns;
  for (;;) {
    if (threadIdx.x == 0)
      s_more = dev::ld_acq64(&g.ctrl->freed.v) + dev::ld_acq_sys64(g.skipped) < dev::ld_acq64(&g.ctrl->ring_tail.v) &&
               dev::now_ns() < dl;
    __syncthreads();
    const int more = s_more;
    __syncthreads();
    if (!more) break;
    if (!dev::block_help(g, -1, true) && threadIdx.x == 0) __nanosleep(1000);
  }
}

__global__ void k_reset(DevHandle g) {
  const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (size_t)gridDim.x * blockDim.x;
  for (size_t f = tid; f < g.n_frames; f += nt) {
    g.fkey[f] = KEY_NONE;
    g.fstate[f] = FR_EMPTY;
    g.fpins[f] = 0;
    g.fconsumed[f] = 0;
    g.fvalid[f] = 0;
    g.fwindow[f] = 0;
    g.fmark[f] = 0;
    g.faseq[f] = ~0ull;
    if (g.fsrc) g.fsrc[f] = SRC_NONE;
  }
  const size_t nslots = (size_t)g.nbuckets * BUCKET;
  for (size_t i = tid; i < nslots; i += nt) g.tab[i] = ENTRY_EMPTY;
  for (size_t i = tid; i < g.nbuckets; i += nt) {
    g.tlock[i] = 0;
    g.tovf[i] = 0;
  }
  for (size_t i = tid; i < g.fifo_cap; i += nt) {
    g.fifo[i] = ((unsigned long long)i << FRAME_BITS) | MAX_FRAMES;
    g.ret[i] = ((unsigned long long)i << FRAME_BITS) | MAX_FRAMES;
  }
  const size_t nle = (size_t)g.max_streams * g.max_files;
  for (size_t i = tid; i < nle; i += nt) g.last_end[i] = 0;
  if (g.fetch_count)
    for (size_t i = tid; i < g.debug_pages; i += nt) g.fetch_count[i] = 0;
  if (tid == 0) {
    g.ctrl->next_unused.v = 0;
    g.ctrl->alloc_counter.v = 0;
    g.ctrl->fifo_head.v = 0;
    g.ctrl->fifo_tail.v = 0;
    g.ctrl->ret_head.v = 0;
    g.ctrl->ret_tail.v = 0;
    g.ctrl->ticket.v = 0;
    g.ctrl->trace_rpc_n.v = 0;
    g.ctrl->trace_evict_n.v = 0;
    g.ctrl->lat_n.v = 0;
    for (int i = 0; i < ST_COUNT; ++i) g.ctrl->stat[i] = 0;
    // ring_tail and freed keep counting across resets (requests still map to slots)
    // ring_tail is left alone: the ring keeps its position across resets
  }
}

// CPU-I/O baseline consumer: per-stride checksums of a file already in device memory.
__global__ void __launch_bounds__(512) k_checksum(const uint8_t* file, unsigned long long size,
                                                  unsigned long long stride, unsigned long long read_len,
                                                  unsigned long long nstrides, long long* cnt,
                                                  unsigned long long* sum, unsigned long long* hash) {
  for (unsigned long long s = blockIdx.x; s < nstrides; s += gridDim.x) {
    const unsigned long long off = s * stride;
    const unsigned long long n = off >= size ? 0 : (read_len < size - off ? read_len : size - off);
    Sums acc{0ull, 0ull};
    if ((off & 15) == 0) {
      checksum_range(file + off, n, off, acc);
    } else {
      for (unsigned long long j = threadIdx.x; j < n; j += blockDim.x) dev::sums_add1(acc, file[off + j], off + j);
    }
    dev::block_sum2(acc.sum, acc.hash);
    if (threadIdx.x == 0) {
      cnt[s] = (long long)n;
      sum[s] = acc.sum;
      hash[s] = acc.hash;
    }
    __syncthreads();
  }
}

// Link probe: GPU threads copy mapped host memory into device memory.
__global__ void __launch_bounds__(512) k_pull_probe(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                   unsigned long long n16) {
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n16;
       i += (unsigned long long)gridDim.x * blockDim.x)
    dst[i] = __ldcg(src + i);
}

static int cuda_err(cudaError_t e) {
  if (e == cudaSuccess) return 0;
  if (e == cudaErrorMemoryAllocation) return -12;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return -19;
  return -22;
}

int launch_reset(const DevHandle& g, cudaStream_t s) {
  k_reset<<<304, 512, 0, s>>>(g);
  return cuda_err(cudaGetLastError());
}

int launch_drain(const DevHandle& g, cudaStream_t s) {
  k_drain<<<32, 256, 0, s>>>(g);
  return cuda_err(cudaGetLastError());
}

// Which instance a launch uses: 0 = <512, 1> (512 threads, or at most two
// blocks per SM); 1 = <256, 4> (256 threads or fewer, more blocks).
static int scan_variant(uint32_t threads, uint32_t blocks, int device) {
  static int sms[64] = {};
  if (threads > 256) return 0;
  int n = device >= 0 && device < 64 ? sms[device] : 0;
  if (n == 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || n <= 0) return 1;
    if (device >= 0 && device < 64) sms[device] = n;
  }
  return blocks <= 2u * (uint32_t)n ? 0 : 1;
}

int launch_scan(const DevHandle& g, int fid, const gfs_scan_args& a, unsigned long long nstrides, uint8_t* bufs,
                uint64_t buf_stride, int64_t* d_count, uint64_t* d_sum, uint64_t* d_hash, cudaStream_t s) {
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return -19;
  if (scan_variant(a.threads, a.blocks, device) == 0)
    launch_scan_wide(g, fid, a, nstrides, bufs, buf_stride, d_count, d_sum, d_hash, s);
  else
    launch_scan_narrow(g, fid, a, nstrides, bufs, buf_stride, d_count, d_sum, d_hash, s);
  return cuda_err(cudaGetLastError());
}

int launch_scan_path(const DevHandle& g, const PathArg& path, const gfs_scan_args& a, unsigned long long nstrides,
                     uint8_t* bufs, uint64_t buf_stride, int64_t* d_count, uint64_t* d_sum, uint64_t* d_hash,
                     cudaStream_t s) {
  k_scan_path<<<a.blocks, a.threads, 0, s>>>(g, path, a.stride, a.read_len, nstrides, bufs, buf_stride,
                                             (long long*)d_count, (unsigned long long*)d_sum,
                                             (unsigned long long*)d_hash);
  return cuda_err(cudaGetLastError());
}

int launch_purge(const DevHandle& g, uint32_t fid, cudaStream_t s) {
  k_purge<<<152, 256, 0, s>>>(g, fid);
  return cuda_err(cudaGetLastError());
}

int launch_read_many(const DevHandle& g, int fid, uint32_t n, const uint64_t* d_off, const uint64_t* d_len,
                     const uint64_t* d_dst, uint8_t* d_buf, int64_t* d_ret, uint32_t blocks, uint32_t threads,
                     cudaStream_t s) {
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return -19;
  if (scan_variant(threads, blocks, device) == 0)
    launch_read_many_wide(g, fid, n, d_off, d_len, d_dst, d_buf, d_ret, blocks, threads, s);
  else
    launch_read_many_narrow(g, fid, n, d_off, d_len, d_dst, d_buf, d_ret, blocks, threads, s);
  return cuda_err(cudaGetLastError());
}

int launch_checksum(const uint8_t* d_file, uint64_t size, uint64_t stride, uint64_t read_len, int64_t* d_count,
                    uint64_t* d_sum, uint64_t* d_hash, cudaStream_t s) {
  unsigned long long ns = size ? (size + stride - 1) / stride : 0;
  if (ns == 0) return 0;
  unsigned grid = ns < 152ull * 8 ? (unsigned)ns : 152u * 8;
  k_checksum<<<grid, 512, 0, s>>>(d_file, size, stride, read_len, ns, (long long*)d_count,
                                   (unsigned long long*)d_sum, (unsigned long long*)d_hash);
  return cuda_err(cudaGetLastError());
}

int launch_pull_probe(const uint8_t* src, uint8_t* dst, uint64_t n, cudaStream_t s) {
  k_pull_probe<<<304, 512, 0, s>>>((const uint4*)src, (uint4*)dst, n / 16);
  return cuda_err(cudaGetLastError());
}

int scan_max_resident_blocks(uint32_t threads, bool fused, int device, int* out) {
  int per_sm = 0, sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) return cuda_err(e);
  // the largest grid that is resident at once with the instance launch_scan picks for it
  e = scan_occupancy_wide(fused, (int)threads, &per_sm);
  if (e != cudaSuccess) return cuda_err(e);
  int best = per_sm * sms;
  if (threads <= 256) {
    if (best > 2 * sms) best = 2 * sms;  // larger grids use <256, 4>
    e = scan_occupancy_narrow(fused, (int)threads, &per_sm);
    if (e != cudaSuccess) return cuda_err(e);
    if (per_sm * sms > best) best = per_sm * sms;
  }
  *out = best;
  return 0;
}

}  // namespace gfs

// ---------------------------------------------------------------- allocation-free scan
// gfs_scan_static keeps the per-threadblock gread buffers in this file-scope
// device array instead of memory the context allocates, so the call itself never
// allocates.  Every device that loads the library holds the array until exit.
namespace {

constexpr size_t kStaticScratchBytes = 64ull << 20;  // GFS_STATIC_SCRATCH_BYTES in include/gfs.h
static __device__ __align__(256) uint8_t g_scan_scratch[kStaticScratchBytes];

// The context an address was looked up in: a caller that resets the device and
// so creates a new primary context gets the array's address looked up again.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CtxGetCurrentFn g_ctx_current = nullptr;

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};
CUcontext g_scratch_ctx[kMaxDevices] = {};

CUcontext current_context() {
  if (!g_ctx_current) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_ctx_current = (CtxGetCurrentFn)fn;
  }
  CUcontext c = nullptr;
  if (g_ctx_current && g_ctx_current(&c) != CUDA_SUCCESS) c = nullptr;
  return c;
}

// Device address of the scratch array on `device` (current).  In host code the
// array's name is only a host-side stand-in, so the address is looked up once per
// device and context and cached.
int static_scratch(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return -EINVAL;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  const CUcontext cur = current_context();
  if (!g_scratch_addr[device] || g_scratch_ctx[device] != cur) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scan_scratch);
    if (e != cudaSuccess || !p) return e == cudaErrorNoDevice ? -ENODEV : -EINVAL;
    g_scratch_addr[device] = p;
    g_scratch_ctx[device] = cur;
  }
  *out = g_scratch_addr[device];
  return 0;
}

}  // namespace

extern "C" int gfs_scan_static(gfs_ctx* ctx, int fid, const gfs_scan_args* a, int64_t* d_count, uint64_t* d_sum,
                               uint64_t* d_hash, void* stream) {
  if (!ctx || !a) return -EINVAL;
  if (fid < 0 || (size_t)fid >= ctx->files.size() || !ctx->files[fid].open) return -EBADF;
  if (a->stride == 0 || a->read_len == 0 || a->blocks == 0) return -EINVAL;
  if (a->threads != 128 && a->threads != 256 && a->threads != 512) return -EINVAL;
  const uint64_t size = ctx->files[fid].size;
  const uint64_t nstrides = size ? (size + a->stride - 1) / a->stride : 0;
  // a gread never delivers more than the file holds; bound before rounding up
  // and divide instead of multiplying, so that no size wraps around
  const uint64_t per_block = a->read_len < size ? a->read_len : size;
  if (per_block > kStaticScratchBytes) return -ENOSPC;
  const uint64_t buf_stride = (per_block + 255) / 256 * 256;
  if (buf_stride && a->blocks > kStaticScratchBytes / buf_stride) return -ENOSPC;  // beyond the static array
  if (nstrides == 0) return 0;
  if (!d_count || !d_sum || !d_hash) return -EINVAL;
  if (cudaSetDevice(ctx->cfg.device) != cudaSuccess) return -ENODEV;
  if ((ctx->cfg.mode == GFS_MODE_PAPER || ctx->cfg.replacement == GFS_REPL_TB_LRA) &&
      ctx->dev.paper_streams < a->blocks)
    return -ENOTSUP;  // the per-block state would have to be allocated
  void* scratch = nullptr;
  int rc = static_scratch(ctx->cfg.device, &scratch);
  if (rc) return rc;
  gfs::DevHandle g = ctx->dev;
  g.exact_lra = a->serialize ? 1u : 0u;
  const uint64_t pages_per_read = (a->read_len >> ctx->dev.page_shift) + ((a->read_len & (ctx->cfg.page_size - 1)) != 0);
  g.reserve = ctx->cfg.reserve_frames
                  ? ctx->cfg.reserve_frames
                  : (uint32_t)(pages_per_read >= 0xffffffffull / a->blocks ? 0xffffffffull
                                                                             : (uint64_t)a->blocks * pages_per_read + 1);
  cudaStream_t s = (cudaStream_t)stream;
  if (a->serialize) {
    int maxb = 0;
    rc = gfs::scan_max_resident_blocks(a->threads, a->fused != 0, ctx->cfg.device, &maxb);
    if (rc) return rc;
    if ((int)a->blocks > maxb) return -EINVAL;
    if (cudaMemsetAsync(&g.ctrl->ticket.v, 0, 8, s) != cudaSuccess) return -EINVAL;
  }
  return gfs::launch_scan(g, fid, *a, nstrides, (uint8_t*)scratch, buf_stride, d_count, d_sum, d_hash, s);
}
