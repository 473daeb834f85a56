// The stride-scan kernel (Section 6.1 microbenchmark shape: block b greads
// strides b, b+B, ... and checksums each) and the helpers it shares with the
// other kernels.  Its two compiled instances live in translation units of their
// own (gfs_scan_wide.cu, gfs_scan_narrow.cu) so that they compile in parallel.
#pragma once

#include <cuda_runtime.h>

#include "gfs_device.cuh"
#include "gfs_host.h"

namespace gfs {

using dev::Sums;

// Checksums of n bytes at p (file offset `off` of p[0]); p is 16-byte aligned.
__device__ __forceinline__ void checksum_range(const uint8_t* __restrict__ p, unsigned long long n,
                                               unsigned long long off, Sums& acc) {
  const uint32_t tid = threadIdx.x, nt = blockDim.x;
  const unsigned long long n16 = n >> 4;
  const uint4* p4 = reinterpret_cast<const uint4*>(p);
  unsigned long long i = tid;
  for (; i + 3 * nt < n16; i += 4 * nt) {
    uint4 a = p4[i], b = p4[i + nt], c = p4[i + 2 * nt], d = p4[i + 3 * nt];
    dev::sums_add16(acc, a, off + 16 * i);
    dev::sums_add16(acc, b, off + 16 * (i + nt));
    dev::sums_add16(acc, c, off + 16 * (i + 2 * nt));
    dev::sums_add16(acc, d, off + 16 * (i + 3 * nt));
  }
  for (; i < n16; i += nt) dev::sums_add16(acc, p4[i], off + 16 * i);
  for (unsigned long long j = 16 * n16 + tid; j < n; j += nt) dev::sums_add1(acc, p[j], off + j);
}

// Serialized mode: wait (helping in pull mode) until no frame is being filled.
static __device__ void block_quiesce(const DevHandle& g) {
  const unsigned long long dl = dev::now_ns() + g.timeout_ns;
  __shared__ int s_late;
  for (;;) {
    bool busy = false;
    for (uint32_t f = threadIdx.x; f < g.n_frames && !busy; f += blockDim.x) {
      const uint32_t st = dev::ld_acq(&g.fstate[f]);
      busy = st == FR_FILLING || st == FR_COPYING;
    }
    if (threadIdx.x == 0) s_late = dev::now_ns() > dl;
    const int any_busy = __syncthreads_or(busy);
    const int late = s_late;
    __syncthreads();
    if (!any_busy || late) break;
    if (g.xfer != GFS_XFER_DMA && dev::block_help(g, -1, true)) continue;
    if (threadIdx.x == 0) __nanosleep(256);
  }
  __syncthreads();
}

// Pull mode, before a block exits: copy out served requests nobody waits for
// (asynchronous readahead at the end of a scan) so their ring slots free up.
static __device__ void block_help_drain(const DevHandle& g) {
  if (g.xfer == GFS_XFER_DMA) return;
  for (int i = 0; i < 4096; ++i)
    if (!dev::block_help(g, -1, true)) break;
}

// MAXT, MINB: the largest block the instance is compiled for and the blocks per
// SM it must leave room for, which set its register budget.  <512, 1> leaves the
// control path every register it uses (no spills; two 256-thread blocks per SM);
// <256, 4> fits four 256-thread blocks per SM in 64 registers.
template <bool FUSED, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_scan(DevHandle g, int fid, unsigned long long stride,
                                               unsigned long long read_len, unsigned long long nstrides, int serialize,
                                               uint8_t* bufs, unsigned long long buf_stride, long long* cnt,
                                               unsigned long long* sum, unsigned long long* hash) {
  const uint32_t b = blockIdx.x, tid = threadIdx.x;
  uint8_t* buf = bufs + (size_t)b * buf_stride;
  for (unsigned long long s = b; s < nstrides; s += gridDim.x) {
    const unsigned long long off = s * stride;
    if (serialize) {  // one gread at a time, in stride order
      if (tid == 0) {
        const unsigned long long dl = dev::now_ns() + g.timeout_ns;
        while (dev::ld_acq64(&g.ctrl->ticket.v) != s) {
          if (dev::now_ns() > dl) {
            dev::stat_add(g, ST_TIMEOUTS, 1);
            break;
          }
          __nanosleep(128);
        }
      }
      __syncthreads();
    }
    Sums acc{0ull, 0ull};
    long long r = dev::gread_impl<FUSED>(g, (int)b, fid, off, read_len, buf, acc);
    if (serialize) {  // wait until every request of this gread has been served
      block_quiesce(g);
      if (tid == 0) dev::st_rel64(&g.ctrl->ticket.v, s + 1);
    }
    if (!FUSED && r > 0) checksum_range(buf, (unsigned long long)r, off, acc);
    dev::block_sum2(acc.sum, acc.hash);
    if (tid == 0) {
      cnt[s] = r;
      sum[s] = r > 0 ? acc.sum : 0ull;
      hash[s] = r > 0 ? acc.hash : 0ull;
    }
    __syncthreads();
  }
  block_help_drain(g);
}

// Independent greads (Section 2.2): block b serves reads b, b + B, ...; read i
// copies len[i] bytes at off[i] to buf + dst[i] and stores the return value in
// ret[i].  MAXT, MINB as for k_scan: a small read costs a block mostly control-path
// latency, so the reads in flight grow with the blocks resident per SM.
template <int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) k_read_many(DevHandle g, int fid, uint32_t n, const uint64_t* off,
                                                    const uint64_t* len, const uint64_t* dst, uint8_t* buf,
                                                    long long* ret) {
  for (uint32_t i = blockIdx.x; i < n; i += gridDim.x) {
    long long r = dev::gread(g, (int)blockIdx.x, fid, off[i], len[i], buf + dst[i]);
    if (threadIdx.x == 0) ret[i] = r;
    __syncthreads();
  }
  block_help_drain(g);
}

template <bool FUSED, int MAXT, int MINB>
inline void launch_scan_as(const DevHandle& g, int fid, const gfs_scan_args& a, unsigned long long nstrides,
                           uint8_t* bufs, uint64_t buf_stride, int64_t* d_count, uint64_t* d_sum, uint64_t* d_hash,
                           cudaStream_t s) {
  k_scan<FUSED, MAXT, MINB><<<a.blocks, a.threads, 0, s>>>(g, fid, a.stride, a.read_len, nstrides, (int)a.serialize,
                                                           bufs, buf_stride, (long long*)d_count,
                                                           (unsigned long long*)d_sum, (unsigned long long*)d_hash);
}

// Launchers and occupancy of the two instances of k_scan and k_read_many
// (gfs_scan_wide.cu: <512, 1>; gfs_scan_narrow.cu: <256, 4>).
void launch_scan_wide(const DevHandle& g, int fid, const gfs_scan_args& a, unsigned long long nstrides, uint8_t* bufs,
                      uint64_t buf_stride, int64_t* d_count, uint64_t* d_sum, uint64_t* d_hash, cudaStream_t s);
void launch_scan_narrow(const DevHandle& g, int fid, const gfs_scan_args& a, unsigned long long nstrides,
                        uint8_t* bufs, uint64_t buf_stride, int64_t* d_count, uint64_t* d_sum, uint64_t* d_hash,
                        cudaStream_t s);
cudaError_t scan_occupancy_wide(bool fused, int threads, int* per_sm);
cudaError_t scan_occupancy_narrow(bool fused, int threads, int* per_sm);
void launch_read_many_wide(const DevHandle& g, int fid, uint32_t n, const uint64_t* d_off, const uint64_t* d_len,
                           const uint64_t* d_dst, uint8_t* d_buf, int64_t* d_ret, uint32_t blocks, uint32_t threads,
                           cudaStream_t s);
void launch_read_many_narrow(const DevHandle& g, int fid, uint32_t n, const uint64_t* d_off, const uint64_t* d_len,
                             const uint64_t* d_dst, uint8_t* d_buf, int64_t* d_ret, uint32_t blocks, uint32_t threads,
                             cudaStream_t s);

}  // namespace gfs
