// Application-shaped consumers of the read path (the paper evaluates GPU
// applications that read their input files through GPUfs, Section 6.2):
//   gfs_rowdot     a row-major float32 matrix streamed by stripes of rows into
//                  per-row dot products with a resident vector;
//   gfs_histogram  an int32 array streamed into a histogram.
// Both gread their input in read_len pieces through the page cache, so every
// byte they consume came through the same path as the stride scan; both also
// report checksums of the bytes they consumed.
#include <cuda_runtime.h>
#include <errno.h>

#include "gfs_device.cuh"
#include "gfs_host.h"

namespace gfs {
namespace {

constexpr uint32_t kThreads = 256;
constexpr uint32_t kSmemBins = 8192;  // histogram bins kept in shared memory (the heavy head of a Zipf law)

// Block b reads stripes b, b + B, ...; a stripe is `stripe_rows` rows and is read
// in pieces of `read_len` bytes (whole rows).  Each warp takes rows of the piece.
__global__ void __launch_bounds__(kThreads) k_rowdot(DevHandle g, int fid, uint32_t rows, uint32_t cols,
                                                     const float* __restrict__ vec, float* __restrict__ out,
                                                     uint32_t stripe_rows, unsigned long long read_len, uint8_t* bufs,
                                                     unsigned long long buf_stride, unsigned long long* stripe_sum,
                                                     unsigned long long* stripe_hash, long long* status) {
  uint8_t* buf = bufs + (size_t)blockIdx.x * buf_stride;
  const unsigned long long row_bytes = (unsigned long long)cols * 4;
  const uint32_t rows_per_piece = (uint32_t)(read_len / row_bytes);
  const uint32_t nstripes = (rows + stripe_rows - 1) / stripe_rows;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (uint32_t st = blockIdx.x; st < nstripes; st += gridDim.x) {
    const uint32_t r0 = st * stripe_rows;
    const uint32_t r1 = r0 + stripe_rows < rows ? r0 + stripe_rows : rows;
    dev::Sums acc{0ull, 0ull};
    long long err = 0;
    for (uint32_t pr = r0; pr < r1; pr += rows_per_piece) {
      const uint32_t nr = pr + rows_per_piece < r1 ? rows_per_piece : r1 - pr;
      const unsigned long long off = (unsigned long long)pr * row_bytes;
      const long long n = dev::gread_impl<true>(g, (int)blockIdx.x, fid, off, nr * row_bytes, buf, acc);
      if (n != (long long)(nr * row_bytes)) {
        err = n < 0 ? n : -5;
        break;
      }
      for (uint32_t r = warp; r < nr; r += nwarps) {
        const float4* a = reinterpret_cast<const float4*>(buf + (size_t)r * row_bytes);
        const float4* v = reinterpret_cast<const float4*>(vec);
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
        for (uint32_t c = lane; c < cols / 4; c += 32) {
          const float4 x = a[c], y = __ldg(v + c);
          s0 = fmaf(x.x, y.x, s0);
          s1 = fmaf(x.y, y.y, s1);
          s2 = fmaf(x.z, y.z, s2);
          s3 = fmaf(x.w, y.w, s3);
        }
        float s = (s0 + s1) + (s2 + s3);
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(dev::kFull, s, o);
        if (lane == 0) out[pr + r] = s;
      }
      __syncthreads();
    }
    dev::block_sum2(acc.sum, acc.hash);
    if (threadIdx.x == 0) {
      stripe_sum[st] = acc.sum;
      stripe_hash[st] = acc.hash;
      if (err) atomicCAS((unsigned long long*)status, 0ull, (unsigned long long)err);
    }
    __syncthreads();
  }
  if (g.xfer != GFS_XFER_DMA)
    for (int i = 0; i < 4096; ++i)
      if (!dev::block_help(g, -1, true)) break;
}

// One value of the histogram (warp-collective: every lane calls it, `have` says
// whether the lane holds a value).  Bins below kSmemBins go to shared memory; the
// rest to global memory, lanes holding the same value adding once; values at or
// above nbins are counted in `bad`.
__device__ __forceinline__ void count_value(uint32_t* sh, uint32_t* hist, uint32_t nbins, uint32_t v, bool have,
                                            unsigned long long& bad) {
  if (have && v < kSmemBins && v < nbins) atomicAdd(&sh[v], 1u);
  if (have && v >= nbins) ++bad;
  const bool far = have && v >= kSmemBins && v < nbins;
  const unsigned fm = __ballot_sync(dev::kFull, far);
  if (far) {
    const unsigned same = __match_any_sync(fm, v);
    if ((threadIdx.x & 31) == (uint32_t)(__ffs(same) - 1)) atomicAdd(&hist[v], (uint32_t)__popc(same));
  }
}

// Block b reads pieces b, b + B, ... of the int32 file and counts values.  Bins
// below kSmemBins are counted in shared memory; the rest with warp-aggregated
// global atomics (lanes holding the same value add once).
__global__ void __launch_bounds__(kThreads) k_histogram(DevHandle g, int fid, unsigned long long size, uint32_t nbins,
                                                        uint32_t* __restrict__ hist, unsigned long long read_len,
                                                        uint8_t* bufs, unsigned long long buf_stride,
                                                        unsigned long long* sums, long long* status) {
  __shared__ uint32_t sh[kSmemBins];
  for (uint32_t i = threadIdx.x; i < kSmemBins; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  uint8_t* buf = bufs + (size_t)blockIdx.x * buf_stride;
  const unsigned long long npieces = (size + read_len - 1) / read_len;
  dev::Sums acc{0ull, 0ull};
  unsigned long long bad = 0;
  for (unsigned long long pc = blockIdx.x; pc < npieces; pc += gridDim.x) {
    const unsigned long long off = pc * read_len;
    const long long n = dev::gread_impl<true>(g, (int)blockIdx.x, fid, off, read_len, buf, acc);
    if (n < 0) {
      if (threadIdx.x == 0) atomicCAS((unsigned long long*)status, 0ull, (unsigned long long)n);
      break;
    }
    const uint32_t nv = (uint32_t)(n / 4);
    const uint32_t* vals = reinterpret_cast<const uint32_t*>(buf);
    // 16-byte loads, two per thread in flight (the buffer is 256-byte aligned), then
    // the values left over after the last whole 16 bytes one per thread; every
    // trip count is block-uniform (the far-bin path is warp-collective)
    const uint4* v4 = reinterpret_cast<const uint4*>(buf);
    const uint32_t n4 = nv / 4, nt = blockDim.x;
    for (uint32_t base = 0; base < n4; base += 2 * nt) {
      const uint32_t i = base + threadIdx.x, j = i + nt;
      const uint4 a = i < n4 ? v4[i] : make_uint4(0u, 0u, 0u, 0u);
      const uint4 b = j < n4 ? v4[j] : make_uint4(0u, 0u, 0u, 0u);
      count_value(sh, hist, nbins, a.x, i < n4, bad);
      count_value(sh, hist, nbins, a.y, i < n4, bad);
      count_value(sh, hist, nbins, a.z, i < n4, bad);
      count_value(sh, hist, nbins, a.w, i < n4, bad);
      count_value(sh, hist, nbins, b.x, j < n4, bad);
      count_value(sh, hist, nbins, b.y, j < n4, bad);
      count_value(sh, hist, nbins, b.z, j < n4, bad);
      count_value(sh, hist, nbins, b.w, j < n4, bad);
    }
    for (uint32_t base = 4 * n4; base < nv; base += nt) {
      const uint32_t i = base + threadIdx.x;
      count_value(sh, hist, nbins, i < nv ? vals[i] : 0u, i < nv, bad);
    }
    __syncthreads();
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < kSmemBins && i < nbins; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
  unsigned long long b2 = bad;
  dev::block_sum2(acc.sum, b2);
  if (threadIdx.x == 0) {
    atomicAdd(&sums[0], acc.sum);
    atomicAdd(&sums[1], b2);
  }
  if (g.xfer != GFS_XFER_DMA)
    for (int i = 0; i < 4096; ++i)
      if (!dev::block_help(g, -1, true)) break;
}

}  // namespace
}  // namespace gfs

using namespace gfs;

extern "C" int gfs_rowdot(gfs_ctx* ctx, int fid, uint32_t rows, uint32_t cols, const float* d_vec, float* d_out,
                          uint32_t stripe_rows, uint64_t read_len, uint32_t blocks, uint64_t* d_stripe_sum,
                          uint64_t* d_stripe_hash, int64_t* d_status, void* stream) {
  if (!ctx || !d_vec || !d_out || !d_stripe_sum || !d_stripe_hash || !d_status) return -EINVAL;
  if (fid < 0 || (size_t)fid >= ctx->files.size() || !ctx->files[fid].open) return -EBADF;
  if (rows == 0 || cols == 0 || cols % 4 || stripe_rows == 0 || blocks == 0) return -EINVAL;
  const uint64_t row_bytes = (uint64_t)cols * 4;
  if (read_len < row_bytes || read_len % row_bytes) return -EINVAL;  // pieces of whole rows
  if ((uint64_t)rows * row_bytes > ctx->files[fid].size) return -EINVAL;
  const uint64_t stride = (read_len + 255) / 256 * 256;
  int rc = ensure_scan_buf(ctx, (size_t)blocks * stride);
  if (!rc) rc = ensure_paper_state(ctx, blocks);
  if (rc) return rc;
  DevHandle g = ctx->dev;
  g.reserve = ctx->cfg.reserve_frames ? ctx->cfg.reserve_frames
                                      : blocks * (uint32_t)((read_len + ctx->cfg.page_size - 1) / ctx->cfg.page_size) + 1;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_status, 0, 8, s) != cudaSuccess) return -EINVAL;
  k_rowdot<<<blocks, kThreads, 0, s>>>(g, fid, rows, cols, d_vec, d_out, stripe_rows, read_len, ctx->d_scan_buf,
                                       stride, (unsigned long long*)d_stripe_sum,
                                       (unsigned long long*)d_stripe_hash, (long long*)d_status);
  return cudaGetLastError() == cudaSuccess ? 0 : -EINVAL;
}

extern "C" int gfs_histogram(gfs_ctx* ctx, int fid, uint32_t nbins, uint32_t* d_hist, uint64_t read_len,
                             uint32_t blocks, uint64_t* d_sums, int64_t* d_status, void* stream) {
  if (!ctx || !d_hist || !d_sums || !d_status) return -EINVAL;
  if (fid < 0 || (size_t)fid >= ctx->files.size() || !ctx->files[fid].open) return -EBADF;
  if (nbins == 0 || read_len == 0 || read_len % 16 || blocks == 0) return -EINVAL;
  const uint64_t stride = (read_len + 255) / 256 * 256;
  int rc = ensure_scan_buf(ctx, (size_t)blocks * stride);
  if (!rc) rc = ensure_paper_state(ctx, blocks);
  if (rc) return rc;
  DevHandle g = ctx->dev;
  g.reserve = ctx->cfg.reserve_frames ? ctx->cfg.reserve_frames
                                      : blocks * (uint32_t)((read_len + ctx->cfg.page_size - 1) / ctx->cfg.page_size) + 1;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(d_hist, 0, (size_t)nbins * 4, s) != cudaSuccess) return -EINVAL;
  if (cudaMemsetAsync(d_sums, 0, 16, s) != cudaSuccess) return -EINVAL;
  if (cudaMemsetAsync(d_status, 0, 8, s) != cudaSuccess) return -EINVAL;
  k_histogram<<<blocks, kThreads, 0, s>>>(g, fid, ctx->files[fid].size, nbins, d_hist, read_len, ctx->d_scan_buf,
                                          stride, (unsigned long long*)d_sums, (long long*)d_status);
  return cudaGetLastError() == cudaSuccess ? 0 : -EINVAL;
}
