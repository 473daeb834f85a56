// The stride-scan and read kernel instances <512, 1>: 512-thread blocks, or grids of at
// most two blocks per SM.
#include "gfs_scan.cuh"

namespace gfs {

void launch_scan_wide(const DevHandle& g, int fid, const gfs_scan_args& a, unsigned long long nstrides, uint8_t* bufs,
                    uint64_t buf_stride, int64_t* d_count, uint64_t* d_sum, uint64_t* d_hash, cudaStream_t s) {
  if (a.fused) launch_scan_as<true, 512, 1>(g, fid, a, nstrides, bufs, buf_stride, d_count, d_sum, d_hash, s);
  else launch_scan_as<false, 512, 1>(g, fid, a, nstrides, bufs, buf_stride, d_count, d_sum, d_hash, s);
}

cudaError_t scan_occupancy_wide(bool fused, int threads, int* per_sm) {
  return fused ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_scan<true, 512, 1>, threads, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_scan<false, 512, 1>, threads, 0);
}

void launch_read_many_wide(const DevHandle& g, int fid, uint32_t n, const uint64_t* d_off, const uint64_t* d_len,
                      const uint64_t* d_dst, uint8_t* d_buf, int64_t* d_ret, uint32_t blocks, uint32_t threads,
                      cudaStream_t s) {
  k_read_many<512, 1><<<blocks, threads, 0, s>>>(g, fid, n, d_off, d_len, d_dst, d_buf, (long long*)d_ret);
}

}  // namespace gfs
