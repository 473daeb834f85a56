// The stride-scan kernel instance <256, 4>: grids of more than two 256-thread blocks per SM.
#include "gfs_scan.cuh"

namespace gfs {

void launch_scan_narrow(const DevHandle& g, int fid, const gfs_scan_args& a, unsigned long long nstrides, uint8_t* bufs,
                    uint64_t buf_stride, int64_t* d_count, uint64_t* d_sum, uint64_t* d_hash, cudaStream_t s) {
  if (a.fused) launch_scan_as<true, 256, 4>(g, fid, a, nstrides, bufs, buf_stride, d_count, d_sum, d_hash, s);
  else launch_scan_as<false, 256, 4>(g, fid, a, nstrides, bufs, buf_stride, d_count, d_sum, d_hash, s);
}

cudaError_t scan_occupancy_narrow(bool fused, int threads, int* per_sm) {
  return fused ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_scan<true, 256, 4>, threads, 0)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_scan<false, 256, 4>, threads, 0);
}

}  // namespace gfs
