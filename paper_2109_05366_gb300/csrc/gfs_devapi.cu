// The device-side file API of include/gfs_device.h, compiled as relocatable
// device code into libgfs_device.a: user kernels include the public header
// only and link this library (nvcc -rdc=true).  Each call forwards to the
// device runtime (gfs_device.cuh) with the opaque handle viewed as the
// context's DevHandle.
#include "gfs_device.cuh"

#include "../../include/gfs_device.h"

static_assert(sizeof(gfs::DevHandle) <= GFS_DEV_HANDLE_BYTES, "the device handle outgrew gfs_dev");
static_assert(alignof(gfs::DevHandle) <= alignof(gfs_dev), "gfs_dev is not aligned for the device handle");

namespace {

__device__ __forceinline__ const gfs::DevHandle& handle_of(const gfs_dev* h) {
  return *reinterpret_cast<const gfs::DevHandle*>(h);
}

// The reader identity of a threadblock: its linear index in the grid.
__device__ __forceinline__ int block_reader() {
  return (int)(blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z));
}

}  // namespace

extern "C" __device__ int gopen(const gfs_dev* h, const char* path, int flags) {
  return gfs::dev::gopen(handle_of(h), path, flags);
}

extern "C" __device__ long long gread(const gfs_dev* h, int fid, unsigned long long off, unsigned long long len,
                                      void* buf) {
  return gfs::dev::gread(handle_of(h), block_reader(), fid, off, len, buf);
}

extern "C" __device__ long long gread_as(const gfs_dev* h, int reader, int fid, unsigned long long off,
                                         unsigned long long len, void* buf) {
  return gfs::dev::gread(handle_of(h), reader, fid, off, len, buf);
}

extern "C" __device__ int gclose(const gfs_dev* h, int fid) { return gfs::dev::gclose(handle_of(h), fid); }

extern "C" __device__ int gfstat(const gfs_dev* h, int fid, gfs_stat* st) {
  return gfs::dev::gfstat(handle_of(h), fid, st);
}

extern "C" __device__ int gfadvise(const gfs_dev* h, int fid, int advice) {
  return gfs::dev::gfadvise(handle_of(h), fid, advice);
}
