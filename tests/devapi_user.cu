// A kernel written the way a user of the library writes one: it includes the
// public device API (include/gfs_device.h) and nothing else of the library, and
// links libgfs_device.a (relocatable device code).  In user_scan every threadblock
// opens the file (gopen), optionally sets an access hint (gfadvise), checks
// gfstat, reads its strides with gread into its own buffer, sums the bytes, and
// closes the file (gclose).  In user_replay one threadblock replays a list of
// greads one at a time, each under its own reader identity (gread_as).  Built by
// tests/test_gpu_devapi.py with nvcc.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "gfs_device.h"

namespace {

struct UserPath {
  char s[GFS_PATH_MAX];
};

__global__ void __launch_bounds__(256) k_user(const __grid_constant__ gfs_dev g, const __grid_constant__ UserPath path,
                                              int advice, unsigned long long stride, unsigned long long nstrides,
                                              uint8_t* bufs, long long* cnt, unsigned long long* sum, long long* info) {
  uint8_t* buf = bufs + (size_t)blockIdx.x * stride;
  const int fid = gopen(&g, path.s, GFS_RDONLY);
  int arc = 0;
  if (fid >= 0 && advice >= 0) arc = gfadvise(&g, fid, advice);
  gfs_stat st{};
  const int src = fid >= 0 ? gfstat(&g, fid, &st) : fid;
  for (unsigned long long s = blockIdx.x; s < nstrides; s += gridDim.x) {
    const long long r = fid >= 0 ? gread(&g, fid, s * stride, stride, buf) : fid;
    unsigned long long acc = 0;
    for (long long i = threadIdx.x; i < r; i += blockDim.x) acc += buf[i];
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ unsigned long long s_part[8];
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long t = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
      cnt[s] = r;
      sum[s] = t;
    }
    __syncthreads();
  }
  const int crc = fid >= 0 ? gclose(&g, fid) : 0;
  if (threadIdx.x == 0) {
    long long* mine = info + 8 * blockIdx.x;
    mine[0] = fid;
    mine[1] = arc;
    mine[2] = src;
    mine[3] = (long long)st.size;
    mine[4] = st.page_size;
    mine[5] = st.advice;
    mine[6] = st.flags;
    mine[7] = crc;
  }
}

// One threadblock: read i copies len[i] bytes at off[i] of file `fid` into
// buf + dst[i] as reader reader[i], and stores the return value in ret[i].
__global__ void __launch_bounds__(256) k_replay(const __grid_constant__ gfs_dev g, int fid, uint32_t n,
                                                const int* reader, const unsigned long long* off,
                                                const unsigned long long* len, const unsigned long long* dst,
                                                uint8_t* buf, long long* ret) {
  for (uint32_t i = 0; i < n; ++i) {
    const long long r = gread_as(&g, reader[i], fid, off[i], len[i], buf + dst[i]);
    if (threadIdx.x == 0) ret[i] = r;
    __syncthreads();
  }
}

}  // namespace

// handle: the bytes gfs_device_handle wrote; fid: a file id open in the context;
// reader, off, len, dst, ret: n entries each (device memory); buf: device memory
// covering every dst[i] + len[i].  Returns a cudaError_t.
extern "C" int user_replay(const void* handle, uint64_t handle_bytes, int fid, uint32_t n, const void* reader,
                           const void* off, const void* len, const void* dst, void* buf, void* ret, void* stream) {
  if (handle_bytes == 0 || handle_bytes > sizeof(gfs_dev)) return (int)cudaErrorInvalidValue;
  gfs_dev g;
  memset(&g, 0, sizeof(g));
  memcpy(&g, handle, handle_bytes);
  k_replay<<<1, 256, 0, (cudaStream_t)stream>>>(g, fid, n, (const int*)reader, (const unsigned long long*)off,
                                                (const unsigned long long*)len, (const unsigned long long*)dst,
                                                (uint8_t*)buf, (long long*)ret);
  return (int)cudaGetLastError();
}

// handle: the bytes gfs_device_handle wrote; bufs: blocks * stride bytes;
// cnt, sum: nstrides entries; info: 8 * blocks entries.  Returns a cudaError_t.
extern "C" int user_scan(const void* handle, uint64_t handle_bytes, const char* path, int advice, uint64_t stride,
                         uint64_t nstrides, uint32_t blocks, void* bufs, void* cnt, void* sum, void* info,
                         void* stream) {
  if (handle_bytes == 0 || handle_bytes > sizeof(gfs_dev)) return (int)cudaErrorInvalidValue;
  if (strlen(path) >= GFS_PATH_MAX) return (int)cudaErrorInvalidValue;
  gfs_dev g;
  memset(&g, 0, sizeof(g));
  memcpy(&g, handle, handle_bytes);
  UserPath p;
  memset(p.s, 0, sizeof(p.s));
  strcpy(p.s, path);
  k_user<<<blocks, 256, 0, (cudaStream_t)stream>>>(g, p, advice, stride, nstrides, (uint8_t*)bufs, (long long*)cnt,
                                                   (unsigned long long*)sum, (long long*)info);
  return (int)cudaGetLastError();
}
