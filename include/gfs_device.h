/*
 * gfs_device.h -- device-side file API of the GB300 GPU file-read path.
 *
 * Section 2.2 of "A readahead prefetcher for GPU file system layer" (GPUfs):
 * GPU threads open, read and close files with POSIX-like calls; a read is
 * called by every thread of a threadblock together with the same arguments,
 * the request is split into pages of the GPU page cache, hits are copied to
 * the caller's buffer and misses go to the host over the request queue.
 * Section 4.1 adds the readahead prefetcher behind the same read call, and
 * Section 4.4 the access hint that turns it off.
 *
 * Use from CUDA C++ (nvcc, sm_103a), with relocatable device code:
 *
 *   #include "gfs_device.h"
 *   __global__ void k(const __grid_constant__ gfs_dev h, ...) {
 *     int fid = gopen(&h, path, GFS_RDONLY);
 *     long long n = gread(&h, fid, off, len, buf);
 *     gclose(&h, fid);
 *   }
 *
 *   nvcc -gencode arch=compute_103a,code=sm_103a -rdc=true -I include \
 *        k.cu paper_2109_05366_gb300/libgfs_device.a ...
 *
 * The host fills the handle with gfs_device_handle() (include/gfs.h) and
 * passes it to the kernel by value.  Declare the kernel parameter
 * `const __grid_constant__ gfs_dev` so that &h refers to the parameter itself
 * (a plain by-value parameter whose address is taken is copied to each
 * thread's local memory); a handle copied to device memory works too.  The
 * handle stays valid until gfs_shutdown; the kernel must run on the context's
 * device, and gfs_close / gfs_reset_cache / gfs_shutdown must not be called
 * while it runs.
 *
 * Every call below is threadblock-collective: all threads of the block call it
 * with the same arguments, and it returns the same value in every thread.
 * Nothing traps: each wait has the context's device deadline
 * (gfs_config.timeout_ns) and gives up with -ETIMEDOUT.  Errors are negative
 * errno values.
 */
#ifndef GFS_DEVICE_H_
#define GFS_DEVICE_H_

#include "gfs.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Bytes of the device handle gfs_device_handle() writes (at most this many). */
#define GFS_DEV_HANDLE_BYTES 1024

/* The context's device handle: plain data, opaque to the caller.  Pass it to
 * kernels by value; pass its address to the calls below. */
typedef struct gfs_dev {
  unsigned long long opaque[GFS_DEV_HANDLE_BYTES / 8];
} gfs_dev;

#if defined(__CUDACC__)

/* Open `path` for reading (Section 2.2: open travels over the request queue to
 * the host like a read).  path: NUL-terminated, readable by the device, shorter
 * than GFS_PATH_MAX.  flags: GFS_RDONLY (readahead on, Section 4.4) or GFS_RDWR
 * (readahead off; the path never writes).  Blocks that open a path already open
 * on the device with the same flags share its file id (reference counted); a
 * path whose last reference was closed gets its id back as long as the host has
 * not dropped that id's pages yet (gfs_reset_cache), so blocks that open and
 * close one file at different times still share one id.
 * Returns the file id (>= 0) or -EINVAL, -ENAMETOOLONG, -EMFILE (every id in
 * use), -ENOTSUP (GFS_MODE_PAPER), an error of the host open (-ENOENT, ...),
 * -ETIMEDOUT. */
__device__ int gopen(const gfs_dev* h, const char* path, int flags);

/* Read [off, off + len) of file `fid` into buf (Section 2.2; Section 4.1 may
 * fetch more pages than asked for, which later reads find in the cache).
 * buf: device memory of at least min(len, size - off) bytes, owned by the
 * caller.  The reader identity used to detect sequential access (Section 2.3)
 * is the threadblock (its linear index in the grid).  Returns the byte count
 * (short at end of file, 0 at or past it) or -EBADF (fid not open), -EIO (the
 * host read failed), -ENOMEM (no frame could be freed for a page before the
 * deadline), -ETIMEDOUT. */
__device__ long long gread(const gfs_dev* h, int fid, unsigned long long off, unsigned long long len, void* buf);

/* gread with an explicit reader identity (0 .. max_streams - 1 are tracked),
 * for kernels whose blocks serve several logical readers in turn (a persistent
 * kernel that takes work items, for example). */
__device__ long long gread_as(const gfs_dev* h, int reader, int fid, unsigned long long off,
                              unsigned long long len, void* buf);

/* Close a file id opened with gopen (Section 2.2).  After the last reference
 * the id reads as closed; its pages stay cached, unreachable, until the host
 * drops them (gfs_reset_cache, or reuse of the id) or a gopen of the same path
 * opens the id again.  Returns 0, -EBADF, -ETIMEDOUT. */
__device__ int gclose(const gfs_dev* h, int fid);

/* Size, page size, open flags, hint and mapping of an open file id (no request
 * is sent).  Returns 0 or -EBADF. */
__device__ int gfstat(const gfs_dev* h, int fid, gfs_stat* st);

/* Access hint (Section 4.4): GFS_ADV_RANDOM turns readahead off for the file id,
 * GFS_ADV_NORMAL / GFS_ADV_SEQUENTIAL turn it back on for read-only opens.
 * Applies to greads that start after the call returns, in every block.
 * Returns 0, -EBADF, -EINVAL, -ETIMEDOUT. */
__device__ int gfadvise(const gfs_dev* h, int fid, int advice);

#endif /* __CUDACC__ */

#ifdef __cplusplus
}
#endif
#endif /* GFS_DEVICE_H_ */
