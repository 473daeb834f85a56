/*
 * gfs.h -- C ABI of the GB300 GPU file-read path: a GPU-resident page cache fed
 * by a GPU-side readahead prefetcher, with streaming replacement for files larger
 * than the cache, served by host I/O threads over a request ring.
 *
 * Method: "A readahead prefetcher for GPU file system layer" (Dimitsas and
 * Silberstein).  Section 2.2 defines the read path (GPUfs): every thread of a
 * threadblock calls a POSIX-like read together; the request is split into pages
 * of the GPU page cache; hits are copied to the user buffer, misses go to the CPU
 * over a shared request queue, the CPU preads the file and sends the data to the
 * GPU.  Section 4.1 adds the readahead prefetcher (one request of PAGE_SIZE +
 * PREFETCH_SIZE on a miss; CPU delivers several pages from one pread; read-only
 * files only; an fadvise-style hint turns it off).  Section 5.1 adds the
 * least-recently-allocated replacement for files larger than the cache.
 *
 * Conventions for every call:
 *   - Return 0 (or a count >= 0) on success and a negative errno on failure
 *     (-EINVAL bad argument, -EBADF bad file id, -ENOMEM allocation failed,
 *     -EIO host read failed, -ENODEV no CUDA device, -ETIMEDOUT a device wait
 *     gave up).  No call aborts the process.
 *   - "stream" arguments are cudaStream_t values passed as void*; NULL is the
 *     legacy default stream.  Launch calls are asynchronous on that stream.
 *   - Pointers named d_* are device pointers (cudaMalloc or equivalent) owned by
 *     the caller; h_* pointers are host memory owned by the caller.
 *   - A gfs_ctx is owned by the library from gfs_init to gfs_shutdown; it is
 *     not safe to call gfs_* on one context from several host threads at once.
 *     Contexts are independent of one another (each its own cache, ring and I/O
 *     threads): several may run at once on one device, on their own streams.
 */
#ifndef GFS_H_
#define GFS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GFS_ABI_VERSION 3

/* Cache policy modes. */
#define GFS_MODE_READAHEAD 0 /* Section 4.1 prefetcher + Section 2.3 window growth */
#define GFS_MODE_ONDEMAND 1  /* original GPUfs (Section 2.2): one page per request */
#define GFS_MODE_PAPER 2     /* the paper's own prefetcher (Section 4.1): per-threadblock private buffer,
                              * one request of 1 + ra_cap_pages pages on a miss; GFS_XFER_PULL / MAPPED only */

/* Replacement (gfs_config.replacement). */
#define GFS_REPL_FIFO 0   /* never-used, then consumed FIFO, then least recently allocated (rule R6) */
#define GFS_REPL_TB_LRA 1 /* Section 5.1: per-threadblock least-recently-allocated queues of F / blocks frames;
                           * with GFS_MODE_READAHEAD every frame a request takes, demand or readahead, comes
                           * from the requesting block's queue (the quota replaces the readahead reserve) */

/* Open flags (Section 4.4, "Page cache coherency": readahead for read-only opens only). */
#define GFS_RDONLY 0
#define GFS_RDWR 2 /* accepted for the hint semantics only; the path never writes */
#define GFS_DIRECT 0x100 /* or-ed into the flags of gfs_open: the host I/O threads read the file with
                          * O_DIRECT, bypassing the host page cache (a cold read from storage every
                          * time, Section 6: the paper flushes the page cache before each run).  The
                          * file is never mapped (GFS_XFER_MAPPED serves it by pread staging);
                          * gfs_open returns the error of open(2) where the file system refuses
                          * O_DIRECT (tmpfs, for one) */

/* fadvise hints (Section 4.4: the user may turn the prefetcher off). */
#define GFS_ADV_NORMAL 0
#define GFS_ADV_SEQUENTIAL 1
#define GFS_ADV_RANDOM 2

/* How a served request reaches the cache frames.
 * In GFS_XFER_PULL and GFS_XFER_MAPPED the host I/O threads make no CUDA call:
 * the GPU copies every page itself, so a kernel waiting for a page depends only
 * on host threads and its own blocks.  In GFS_XFER_DMA the waiting kernel
 * depends on copies the host threads issue on side streams while it runs;
 * anything that serialises GPU work (a profiler's kernel replay or launch
 * capture, a debugger, some MPS set-ups) then holds those copies back until the
 * kernel's device deadline expires (-ETIMEDOUT).  Use DMA only where kernels
 * and copies run concurrently. */
#define GFS_XFER_DMA 0  /* host: pread -> pinned staging -> cudaMemcpyAsync -> stream write of the frame state */
#define GFS_XFER_PULL 1 /* host: pread -> pinned staging; GPU copies staging -> frames over the host link */
#define GFS_XFER_MAPPED 2 /* default.  The file's page cache is mapped for the GPU; the host serves a
                           * request by publishing where its pages are and the GPU copies them into
                           * frames over the host link.  Only a file whose pages are all resident in
                           * the host page cache at gfs_open is mapped (else a page not yet read would
                           * be read from storage where no read is timed).  Where the device reads
                           * pageable host memory through the host's page tables (device attribute
                           * cudaDevAttrPageableMemoryAccessUsesHostPageTables; GB300 with Grace), the
                           * mapping is read-only, of the read-only descriptor, and nothing is pinned
                           * (gfs_stat.mapped = 2); files on any file system qualify, and files opened
                           * on the device (gopen) are mapped too.  Elsewhere, or with
                           * gfs_config.map_pinned, the mapping is registered with CUDA, which pins
                           * every page inside gfs_open (gfs_stat.mapped = 1); registration of
                           * read-only mappings is not available on every platform, so that mapping
                           * is opened read-write (the library never writes through it), and file
                           * systems whose pages cannot be pinned (other than tmpfs) refuse it.  A
                           * file that is not mapped (gfs_stat.mapped = 0) is served as in
                           * GFS_XFER_PULL.  Do not truncate a file while it is open: the GPU reads
                           * its pages where they were mapped, as any reader of a mapping does. */

/* How requests are placed in the ring and how host threads find them (gfs_config.queue). */
#define GFS_QUEUE_SHARED 0 /* one shared ring: the GPU takes the next ticket, any host thread serves any
                            * ticket (every thread busy while requests wait) */
#define GFS_QUEUE_STATIC 1 /* GPUfs as Section 3.2 describes it: a threadblock uses slot
                            * (block index mod rpc_slots) and host thread k polls only its contiguous
                            * share of the slots, so threads whose slots belong to blocks that are not
                            * running stay idle */

/* Request kinds in the RPC trace. */
#define GFS_KIND_DEMAND 0
#define GFS_KIND_SYNC_RA 1
#define GFS_KIND_ASYNC_RA 2

typedef struct gfs_ctx gfs_ctx;

/* Configuration.  gfs_config_default() fills every field; change what you need. */
typedef struct gfs_config {
  uint64_t cache_bytes;    /* GPU page cache size (frames = cache_bytes / page_size) */
  uint64_t timeout_ns;     /* deadline of every device-side wait (default 10 s) */
  uint32_t page_size;      /* bytes per page, power of two, 4 KiB .. 64 MiB */
  uint32_t mode;           /* GFS_MODE_* */
  uint32_t ra_cap_pages;   /* Wmax: readahead pages beyond the demand run (Section 4.1 PREFETCH_SIZE / page) */
  uint32_t async_ra;       /* 1: asynchronous readahead at the readahead mark (Section 2.3); 0: synchronous only (Section 4.1) */
  uint32_t reserve_frames; /* frames readahead must leave for demand misses; 0 = B * ceil(len/P) + 1 per launch */
  uint32_t rpc_slots;      /* request ring slots, 2 or more (Section 2.2 request queue; 128 in GPUfs) */
  uint32_t max_rpc_pages;  /* pages per request at most (1 .. 256) */
  uint32_t host_threads;   /* host I/O threads (Section 2.2; 4 in GPUfs) */
  uint32_t staging_bytes;  /* pinned staging per host thread and buffer (rounded up to whole pages) */
  uint32_t max_streams;    /* distinct gread stream ids (threadblocks) tracked for sequential detection */
  uint32_t max_files;      /* open files at once (<= 255) */
  uint32_t trace_capacity; /* entries kept in the RPC and eviction traces (0 = off) */
  uint32_t xfer;           /* GFS_XFER_* */
  uint32_t debug_counts;   /* 1: keep per-page fetch counts for file id 0 */
  int32_t device;          /* CUDA device ordinal */
  uint32_t latency_capacity; /* greads whose latency (globaltimer ns, entry to exit) is kept; 0 = off */
  uint32_t replacement;    /* GFS_REPL_* */
  uint32_t queue;          /* GFS_QUEUE_* */
  uint32_t host_merge_pages; /* GFS_QUEUE_SHARED: a host thread that takes a read also takes the next
                              * requests already waiting in the ring that continue the same file range,
                              * up to this many pages in all, and serves them with one read into staging
                              * (Section 4.1's several pages from one pread, across threadblocks).
                              * 0 = one staging buffer's worth; 1 = one request at a time */
  uint32_t map_pinned;     /* GFS_XFER_MAPPED: 1 = always register (pin) the mapping; 0 = read it through
                            * the host page tables where the device can (see GFS_XFER_MAPPED) */
  uint32_t self_serve;     /* GFS_XFER_MAPPED: 1 (default) = a request for a mapped file is served by the
                            * threadblock that makes it, which copies the pages from the mapping into
                            * their frames itself (no host thread, no ring slot); 0 = by the host I/O
                            * threads like any other.  Off while host faults are injected
                            * (gfs_set_faults), which only reach requests the host serves */
  uint32_t reserved[1];
} gfs_config;

typedef struct gfs_stat {
  uint64_t size;      /* file size in bytes */
  uint32_t page_size; /* cache page size */
  uint32_t flags;     /* open flags */
  uint32_t advice;    /* current fadvise hint */
  uint32_t mapped;    /* GFS_XFER_MAPPED: 0 not mapped (pread staging), 1 mapped and pinned, 2 mapped
                       * read-only through the host page tables (nothing pinned) */
} gfs_stat;

/* Counters since the last gfs_reset_cache (device side and host side). */
typedef struct gfs_stats {
  uint64_t greads, hits, misses, coalesced_waits;
  uint64_t rpcs, pages_fetched, bytes_fetched, ra_pages_sync, ra_pages_async;
  uint64_t evictions, unconsumed_evictions, retries;
  uint64_t timeouts, eio, enomem;
  uint64_t host_requests, host_preads, host_bytes, host_copies, host_errors;
  uint64_t trace_rpc_count, trace_evict_count;
  uint64_t host_ns_pread;     /* host I/O threads: time inside pread, summed over threads */
  uint64_t host_ns_wait_buf;  /* time waiting for a staging buffer to be copied out (pull) */
  uint64_t host_ns_idle;      /* time waiting for a request */
  uint64_t buffer_hits;       /* GFS_MODE_PAPER: misses served from the private buffer */
  uint64_t host_controls;     /* opens and closes requested by the device (gopen, gclose) */
  uint64_t host_merged;       /* requests a host thread served together with the request before them */
  uint64_t run_cuts;          /* requests cut short because another gread mapped one of their pages
                               * while they were being installed (the rest requested separately) */
  uint64_t reserved[1];
} gfs_stats;

/* Per host I/O thread counters since the last gfs_reset_cache (Section 3.2: the
 * GPUfs host threads' polling before their first request). */
typedef struct gfs_thread_stat {
  uint64_t requests;           /* requests this thread served (reads, opens, closes, hints) */
  uint64_t polls_before_first; /* empty polls (of its ticket or of its slots) before its first request */
  uint64_t first_request_ns;   /* from the reset (or start) to its first request; 0 if none */
  uint64_t idle_ns;            /* time spent waiting for requests */
  uint64_t pread_ns;           /* time spent in pread */
  uint64_t bytes;              /* file bytes it delivered */
} gfs_thread_stat;

/* One entry of the host I/O trace: a file range a host thread served (read with
 * pread in the staging transfers, published for the GPU in the mapped one). */
typedef struct gfs_io_rec {
  uint64_t offset, bytes;
  uint32_t fid, thread;
  uint64_t t_ns; /* when the thread took the request (CLOCK_MONOTONIC) */
} gfs_io_rec;

/* One entry of the RPC trace: a request as the GPU issued it. */
typedef struct gfs_rpc_rec {
  uint32_t fid, kind, npages, reserved;
  uint64_t page_lo;
} gfs_rpc_rec;

/* One entry of the eviction trace. */
typedef struct gfs_evict_rec {
  uint32_t frame, old_fid, new_fid, reserved;
  uint64_t old_page, new_page;
} gfs_evict_rec;

/* Arguments of the stride scan (Section 6.1 microbenchmark): block b of
 * `blocks` greads strides b, b+blocks, ...; stride s covers
 * [s*stride, s*stride + read_len) clipped at EOF. */
typedef struct gfs_scan_args {
  uint64_t stride;    /* bytes between stride starts */
  uint64_t read_len;  /* bytes per gread (usually == stride) */
  uint32_t blocks;    /* threadblocks (gread streams) */
  uint32_t threads;   /* threads per block: 128, 256 or 512 */
  uint32_t serialize; /* 1: one gread at a time in stride order, each waiting for its requests (exact policy traces) */
  uint32_t fused;     /* 1: checksum while copying out of the cache (no user-buffer re-read) */
  uint32_t reserved[4];
} gfs_scan_args;

/* Fill *cfg with defaults: 1 GiB cache, 512 KiB pages, readahead, Wmax 8,
 * async readahead on, 128 slots, 64 pages per request, 16 host threads,
 * 4 MiB staging, 4096 streams, 16 files, no trace, mapped transfer
 * (GFS_XFER_MAPPED, falling back to pread staging per file) with requests for
 * mapped files served by the GPU itself, device 0. */
int gfs_config_default(gfs_config* cfg);

/* Create a context: allocates the cache frames and metadata in device memory,
 * the request ring (mapped pinned host memory) and pinned staging, and starts
 * the host I/O threads.  *out is set only on success. */
int gfs_init(const gfs_config* cfg, gfs_ctx** out);

/* Stop the I/O threads and free everything.  No kernel using the context may
 * still be running.  Accepts NULL. */
int gfs_shutdown(gfs_ctx* ctx);

/* Open `path` read-only; *fid (0 .. max_files-1) names it on host and device.
 * Readahead applies only with GFS_RDONLY (Section 4.4).  With GFS_XFER_MAPPED
 * the open also maps the file when it is fully resident in the host page cache
 * (see GFS_XFER_MAPPED); where the mapping is pinned, that takes time in
 * proportion to the file's size, and gfs_close unpins it. */
int gfs_open(gfs_ctx* ctx, const char* path, int flags, int* fid);

/* Close a file id and drop its cached pages, so that a file opened later under
 * the same id never sees them.  Waits for the device and the host I/O threads
 * to finish the requests in flight (no kernel of the context may be running or
 * queued).  Also closes a file opened on the device (gopen), whatever its
 * reference count. */
int gfs_close(gfs_ctx* ctx, int fid);

/* Set the access hint of a file (Section 4.4): GFS_ADV_RANDOM turns readahead off. */
int gfs_fadvise(gfs_ctx* ctx, int fid, int advice);

/* File size and cache page size. */
int gfs_fstat(gfs_ctx* ctx, int fid, gfs_stat* st);

/* Host-side fault injection for tests (never a device fault): every
 * eio_every-th pread fails with EIO, every short_every-th returns half of what
 * was asked, every pread first sleeps delay_us.  0 disables each.  While any is
 * set, requests for mapped files are served by the host too (gfs_config.self_serve),
 * from the next launch on. */
int gfs_set_faults(gfs_ctx* ctx, uint32_t eio_every, uint32_t short_every, uint32_t delay_us);

/* Drop every cached page, clear the counters, traces and stream history.
 * Synchronises `stream`, then waits until every request issued so far has been
 * served (or skipped: a device wait that ran out before its request got a ring
 * slot posts the request's cancellation, and the host skips it), copies out
 * what was served but never read (GPU copy transfers), and clears the cache on
 * `stream`.  No kernel of the context may be running on another stream.
 * -ETIMEDOUT if the host does not finish within timeout_ns + 5 s (the context
 * is then unusable and should be shut down). */
int gfs_reset_cache(gfs_ctx* ctx, void* stream);

/* Read the counters (synchronises `stream`). */
int gfs_get_stats(gfs_ctx* ctx, gfs_stats* out, void* stream);

/* Copy up to `cap` trace entries to host arrays (either may be NULL);
 * *n_rpc / *n_evict receive the totals recorded (may exceed cap). */
int gfs_get_trace(gfs_ctx* ctx, gfs_rpc_rec* h_rpc, gfs_evict_rec* h_evict, uint32_t cap,
                  uint64_t* n_rpc, uint64_t* n_evict, void* stream);

/* Latencies (ns) of the greads recorded since the last reset (latency_capacity
 * > 0): copies min(cap, recorded) values to h_ns; *n receives the number of
 * greads that finished (may exceed the capacity). */
int gfs_get_latencies(gfs_ctx* ctx, uint64_t* h_ns, uint64_t cap, uint64_t* n, void* stream);

/* Per host I/O thread counters; copies min(cap, host_threads) entries and
 * returns host_threads. */
int gfs_get_thread_stats(gfs_ctx* ctx, gfs_thread_stat* h_out, uint32_t cap);

/* Host I/O trace (trace_capacity > 0): copies min(cap, recorded, trace_capacity)
 * entries in the order the host threads took the requests; *n = ranges recorded. */
int gfs_get_io_trace(gfs_ctx* ctx, gfs_io_rec* h_out, uint64_t cap, uint64_t* n);

/* Replay a host I/O trace on the CPU without the GPU (Section 3.2: the GPU I/O
 * trace replayed by CPU threads isolates the file access pattern from the
 * CPU-GPU interaction): `threads` threads take the records in order and pread
 * each range of `path` into a private buffer.  *seconds = wall time, *bytes =
 * bytes read. */
int gfs_replay_io(const char* path, const gfs_io_rec* recs, uint64_t n, uint32_t threads, double* seconds,
                  uint64_t* bytes);

/* Per-page fetch counts of file id 0 (debug_counts=1); copies min(cap, pages). */
int gfs_get_fetch_counts(gfs_ctx* ctx, uint32_t* h_counts, uint64_t cap, void* stream);

/* The stride scan: launches `args->blocks` threadblocks that gread their strides
 * through the page cache and write, per stride s, d_count[s] (bytes delivered or
 * -errno), d_sum[s] = sum of the bytes mod 2^64 and d_hash[s] = sum of
 * byte * (file offset + 1) mod 2^64.  Arrays hold ceil(size/stride) entries. */
int gfs_scan(gfs_ctx* ctx, int fid, const gfs_scan_args* args, int64_t* d_count,
             uint64_t* d_sum, uint64_t* d_hash, void* stream);

/* Same as gfs_scan with host output arrays: the device results are copied back
 * (through a pinned buffer the context keeps) and `stream` is synchronised
 * before return.
 * While a kernel that calls gread is running, other host threads of the
 * process must not issue blocking CUDA calls that take the driver lock (for
 * example a device-to-pageable-host cudaMemcpy): the host I/O threads need the
 * driver to complete the requests the kernel waits for (GFS_XFER_DMA). */
int gfs_scan_host(gfs_ctx* ctx, int fid, const gfs_scan_args* args, int64_t* h_count,
                  uint64_t* h_sum, uint64_t* h_hash, void* stream);

/* Allocation-free variant of gfs_scan.  The paper has no counterpart: this is a
 * service of this library.  Some callers cannot call cudaMalloc while they
 * run: serving loops that must not stall other streams (cudaMalloc and cudaFree
 * can synchronise the device), and code that owns all of a device's memory
 * through its own allocator and budget.  gfs_scan may allocate its
 * per-threadblock gread buffers on first use or growth; this call never
 * allocates (no cudaMalloc, cudaFree or allocating library routine): the
 * buffers live in a file-scope device array of GFS_STATIC_SCRATCH_BYTES that
 * every device loading the library holds until the process exits.
 *   - blocks * round_up(min(read_len, file size), 256) must fit in
 *     GFS_STATIC_SCRATCH_BYTES, else the call returns -ENOSPC and launches
 *     nothing.
 *   - The first call on a device looks the array's device address up (with that
 *     device made current) and caches it per device and CUDA context; make that
 *     first call before any stream capture.  A caller that resets the device
 *     (cudaDeviceReset) loses every context of this library anyway; the address
 *     is then looked up again in the new context.
 *   - Every call shares the one array and leaves its contents behind; nothing
 *     in it needs to start at zero.  Calls whose kernels overlap on the GPU
 *     race on the array: serialise them (one stream, or events).
 *   - With GFS_MODE_PAPER or GFS_REPL_TB_LRA the context keeps per-threadblock
 *     state that an allocating call sizes: -ENOTSUP until a gfs_scan (or
 *     gfs_scan_path, gfs_read_many) with at least `blocks` threadblocks has run
 *     on the context.
 * Arguments and outputs are those of gfs_scan; its other errors apply too. */
#define GFS_STATIC_SCRATCH_BYTES (64ull << 20)
int gfs_scan_static(gfs_ctx* ctx, int fid, const gfs_scan_args* args, int64_t* d_count, uint64_t* d_sum,
                    uint64_t* d_hash, void* stream);

/* The steady loop of gfs_scan captured in a CUDA graph: `reps` times
 * (copy out requests in flight, clear the cache, scan), launched as one graph on
 * `stream`.  Every repetition starts from an empty cache and rewrites the same
 * outputs.  Needs GFS_XFER_MAPPED or GFS_XFER_PULL (the DMA transfer's reset
 * waits on the host); -ENOTSUP otherwise.  The graph is cached in the context
 * and rebuilt when fid, args, reps or outputs change. */
int gfs_scan_graph(gfs_ctx* ctx, int fid, const gfs_scan_args* args, uint32_t reps, int64_t* d_count,
                   uint64_t* d_sum, uint64_t* d_hash, void* stream);

/* The stride scan with the file opened on the device: every threadblock calls
 * gopen(path, GFS_RDONLY) (the open travels over the request ring to the host
 * like a read, Section 2.2), gfstat for the size, greads its strides and calls
 * gclose.  All threadblocks share one file id (host-side reference count).
 * Outputs as gfs_scan, sized ceil(size/stride) for the size of `path` at the
 * time of the call; if a threadblock's gopen fails, every stride of that block
 * reports the error.  path: host string, at most GFS_PATH_MAX - 1 bytes.
 * GFS_MODE_PAPER: -ENOTSUP.  A file closed on the device keeps its file id
 * (and its cached pages) until gfs_reset_cache, or until gfs_open or gopen
 * needs the id and drops the pages first (gfs_open at a quiet point only). */
#define GFS_PATH_MAX 1024
int gfs_scan_path(gfs_ctx* ctx, const char* path, const gfs_scan_args* args, int64_t* d_count,
                  uint64_t* d_sum, uint64_t* d_hash, void* stream);

/* Copy the context's device handle (the plain-data gfs_dev of
 * include/gfs_device.h that every kernel calling the device API -- gopen,
 * gread, gclose, gfstat, gfadvise -- receives by value) into `out`, which holds
 * `cap` bytes (GFS_DEV_HANDLE_BYTES, i.e. sizeof(gfs_dev), always suffices).
 * `blocks` and `read_len` size the readahead reserve (blocks * ceil(read_len /
 * page) + 1 frames kept free for demand misses) unless
 * gfs_config.reserve_frames is set.  Returns the number of bytes written;
 * -ENOSPC (nothing copied) when cap is smaller.  The handle stays valid until
 * gfs_shutdown; a later gfs_open does not change it. */
int gfs_device_handle(gfs_ctx* ctx, uint32_t blocks, uint64_t read_len, void* out, uint64_t cap);

/* n independent greads: request i reads [d_off[i], d_off[i]+d_len[i]) into
 * d_buf + d_dst[i] and writes its return value to d_ret[i]; `blocks`
 * threadblocks take requests i = b, b+blocks, ...; gread stream id = block
 * index. */
int gfs_read_many(gfs_ctx* ctx, int fid, uint32_t n, const uint64_t* d_off, const uint64_t* d_len,
                  const uint64_t* d_dst, uint8_t* d_buf, int64_t* d_ret, uint32_t blocks,
                  uint32_t threads, void* stream);

/* ---------------------------------------------------------------- serving
 * A persistent kernel runs many sequential-scan requests at once through the
 * shared page cache (continuous batching).  Requests wait in a submission ring
 * and are admitted in arrival order while their frame reservation
 * (min(units, units_in_flight) * pages per unit) fits the frame budget; CTAs
 * take units of the admitted requests round-robin, so requests that arrive
 * while others run share the GPU with them.  Each request reports the byte sum
 * and position hash of its range (the stride-scan checksums), the bytes read
 * and device timestamps.  The paper has no serving loop: this extends its
 * read path (Sections 2.2, 4, 5) to many concurrent readers. */
typedef struct gfs_serve_config {
  uint32_t ctas;            /* persistent CTAs; all must be resident at once */
  uint32_t threads;         /* 128, 256 or 512 */
  uint64_t unit_bytes;      /* bytes per unit of work (one gread) */
  uint32_t max_requests;    /* requests active at once */
  uint32_t queue_slots;     /* submission and completion ring slots (2 or more) */
  uint32_t units_in_flight; /* per-request reservation in units (0 = 16) */
  uint32_t frame_budget;    /* frames admission may reserve (0 = cache frames - ctas * pages per unit) */
  uint32_t idle_exit_ms;    /* the kernel ends after this long with no work (0 = 60 s) */
  uint32_t reserved[5];
} gfs_serve_config;

typedef struct gfs_completion {
  uint64_t tag;        /* the caller's tag */
  int64_t status;      /* 0, or the first -errno of a unit */
  uint64_t sum, hash;  /* sum of bytes, sum of byte * (offset + 1), mod 2^64, over the range */
  uint64_t bytes;      /* bytes read */
  uint64_t t_admit_ns, t_done_ns; /* %globaltimer at admission and completion */
} gfs_completion;

/* Launch the serving kernel on `stream` (asynchronous).  -EBUSY if one runs. */
int gfs_serve_start(gfs_ctx* ctx, const gfs_serve_config* cfg, void* stream);
/* Queue a scan of [off, off+len) of fid; -EAGAIN when the submission ring is full. */
int gfs_submit_scan(gfs_ctx* ctx, int fid, uint64_t off, uint64_t len, uint64_t tag);
/* Copy up to `max` completions (in completion order); returns how many. */
int gfs_poll(gfs_ctx* ctx, gfs_completion* out, int max);
/* Ask the kernel to finish once every submitted request is done, wait, free.
 * Completions not polled by then are discarded.  A completion the device could
 * not post because the host left the completion ring full for longer than the
 * device deadline is dropped, not written over an unread one; gfs_serve_stop
 * then returns -ENOBUFS. */
int gfs_serve_stop(gfs_ctx* ctx);

/* ---------------------------------------------------------------- application streams
 * Consumers shaped like the paper's GPU applications (Section 6.2), reading their
 * input through the page cache.
 *
 * gfs_rowdot: file fid holds a row-major float32 matrix (rows x cols, cols a
 * multiple of 4).  Block b takes stripes b, b+blocks, ... of stripe_rows rows and
 * greads each stripe in pieces of read_len bytes (a multiple of the row size);
 * d_out[r] = sum_c A[r][c] * d_vec[c] in float32 (FMA, any summation order);
 * d_stripe_sum / d_stripe_hash[s] = the byte checksums of stripe s (as in
 * gfs_scan); *d_status = 0 or the first -errno.  d_vec holds cols floats. */
int gfs_rowdot(gfs_ctx* ctx, int fid, uint32_t rows, uint32_t cols, const float* d_vec, float* d_out,
               uint32_t stripe_rows, uint64_t read_len, uint32_t blocks, uint64_t* d_stripe_sum,
               uint64_t* d_stripe_hash, int64_t* d_status, void* stream);

/* gfs_histogram: file fid holds int32 values; d_hist[nbins] (zeroed by the call)
 * receives the count of each value v < nbins; d_sums[0] = sum of all bytes read
 * mod 2^64, d_sums[1] = values >= nbins; *d_status = 0 or the first -errno.
 * Block b greads pieces b, b+blocks, ... of read_len bytes (a multiple of 16). */
int gfs_histogram(gfs_ctx* ctx, int fid, uint32_t nbins, uint32_t* d_hist, uint64_t read_len, uint32_t blocks,
                  uint64_t* d_sums, int64_t* d_status, void* stream);

/* CPU-I/O baseline (Section 6.2 comparison): `threads` host threads pread the
 * file in `chunk` pieces into pinned buffers and cudaMemcpyAsync them into
 * d_file (>= size bytes, caller-owned); then the same per-stride checksum
 * kernel runs.  threads == 1 and chunk >= size is the whole-file variant.
 * *seconds receives the wall time from first pread to results ready. */
int gfs_cpuio_scan(const char* path, uint64_t stride, uint64_t read_len, uint32_t threads,
                   uint64_t chunk, uint8_t* d_file, int64_t* d_count, uint64_t* d_sum,
                   uint64_t* d_hash, void* stream, double* seconds);

/* CPU-only scan, a context figure beside the GPU path (no CUDA call): `threads`
 * host threads pread strides of the file (stride s is [s*stride, s*stride +
 * read_len), clipped at EOF; Section 6.1's per-stride checksums) and compute
 * h_count[s], h_sum[s] (sum of the bytes mod 2^64) and h_hash[s] (sum of byte *
 * (file offset + 1) mod 2^64), the same values the stride scan returns.
 * h_count, h_sum, h_hash: caller-owned host arrays of ceil(size / stride)
 * entries.  *seconds receives the wall time of the scan.  Returns 0, -EINVAL,
 * -ENOMEM, -EAGAIN (no host thread could be started) or the -errno of open; a
 * stride whose pread failed gets that -errno in h_count[s]. */
int gfs_cpu_scan(const char* path, uint64_t stride, uint64_t read_len, uint32_t threads, int64_t* h_count,
                 uint64_t* h_sum, uint64_t* h_hash, double* seconds);

/* Host-link probes for the roofline: pinned host->device copy GB/s with
 * `chunk`-byte copies over `bytes`, and multi-thread pread GB/s of a file. */
int gfs_probe_h2d(uint64_t bytes, uint64_t chunk, int reps, double* gbps);
int gfs_probe_pread(const char* path, uint32_t threads, uint64_t chunk, int reps, double* gbps);
/* GB/s of GPU threads copying `bytes` of mapped pinned host memory into device
 * memory (the link GFS_XFER_MAPPED and GFS_XFER_PULL move data over). */
int gfs_probe_pull(uint64_t bytes, int reps, double* gbps);

/* Self-test of the request ring and the host I/O service without a GPU: a host
 * thread plays the device client (same slot protocol), the service preads the
 * file into host frames; returns 0 when every page matches pread.  queue:
 * GFS_QUEUE_*; with GFS_QUEUE_STATIC request i comes from client block
 * i mod client_blocks and uses that block's slot.  Every other request of a
 * batch continues the file range of the one before it; merge_pages is the
 * service's host_merge_pages (<= 1: no merging).  *h_served = requests the
 * service handed to its sinks; *h_merged (or NULL) = requests it served merged
 * with the one before; h_thread_requests (threads entries, or NULL) gets each
 * host thread's request count. */
int gfs_selftest_ring(const char* path, uint32_t page_size, uint32_t frames, uint32_t requests,
                      uint32_t max_pages, uint32_t threads, uint32_t slots, uint32_t queue,
                      uint32_t client_blocks, uint64_t seed, uint32_t merge_pages, uint64_t* h_served,
                      uint64_t* h_thread_requests, uint64_t* h_merged);

/* Library ABI version (GFS_ABI_VERSION). */
int gfs_abi_version(void);

/* Human-readable text for a negative return value. */
const char* gfs_strerror(int err);

#ifdef __cplusplus
}
#endif
#endif /* GFS_H_ */
