// Layouts shared by the host runtime and the device code of the GPU file-read path.
//
// Everything the GPU touches lives in two places:
//   * one device arena (cudaMalloc): cache frames, per-frame metadata, the page
//     table, the consumed FIFO, control counters, traces;
//   * the request ring in mapped pinned host memory, written by the GPU and
//     served by the host I/O threads (Section 2.2: the request queue GPU and host share).
#pragma once

#include <stdint.h>

#include "../../include/gfs.h"

#if defined(__CUDACC__)
#define GFS_HD __host__ __device__
#else
#define GFS_HD
#endif

namespace gfs {

// Frame states.  RECLAIM = claimed by an evictor, not yet reinstalled;
// COPYING = (GFS_XFER_PULL) a threadblock is copying the page out of host staging.
enum : uint32_t { FR_EMPTY = 0, FR_FILLING = 1, FR_READY = 2, FR_ERROR = 3, FR_RECLAIM = 4, FR_COPYING = 5 };
constexpr uint32_t SRC_NONE = 0xffffffffu;
constexpr uint32_t BUF_MAPPED = 0xffffffffu;  // PullPage.buf: src is a device address in a mapped file

constexpr uint64_t KEY_NONE = ~0ull;
constexpr uint64_t ENTRY_EMPTY = ~0ull;
constexpr uint32_t FRAME_BITS = 24;               // frame index bits in a table entry
constexpr uint32_t MAX_FRAMES = (1u << FRAME_BITS) - 1;
constexpr uint32_t MAX_FILES = 255;               // fid 255 reserved (all-ones entry)
constexpr uint32_t BUCKET = 32;                   // slots per bucket = one warp
constexpr uint32_t MAX_RPC_PAGES = 256;
// Cancellations are kept per ticket in a table this much longer than the ring.
// Tickets taken but neither published nor skipped yet: one waiting per resident
// threadblock (2048 at most), plus cancelled ones the host has not reached; a
// block cancels at most one ticket per device deadline, so even every block of a
// full GPU timing out over and over needs tens of seconds of a stalled host to
// come near this span.
constexpr uint32_t CANCEL_SPAN = 65536;

// Page key: (fid, page), 8 + 32 bits.
GFS_HD inline uint64_t make_key(uint32_t fid, uint64_t page) { return ((uint64_t)fid << 32) | (page & 0xffffffffull); }
GFS_HD inline uint32_t key_fid(uint64_t key) { return (uint32_t)(key >> 32); }
GFS_HD inline uint64_t key_page(uint64_t key) { return key & 0xffffffffull; }

// Statistic slots in the device counter block (order = gfs_stats fields).
enum : int {
  ST_GREADS = 0, ST_HITS, ST_MISSES, ST_COALESCED, ST_RPCS, ST_PAGES, ST_BYTES, ST_RA_SYNC, ST_RA_ASYNC,
  ST_EVICT, ST_EVICT_UNCONSUMED, ST_RETRIES, ST_TIMEOUTS, ST_EIO, ST_ENOMEM, ST_BUFHITS, ST_RUN_CUTS, ST_COUNT
};

// Control counters in device memory (one 128-byte line per hot counter).
struct alignas(128) Line { unsigned long long v; unsigned long long pad[15]; };
struct Ctrl {
  Line next_unused;    // never-used frames handed out (victim class 1)
  Line alloc_counter;  // allocation sequence
  Line fifo_head;      // consumed FIFO pop position
  Line fifo_tail;      // consumed FIFO push position
  Line ret_head;       // returned-frame ring pop position
  Line ret_tail;       // returned-frame ring push position
  Line ring_tail;      // request ring: next ticket the GPU takes
  Line ticket;         // serialized mode: next stride allowed to gread
  Line trace_rpc_n;
  Line trace_evict_n;
  Line freed;          // GFS_XFER_PULL: requests whose pages have all been copied out of staging
  Line lat_n;          // greads whose latency was recorded
  unsigned long long stat[ST_COUNT];
};

// GFS_XFER_PULL completion record of a slot, in mapped pinned memory, written by
// the host once every page of the request is published: result (bytes read or
// -errno), then done = ticket + 1.
struct PullDone {
  unsigned long long done;
  long long result;
};

// GFS_XFER_PULL per-page descriptor (mapped pinned), written by the host after
// the pread of the chunk holding the page: where the page sits in the staging
// arena, whether it holds all its bytes, then tag = ticket + 1.
struct PullPage {
  unsigned long long tag;
  unsigned long long src;  // byte offset in the staging arena, or (buf == BUF_MAPPED) a device address
  uint32_t buf;            // staging buffer (host thread * buffers per thread + k), or BUF_MAPPED
  uint32_t ok;
  uint32_t pad[2];
};

// GFS_MODE_PAPER: the pages a stream's private buffer holds ([first, first+count) of fid).
struct PrivBuf {
  unsigned long long first;
  uint32_t fid, count;
};

// Per-file device state.
// Written only by the host (also for the device's gopen, gfadvise and gclose,
// before it answers them); read with relaxed loads at the start of each gread.
struct FileDev {
  unsigned long long size;
  unsigned long long npages;
  uint32_t open;     // 1 if the fid is open
  uint32_t ra;       // readahead enabled (read-only, not ADV_RANDOM)
  uint32_t* fetched; // one bit per page: fetched since the last reset (readahead skips those)
  uint32_t flags;    // open flags
  uint32_t advice;   // GFS_ADV_*
  uint32_t mapped;   // the file's page cache is mapped for the GPU: 1 pinned, 2 through the host page tables
  uint32_t pad;
  unsigned long long dev_map;  // device address of that mapping (0: not mapped)
};
static_assert(sizeof(FileDev) == 56, "FileDev");

// One request-ring slot in mapped pinned memory (64-byte header + frame list).
// Vyukov bounded MPMC protocol on `seq`: slot i starts at seq = i; the GPU
// producer with ticket t waits for seq == t, fills the slot and publishes
// seq = t + 1; the host consumer with ticket h waits for seq == h + 1, copies the
// request out and frees the slot with seq = h + R (in the GPU copy transfers the
// GPU frees it once every page is copied).  A producer whose wait runs out posts
// cancel[t % cancel_n] = t + 1; the host consumer of ticket t then skips it once
// the slot is free for it (seq = t + R), so no host thread waits for a ticket
// nobody will publish.  Tickets of slot i are
// i, i + R, i + 2R, ...: GFS_QUEUE_SHARED hands out tickets in order from one
// counter (slot = ticket mod R); GFS_QUEUE_STATIC picks the slot from the
// threadblock and numbers that slot's uses (ticket = lap * R + slot).
struct RingSlot {
  unsigned long long seq;
  uint32_t fid;
  uint32_t npages;
  unsigned long long page_lo;
  uint32_t kind;
  uint32_t op;         // OP_READ, OP_OPEN, OP_CLOSE
  unsigned long long issue_ns;
  uint32_t pad[6];
  uint32_t frames[1];  // npages entries follow (slot stride covers max_rpc_pages)
};

// Request kinds of a ring slot.  OPEN, CLOSE and ADVISE carry no frames: their
// payload (where the frame list of a read would be) is a CtlMsg, the path of an
// OPEN sits in the slot's GFS_PATH_MAX-byte path buffer, and the requesting
// warp frees the slot after it has read the host's answer.  The host makes
// every change to a file's FileDev itself (a copy on a stream of its own) before
// it answers, so the device sees one order of opens, closes and hints.
enum : uint32_t { OP_READ = 1, OP_OPEN = 2, OP_CLOSE = 3, OP_ADVISE = 4 };

// Payload of an OPEN / CLOSE / ADVISE slot.
struct CtlMsg {
  uint32_t done;    // host: 1 once the answer is written (release)
  int32_t status;   // host: fid (OPEN) or 0, else -errno
  uint32_t arg;     // GPU: open flags (OPEN) or advice (ADVISE)
  uint32_t last;    // host: 1 if the CLOSE dropped the last device reference
};
static_assert(sizeof(CtlMsg) == 16, "CtlMsg");
static_assert(sizeof(unsigned long long) == 8, "u64");

GFS_HD inline uint32_t slot_stride(uint32_t max_pages) {
  uint32_t b = 64 + 4 * max_pages;
  return (b + 63) & ~63u;
}

// Handle passed by value to every kernel.  Plain data only.
struct DevHandle {
  // configuration
  unsigned long long timeout_ns;
  unsigned long long cache_bytes;
  uint32_t page_size, page_shift, n_frames, mode;
  uint32_t ra_cap, async_ra, max_rpc_pages, reserve;
  uint32_t nbuckets, max_streams, max_files, trace_cap;
  uint32_t rpc_slots, slot_stride, fifo_cap, debug_pages;
  // cache frames and per-frame metadata (structure of arrays)
  uint8_t* frames;
  unsigned long long* fkey;
  uint32_t* fstate;
  uint32_t* fpins;
  uint32_t* fconsumed;
  uint32_t* fvalid;
  uint32_t* fwindow;
  uint32_t* fmark;            // readahead mark: end page + 1, 0 = none
  unsigned long long* faseq;  // allocation sequence
  // page table: nbuckets * 32 entries of (key << 24 | frame); per-bucket lock and overflow flag
  unsigned long long* tab;
  uint32_t* tlock;
  uint32_t* tovf;
  // consumed FIFO cells: (position << 24 | frame)
  unsigned long long* fifo;
  // returned-frame ring cells, same layout and capacity: frames a gread took for a
  // page that another gread mapped first (only concurrent greads return one)
  unsigned long long* ret;
  Ctrl* ctrl;
  FileDev* files;
  unsigned long long* last_end;  // per stream: (fid << 32 | end page), ~0 = none
  // request ring (device view of mapped pinned memory) and its per-slot path buffers
  uint8_t* ring;
  char* paths;                   // rpc_slots * GFS_PATH_MAX bytes, mapped pinned
  uint32_t queue;                // GFS_QUEUE_*
  unsigned long long* slot_lap;  // GFS_QUEUE_STATIC: per slot, requests placed in it so far
  unsigned long long* slot_free; // GPU copy transfers: per slot, the ticket it is free for (device
                                 // mirror of `seq` after the GPU frees it; slot i starts at i)
  unsigned long long* cancel;    // mapped pinned, cancel_n entries: at t % cancel_n, t + 1 for a ticket t
                                 // whose producer gave up waiting for its slot (the host skips it)
  uint32_t cancel_n;             // rpc_slots + CANCEL_SPAN entries
  unsigned long long* skipped;   // mapped pinned: tickets the host skipped (drain counts them as freed)
  // traces
  gfs_rpc_rec* trace_rpc;
  gfs_evict_rec* trace_evict;
  uint32_t* fetch_count;  // per page of fid 0
  // GFS_XFER_PULL: host staging per slot (device view), completion records, and
  // the device copy of each in-flight request
  uint32_t xfer;
  uint32_t nbufs;                 // staging buffers in the arena (host threads * buffers per thread)
  unsigned long long chunk_bytes; // bytes per staging buffer (whole pages)
  uint8_t* staging;               // staging arena (device view), nbufs * chunk_bytes, mapped pinned
  PullDone* done;                 // rpc_slots records, mapped pinned
  PullPage* pages;                // rpc_slots * max_rpc_pages descriptors, mapped pinned
  uint32_t* bcount;               // per staging buffer: pages not yet copied out (GPU decrements)
  unsigned long long* dticket;    // ticket of the request in each slot
  uint32_t* dnpages;              // pages of that request
  uint32_t* dcopied;              // pages copied out so far
  uint32_t* dframes;              // rpc_slots * max_rpc_pages frame indices
  uint32_t* fsrc;                 // per frame: slot * max_rpc_pages + page index, SRC_NONE when not in flight
  // gread latency trace (ns), lat_cap entries
  unsigned long long* lat;
  uint32_t lat_cap;
  // GFS_MODE_PAPER: per-stream private buffers and per-stream LRA queues
  uint32_t repl;                  // GFS_REPL_*
  uint32_t paper_streams;         // streams (threadblocks) with state below
  uint32_t quota;                 // frames per stream LRA queue
  uint8_t* pbuf;                  // paper_streams * ra_cap pages
  PrivBuf* pmeta;                 // per stream: which pages the private buffer holds
  uint32_t* lra;                  // paper_streams * quota frames, ring per stream
  uint32_t* lra_head;             // per stream: ring position of the oldest frame
  uint32_t* lra_len;              // per stream: frames in the ring
  // a request for a mapped file is served by the requesting block (it copies the
  // pages from the mapping itself) instead of by the host I/O threads
  uint32_t self_serve;
  // 1: one gread at a time (serialized scan): the demand fallback takes the exact
  // least recently allocated frame of the whole cache, not of a window
  uint32_t exact_lra;
};

}  // namespace gfs
