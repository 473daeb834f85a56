// Device runtime of the GPU file-read path (sm_103a).
//
// gread() is threadblock-collective (Section 2.2: every thread of a threadblock
// calls the read together).  Warp 0 runs the page-cache control for one page at a
// time; then all threads copy the page slice to the user buffer.
//
//   page table      lock-free warp-cooperative lookup in 32-slot buckets of
//                   (key << 24 | frame); inserts and removals take a per-bucket
//                   lock bit so one key is never mapped twice.
//   frames          per-frame state word (EMPTY/FILLING/READY/ERROR/RECLAIM), pin
//                   count, consumed bytes, recorded readahead window, readahead
//                   mark, allocation sequence.
//   miss coalescing the warp that installs a page as FILLING requests it; every
//                   other reader pins the frame and waits on its state word.
//   readahead       Sections 2.3 / 4.1: sequential test, window growth
//                   min(d + Wmax, max(4d, 2 Tprev)), mark for asynchronous
//                   readahead, cut at EOF / present page / reserve.
//   replacement     Section 5.1: never-used frames, then the consumed FIFO (pages
//                   read once, in consumption order), then for demand misses only
//                   the least-recently-allocated unconsumed frame.
//   request ring    Vyukov slots in mapped pinned memory, system-scope release /
//                   acquire; any host thread serves any slot.
//
// Every wait has a %globaltimer deadline; on expiry the call returns -ETIMEDOUT.
// Nothing traps.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gfs_internal.h"

namespace gfs {
namespace dev {

constexpr int kEIO = 5, kEBADF = 9, kEAGAIN = 11, kENOMEM = 12, kEINVAL = 22, kEMFILE = 24, kENAMETOOLONG = 36,
              kENOTSUP = 95, kETIMEDOUT = 110;
constexpr unsigned kFull = 0xffffffffu;

// A gread's allocation context and every frame's allocation record share one
// encoding: (allocation sequence << kOwnerBits) | owner, owner = stream + 1
// (0 = no stream).  Ordering by the value orders by allocation sequence.
constexpr uint32_t kOwnerBits = 20;
constexpr unsigned long long kOwnerMask = (1ull << kOwnerBits) - 1;
__device__ __forceinline__ unsigned long long owner_of(int stream) {
  return stream >= 0 ? ((unsigned long long)stream + 1) & kOwnerMask : 0ull;
}
// Frames the demand fallback scans per attempt; a cache of at most this many
// frames is scanned whole (exact least recently allocated).
constexpr uint32_t kLraWindow = 1024;

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t ld_acq(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_rlx(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acq64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_rlx64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_rel64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_rlx(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_rlx64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Mapped pinned host memory (request ring): system scope.
__device__ __forceinline__ unsigned long long ld_acq_sys64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_acq_sys32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel_sys64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_sys32(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.sys.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_sys64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Four consecutive table entries (32 bytes, 32-byte aligned), one load.
__device__ __forceinline__ void ld_rlx_v4(const unsigned long long* p, unsigned long long* v) {
  asm volatile("ld.relaxed.gpu.global.v4.u64 {%0, %1, %2, %3}, [%4];"
               : "=l"(v[0]), "=l"(v[1]), "=l"(v[2]), "=l"(v[3])
               : "l"(p)
               : "memory");
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ int bcast(int v) { return __shfl_sync(kFull, v, 0); }
__device__ __forceinline__ unsigned long long bcast64(unsigned long long v) { return __shfl_sync(kFull, v, 0); }

__device__ __forceinline__ void stat_add(const DevHandle& g, int i, unsigned long long v) {
  if (v) atomicAdd(&g.ctrl->stat[i], v);
}

// SplitMix64 finaliser (Steele, Lea, Flood 2014) as the bucket hash.
__device__ __forceinline__ uint32_t bucket_of(unsigned long long key, uint32_t nb) {
  unsigned long long z = key + 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  z ^= z >> 31;
  return (uint32_t)z & (nb - 1);
}

__device__ __forceinline__ uint32_t expected_valid(const DevHandle& g, const FileDev& fi, unsigned long long page) {
  unsigned long long base = page << g.page_shift;
  unsigned long long rem = fi.size - base;
  return rem < g.page_size ? (uint32_t)rem : g.page_size;
}

// The file's device state, read with relaxed loads (the device API may have
// rewritten it since this SM last read it).
__device__ __forceinline__ FileDev load_file(const DevHandle& g, int fid) {
  const FileDev* p = &g.files[fid];
  FileDev f;
  f.size = ld_rlx64(&p->size);
  f.npages = ld_rlx64(&p->npages);
  f.open = ld_rlx(&p->open);
  f.ra = ld_rlx(&p->ra);
  f.fetched = (uint32_t*)ld_rlx64((const unsigned long long*)&p->fetched);
  f.flags = ld_rlx(&p->flags);
  f.advice = ld_rlx(&p->advice);
  f.mapped = ld_rlx(&p->mapped);
  f.pad = 0;
  f.dev_map = ld_rlx64(&p->dev_map);
  return f;
}

// ---------------------------------------------------------------- page table
// Warp-cooperative lookup: each lane reads one slot of the bucket (256 B).
static __device__ int tab_lookup(const DevHandle& g, unsigned long long key) {
  const int lane = lane_id();
  uint32_t b = bucket_of(key, g.nbuckets);
  for (uint32_t probe = 0; probe < g.nbuckets; ++probe) {
    unsigned long long e = ld_rlx64(&g.tab[(size_t)b * BUCKET + lane]);
    int ovf = 0;
    if (lane == 0) ovf = (int)ld_rlx(&g.tovf[b]);  // in flight with the bucket
    bool hit = e != ENTRY_EMPTY && (e >> FRAME_BITS) == key;
    unsigned m = __ballot_sync(kFull, hit);
    if (m) {
      unsigned long long w = __shfl_sync(kFull, e, __ffs(m) - 1);
      return (int)(w & MAX_FRAMES);
    }
    if (!bcast(ovf)) return -1;
    b = (b + 1) & (g.nbuckets - 1);
  }
  return -1;
}

// Warp: how many of the pages p, p + 1, ..., p + k - 1 (k <= 32), counted from p,
// are not in the table before the first that is.  Eight keys are looked up at a
// time (eight bucket loads in flight, with their overflow flags); a key missing
// from a bucket that overflowed is followed along the chain by tab_lookup.
static __device__ uint32_t absent_prefix(const DevHandle& g, uint32_t fid, unsigned long long p, uint32_t k) {
  const int lane = lane_id();
  for (uint32_t q0 = 0; q0 < k; q0 += 8) {
    unsigned long long e[8];
#pragma unroll
    for (uint32_t j = 0; j < 8; ++j) {
      const uint32_t b = bucket_of(make_key(fid, p + q0 + j), g.nbuckets);
      e[j] = q0 + j < k ? ld_rlx64(&g.tab[(size_t)b * BUCKET + lane]) : ENTRY_EMPTY;
    }
    const uint32_t jb = bucket_of(make_key(fid, p + q0 + (lane & 7)), g.nbuckets);
    const uint32_t ovf = lane < 8 && q0 + lane < k ? ld_rlx(&g.tovf[jb]) : 0u;
#pragma unroll
    for (uint32_t j = 0; j < 8; ++j) {
      if (q0 + j >= k) return k;
      const unsigned long long key = make_key(fid, p + q0 + j);
      bool present = __ballot_sync(kFull, e[j] != ENTRY_EMPTY && (e[j] >> FRAME_BITS) == key) != 0u;
      if (!present && __shfl_sync(kFull, ovf, (int)j) != 0u) present = tab_lookup(g, key) >= 0;
      if (present) return q0 + j;
    }
  }
  return k;
}

static __device__ bool bucket_lock(const DevHandle& g, uint32_t b, unsigned long long deadline) {
  // lane 0 only
  while (atomicCAS(&g.tlock[b], 0u, 1u) != 0u) {
    if (now_ns() > deadline) return false;
    __nanosleep(32);
  }
  __threadfence();
  return true;
}
static __device__ void bucket_unlock(const DevHandle& g, uint32_t b) {
  __threadfence();
  atomicExch(&g.tlock[b], 0u);
}

// Map key -> f unless key is already mapped.  Returns the frame now mapped for
// the key (f if this call inserted it), -ETIMEDOUT, or -ENOMEM (table full).
static __device__ int tab_insert(const DevHandle& g, unsigned long long key, uint32_t f, unsigned long long deadline) {
  const int lane = lane_id();
  const uint32_t home = bucket_of(key, g.nbuckets);
  int ok = 0;
  if (lane == 0) ok = bucket_lock(g, home, deadline);
  if (!bcast(ok)) return -kETIMEDOUT;
  int result = -kENOMEM;
  uint32_t b = home;
  for (uint32_t probe = 0; probe < g.nbuckets; ++probe) {  // already present?
    unsigned long long e = ld_rlx64(&g.tab[(size_t)b * BUCKET + lane]);
    unsigned m = __ballot_sync(kFull, e != ENTRY_EMPTY && (e >> FRAME_BITS) == key);
    if (m) {
      result = (int)(__shfl_sync(kFull, e, __ffs(m) - 1) & MAX_FRAMES);
      break;
    }
    int ovf = 0;
    if (lane == 0) ovf = (int)ld_rlx(&g.tovf[b]);
    if (!bcast(ovf)) break;
    b = (b + 1) & (g.nbuckets - 1);
  }
  if (result < 0) {
    const unsigned long long entry = (key << FRAME_BITS) | f;
    b = home;
    for (uint32_t probe = 0; probe < g.nbuckets && result < 0; ++probe) {
      unsigned long long* slot = &g.tab[(size_t)b * BUCKET + lane];
      unsigned em = __ballot_sync(kFull, ld_rlx64(slot) == ENTRY_EMPTY);
      while (em) {
        int src = __ffs(em) - 1;
        unsigned long long old = 0;
        if (lane == src) old = atomicCAS(slot, ENTRY_EMPTY, entry);
        old = __shfl_sync(kFull, old, src);
        if (old == ENTRY_EMPTY) { result = (int)f; break; }
        em &= ~(1u << src);
      }
      if (result < 0) {  // bucket full: later lookups must continue past it
        if (lane == 0) { atomicExch(&g.tovf[b], 1u); __threadfence(); }
        __syncwarp();
        b = (b + 1) & (g.nbuckets - 1);
      }
    }
  }
  __syncwarp();
  if (lane == 0) bucket_unlock(g, home);
  __syncwarp();
  return result;
}

// Remove the mapping key -> f if present.
static __device__ void tab_remove(const DevHandle& g, unsigned long long key, uint32_t f, unsigned long long deadline) {
  const int lane = lane_id();
  const uint32_t home = bucket_of(key, g.nbuckets);
  int ok = 0;
  if (lane == 0) ok = bucket_lock(g, home, deadline);
  ok = bcast(ok);
  const unsigned long long entry = (key << FRAME_BITS) | f;
  uint32_t b = home;
  for (uint32_t probe = 0; probe < g.nbuckets; ++probe) {
    unsigned long long* slot = &g.tab[(size_t)b * BUCKET + lane];
    unsigned m = __ballot_sync(kFull, ld_rlx64(slot) == entry);
    if (m) {
      if (lane == __ffs(m) - 1) atomicCAS(slot, entry, ENTRY_EMPTY);
      break;
    }
    int ovf = 0;
    if (lane == 0) ovf = (int)ld_rlx(&g.tovf[b]);
    if (!bcast(ovf)) break;
    b = (b + 1) & (g.nbuckets - 1);
  }
  __syncwarp();
  if (lane == 0 && ok) bucket_unlock(g, home);
  __syncwarp();
}

// ---------------------------------------------------------------- lane-level table updates
// One lane, one key: the counterparts of tab_remove and tab_insert for the pages
// of a run, which update the table a lane per page instead of one page at a
// time.  A lane reads a whole bucket with eight 32-byte loads.  A lane holds at
// most one bucket lock at a time (lanes whose keys share a home bucket take it
// in turn, and independent thread scheduling lets the holder go on), so no two
// lanes or warps ever wait on each other in a cycle.

// One lane's view of bucket b: the first entry for `key` (hit, its slot, -1 if
// none) and the first empty slot (-1 if none).
struct LaneScan {
  int hit, empty;
  unsigned long long entry;
};
static __device__ __noinline__ LaneScan lane_scan(const DevHandle& g, uint32_t b, unsigned long long key) {
  const unsigned long long* base = &g.tab[(size_t)b * BUCKET];
  LaneScan r{-1, -1, 0ull};
#pragma unroll
  for (int h = 0; h < 2; ++h) {  // two halves of 16 slots, four loads in flight each
    unsigned long long v[16];
#pragma unroll
    for (int q = 0; q < 4; ++q) ld_rlx_v4(base + 16 * h + 4 * q, v + 4 * q);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const unsigned long long e = v[i];
      if (r.hit < 0 && e != ENTRY_EMPTY && (e >> FRAME_BITS) == key) {
        r.hit = 16 * h + i;
        r.entry = e;
      }
      if (r.empty < 0 && e == ENTRY_EMPTY) r.empty = 16 * h + i;
    }
  }
  return r;
}

// Remove the mapping key -> f if present (one lane).  No lock: the entry's value
// is unique to (key, frame), so one compare-and-swap on its slot removes exactly
// it, and an insert holding the bucket's lock only ever fills empty slots.
static __device__ void lane_tab_remove(const DevHandle& g, unsigned long long key, uint32_t f) {
  const unsigned long long entry = (key << FRAME_BITS) | f;
  uint32_t b = bucket_of(key, g.nbuckets);
  for (uint32_t probe = 0; probe < g.nbuckets; ++probe) {
    const LaneScan r = lane_scan(g, b, key);
    if (r.hit >= 0 && r.entry == entry) {
      atomicCAS(&g.tab[(size_t)b * BUCKET + r.hit], entry, ENTRY_EMPTY);
      return;
    }
    if (r.hit >= 0) {  // another mapping of the key first: look at every slot of the bucket
      for (uint32_t i = 0; i < BUCKET; ++i)
        if (ld_rlx64(&g.tab[(size_t)b * BUCKET + i]) == entry) {
          atomicCAS(&g.tab[(size_t)b * BUCKET + i], entry, ENTRY_EMPTY);
          return;
        }
    }
    if (ld_rlx(&g.tovf[b]) == 0u) return;
    b = (b + 1) & (g.nbuckets - 1);
  }
}

// Map key -> f unless key is already mapped (one lane; tab_insert's rule under
// the home bucket's lock).  Returns the frame now mapped for the key (f if this
// call inserted it), -ETIMEDOUT or -ENOMEM.
static __device__ __noinline__ int lane_tab_insert(const DevHandle& g, unsigned long long key, uint32_t f,
                                                   unsigned long long deadline) {
  const uint32_t home = bucket_of(key, g.nbuckets);
  if (!bucket_lock(g, home, deadline)) return -kETIMEDOUT;
  int result = -kENOMEM;
  int first_b = -1, first_i = -1;  // the first empty slot from the home bucket on
  uint32_t b = home;
  for (uint32_t probe = 0; probe < g.nbuckets; ++probe) {  // already present?
    const LaneScan r = lane_scan(g, b, key);
    if (r.hit >= 0) {
      result = (int)(r.entry & MAX_FRAMES);
      break;
    }
    if (first_b < 0 && r.empty >= 0) {
      first_b = (int)b;
      first_i = r.empty;
    }
    if (ld_rlx(&g.tovf[b]) == 0u) break;
    b = (b + 1) & (g.nbuckets - 1);
  }
  if (result < 0) {
    const unsigned long long entry = (key << FRAME_BITS) | f;
    // an insert under another home's lock may fill an empty slot of an overflow
    // bucket first: a failed CAS moves on to the next empty slot
    if (first_b >= 0 && atomicCAS(&g.tab[(size_t)first_b * BUCKET + first_i], ENTRY_EMPTY, entry) == ENTRY_EMPTY)
      result = (int)f;
    b = home;
    for (uint32_t probe = 0; probe < g.nbuckets && result < 0; ++probe) {
      for (uint32_t i = 0; i < BUCKET && result < 0; ++i) {
        unsigned long long* slot = &g.tab[(size_t)b * BUCKET + i];
        if (ld_rlx64(slot) == ENTRY_EMPTY && atomicCAS(slot, ENTRY_EMPTY, entry) == ENTRY_EMPTY) result = (int)f;
      }
      if (result < 0) {  // bucket full: later lookups must continue past it
        atomicExch(&g.tovf[b], 1u);
        __threadfence();
        b = (b + 1) & (g.nbuckets - 1);
      }
    }
  }
  bucket_unlock(g, home);
  return result;
}

// ---------------------------------------------------------------- consumed FIFO, returned frames
// Bounded MPMC queue over fifo_cap cells; each frame is in it at most once.  Cell
// t % cap holds (seq << FRAME_BITS) | frame: seq = t while free for the push of
// ticket t, t + 1 once that push landed, t + cap once popped (free for the next
// lap).  Both ends take tickets by fetch-and-add (one atomic per operation, no
// retry loop every block contends on).  A pop whose ticket ran past the tail
// gives the ticket up by moving its cell straight to t + cap; the push that later
// draws that ticket sees a cell already past it and draws another.  Give-ups only
// happen when the queue is empty, so the order of the frames in it is kept.

// A ticket ring of frames: the consumed FIFO, or the ring of returned frames
// (same protocol and capacity).
struct FrameRing {
  unsigned long long* cells;
  unsigned long long* head;
  unsigned long long* tail;
};
__device__ __forceinline__ FrameRing fifo_ring(const DevHandle& g) {
  return FrameRing{g.fifo, &g.ctrl->fifo_head.v, &g.ctrl->fifo_tail.v};
}
__device__ __forceinline__ FrameRing ret_ring(const DevHandle& g) {
  return FrameRing{g.ret, &g.ctrl->ret_head.v, &g.ctrl->ret_tail.v};
}
// Frames in a ring that no pop has drawn yet.
__device__ __forceinline__ unsigned long long ring_size(const FrameRing& q) {  // one thread
  const unsigned long long h = ld_rlx64(q.head), t = ld_rlx64(q.tail);
  return t > h ? t - h : 0;
}

// Store frame f into cell t, a ticket the caller took from the ring's tail
// (another if a pop gave that one up).
static __device__ bool ring_put(const DevHandle& g, const FrameRing& q, unsigned long long t, uint32_t f,
                                unsigned long long deadline) {  // one thread
  __threadfence();  // the frame's state before its entry
  for (;;) {
    unsigned long long* c = &q.cells[t % g.fifo_cap];
    const unsigned long long v = ld_acq64(c), s = v >> FRAME_BITS;
    if (s == t) {  // a CAS: a pop may give this ticket up at the same time
      if (atomicCAS(c, v, ((t + 1) << FRAME_BITS) | f) == v) return true;
      continue;
    }
    if (s > t) {  // given up by a pop
      t = atomicAdd(q.tail, 1ull);
      continue;
    }
    if (now_ns() > deadline) { stat_add(g, ST_TIMEOUTS, 1); return false; }
    __nanosleep(32);
  }
}
static __device__ bool ring_push(const DevHandle& g, const FrameRing& q, uint32_t f,
                                 unsigned long long deadline) {  // one thread
  return ring_put(g, q, atomicAdd(q.tail, 1ull), f, deadline);
}

// The frame of ticket h, drawn by the caller from the ring's head: -1 when the
// ticket was given up (no push held it), -ETIMEDOUT.
static __device__ int ring_take(const DevHandle& g, const FrameRing& q, unsigned long long h,
                                unsigned long long deadline) {  // one thread
  unsigned long long* c = &q.cells[h % g.fifo_cap];
  const unsigned long long gone = ((h + g.fifo_cap) << FRAME_BITS) | MAX_FRAMES;
  for (;;) {
    const unsigned long long v = ld_acq64(c), s = v >> FRAME_BITS;
    if (s == h + 1) {
      st_rel64(c, gone);
      return (int)(v & MAX_FRAMES);
    }
    const bool late = now_ns() > deadline;
    // not pushed: give the ticket up if no push holds it (the ring was empty),
    // or when out of time
    if (s == h && (late || ld_acq64(q.tail) <= h)) {
      if (atomicCAS(c, v, gone) == v) {
        if (!late) return -1;
        stat_add(g, ST_TIMEOUTS, 1);
        return -kETIMEDOUT;
      }
      continue;  // the push landed first
    }
    if (late) { stat_add(g, ST_TIMEOUTS, 1); return -kETIMEDOUT; }
    __nanosleep(32);
  }
}

// Returns a frame, -1 when empty, -ETIMEDOUT.
static __device__ int ring_pop(const DevHandle& g, const FrameRing& q, unsigned long long deadline) {  // one thread
  if (ld_rlx64(q.head) >= ld_rlx64(q.tail)) return -1;
  return ring_take(g, q, atomicAdd(q.head, 1ull), deadline);
}

static __device__ bool fifo_put(const DevHandle& g, unsigned long long t, uint32_t f,
                                unsigned long long deadline) {  // one thread
  return ring_put(g, fifo_ring(g), t, f, deadline);
}
static __device__ bool fifo_push(const DevHandle& g, uint32_t f, unsigned long long deadline) {  // one thread
  return ring_push(g, fifo_ring(g), f, deadline);
}
static __device__ int fifo_take(const DevHandle& g, unsigned long long h, unsigned long long deadline) {  // one thread
  return ring_take(g, fifo_ring(g), h, deadline);
}

// ---------------------------------------------------------------- frames
// Pin frame f for key.  Returns its state, or -1 if the mapping went stale.
static __device__ int frame_pin(const DevHandle& g, int f, unsigned long long key) {  // one thread
  atomicAdd(&g.fpins[f], 1u);
  __threadfence();
  uint32_t st = ld_acq(&g.fstate[f]);
  if (st == FR_RECLAIM || st == FR_EMPTY || ld_rlx64(&g.fkey[f]) != key) {
    atomicSub(&g.fpins[f], 1u);
    return -1;
  }
  return (int)st;
}

static __device__ void frame_unpin(const DevHandle& g, int f) {  // one thread
  __threadfence();
  atomicSub(&g.fpins[f], 1u);
}

// Claim frame f for eviction.  from_fifo: only a still-consumed READY frame or a
// returned (EMPTY, keyless) frame qualifies.  Returns 1 claimed, 0 pinned (try
// later), -1 not a victim (stale entry).
static __device__ int frame_claim(const DevHandle& g, int f, bool from_fifo) {  // one thread
  uint32_t st = ld_acq(&g.fstate[f]);
  if (from_fifo) {
    if (st == FR_READY) {
      if (ld_rlx(&g.fconsumed[f]) < ld_rlx(&g.fvalid[f])) return -1;
    } else if (!(st == FR_EMPTY && ld_rlx64(&g.fkey[f]) == KEY_NONE)) {
      return -1;
    }
  } else if (st != FR_READY && st != FR_ERROR) {
    return -1;
  }
  if (atomicCAS(&g.fstate[f], st, (uint32_t)FR_RECLAIM) != st) return -1;
  __threadfence();
  if (ld_rlx(&g.fpins[f]) != 0u) {
    st_rel(&g.fstate[f], st);
    return 0;
  }
  return 1;
}

// Unmap a claimed frame's old page and record the eviction.
static __device__ void evict_key(const DevHandle& g, int f, unsigned long long new_key, unsigned long long deadline) {
  const int lane = lane_id();
  unsigned long long old = 0;
  uint32_t consumed = 0, valid = 0;
  if (lane == 0) {
    old = ld_rlx64(&g.fkey[f]);
    consumed = ld_rlx(&g.fconsumed[f]);
    valid = ld_rlx(&g.fvalid[f]);
  }
  old = bcast64(old);
  if (old == KEY_NONE) return;
  tab_remove(g, old, (uint32_t)f, deadline);
  if (lane == 0) {
    st_rlx64(&g.fkey[f], KEY_NONE);
    stat_add(g, ST_EVICT, 1);
    if (consumed < valid || valid == 0) stat_add(g, ST_EVICT_UNCONSUMED, 1);
    if (g.trace_cap) {
      unsigned long long i = atomicAdd(&g.ctrl->trace_evict_n.v, 1ull);
      if (i < g.trace_cap) {
        gfs_evict_rec r;
        r.frame = (uint32_t)f;
        r.old_fid = key_fid(old);
        r.new_fid = key_fid(new_key);
        r.reserved = 0;
        r.old_page = key_page(old);
        r.new_page = key_page(new_key);
        g.trace_evict[i] = r;
      }
    }
  }
  __syncwarp();
}

// Warp: unmap the old pages of the n claimed frames[0 .. n) and record the
// evictions, a lane per frame; frame j is about to hold page q0 + j of fid.  The
// eviction records keep frame order (one ticket add per 32 frames), so a run
// records exactly what one evict_key per frame, in order, would.
static __device__ void evict_run(const DevHandle& g, const uint32_t* frames, uint32_t n, uint32_t fid,
                                 unsigned long long q0) {
  const int lane = lane_id();
  for (uint32_t j0 = 0; j0 < n; j0 += 32) {
    const uint32_t j = j0 + (uint32_t)lane;
    unsigned long long old = KEY_NONE;
    uint32_t f = 0, consumed = 0, valid = 0;
    if (j < n) {
      f = frames[j];
      old = ld_rlx64(&g.fkey[f]);
      consumed = ld_rlx(&g.fconsumed[f]);
      valid = ld_rlx(&g.fvalid[f]);
    }
    const bool has = j < n && old != KEY_NONE;
    if (has) {
      lane_tab_remove(g, old, f);
      st_rlx64(&g.fkey[f], KEY_NONE);
    }
    const unsigned hm = __ballot_sync(kFull, has);
    const unsigned um = __ballot_sync(kFull, has && (consumed < valid || valid == 0));
    if (lane == 0) {
      stat_add(g, ST_EVICT, (unsigned long long)__popc(hm));
      stat_add(g, ST_EVICT_UNCONSUMED, (unsigned long long)__popc(um));
    }
    if (g.trace_cap && hm) {
      unsigned long long t0 = 0;
      if (lane == 0) t0 = atomicAdd(&g.ctrl->trace_evict_n.v, (unsigned long long)__popc(hm));
      t0 = bcast64(t0);
      const unsigned long long i = t0 + (unsigned long long)__popc(hm & ((1u << lane) - 1u));
      if (has && i < g.trace_cap) {
        gfs_evict_rec r;
        r.frame = f;
        r.old_fid = key_fid(old);
        r.new_fid = fid;
        r.reserved = 0;
        r.old_page = key_page(old);
        r.new_page = key_page(make_key(fid, q0 + j));
        g.trace_evict[i] = r;
      }
    }
  }
  __syncwarp();
}

// Readahead may only use free / returned / consumed frames above the reserve
// (victim classes 1, 2).
static __device__ bool ra_allowed(const DevHandle& g) {  // one thread
  unsigned long long used = ld_rlx64(&g.ctrl->next_unused.v);
  unsigned long long never = used >= g.n_frames ? 0 : g.n_frames - used;
  return never + ring_size(ret_ring(g)) + ring_size(fifo_ring(g)) > g.reserve;
}

// Victim selection (Section 5.1 restated; classes 1-3).  Returns a frame owned
// by the caller with its old mapping removed, -1 if none (readahead), or a
// negative errno.
static __device__ int take_frame(const DevHandle& g, bool for_ra, unsigned long long seq0, unsigned long long new_key,
                          unsigned long long deadline, bool fallback = true) {
  const int lane = lane_id();
  int r = 0;
  if (for_ra) {
    if (lane == 0) r = ra_allowed(g) ? 1 : 0;
    if (!bcast(r)) return -1;
  }
  // (1) never-used frames, lowest index first
  int f = -1;
  if (lane == 0 && ld_rlx64(&g.ctrl->next_unused.v) < g.n_frames) {
    unsigned long long u = atomicAdd(&g.ctrl->next_unused.v, 1ull);
    if (u < g.n_frames) f = (int)u;
  }
  f = bcast(f);
  if (f >= 0) return f;
  // (1b) frames returned by greads that lost a page to another gread (keyless),
  // then (2) the consumed FIFO, oldest first; a pinned entry goes back to its tail
  for (int which = 0; which < 2; ++which) {
    const FrameRing q = which == 0 ? ret_ring(g) : fifo_ring(g);
    for (uint32_t it = 0; it <= g.fifo_cap; ++it) {
      int c = -1, claimed = -1;
      if (lane == 0) {
        c = ring_pop(g, q, deadline);
        if (c >= 0) {
          claimed = frame_claim(g, c, true);
          if (claimed == 0) ring_push(g, q, (uint32_t)c, deadline);
        }
      }
      c = bcast(c);
      claimed = bcast(claimed);
      if (c == -1) break;
      if (c < 0) return c;
      if (claimed == 1) {
        evict_key(g, c, new_key, deadline);
        return c;
      }
    }
  }
  if (for_ra || !fallback) return -1;
  // (3) only for the page a gread waits for (later pages of a demand run end the
  //     request instead of evicting unconsumed pages): the least recently
  //     allocated unconsumed frame that this gread did not allocate.  A cache of
  //     at most kLraWindow frames, or any cache when greads run one at a time
  //     (exact_lra), is scanned whole.  A larger one is scanned a window of
  //     kLraWindow frames at a time,
  //     from a place that depends on the gread, and the oldest frame of the first
  //     window that has one is taken: concurrent greads then pick different
  //     victims instead of all racing for the single oldest frame.
  const uint32_t W = (g.exact_lra || g.n_frames < kLraWindow) ? g.n_frames : kLraWindow;
  const uint32_t nwin = (g.n_frames + W - 1) / W;
  uint32_t base = 0;
  if (nwin > 1) {
    unsigned long long z = seq0 + 0x9e3779b97f4a7c15ull * (1ull + blockIdx.x);
    z = (z ^ (z >> 31)) * 0xbf58476d1ce4e5b9ull;
    base = (uint32_t)((z ^ (z >> 29)) % g.n_frames);
  }
  const unsigned long long my_seq = seq0 >> kOwnerBits, my_owner = seq0 & kOwnerMask;
  uint32_t empty_windows = 0;
  for (uint32_t attempt = 0; attempt < nwin + 8; ++attempt) {
    const uint32_t start = nwin > 1 ? (uint32_t)((base + (unsigned long long)attempt * W) % g.n_frames) : 0u;
    unsigned long long best = ~0ull;
    int bf = -1;
    for (uint32_t k = lane; k < W; k += 32) {
      uint32_t i = start + k;
      if (i >= g.n_frames) i -= g.n_frames;
      uint32_t st = ld_rlx(&g.fstate[i]);
      if (st != FR_READY && st != FR_ERROR) continue;
      if (ld_rlx(&g.fpins[i]) != 0u) continue;
      unsigned long long a = ld_rlx64(&g.faseq[i]);
      if ((a >> kOwnerBits) >= my_seq && (a & kOwnerMask) == my_owner) continue;  // allocated by this gread
      if (st == FR_READY && ld_rlx(&g.fconsumed[i]) >= ld_rlx(&g.fvalid[i])) continue;  // belongs to the FIFO
      if (a < best) { best = a; bf = (int)i; }
    }
    for (int o = 16; o; o >>= 1) {
      unsigned long long ob = __shfl_xor_sync(kFull, best, o);
      int of = __shfl_xor_sync(kFull, bf, o);
      if (ob < best || (ob == best && of >= 0 && (bf < 0 || of < bf))) { best = ob; bf = of; }
    }
    if (bf < 0) {
      if (++empty_windows >= nwin) return -kENOMEM;  // no candidate anywhere
      continue;
    }
    empty_windows = 0;
    int claimed = 0;
    if (lane == 0) claimed = frame_claim(g, bf, false);
    if (bcast(claimed) == 1) {
      evict_key(g, bf, new_key, deadline);
      return bf;
    }
  }
  return -kEAGAIN;
}

// Give a frame that lost an insert race back, keyless: to the returned-frame ring,
// taken again before any consumed page is evicted, unless it sits in the
// requesting block's own LRA queue (Section 5.1), which reuses it from there (a
// ring entry too would let the queue's reuses push it again and again).
static __device__ void frame_return(const DevHandle& g, int f, bool pinned, bool in_own_queue,
                                    unsigned long long deadline) {  // one thread
  if (pinned) atomicSub(&g.fpins[f], 1u);
  st_rlx64(&g.fkey[f], KEY_NONE);
  st_rel(&g.fstate[f], FR_EMPTY);
  if (!in_own_queue) ring_push(g, ret_ring(g), (uint32_t)f, deadline);
}

// ---------------------------------------------------------------- pull transfer (GFS_XFER_PULL)
// The host preads a request into the slot's staging (mapped pinned memory) and
// publishes a completion record; GPU threads copy each page into its frame over
// the host link.  A page is claimed by CAS FILLING -> COPYING on its frame state,
// so exactly one group copies it; the group that copies a request's last page
// frees the ring slot.
struct PullJob {
  int f;                   // frame to fill, -1 = no job
  uint32_t s, i;           // slot and page index within the request
  uint32_t buf, ok;        // staging buffer holding the page; page complete
  unsigned long long t;    // ticket of the request
  unsigned long long src;  // byte offset of the page in the staging arena
};

__device__ __forceinline__ RingSlot* ring_slot(const DevHandle& g, uint32_t s) {
  return (RingSlot*)(g.ring + (size_t)s * g.slot_stride);
}

__device__ __forceinline__ void pull_read_page(const DevHandle& g, PullJob& j) {
  const PullPage* pp = &g.pages[(size_t)j.s * g.max_rpc_pages + j.i];
  j.src = ld_rlx64((const unsigned long long*)&pp->src);
  j.buf = ld_rlx((const uint32_t*)&pp->buf);
  j.ok = ld_rlx((const uint32_t*)&pp->ok);
}

// One thread: claim frame f if its page has been published.
static __device__ PullJob pull_claim_frame(const DevHandle& g, int f) {
  PullJob j{-1, 0, 0, 0, 0, 0, 0};
  const uint32_t src = ld_acq(&g.fsrc[f]);
  if (src == SRC_NONE) return j;
  const uint32_t s = src / g.max_rpc_pages, i = src % g.max_rpc_pages;
  const unsigned long long t = ld_rlx64(&g.dticket[s]);
  if (ld_acq_sys64(&g.pages[(size_t)s * g.max_rpc_pages + i].tag) != t + 1) return j;
  if (atomicCAS(&g.fstate[f], (uint32_t)FR_FILLING, (uint32_t)FR_COPYING) != FR_FILLING) return j;
  j.f = f;
  j.s = s;
  j.i = i;
  j.t = t;
  pull_read_page(g, j);
  return j;
}

// One warp: find a request with published pages still FILLING and claim one
// page.  A request counts once its first page is published: a host thread
// waiting for one of its staging buffers may be in the middle of the request,
// and only a copy of the pages already published lets it go on.  Scans 32
// slots starting at `start`.
static __device__ PullJob pull_claim_any(const DevHandle& g, uint32_t start) {
  const int lane = lane_id();
  PullJob j{-1, 0, 0, 0, 0, 0, 0};
  const uint32_t s = (start + lane) % g.rpc_slots;
  bool cand = false;
  unsigned long long t = 0;
  if ((uint32_t)lane < g.rpc_slots) {
    t = ld_rlx64(&g.dticket[s]);
    cand = ld_rlx(&g.dcopied[s]) < ld_rlx(&g.dnpages[s]) &&
           ld_acq_sys64(&g.pages[(size_t)s * g.max_rpc_pages].tag) == t + 1;
  }
  unsigned m = __ballot_sync(kFull, cand);
  while (m) {
    const int src = __ffs(m) - 1;
    m &= m - 1;
    const uint32_t ss = (uint32_t)__shfl_sync(kFull, (int)s, src);
    const unsigned long long tt = __shfl_sync(kFull, t, src);
    const uint32_t np = ld_rlx(&g.dnpages[ss]);
    int got = -1;
    for (uint32_t base = 0; base < np && got < 0; base += 32) {
      const uint32_t i = base + lane;
      int f = -1;
      if (i < np) {
        f = (int)ld_rlx(&g.dframes[(size_t)ss * g.max_rpc_pages + i]);
        if (f >= (int)g.n_frames || ld_rlx(&g.fstate[f]) != FR_FILLING ||
            ld_acq(&g.fsrc[f]) != ss * g.max_rpc_pages + i ||
            ld_acq_sys64(&g.pages[(size_t)ss * g.max_rpc_pages + i].tag) != tt + 1)
          f = -1;
      }
      unsigned fm = __ballot_sync(kFull, f >= 0);
      while (fm && got < 0) {
        const int l = __ffs(fm) - 1;
        fm &= fm - 1;
        int ok = 0;
        if (lane == l && atomicCAS(&g.fstate[f], (uint32_t)FR_FILLING, (uint32_t)FR_COPYING) == FR_FILLING) {
          // the slot may have been freed and reused since it was found served:
          // the claim only stands for the request that was checked
          __threadfence();
          ok = ld_rlx64(&g.dticket[ss]) == tt;
          if (!ok) st_rel(&g.fstate[f], (uint32_t)FR_FILLING);
        }
        if (__shfl_sync(kFull, ok, l)) got = (int)(base + l);
      }
      if (got >= 0) {
        j.f = (int)ld_rlx(&g.dframes[(size_t)ss * g.max_rpc_pages + got]);
        j.s = ss;
        j.i = (uint32_t)got;
        j.t = tt;
        pull_read_page(g, j);
      }
    }
    if (got >= 0) break;
  }
  return j;
}

// Copy n bytes of host staging into a frame with `nt` threads (rank `r`).
// Staging is read through L2 (ld.global.cg), never L1: the host rewrites a
// buffer every lap and only L2 is kept coherent with the host over C2C.
__device__ __forceinline__ void copy_in(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, uint32_t n,
                                        uint32_t r, uint32_t nt) {
  const uint32_t n16 = n >> 4;
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
  uint4* d4 = reinterpret_cast<uint4*>(dst);
  uint32_t i = r;
  for (; i + 7 * nt < n16; i += 8 * nt) {
    uint4 v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = __ldcg(s4 + i + u * nt);
#pragma unroll
    for (int u = 0; u < 8; ++u) d4[i + u * nt] = v[u];
  }
  for (; i < n16; i += nt) d4[i] = __ldcg(s4 + i);
  for (uint32_t b = 16 * n16 + r; b < n; b += nt) dst[b] = __ldcg(src + b);
}

// Copy a claimed page (all `nt` threads of the group), without the completion.
__device__ __forceinline__ bool pull_copy(const DevHandle& g, const PullJob& j, uint32_t r, uint32_t nt) {
  const uint32_t valid = ld_rlx(&g.fvalid[j.f]);
  const bool ok = j.ok != 0;
  if (ok) {
    const uint8_t* src = j.buf == BUF_MAPPED ? (const uint8_t*)j.src : g.staging + j.src;
    copy_in(src, g.frames + ((size_t)j.f << g.page_shift), valid, r, nt);
  }
  __threadfence();
  return ok;
}

// One thread, after the group's copy: publish the page, give the staging buffer
// back to its host thread, and free the slot after the request's last page.
__device__ __forceinline__ void pull_finish(const DevHandle& g, const PullJob& j, bool ok) {
  st_rlx(&g.fsrc[j.f], SRC_NONE);
  st_rel(&g.fstate[j.f], ok ? (uint32_t)FR_READY : (uint32_t)FR_ERROR);
  if (j.buf != BUF_MAPPED) {
    __threadfence_system();
    atomicAdd_system(&g.bcount[j.buf], 0xffffffffu);  // -1: the host may reuse the buffer once 0
  }
  // the page count is read while this page's claim still keeps the slot from
  // being freed: after the increment a later request may own the slot
  const uint32_t np = ld_rlx(&g.dnpages[j.s]);
  const uint32_t c = atomicAdd(&g.dcopied[j.s], 1u) + 1;
  if (c == np) {
    __threadfence_system();
    st_rel_sys64(&ring_slot(g, j.s)->seq, j.t + g.rpc_slots);
    st_rel64(&g.slot_free[j.s], j.t + g.rpc_slots);
    atomicAdd(&g.ctrl->freed.v, 1ull);
  }
}

// One warp: help with one served page.  Returns true if it copied one.
static __device__ bool warp_help(const DevHandle& g, uint32_t start) {
  PullJob j = pull_claim_any(g, start);
  if (j.f < 0) return false;
  bool ok = pull_copy(g, j, (uint32_t)lane_id(), 32);
  __syncwarp();
  if (lane_id() == 0) pull_finish(g, j, ok);
  __syncwarp();
  return true;
}

// One warp, after claiming page j.i of request (j.s, ticket j.t): claim up to
// `want` more published pages of the same request (their frames FILLING ->
// COPYING, as one claim each).  Claimed pages go to out[0 .. count).
static __device__ int pull_claim_more(const DevHandle& g, const PullJob& j, int want, PullJob* out) {
  const int lane = lane_id();
  const uint32_t np = ld_rlx(&g.dnpages[j.s]);
  int got = 0;
  for (uint32_t base = 0; base < np && got < want; base += 32) {
    const uint32_t i = base + (uint32_t)lane;
    int f = -1;
    if (i < np && i != j.i) {
      f = (int)ld_rlx(&g.dframes[(size_t)j.s * g.max_rpc_pages + i]);
      if (f >= (int)g.n_frames || ld_rlx(&g.fstate[f]) != FR_FILLING ||
          ld_acq(&g.fsrc[f]) != j.s * g.max_rpc_pages + i ||
          ld_acq_sys64(&g.pages[(size_t)j.s * g.max_rpc_pages + i].tag) != j.t + 1)
        f = -1;
    }
    const unsigned cm = __ballot_sync(kFull, f >= 0);
    const int rank = __popc(cm & ((1u << lane) - 1u));
    bool mine = false;
    if (f >= 0 && rank < want - got &&
        atomicCAS(&g.fstate[f], (uint32_t)FR_FILLING, (uint32_t)FR_COPYING) == FR_FILLING) {
      __threadfence();
      mine = ld_rlx64(&g.dticket[j.s]) == j.t;  // the claim stands for the request that was checked
      if (!mine) st_rel(&g.fstate[f], (uint32_t)FR_FILLING);
    }
    const unsigned mm = __ballot_sync(kFull, mine);
    if (mine) {
      PullJob k{f, j.s, i, 0, 0, j.t, 0};
      pull_read_page(g, k);
      out[got + __popc(mm & ((1u << lane) - 1u))] = k;
    }
    got += __popc(mm);
  }
  return got;
}

// Pages of one request a helping block copies in one pass: small pages are
// copied a warp per page, many at once, so their claim, descriptor and copy
// round trips overlap; large pages keep one page per pass, the whole block on it.
__device__ __forceinline__ int help_batch(const DevHandle& g) {
  if (g.page_size <= (16u << 10)) return 32;
  if (g.page_size <= (64u << 10)) return 4;
  return 1;
}

// Whole block: copy frame f if served (target >= 0), else help with any served
// page; with small pages, also further served pages of the same request.
// Returns true if the block copied a page.  Block-uniform.
static __device__ bool block_help(const DevHandle& g, int target, bool any) {
  __shared__ PullJob s_job;
  __shared__ PullJob s_more[31];
  __shared__ int s_nmore;
  __shared__ uint32_t s_ok[32];
  const uint32_t tid = threadIdx.x;
  const int batch = help_batch(g);
  if (tid < 32) {
    PullJob j{-1, 0, 0, 0, 0, 0, 0};
    if (target >= 0 && tid == 0) j = pull_claim_frame(g, target);
    j.f = bcast(j.f);
    if (j.f < 0 && any) {
      const uint32_t start = (uint32_t)((blockIdx.x * 37u + (uint32_t)(now_ns() >> 10)) % g.rpc_slots);
      j = pull_claim_any(g, start);
    }
    int nmore = 0;
    if (j.f >= 0 && batch > 1) {
      // every lane needs the claimed job (lane 0 or the claiming lane filled it)
      PullJob b;
      b.f = __shfl_sync(kFull, j.f, 0);
      b.s = __shfl_sync(kFull, j.s, 0);
      b.i = __shfl_sync(kFull, j.i, 0);
      b.t = __shfl_sync(kFull, j.t, 0);
      b.buf = 0;
      b.ok = 0;
      b.src = 0;
      nmore = pull_claim_more(g, b, batch - 1, s_more);
    }
    if (tid == 0) {
      s_job = j;
      s_nmore = nmore;
    }
  }
  __syncthreads();
  const PullJob j = s_job;
  const int nmore = s_nmore;
  __syncthreads();
  if (j.f < 0) return false;
  if (nmore == 0) {
    const bool ok = pull_copy(g, j, tid, blockDim.x);
    __syncthreads();
    if (tid == 0) pull_finish(g, j, ok);
    return true;
  }
  const uint32_t nw = blockDim.x >> 5, w = tid >> 5, lane = tid & 31u;
  if (g.page_size <= (16u << 10)) {  // a warp per page
    for (int k = (int)w; k <= nmore; k += (int)nw) {
      const PullJob jk = k == 0 ? j : s_more[k - 1];
      const bool ok = pull_copy(g, jk, lane, 32);
      if (lane == 0) s_ok[k] = ok ? 1u : 0u;
    }
  } else {  // the whole block on each page in turn
    for (int k = 0; k <= nmore; ++k) {
      const PullJob jk = k == 0 ? j : s_more[k - 1];
      const bool ok = pull_copy(g, jk, tid, blockDim.x);
      if (tid == 0) s_ok[k] = ok ? 1u : 0u;
    }
  }
  __syncthreads();
  if (tid <= (uint32_t)nmore) pull_finish(g, tid == 0 ? j : s_more[tid - 1], s_ok[tid] != 0u);
  return true;
}

// ---------------------------------------------------------------- request ring
// Take the next ticket of the ring and wait until its slot is free for this
// lap (one warp).  GFS_QUEUE_SHARED: the next ticket of ring_tail.
// GFS_QUEUE_STATIC (Section 3.2): the threadblock's own slot, numbered by its
// lap counter (ring_tail then only counts requests).  In the GPU copy transfers
// the GPU frees slots itself and keeps a device copy of the ticket each is free
// for, read before the ring word in host memory.  Returns 0 with *t and *si set;
// a wait that runs out posts the ticket's cancellation for the host and returns
// -ETIMEDOUT.
static __device__ int ring_acquire(const DevHandle& g, unsigned long long* t_out, uint32_t* si_out,
                                   unsigned long long deadline) {
  const int lane = lane_id();
  unsigned long long t = 0;
  if (lane == 0) {
    const unsigned long long k = atomicAdd(&g.ctrl->ring_tail.v, 1ull);  // requests issued (drain counts them)
    if (g.queue == GFS_QUEUE_STATIC) {
      const uint32_t slot = blockIdx.x % g.rpc_slots;
      t = atomicAdd(&g.slot_lap[slot], 1ull) * g.rpc_slots + slot;
    } else {
      t = k;
    }
  }
  t = bcast64(t);
  const uint32_t si = (uint32_t)(t % g.rpc_slots);
  RingSlot* s = ring_slot(g, si);
  *t_out = t;
  *si_out = si;
  for (unsigned ns = 64;;) {
    int free_ = 0, late = 0;
    if (lane == 0) {
      free_ = (g.xfer != GFS_XFER_DMA && ld_acq64(&g.slot_free[si]) == t) || ld_acq_sys64(&s->seq) == t;
      if (!free_ && now_ns() > deadline) {
        late = 1;
        st_rel_sys64(&g.cancel[t % g.cancel_n], t + 1);  // the host consumer of ticket t skips it
        stat_add(g, ST_TIMEOUTS, 1);
      }
    }
    if (bcast(free_)) return 0;
    if (bcast(late)) return -kETIMEDOUT;
    // in the GPU copy transfers slots are freed by GPU copies: help instead of idling
    if (g.xfer != GFS_XFER_DMA && warp_help(g, si)) continue;
    if (lane == 0) __nanosleep(ns);
    __syncwarp();
    if (ns < 2048) ns <<= 1;
  }
}

// Count a request and record it in the RPC trace (one thread).
static __device__ void rpc_record(const DevHandle& g, uint32_t fid, unsigned long long page_lo, uint32_t n,
                                  uint32_t kind) {
  stat_add(g, ST_RPCS, 1);
  if (g.trace_cap) {
    unsigned long long i = atomicAdd(&g.ctrl->trace_rpc_n.v, 1ull);
    if (i < g.trace_cap) {
      gfs_rpc_rec r;
      r.fid = fid;
      r.kind = kind;
      r.npages = n;
      r.reserved = 0;
      r.page_lo = page_lo;
      g.trace_rpc[i] = r;
    }
  }
}

// ---------------------------------------------------------------- requests the GPU serves itself
// With GFS_XFER_MAPPED a mapped file's pages sit in host memory the GPU reads,
// at dev_map + page * P: serving a request needs no host read and no host
// thread, only the copy.  The block that makes such a request copies its pages
// into their frames right after warp 0 has installed them (block_self_serve);
// readers of those pages meanwhile wait on the frames' state words, as for any
// page being filled.  At most one such request is pending per block.
struct SelfJob {
  unsigned long long page_lo;
  uint32_t n;
};
__device__ __forceinline__ SelfJob& self_job() {
  __shared__ SelfJob j;
  return j;
}

static __device__ int rpc_submit(const DevHandle& g, uint32_t fid, unsigned long long page_lo, uint32_t n, uint32_t kind,
                          const uint32_t* s_frames, unsigned long long deadline, unsigned long long* ticket_out = nullptr) {
  const int lane = lane_id();
  unsigned long long t = 0;
  uint32_t si = 0;
  const int arc = ring_acquire(g, &t, &si, deadline);
  if (arc) return arc;
  RingSlot* s = ring_slot(g, si);
  if (g.xfer != GFS_XFER_DMA && !s_frames) {  // paper mode: the requesting block copies every page itself
    if (lane == 0) {
      st_rlx64(&g.dticket[si], t);
      st_rlx(&g.dnpages[si], 0u);  // helpers skip it
      st_rlx(&g.dcopied[si], 0u);
    }
    __syncwarp();
    __threadfence();
    __syncwarp();
  } else if (g.xfer != GFS_XFER_DMA) {
    for (uint32_t i = lane; i < n; i += 32) g.dframes[(size_t)si * g.max_rpc_pages + i] = s_frames[i];
    if (lane == 0) {
      st_rlx64(&g.dticket[si], t);
      st_rlx(&g.dnpages[si], n);
      st_rlx(&g.dcopied[si], 0u);
    }
    __syncwarp();
    __threadfence();
    __syncwarp();
    for (uint32_t i = lane; i < n; i += 32) st_rel(&g.fsrc[s_frames[i]], si * g.max_rpc_pages + i);
  } else {
    for (uint32_t i = lane; i < n; i += 32) st_sys32(&s->frames[i], s_frames[i]);
  }
  if (lane == 0) {
    st_sys32(&s->fid, fid);
    st_sys32(&s->npages, n);
    st_sys64(&s->page_lo, page_lo);
    st_sys32(&s->kind, kind);
    st_sys32(&s->op, OP_READ);
    st_sys64(&s->issue_ns, now_ns());
  }
  __syncwarp();
  __threadfence_system();
  __syncwarp();
  if (ticket_out) *ticket_out = t;
  if (lane == 0) {
    st_rel_sys64(&s->seq, t + 1);
    rpc_record(g, fid, page_lo, n, kind);
  }
  __syncwarp();
  return 0;
}

// Warp: frames for pages 1 .. L of a request (page i of the request is a
// readahead page when i >= demand), victim classes 1 and 2 only, taken in page
// order into s_frames[1 ..] exactly as one take_frame per page would take them:
// never-used frames first (one fetch-and-add for the run), then returned frames,
// then the consumed FIFO (one ticket add per round).  A readahead page needs
// never + returned + consumed > reserve at its turn, and every page before it in
// the run has taken one frame since page 0 did.  Returns how many pages, from page 1 on, got a frame; claimed victims
// still hold their old keys.
static __device__ uint32_t take_run(const DevHandle& g, uint32_t L, uint32_t demand, unsigned long long deadline,
                                    uint32_t* s_frames) {
  const int lane = lane_id();
  const uint32_t first_ra = demand > 1 ? demand : 1u;
  if (L >= first_ra) {  // ra_allowed at page i: N0 - (i - 1) > reserve, i.e. i <= N0 - reserve
    long long lim = 0;
    if (lane == 0) {
      const unsigned long long used = ld_rlx64(&g.ctrl->next_unused.v);
      const unsigned long long never = used >= g.n_frames ? 0 : g.n_frames - used;
      lim = (long long)(never + ring_size(ret_ring(g)) + ring_size(fifo_ring(g))) - (long long)g.reserve;
    }
    lim = (long long)bcast64((unsigned long long)lim);
    const long long last = lim > (long long)first_ra - 1 ? lim : (long long)first_ra - 1;
    if ((long long)L > last) L = (uint32_t)last;
  }
  if (L == 0) return 0;
  // class 1: never-used frames, lowest index first
  unsigned long long u0 = 0;
  uint32_t got = 0;
  if (lane == 0 && ld_rlx64(&g.ctrl->next_unused.v) < g.n_frames) {
    u0 = atomicAdd(&g.ctrl->next_unused.v, (unsigned long long)L);
    if (u0 < g.n_frames) got = g.n_frames - u0 < L ? (uint32_t)(g.n_frames - u0) : L;
  }
  got = (uint32_t)bcast((int)got);
  u0 = bcast64(u0);
  for (uint32_t j = lane; j < got; j += 32) s_frames[1 + j] = (uint32_t)(u0 + j);
  // class 1b: returned (keyless) frames, then class 2: the consumed FIFO, oldest
  // first; a pinned entry goes back to its ring's tail
  for (int which = 0; which < 2 && got < L; ++which) {
    const FrameRing q = which == 0 ? ret_ring(g) : fifo_ring(g);
    for (uint32_t round = 0; got < L && round < 8; ++round) {
      unsigned long long h0 = 0;
      uint32_t take = 0;
      if (lane == 0) {
        const unsigned long long avail = ring_size(q);
        take = avail < L - got ? (uint32_t)avail : L - got;
        if (take) h0 = atomicAdd(q.head, (unsigned long long)take);
      }
      take = (uint32_t)bcast((int)take);
      h0 = bcast64(h0);
      if (take == 0) break;
      for (uint32_t j0 = 0; j0 < take; j0 += 32) {
        int c = -1, claimed = -1;
        if (j0 + lane < take) {
          c = ring_take(g, q, h0 + j0 + lane, deadline);
          if (c >= 0) {
            claimed = frame_claim(g, c, true);
            if (claimed == 0) ring_push(g, q, (uint32_t)c, deadline);
          }
        }
        const unsigned m = __ballot_sync(kFull, claimed == 1);
        if (claimed == 1) s_frames[1 + got + __popc(m & ((1u << lane) - 1u))] = (uint32_t)c;
        got += (uint32_t)__popc(m);
      }
    }
  }
  __syncwarp();
  return got;
}

static __device__ int finish_request(const DevHandle& g, uint32_t fid, const FileDev& fi, unsigned long long p,
                                     uint32_t n, uint32_t demand, uint32_t window, uint32_t kind,
                                     unsigned long long mark_end, int mark_idx, const uint32_t* s_frames,
                                     unsigned long long deadline, bool allow_self);

static __device__ uint32_t take_run_lra(const DevHandle& g, int stream, uint32_t L, uint32_t* s_frames);

// Whether the frames of `stream`'s requests come from its own LRA queue (Section 5.1).
__device__ __forceinline__ bool own_queue(const DevHandle& g, int stream) {
  return g.repl == GFS_REPL_TB_LRA && stream >= 0 && (uint32_t)stream < g.paper_streams;
}

// Warp: pages 1 .. of a request whose page 0 is installed (page i is p + i, a
// readahead page when i >= demand).  The run is cut, as one page at a time would
// cut it, at EOF, at the first page already in the table and at the first
// readahead page fetched since the last reset (R8), then by take_run.  Victims
// lose their old pages in page order, metadata is written a lane per page (one
// sequence-number add), and the table entries go in in page order.  Frames come
// from take_run, or from the stream's own LRA queue (take_run_lra).  Returns how
// many pages from page 1 on were installed; their frames are in s_frames[1 ..].
static __device__ uint32_t install_run(const DevHandle& g, int stream, uint32_t fid, const FileDev& fi,
                                       unsigned long long p, uint32_t want, uint32_t demand, unsigned long long seq0,
                                       unsigned long long deadline, uint32_t* s_frames) {
  const int lane = lane_id();
  unsigned long long lim = want - 1ull;
  if (p + 1 + lim > fi.npages) lim = fi.npages > p + 1 ? fi.npages - p - 1 : 0;
  // pages 1 .. demand-1 are the demand run that R2 just found absent (a page
  // another gread maps meanwhile is caught by its insert below)
  uint32_t L = demand > 1 ? (demand - 1 < lim ? demand - 1 : (uint32_t)lim) : 0u;
  while (L < lim) {
    const uint32_t k = lim - L < 32ull ? (uint32_t)(lim - L) : 32u;
    const uint32_t a = absent_prefix(g, fid, p + 1 + L, k);
    L += a;
    if (a < k) break;
  }
  if (fi.fetched) {  // R8
    for (uint32_t i0 = demand > 1 ? demand : 1u; i0 <= L; i0 += 32) {
      const uint32_t i = i0 + (uint32_t)lane;
      const unsigned long long q = p + i;
      const bool done = i <= L && ((ld_rlx(&fi.fetched[q >> 5]) >> (q & 31)) & 1u);
      const unsigned m = __ballot_sync(kFull, done);
      if (m) {
        L = i0 + (uint32_t)__ffs(m) - 2;
        break;
      }
    }
  }
  L = own_queue(g, stream) ? take_run_lra(g, stream, L, s_frames) : take_run(g, L, demand, deadline, s_frames);
  if (L == 0) return 0;
  evict_run(g, s_frames + 1, L, fid, p + 1);
  unsigned long long a0 = 0;
  if (lane == 0) a0 = atomicAdd(&g.ctrl->alloc_counter.v, (unsigned long long)L);
  a0 = bcast64(a0);
  for (uint32_t j = 1 + (uint32_t)lane; j <= L; j += 32) {  // metadata first, then FILLING, then the table
    const uint32_t f = s_frames[j];
    const unsigned long long q = p + j;
    st_rlx64(&g.fkey[f], make_key(fid, q));
    st_rlx(&g.fconsumed[f], 0u);
    st_rlx(&g.fwindow[f], 0u);
    st_rlx(&g.fmark[f], 0u);
    st_rlx(&g.fvalid[f], expected_valid(g, fi, q));
    st_rlx64(&g.faseq[f], ((a0 + j - 1) << kOwnerBits) | (seq0 & kOwnerMask));
    if (g.fsrc) st_rlx(&g.fsrc[f], SRC_NONE);
  }
  __threadfence();
  for (uint32_t j = 1 + (uint32_t)lane; j <= L; j += 32) st_rel(&g.fstate[s_frames[j]], FR_FILLING);
  __syncwarp();
  // the table entries, a lane per page; a page another gread mapped meanwhile
  // (its insert finds the key) cuts the request there and its frame goes back
  uint32_t cut = L + 1;  // the first page, from 1 on, whose insert failed
  for (uint32_t j0 = 1; j0 <= L; j0 += 32) {
    const uint32_t j = j0 + (uint32_t)lane;
    bool ok = true;
    if (j <= L) {
      const uint32_t f = s_frames[j];
      ok = lane_tab_insert(g, make_key(fid, p + j), f, deadline) == (int)f;
      if (!ok) frame_return(g, (int)f, false, own_queue(g, stream), deadline);  // never reachable: not in the table
      else {
        const unsigned long long q = p + j;
        if (fi.fetched) atomicOr(&fi.fetched[q >> 5], 1u << (q & 31));
        if (g.fetch_count && fid == 0 && q < g.debug_pages) atomicAdd(&g.fetch_count[q], 1u);
      }
    }
    const unsigned bad = __ballot_sync(kFull, !ok);
    if (bad && cut > L) cut = j0 + (uint32_t)(__ffs(bad) - 1);
    if (j <= L && !ok) s_frames[j] |= 0x80000000u;  // marks the page as not mapped
  }
  __syncwarp();
  if (cut <= L) {
    if (lane == 0) stat_add(g, ST_RUN_CUTS, 1);
    // Pages after the cut that did go into the table are mapped and FILLING:
    // readers may already wait for them, so each maximal run of them is requested
    // on its own (only concurrent greads race like this; one gread at a time never does).
    uint32_t a = cut + 1;
    while (a <= L) {
      if (s_frames[a] & 0x80000000u) {
        ++a;
        continue;
      }
      uint32_t e = a;
      while (e + 1 <= L && !(s_frames[e + 1] & 0x80000000u)) ++e;
      const uint32_t n = e - a + 1;
      const uint32_t kind = a < demand ? (uint32_t)GFS_KIND_DEMAND
                                       : (demand == 0 ? (uint32_t)GFS_KIND_ASYNC_RA : (uint32_t)GFS_KIND_SYNC_RA);
      finish_request(g, fid, fi, p + a, n, a < demand ? demand - a : 0u, n, kind, 0, -1, s_frames + a, deadline,
                     false);
      a = e + 1;
    }
    L = cut - 1;
  }
  return L;
}

// Allocate and install frames for [p, p + want): the first `demand` pages are
// demand pages, the rest readahead.  Cut at EOF, at the first present page and
// when no readahead victim is allowed.  Frames go to s_frames; the first is
// pinned when pin_first.  Returns the page count, -EAGAIN when page p was
// inserted by someone else meanwhile, or a negative errno.
static __device__ int take_frame_lra(const DevHandle& g, int stream, bool for_ra, unsigned long long seq0,
                                     unsigned long long new_key, unsigned long long deadline);

// A frame for a request of `stream`: with GFS_REPL_TB_LRA from the stream's own
// queue (Section 5.1), else by victim classes 1-3 (class 3 only for the page the
// gread waits for, `awaited`).
static __device__ int take_for(const DevHandle& g, int stream, bool for_ra, bool awaited, unsigned long long seq0,
                               unsigned long long new_key, unsigned long long deadline) {
  if (own_queue(g, stream)) return take_frame_lra(g, stream, for_ra, seq0, new_key, deadline);
  return take_frame(g, for_ra, seq0, new_key, deadline, awaited);
}

static __device__ int request_range(const DevHandle& g, int stream, uint32_t fid, const FileDev& fi,
                                    unsigned long long p, uint32_t want,
                             uint32_t demand, bool pin_first, unsigned long long seq0, unsigned long long deadline,
                             uint32_t* s_frames) {
  const int lane = lane_id();
  if (want > g.max_rpc_pages) want = g.max_rpc_pages;
  uint32_t n = 0;
  for (uint32_t i = 0; i < want; ++i) {
    // the pages after the first are taken and installed as one run
    if (i == 1) return 1 + (int)install_run(g, stream, fid, fi, p, want, demand, seq0, deadline, s_frames);
    const unsigned long long q = p + i;
    if (q >= fi.npages) break;
    const unsigned long long key = make_key(fid, q);
    if (i > 0 && tab_lookup(g, key) >= 0) break;
    const bool is_ra = i >= demand;
    // R8: readahead does not fetch a page again once fetched (sequential data is used once)
    if (is_ra && fi.fetched && (ld_rlx(&fi.fetched[q >> 5]) >> (q & 31)) & 1u) break;
    int f = take_for(g, stream, is_ra, i == 0, seq0, key, deadline);
    while (f < 0 && !is_ra && i == 0) {  // the first demand page waits for a victim
      int late = 0;
      if (lane == 0) late = now_ns() > deadline;
      if (bcast(late)) {
        if (lane == 0) stat_add(g, ST_ENOMEM, 1);
        return -kENOMEM;
      }
      // pull mode: frames may all be waiting to be copied out of staging
      if (!(g.xfer != GFS_XFER_DMA && warp_help(g, (uint32_t)(q % g.rpc_slots)))) {
        if (lane == 0) __nanosleep(256);
        __syncwarp();
      }
      f = take_for(g, stream, false, true, seq0, key, deadline);
    }
    if (f < 0) break;
    const bool pin = pin_first && i == 0;
    if (lane == 0) {  // install: metadata first, then FILLING, then the table entry
      st_rlx64(&g.fkey[f], key);
      st_rlx(&g.fconsumed[f], 0u);
      st_rlx(&g.fwindow[f], 0u);
      st_rlx(&g.fmark[f], 0u);
      st_rlx(&g.fvalid[f], expected_valid(g, fi, q));
      st_rlx64(&g.faseq[f], (atomicAdd(&g.ctrl->alloc_counter.v, 1ull) << kOwnerBits) | (seq0 & kOwnerMask));
      if (g.fsrc) st_rlx(&g.fsrc[f], SRC_NONE);
      __threadfence();
      if (pin) atomicAdd(&g.fpins[f], 1u);
      st_rel(&g.fstate[f], FR_FILLING);
    }
    __syncwarp();
    int r = tab_insert(g, key, (uint32_t)f, deadline);
    if (r != f) {
      if (lane == 0) frame_return(g, f, pin, own_queue(g, stream), deadline);
      __syncwarp();
      if (i == 0) return r < 0 ? r : -kEAGAIN;
      break;
    }
    if (lane == 0) {
      s_frames[n] = (uint32_t)f;
      if (fi.fetched) atomicOr(&fi.fetched[q >> 5], 1u << (q & 31));
      if (g.fetch_count && fid == 0 && q < g.debug_pages) atomicAdd(&g.fetch_count[q], 1u);
    }
    __syncwarp();
    ++n;
  }
  return (int)n;
}

// Finish a request: record windows and the readahead mark, send it (or, with
// allow_self, leave it to the requesting block when the file is mapped and no
// other such request is pending: its frame list must stay in s_frames until the
// block copies it), count it.
static __device__ int finish_request(const DevHandle& g, uint32_t fid, const FileDev& fi, unsigned long long p, uint32_t n,
                              uint32_t demand, uint32_t window, uint32_t kind, unsigned long long mark_end,
                              int mark_idx, const uint32_t* s_frames, unsigned long long deadline, bool allow_self) {
  const int lane = lane_id();
  for (uint32_t i = lane; i < n; i += 32) st_rlx(&g.fwindow[s_frames[i]], window);
  if (lane == 0) {
    if (mark_idx >= 0) st_rlx(&g.fmark[s_frames[mark_idx]], (uint32_t)(mark_end + 1));
    unsigned long long bytes = 0;
    for (uint32_t i = 0; i < n; ++i) bytes += expected_valid(g, fi, p + i);
    stat_add(g, ST_PAGES, n);
    stat_add(g, ST_BYTES, bytes);
    if (kind == GFS_KIND_SYNC_RA) stat_add(g, ST_RA_SYNC, n - demand);
    if (kind == GFS_KIND_ASYNC_RA) stat_add(g, ST_RA_ASYNC, n);
    __threadfence();
  }
  __syncwarp();
  int self = 0;
  if (lane == 0 && allow_self && g.self_serve && fi.dev_map && self_job().n == 0) {
    self_job().page_lo = p;
    self_job().n = n;
    rpc_record(g, fid, p, n, kind);
    self = 1;
  }
  if (bcast(self)) return 0;
  return rpc_submit(g, fid, p, n, kind, s_frames, deadline);
}

// Whole block: copy the pages of the pending self-served request (frames in
// frames[0 .. n), pages page_lo ..) from the file's mapping into their frames and
// publish them READY.  No-op when none is pending.  Block-uniform.
static __device__ void block_self_serve(const DevHandle& g, const FileDev& fi, const uint32_t* frames) {
  SelfJob& j = self_job();
  const uint32_t n = j.n;
  if (n == 0) return;
  const unsigned long long p0 = j.page_lo;
  const uint32_t tid = threadIdx.x, nt = blockDim.x;
  if (g.page_size <= (16u << 10)) {  // small pages: a warp per page, many in flight
    const uint32_t w = tid >> 5, nw = nt >> 5, lane = tid & 31u;
    for (uint32_t i = w; i < n; i += nw) {
      const uint32_t f = frames[i];
      copy_in((const uint8_t*)(fi.dev_map + ((p0 + i) << g.page_shift)), g.frames + ((size_t)f << g.page_shift),
              ld_rlx(&g.fvalid[f]), lane, 32);
    }
  } else {
    for (uint32_t i = 0; i < n; ++i) {
      const uint32_t f = frames[i];
      copy_in((const uint8_t*)(fi.dev_map + ((p0 + i) << g.page_shift)), g.frames + ((size_t)f << g.page_shift),
              ld_rlx(&g.fvalid[f]), tid, nt);
    }
  }
  __threadfence();
  __syncthreads();
  for (uint32_t i = tid; i < n; i += nt) st_rel(&g.fstate[frames[i]], FR_READY);
  __syncthreads();
  if (tid == 0) j.n = 0;
  __syncthreads();
}

// R4: asynchronous readahead of [end, end + min(Wmax, 2T)) from a readahead mark.
static __device__ void async_readahead(const DevHandle& g, int stream, uint32_t fid, const FileDev& fi,
                                       unsigned long long end, uint32_t t, unsigned long long seq0,
                                       unsigned long long deadline, uint32_t* s_frames) {
  if (end >= fi.npages) return;
  if (fi.fetched && (ld_rlx(&fi.fetched[end >> 5]) >> (end & 31)) & 1u) return;  // R8
  if (tab_lookup(g, make_key(fid, end)) >= 0) return;
  uint32_t want = 2 * t < g.ra_cap ? 2 * t : g.ra_cap;
  if (want == 0) return;
  int n = request_range(g, stream, fid, fi, end, want, 0, false, seq0, deadline, s_frames);
  if (n <= 0) return;
  finish_request(g, fid, fi, end, (uint32_t)n, 0, (uint32_t)n, GFS_KIND_ASYNC_RA, end + (uint32_t)n, 0, s_frames,
                 deadline, true);
}

// R1-R3: a miss on page p (p1 = last page of the gread).  Returns the pinned,
// FILLING frame of page p, -EAGAIN to look p up again, or a negative errno.
static __device__ int handle_miss(const DevHandle& g, int stream, uint32_t fid, const FileDev& fi, unsigned long long p,
                           unsigned long long p1, unsigned long long seq0, unsigned long long deadline,
                           uint32_t* s_frames) {
  const int lane = lane_id();
  if (lane == 0) stat_add(g, ST_MISSES, 1);
  const bool ra = g.mode == GFS_MODE_READAHEAD && fi.ra;
  uint32_t d = 1, T = 1;
  bool seq = false;
  if (ra) {
    // R2: the demand run is p and the absent pages after it, within the gread and a request
    const unsigned long long cap = p1 - p < g.max_rpc_pages - 1ull ? p1 - p : g.max_rpc_pages - 1ull;
    while (d - 1 < cap) {
      const uint32_t k = cap - (d - 1) < 32ull ? (uint32_t)(cap - (d - 1)) : 32u;
      const uint32_t a = absent_prefix(g, fid, p + d, k);
      d += a;
      if (a < k) break;
    }
    int prev = -1;
    seq = p == 0;                                                                              // R3
    if (!seq) {
      prev = tab_lookup(g, make_key(fid, p - 1));
      seq = prev >= 0;
    }
    if (!seq && stream >= 0 && (uint32_t)stream < g.max_streams) {
      unsigned long long le = 0;
      if (lane == 0) le = ld_rlx64(&g.last_end[(size_t)stream * g.max_files + fid]);
      seq = bcast64(le) == p + 1;  // stored as end page + 1
    }
    if (!seq) {
      T = d;
    } else {
      uint32_t tprev = 0;
      if (prev >= 0 && lane == 0) tprev = ld_rlx(&g.fwindow[prev]);
      tprev = (uint32_t)bcast((int)tprev);
      uint32_t grow = 4 * d > 2 * tprev ? 4 * d : 2 * tprev;
      T = d + g.ra_cap < grow ? d + g.ra_cap : grow;
    }
    if (T > g.max_rpc_pages) T = g.max_rpc_pages;
    if (d > T) d = T;
  }
  int n = request_range(g, stream, fid, fi, p, T, d, true, seq0, deadline, s_frames);
  if (n < 0) return n;
  const uint32_t kind = (uint32_t)n > d ? GFS_KIND_SYNC_RA : GFS_KIND_DEMAND;
  const uint32_t window = (ra && seq) ? (uint32_t)n : 0u;
  const int mark_idx = (uint32_t)n > d ? (int)d : -1;
  int f0 = 0;
  if (lane == 0) f0 = (int)s_frames[0];
  f0 = bcast(f0);
  int r = finish_request(g, fid, fi, p, (uint32_t)n, d, window, kind, p + (uint32_t)n, mark_idx, s_frames, deadline,
                         true);
  if (r < 0) {
    if (lane == 0) frame_unpin(g, f0);
    return r;
  }
  return f0;
}

// ---------------------------------------------------------------- paper mode (Sections 4.1, 5.1)
enum : int { PJ_NONE = 0, PJ_BUFFER = 1, PJ_REQUEST = 2 };
struct PaperJob {
  int kind;
  int f;
  uint32_t slot, n;
  unsigned long long t, page, src;
};

// Claim a frame this stream owns for reuse (one thread).  1 claimed, 0 busy, -1 not reusable.
static __device__ int frame_claim_own(const DevHandle& g, int f) {
  const uint32_t st = ld_acq(&g.fstate[f]);
  if (!(st == FR_READY || st == FR_ERROR || (st == FR_EMPTY && ld_rlx64(&g.fkey[f]) == KEY_NONE))) return 0;
  if (atomicCAS(&g.fstate[f], st, (uint32_t)FR_RECLAIM) != st) return 0;
  __threadfence();
  if (ld_rlx(&g.fpins[f]) != 0u) {
    st_rel(&g.fstate[f], st);
    return 0;
  }
  return 1;
}

// Section 5.1: the stream's least-recently-allocated queue (warp).  Below the
// quota a never-used frame joins it; otherwise its frames are tried oldest
// first: the first one not in use (pinned, being filled, or in the request being
// built) is reused, its old page unmapped; every frame tried moves to the newest
// end.  Returns a frame, or -1 when none can be passed (a demand page retries
// until its deadline; readahead stops).  A stream that owns no frame when none
// is unused adopts a victim of classes 1-3.
static __device__ int take_frame_lra(const DevHandle& g, int stream, bool for_ra, unsigned long long seq0,
                                     unsigned long long new_key, unsigned long long deadline) {
  const int lane = lane_id();
  int f = -1, reuse = 0, adopt = 0;
  if (lane == 0) {
    const uint32_t base = (uint32_t)stream * g.quota;
    const uint32_t len = g.lra_len[stream];
    uint32_t head = g.lra_head[stream];
    if (len < g.quota && ld_rlx64(&g.ctrl->next_unused.v) < g.n_frames) {
      const unsigned long long u = atomicAdd(&g.ctrl->next_unused.v, 1ull);
      if (u < g.n_frames) {
        f = (int)u;
        g.lra[base + (head + len) % g.quota] = (uint32_t)f;
        g.lra_len[stream] = len + 1;
      }
    }
    if (f < 0) {
      for (uint32_t k = 0; k < len; ++k) {
        const int cand = (int)g.lra[base + head];
        const int r = frame_claim_own(g, cand);
        g.lra[base + (head + len) % g.quota] = (uint32_t)cand;  // oldest -> newest
        head = (head + 1) % g.quota;
        if (r == 1) {
          f = cand;
          reuse = 1;
          break;
        }
      }
      g.lra_head[stream] = head;
      adopt = f < 0 && len == 0;
    }
  }
  f = bcast(f);
  if (bcast(reuse)) {
    evict_key(g, f, new_key, deadline);
    return f;
  }
  if (f >= 0 || !bcast(adopt)) return f;
  f = take_frame(g, for_ra, seq0, new_key, deadline);
  if (f >= 0 && lane == 0) {
    const uint32_t b2 = (uint32_t)stream * g.quota;
    const uint32_t len = g.lra_len[stream], head = g.lra_head[stream];
    if (len < g.quota) {
      g.lra[b2 + (head + len) % g.quota] = (uint32_t)f;
      g.lra_len[stream] = len + 1;
    }
  }
  return f;
}

// Whether frame f could be claimed by frame_claim_own right now (no side effect).
__device__ __forceinline__ bool lra_claimable(const DevHandle& g, uint32_t f) {
  const uint32_t st = ld_acq(&g.fstate[f]);
  if (!(st == FR_READY || st == FR_ERROR || (st == FR_EMPTY && ld_rlx64(&g.fkey[f]) == KEY_NONE))) return false;
  return ld_rlx(&g.fpins[f]) == 0u;
}

// Warp: frames for pages 1 .. L of a request of `stream` from its own LRA queue
// (Section 5.1), taken into s_frames[1 ..] as one take_frame_lra per page would
// take them after page 0: never-used frames while the queue is below its quota
// (one fetch-and-add for the run), then the queue's frames oldest first, each
// frame tried moving to the newest end, a page giving up after trying every frame
// of the queue once.  A frame taken for an earlier page of the run is in use, so it
// is passed over.  The queue always holds page 0's frame here, so no frame is
// adopted.  The queue is tried 32 entries at a time: every lane tests one entry
// without side effects, lane 0 replays the one-page-at-a-time order on those
// tests, and the entries it picks are claimed in parallel (a claim lost to another
// block counts as a tried entry that was in use).  Returns how many pages, from
// page 1 on, got a frame; claimed victims still hold their old keys.
static __device__ uint32_t take_run_lra(const DevHandle& g, int stream, uint32_t L, uint32_t* s_frames) {
  if (L == 0) return 0;
  const int lane = lane_id();
  const uint32_t base = (uint32_t)stream * g.quota;
  uint32_t len = 0, head = 0, got = 0;
  unsigned long long u0 = 0, nu = 0;  // never-used frames u0 .. u0 + nu - 1 taken by this run
  if (lane == 0) {
    len = g.lra_len[stream];
    head = g.lra_head[stream];
    if (len < g.quota && ld_rlx64(&g.ctrl->next_unused.v) < g.n_frames) {
      const uint32_t want = g.quota - len < L ? g.quota - len : L;
      u0 = atomicAdd(&g.ctrl->next_unused.v, (unsigned long long)want);
      if (u0 < g.n_frames) nu = g.n_frames - u0 < want ? g.n_frames - u0 : want;
      for (uint32_t j = 0; j < (uint32_t)nu; ++j) {
        g.lra[base + (head + len) % g.quota] = (uint32_t)(u0 + j);
        ++len;
        s_frames[1 + got++] = (uint32_t)(u0 + j);
      }
      g.lra_len[stream] = len;
    }
  }
  len = (uint32_t)bcast((int)len);
  head = (uint32_t)bcast((int)head);
  got = (uint32_t)bcast((int)got);
  u0 = bcast64(u0);
  nu = bcast64(nu);
  __syncwarp();
  uint32_t streak = 0;  // entries tried since the last claim (the current page's tries)
  while (got < L && len > 0 && streak < len) {
    const uint32_t m = len < 32u ? len : 32u;
    uint32_t cand = 0;
    bool free_now = false;
    if ((uint32_t)lane < m) {
      cand = g.lra[base + (head + (uint32_t)lane) % g.quota];
      free_now = !(cand >= u0 && cand < u0 + nu) && lra_claimable(g, cand);
    }
    const unsigned pm = __ballot_sync(kFull, free_now);
    // lane 0 replays the order: the entries tried (0 .. end) and the ones to claim
    unsigned want_mask = 0;
    int end = (int)m - 1;
    if (lane == 0) {
      uint32_t k = got, st = streak;
      for (uint32_t j = 0; j < m; ++j) {
        if ((pm >> j) & 1u) {
          want_mask |= 1u << j;
          st = 0;
          if (++k == L) {
            end = (int)j;
            break;
          }
        } else if (++st == len) {
          end = (int)j;
          break;
        }
      }
    }
    want_mask = (unsigned)bcast((int)want_mask);
    end = bcast(end);
    const bool claimed = ((want_mask >> lane) & 1u) && frame_claim_own(g, (int)cand) == 1;
    const unsigned cm = __ballot_sync(kFull, claimed);
    if (claimed) s_frames[1 + got + (uint32_t)__popc(cm & ((1u << lane) - 1u))] = cand;
    // every entry tried moves to the newest end (a no-op when the queue is full)
    if (len < g.quota && lane <= end) g.lra[base + (head + len + (uint32_t)lane) % g.quota] = cand;
    for (int j = 0; j <= end; ++j) streak = ((cm >> j) & 1u) ? 0u : streak + 1u;
    got += (uint32_t)__popc(cm);
    head = (head + (uint32_t)end + 1u) % g.quota;
    __syncwarp();
  }
  if (lane == 0) g.lra_head[stream] = head;
  __syncwarp();
  return got;
}

// Section 4.1 miss: allocate a frame for p, then serve it from the stream's
// private buffer or request PAGE_SIZE + PREFETCH_SIZE (warp).  Returns the
// pinned FILLING frame and the block-level work in *job, -EAGAIN, or -errno.
static __device__ int handle_miss_paper(const DevHandle& g, int stream, uint32_t fid, const FileDev& fi,
                                        unsigned long long p, unsigned long long seq0, unsigned long long deadline,
                                        PaperJob* job) {
  const int lane = lane_id();
  const unsigned long long key = make_key(fid, p);
  if (lane == 0) stat_add(g, ST_MISSES, 1);
  const bool own = g.repl == GFS_REPL_TB_LRA && stream >= 0 && (uint32_t)stream < g.paper_streams;
  int f = own ? take_frame_lra(g, stream, false, seq0, key, deadline) : take_frame(g, false, seq0, key, deadline);
  while (f < 0) {
    int late = 0;
    if (lane == 0) late = now_ns() > deadline;
    if (bcast(late)) {
      if (lane == 0) stat_add(g, ST_ENOMEM, 1);
      return -kENOMEM;
    }
    if (!warp_help(g, (uint32_t)(p % g.rpc_slots))) {
      if (lane == 0) __nanosleep(256);
      __syncwarp();
    }
    f = own ? take_frame_lra(g, stream, false, seq0, key, deadline) : take_frame(g, false, seq0, key, deadline);
  }
  if (lane == 0) {
    st_rlx64(&g.fkey[f], key);
    st_rlx(&g.fconsumed[f], 0u);
    st_rlx(&g.fwindow[f], 0u);
    st_rlx(&g.fmark[f], 0u);
    st_rlx(&g.fvalid[f], expected_valid(g, fi, p));
    st_rlx64(&g.faseq[f], (atomicAdd(&g.ctrl->alloc_counter.v, 1ull) << kOwnerBits) | (seq0 & kOwnerMask));
    st_rlx(&g.fsrc[f], SRC_NONE);
    __threadfence();
    atomicAdd(&g.fpins[f], 1u);
    st_rel(&g.fstate[f], FR_FILLING);
  }
  __syncwarp();
  const int r = tab_insert(g, key, (uint32_t)f, deadline);
  if (r != f) {  // another stream mapped p meanwhile: keep the frame, unused
    if (lane == 0) {
      atomicSub(&g.fpins[f], 1u);
      st_rlx64(&g.fkey[f], KEY_NONE);
      st_rel(&g.fstate[f], FR_EMPTY);
      if (!own) ring_push(g, ret_ring(g), (uint32_t)f, deadline);
    }
    __syncwarp();
    return r < 0 ? r : -kEAGAIN;
  }
  if (lane == 0) {
    if (fi.fetched) atomicOr(&fi.fetched[p >> 5], 1u << (p & 31));
    job->kind = PJ_NONE;
    job->f = f;
    job->page = p;
  }
  // the stream's private buffer
  PrivBuf pb{0, 0, 0};
  if (stream >= 0 && (uint32_t)stream < g.paper_streams) pb = g.pmeta[stream];
  if (pb.count && pb.fid == fid && p >= pb.first && p < pb.first + pb.count) {
    if (lane == 0) {
      job->kind = PJ_BUFFER;
      job->src = ((unsigned long long)stream * g.ra_cap + (p - pb.first)) << g.page_shift;
      stat_add(g, ST_BUFHITS, 1);
    }
    __syncwarp();
    return f;
  }
  unsigned long long n = 1ull + g.ra_cap;
  if (n > fi.npages - p) n = fi.npages - p;
  if (n > g.max_rpc_pages) n = g.max_rpc_pages;
  if (!(stream >= 0 && (uint32_t)stream < g.paper_streams)) n = 1;  // no buffer for this stream
  unsigned long long t = 0;
  const int rc = rpc_submit(g, fid, p, (uint32_t)n, n > 1 ? GFS_KIND_SYNC_RA : GFS_KIND_DEMAND, nullptr, deadline, &t);
  if (rc < 0) {
    if (lane == 0) frame_unpin(g, f);
    return rc;
  }
  if (lane == 0) {
    unsigned long long bytes = 0;
    for (unsigned long long i = 0; i < n; ++i) {
      bytes += expected_valid(g, fi, p + i);
      if (g.fetch_count && fid == 0 && p + i < g.debug_pages) atomicAdd(&g.fetch_count[p + i], 1u);
    }
    stat_add(g, ST_PAGES, n);
    stat_add(g, ST_BYTES, bytes);
    if (n > 1) stat_add(g, ST_RA_SYNC, n - 1);
    job->kind = PJ_REQUEST;
    job->slot = (uint32_t)(t % g.rpc_slots);
    job->t = t;
    job->n = (uint32_t)n;
  }
  __syncwarp();
  return f;
}

// Whole block: finish a paper-mode miss (copy the page from the private buffer,
// or take every page of the request as the host publishes it: page p into its
// frame, the rest into the private buffer).  Returns the frame state or -errno.
static __device__ int block_paper_job(const DevHandle& g, int stream, uint32_t fid, const FileDev& fi,
                                      const PaperJob& j, unsigned long long deadline) {
  __shared__ unsigned long long s_src;
  __shared__ uint32_t s_buf, s_ok;
  __shared__ int s_late;
  const uint32_t tid = threadIdx.x, nt = blockDim.x;
  uint8_t* frame = g.frames + ((size_t)j.f << g.page_shift);
  if (j.kind == PJ_BUFFER) {
    copy_in(g.pbuf + j.src, frame, ld_rlx(&g.fvalid[j.f]), tid, nt);
    __threadfence();
    __syncthreads();
    if (tid == 0) st_rel(&g.fstate[j.f], FR_READY);
    __syncthreads();
    return FR_READY;
  }
  bool first_ok = false;
  uint32_t good = 0;
  bool run = true;
  for (uint32_t i = 0; i < j.n; ++i) {
    if (tid == 0) {
      const PullPage* pp = &g.pages[(size_t)j.slot * g.max_rpc_pages + i];
      int late = 0;
      while (ld_acq_sys64(&pp->tag) != j.t + 1) {
        if (now_ns() > deadline) {
          late = 1;
          stat_add(g, ST_TIMEOUTS, 1);
          break;
        }
        __nanosleep(256);
      }
      s_late = late;
      if (!late) {
        s_src = ld_rlx64((const unsigned long long*)&pp->src);
        s_buf = ld_rlx((const uint32_t*)&pp->buf);
        s_ok = ld_rlx((const uint32_t*)&pp->ok);
      }
    }
    __syncthreads();
    if (s_late) {
      __syncthreads();
      return -kETIMEDOUT;
    }
    const bool ok = s_ok != 0;
    const uint8_t* src = s_buf == BUF_MAPPED ? (const uint8_t*)s_src : g.staging + s_src;
    const uint32_t bytes = expected_valid(g, fi, j.page + i);
    if (ok) {
      uint8_t* dst = i == 0 ? frame : g.pbuf + (((unsigned long long)stream * g.ra_cap + (i - 1)) << g.page_shift);
      copy_in(src, dst, bytes, tid, nt);
    }
    __threadfence();
    __syncthreads();
    if (tid == 0 && s_buf != BUF_MAPPED) {
      __threadfence_system();
      atomicAdd_system(&g.bcount[s_buf], 0xffffffffu);
    }
    if (i == 0) first_ok = ok;
    else if (run && ok) ++good;
    else run = false;
    __syncthreads();
  }
  if (tid == 0) {
    if (stream >= 0 && (uint32_t)stream < g.paper_streams) {
      PrivBuf pb;
      pb.first = j.page + 1;
      pb.fid = fid;
      pb.count = good;
      g.pmeta[stream] = pb;
    }
    __threadfence_system();
    st_rel_sys64(&ring_slot(g, j.slot)->seq, j.t + g.rpc_slots);
    st_rel64(&g.slot_free[j.slot], j.t + g.rpc_slots);
    atomicAdd(&g.ctrl->freed.v, 1ull);
    st_rel(&g.fstate[j.f], first_ok ? (uint32_t)FR_READY : (uint32_t)FR_ERROR);
  }
  __syncthreads();
  return first_ok ? (int)FR_READY : (int)FR_ERROR;
}

// Find or install page p and pin its frame for the caller (warp 0); does not
// wait.  Returns the frame (its state in *state) or -errno.
static __device__ int acquire_begin(const DevHandle& g, int stream, uint32_t fid, const FileDev& fi, unsigned long long p,
                             unsigned long long p1, unsigned long long seq0, unsigned long long deadline,
                             uint32_t* s_frames, int* state, PaperJob* job) {
  const int lane = lane_id();
  const unsigned long long key = make_key(fid, p);
  for (;;) {
    int late = 0;
    if (lane == 0) late = now_ns() > deadline;
    if (bcast(late)) {
      if (lane == 0) stat_add(g, ST_TIMEOUTS, 1);
      return -kETIMEDOUT;
    }
    int f = tab_lookup(g, key);
    if (f >= 0) {
      int st = -1;
      if (lane == 0) {
        st = frame_pin(g, f, key);
        if (st >= 0) {
          stat_add(g, ST_HITS, 1);
          if (st == FR_FILLING || st == FR_COPYING) stat_add(g, ST_COALESCED, 1);
        } else {
          stat_add(g, ST_RETRIES, 1);
        }
      }
      st = bcast(st);
      if (st == -1) continue;
      *state = st;
      return f;
    }
    const bool paper = g.mode == GFS_MODE_PAPER && fi.ra && g.xfer != GFS_XFER_DMA;
    int r = paper ? handle_miss_paper(g, stream, fid, fi, p, seq0, deadline, job)
                  : handle_miss(g, stream, fid, fi, p, p1, seq0, deadline, s_frames);
    if (r == -kEAGAIN) {
      if (lane == 0) stat_add(g, ST_RETRIES, 1);
      continue;
    }
    if (r < 0) return r;
    *state = FR_FILLING;
    return r;
  }
}

// Whole block: wait until pinned frame f leaves FILLING / COPYING (in pull mode
// copying it, or other served pages, meanwhile).  Returns the state or
// -ETIMEDOUT.  Block-uniform.
static __device__ int block_wait_ready(const DevHandle& g, int f, unsigned long long deadline) {
  __shared__ int s_st;
  unsigned ns = 64;
  for (uint32_t it = 0;; ++it) {
    if (threadIdx.x == 0) {
      int st = (int)ld_acq(&g.fstate[f]);
      if ((st == FR_FILLING || st == FR_COPYING || st == FR_RECLAIM) && now_ns() > deadline) {
        stat_add(g, ST_TIMEOUTS, 1);
        st = -kETIMEDOUT;
      }
      s_st = st;
    }
    __syncthreads();
    const int st = s_st;
    __syncthreads();
    // RECLAIM is transient here: an evictor that claimed the frame finds this
    // block's pin and puts the state back
    if (st != FR_FILLING && st != FR_COPYING && st != FR_RECLAIM) return st;
    if (g.xfer != GFS_XFER_DMA) {
      // the page itself first; other served pages only now and then (their
      // completion records are read over the host link)
      if (block_help(g, st == FR_FILLING ? f : -1, (it & 7) == 7)) {
        ns = 64;
        continue;
      }
    }
    if (threadIdx.x == 0) __nanosleep(ns);
    if (ns < 2048) ns <<= 1;
  }
}

// R4 for a READY page just acquired: the first reader of a marked page issues
// the asynchronous window (warp 0).
static __device__ void check_mark(const DevHandle& g, int stream, uint32_t fid, const FileDev& fi, int f,
                                  unsigned long long seq0, unsigned long long deadline, uint32_t* s_frames) {
  const int lane = lane_id();
  if (!(g.mode == GFS_MODE_READAHEAD && g.async_ra && fi.ra)) return;  // no marks in the other modes
  uint32_t m = 0, w = 0;
  if (lane == 0) {
    // a READY page's mark only ever goes from set to clear, and it was set
    // before the page was published: most pages carry none, and only a set
    // mark needs the exchange that lets exactly one reader claim it
    m = ld_rlx(&g.fmark[f]) ? atomicExch(&g.fmark[f], 0u) : 0u;
    if (m) w = ld_rlx(&g.fwindow[f]);
  }
  m = (uint32_t)bcast((int)m);
  w = (uint32_t)bcast((int)w);
  if (m) async_readahead(g, stream, fid, fi, (unsigned long long)m - 1, w, seq0, deadline, s_frames);
}

// R5: account the delivered bytes, unpin, and queue the frame once fully consumed.
static __device__ void release_page(const DevHandle& g, int f, uint32_t nbytes, unsigned long long deadline) {  // one thread
  if (g.repl == GFS_REPL_TB_LRA) {  // per-threadblock LRA queues (Section 5.1) replace the consumed FIFO
    atomicAdd(&g.fconsumed[f], nbytes);  // nothing waits for the old count
    frame_unpin(g, f);
    return;
  }
  uint32_t c = atomicAdd(&g.fconsumed[f], nbytes);
  uint32_t v = ld_rlx(&g.fvalid[f]);
  bool push = c < v && c + nbytes >= v;
  frame_unpin(g, f);
  if (push) fifo_push(g, (uint32_t)f, deadline);
}

// ---------------------------------------------------------------- page runs
// With small pages a page's control chain (lookup, pin, mark check, release)
// costs more than its copy, so a gread takes up to 32 consecutive pages that are
// already in the cache at once, one lane per page.  A run ends before the first
// page that is missing, in error, being reclaimed, or READY with a readahead
// mark still set (R4 stays with the one-page path, at the page's turn).  The
// pages of a run are released in page order, so the consumed FIFO receives the
// same pushes, in the same order, as from pages read one at a time.
constexpr uint32_t kRunMaxShift = 14;  // runs for pages of at most 16 KiB
constexpr uint32_t kRunPages = 32;

// Warp 0: look up and pin pages p .. p + k - 1 (k <= 32).  Returns the length of
// the leading run of pages that are READY without a mark, FILLING or COPYING;
// their frames and states are left in s_f / s_st, pinned.  Pages after the run
// are left unpinned.
static __device__ uint32_t run_begin(const DevHandle& g, uint32_t fid, unsigned long long p, uint32_t k, bool marks,
                                     uint32_t* s_f, int* s_st) {
  const int lane = lane_id();
  int f = -1;  // frame of page p + lane
  // home buckets only, eight keys in flight: a key in an overflow bucket ends the run
  for (uint32_t q0 = 0; q0 < k; q0 += 8) {
    unsigned long long e[8];
#pragma unroll
    for (uint32_t j = 0; j < 8; ++j) {
      const uint32_t b = bucket_of(make_key(fid, p + q0 + j), g.nbuckets);
      e[j] = q0 + j < k ? ld_rlx64(&g.tab[(size_t)b * BUCKET + lane]) : ENTRY_EMPTY;
    }
    bool gap = false;
#pragma unroll
    for (uint32_t j = 0; j < 8; ++j) {
      const unsigned long long key = make_key(fid, p + q0 + j);
      const unsigned m = __ballot_sync(kFull, e[j] != ENTRY_EMPTY && (e[j] >> FRAME_BITS) == key);
      const int fj = m ? (int)(__shfl_sync(kFull, e[j], __ffs(m) - 1) & MAX_FRAMES) : -1;
      if (lane == (int)(q0 + j)) f = fj;
      gap |= q0 + j < k && fj < 0;
    }
    if (gap) break;
  }
  // pin as frame_pin does, one lane per page
  const bool mine = (uint32_t)lane < k && f >= 0;
  if (mine) atomicAdd(&g.fpins[f], 1u);
  __threadfence();
  int st = -1;
  bool ok = false;
  if (mine) {
    st = (int)ld_acq(&g.fstate[f]);
    ok = (st == FR_READY || st == FR_FILLING || st == FR_COPYING) && ld_rlx64(&g.fkey[f]) == make_key(fid, p + lane);
    // a READY page's mark was set before the page was published
    if (ok && st == FR_READY && marks && ld_rlx(&g.fmark[f]) != 0u) ok = false;
  }
  const unsigned okm = __ballot_sync(kFull, ok);
  const uint32_t c = okm == kFull ? 32u : (uint32_t)(__ffs(~okm) - 1);
  if (mine && (uint32_t)lane >= c) atomicSub(&g.fpins[f], 1u);
  if ((uint32_t)lane < c) {
    s_f[lane] = (uint32_t)f;
    s_st[lane] = st;
  }
  __syncwarp();
  return c;
}

// Warp 0, after the block copied the run: R5 for its n pages (page p + i in frame
// s_f[i]; the gread covers [off, end)).  FIFO cells are reserved with one ticket
// add and filled in page order.
static __device__ void run_release(const DevHandle& g, const uint32_t* s_f, uint32_t n, unsigned long long p,
                                   unsigned long long off, unsigned long long end, unsigned long long deadline) {
  const int lane = lane_id();
  const bool mine = (uint32_t)lane < n;
  bool push = false;
  uint32_t f = 0;
  if (mine) {
    f = s_f[lane];
    const unsigned long long base = (p + lane) << g.page_shift;
    const unsigned long long lo = off > base ? off : base;
    const unsigned long long hi = end < base + g.page_size ? end : base + g.page_size;
    const uint32_t nb = (uint32_t)(hi - lo);
    const uint32_t c = atomicAdd(&g.fconsumed[f], nb);
    if (g.repl != GFS_REPL_TB_LRA) {  // per-threadblock LRA queues keep no consumed FIFO
      const uint32_t v = ld_rlx(&g.fvalid[f]);
      push = c < v && c + nb >= v;
    }
  }
  __threadfence();
  if (mine) atomicSub(&g.fpins[f], 1u);
  const unsigned m = __ballot_sync(kFull, push);
  if (!m) return;
  unsigned long long t0 = 0;
  if (lane == 0) t0 = atomicAdd(&g.ctrl->fifo_tail.v, (unsigned long long)__popc(m));
  t0 = bcast64(t0);
  if (push) fifo_put(g, t0 + (unsigned long long)__popc(m & ((1u << lane) - 1u)), f, deadline);
  __syncwarp();
}

// ---------------------------------------------------------------- copy-out
// Checksum accumulators of the stride-scan consumer (per thread).
struct Sums {
  unsigned long long sum, hash;
};

// Add 16 bytes starting at absolute file offset `o` to the checksums:
// sum += sum of bytes, hash += sum of byte_j * (o + j + 1).
__device__ __forceinline__ void sums_add16(Sums& s, uint4 v, unsigned long long o) {
  uint32_t s16 = __dp4a(v.x, 0x01010101u, 0u);
  s16 = __dp4a(v.y, 0x01010101u, s16);
  s16 = __dp4a(v.z, 0x01010101u, s16);
  s16 = __dp4a(v.w, 0x01010101u, s16);
  uint32_t w16 = __dp4a(v.x, 0x03020100u, 0u);
  w16 = __dp4a(v.y, 0x07060504u, w16);
  w16 = __dp4a(v.z, 0x0b0a0908u, w16);
  w16 = __dp4a(v.w, 0x0f0e0d0cu, w16);
  s.sum += s16;
  s.hash += (o + 1) * (unsigned long long)s16 + w16;
}
__device__ __forceinline__ void sums_add1(Sums& s, uint8_t b, unsigned long long o) {
  s.sum += b;
  s.hash += (o + 1) * (unsigned long long)b;
}

// Copy n bytes of a cache frame (src) to the user buffer (dst), thread `tid` of
// the `nt` that share the copy.  Frame data is read through L2 (ld.global.cg):
// frames are rewritten by the copy engine, so L1 may hold an older page.  With
// FUSED the checksums of the copied bytes are accumulated on the way (src_off =
// file offset of src[0]).
template <bool FUSED>
__device__ __forceinline__ void copy_range(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, uint32_t n,
                                           unsigned long long src_off, Sums& acc, uint32_t tid, uint32_t nt) {
  const uint32_t phase_s = (uint32_t)((uintptr_t)src & 15), phase_d = (uint32_t)((uintptr_t)dst & 15);
  if (phase_s == phase_d) {
    uint32_t head = (16 - phase_s) & 15;
    if (head > n) head = n;
    for (uint32_t i = tid; i < head; i += nt) {
      uint8_t b = __ldcg(src + i);
      dst[i] = b;
      if (FUSED) sums_add1(acc, b, src_off + i);
    }
    const uint32_t n16 = (n - head) >> 4;
    const uint4* s4 = reinterpret_cast<const uint4*>(src + head);
    uint4* d4 = reinterpret_cast<uint4*>(dst + head);
    uint32_t i = tid;
    for (; i + 3 * nt < n16; i += 4 * nt) {
      uint4 a = __ldcg(s4 + i), b = __ldcg(s4 + i + nt), c = __ldcg(s4 + i + 2 * nt), d = __ldcg(s4 + i + 3 * nt);
      d4[i] = a;
      d4[i + nt] = b;
      d4[i + 2 * nt] = c;
      d4[i + 3 * nt] = d;
      if (FUSED) {
        const unsigned long long o = src_off + head + 16ull * i;
        sums_add16(acc, a, o);
        sums_add16(acc, b, o + 16ull * nt);
        sums_add16(acc, c, o + 32ull * nt);
        sums_add16(acc, d, o + 48ull * nt);
      }
    }
    for (; i < n16; i += nt) {
      uint4 a = __ldcg(s4 + i);
      d4[i] = a;
      if (FUSED) sums_add16(acc, a, src_off + head + 16ull * i);
    }
    for (uint32_t j = head + 16 * n16 + tid; j < n; j += nt) {
      uint8_t b = __ldcg(src + j);
      dst[j] = b;
      if (FUSED) sums_add1(acc, b, src_off + j);
    }
  } else {
    for (uint32_t j = tid; j < n; j += nt) {
      uint8_t b = __ldcg(src + j);
      dst[j] = b;
      if (FUSED) sums_add1(acc, b, src_off + j);
    }
  }
}

// The whole block copies.
template <bool FUSED>
__device__ __forceinline__ void copy_out(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst, uint32_t n,
                                         unsigned long long src_off, Sums& acc) {
  copy_range<FUSED>(src, dst, n, src_off, acc, threadIdx.x, blockDim.x);
}

// Block-wide sum of two u64 values (mod 2^64); the result is valid in thread 0.
__device__ __forceinline__ void block_sum2(unsigned long long& a, unsigned long long& b) {
  __shared__ unsigned long long ra[32], rb[32];
  for (int o = 16; o; o >>= 1) {
    a += __shfl_xor_sync(kFull, a, o);
    b += __shfl_xor_sync(kFull, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) {
    ra[w] = a;
    rb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    a = l < nw ? ra[l] : 0ull;
    b = l < nw ? rb[l] : 0ull;
    for (int o = 16; o; o >>= 1) {
      a += __shfl_xor_sync(kFull, a, o);
      b += __shfl_xor_sync(kFull, b, o);
    }
  }
}

// ---------------------------------------------------------------- gread
// Whole block: read the run of cached pages that starts at page p (p1 = last
// page of the gread, which covers [off, end) into buf): pin it, wait for pages
// still being filled in page order, copy it a warp per page, release it.  Returns
// the number of pages read (0: page p takes the one-page path) or -errno.
// Kept out of line so that it leaves the one-page path's registers alone.
template <bool FUSED>
__device__ __noinline__ long long read_run(const DevHandle& g, uint32_t fid, unsigned long long p,
                                           unsigned long long p1, unsigned long long off, unsigned long long end,
                                           uint8_t* buf, bool marks, unsigned long long deadline, Sums* part) {
  __shared__ uint32_t s_rf[kRunPages], s_rn;
  __shared__ int s_rst[kRunPages], s_mark;
  const uint32_t tid = threadIdx.x;
  if (tid < 32) {
    const unsigned long long left = p1 - p + 1;
    const uint32_t c = run_begin(g, fid, p, left < kRunPages ? (uint32_t)left : kRunPages, marks, s_rf, s_rst);
    if (tid == 0) s_rn = c;
  }
  __syncthreads();
  uint32_t n = s_rn;
  // a mark found on a waited page once it is READY ends the run before it
  for (uint32_t i = 0; i < n; ++i) {
    if (s_rst[i] == FR_READY) continue;
    const int st = block_wait_ready(g, (int)s_rf[i], deadline);
    if (st != FR_READY) {
      if (tid == 0) {
        for (uint32_t j = 0; j < n; ++j) frame_unpin(g, (int)s_rf[j]);
        stat_add(g, ST_HITS, i + 1);
        if (st == FR_ERROR) stat_add(g, ST_EIO, 1);
      }
      __syncthreads();
      return st < 0 ? st : -kEIO;
    }
    if (marks) {
      if (tid == 0) s_mark = ld_rlx(&g.fmark[s_rf[i]]) != 0u;
      __syncthreads();
      const int mk = s_mark;
      __syncthreads();
      if (mk) {
        if (tid == 0)
          for (uint32_t j = i; j < n; ++j) frame_unpin(g, (int)s_rf[j]);
        n = i;
      }
    }
  }
  if (n == 0) return 0;
  if (tid == 0) {
    uint32_t waited = 0;
    for (uint32_t i = 0; i < n; ++i) waited += s_rst[i] != FR_READY;
    stat_add(g, ST_HITS, n);
    stat_add(g, ST_COALESCED, waited);
  }
  Sums acc{0ull, 0ull};
  const uint32_t lane = tid & 31, nw = blockDim.x >> 5;
  for (uint32_t i = tid >> 5; i < n; i += nw) {  // a warp per page
    const unsigned long long base = (p + i) << g.page_shift;
    const unsigned long long lo = (off > base ? off : base) - base;
    const unsigned long long hi = (end < base + g.page_size ? end : base + g.page_size) - base;
    copy_range<FUSED>(g.frames + ((size_t)s_rf[i] << g.page_shift) + lo, buf + (base + lo - off),
                      (uint32_t)(hi - lo), base + lo, acc, lane, 32);
  }
  if (FUSED) *part = acc;
  __syncthreads();
  if (tid < 32) run_release(g, s_rf, n, p, off, end, deadline);
  return n;
}

// Threadblock-collective read of [off, off + len) of file `fid` into buf.
// Every thread of the block must call it with the same arguments.  `stream`
// identifies the reader for sequential detection (the threadblock).  Returns
// the byte count (short at EOF, 0 at or past EOF) or a negative errno.
template <bool FUSED>
__device__ long long gread_impl(const DevHandle& g, int stream, int fid, unsigned long long off,
                                unsigned long long len, uint8_t* buf, Sums& acc) {
  __shared__ int s_frame, s_state;
  __shared__ unsigned long long s_seq0;
  __shared__ PaperJob s_job;
  __shared__ uint32_t s_frames[MAX_RPC_PAGES];
  const uint32_t tid = threadIdx.x;
  if (fid < 0 || (uint32_t)fid >= g.max_files) return -kEBADF;
  const FileDev fi = load_file(g, fid);
  if (!fi.open) return -kEBADF;
  if (tid == 0) stat_add(g, ST_GREADS, 1);
  if (off >= fi.size || len == 0) return 0;
  const unsigned long long end = (len > fi.size - off) ? fi.size : off + len;
  const unsigned long long p0 = off >> g.page_shift, p1 = (end - 1) >> g.page_shift;
  if (tid == 0) s_seq0 = (ld_rlx64(&g.ctrl->alloc_counter.v) << kOwnerBits) | owner_of(stream);
  __syncthreads();
  const unsigned long long seq0 = s_seq0;
  const unsigned long long deadline = now_ns() + g.timeout_ns;
  long long err = 0;
  const bool runs = g.mode != GFS_MODE_PAPER && g.page_shift <= kRunMaxShift && p1 > p0;
  const bool marks = g.mode == GFS_MODE_READAHEAD && g.async_ra && fi.ra;
  for (unsigned long long p = p0; p <= p1;) {
    if (runs) {
      Sums part{0ull, 0ull};
      const long long n = read_run<FUSED>(g, (uint32_t)fid, p, p1, off, end, buf, marks, deadline, &part);
      if (n < 0) {
        err = n;
        break;
      }
      if (n) {
        if (FUSED) {
          acc.sum += part.sum;
          acc.hash += part.hash;
        }
        p += (unsigned long long)n;
        continue;
      }
    }
    if (tid == 0) {
      s_job.kind = PJ_NONE;
      self_job().n = 0;
    }
    __syncthreads();
    if (tid < 32) {
      int st = 0;
      int r = acquire_begin(g, stream, (uint32_t)fid, fi, p, p1, seq0, deadline, s_frames, &st, &s_job);
      if (tid == 0) {
        s_frame = r;
        s_state = st;
      }
    }
    __syncthreads();
    const int f = s_frame;
    int st = s_state;
    const PaperJob job = s_job;
    __syncthreads();
    block_self_serve(g, fi, s_frames);  // the request the miss just made, when its pages are the block's to copy
    if (f < 0) {
      err = f;
      break;
    }
    if (job.kind != PJ_NONE) st = block_paper_job(g, stream, (uint32_t)fid, fi, job, deadline);
    else if (st == FR_FILLING || st == FR_COPYING) st = block_wait_ready(g, f, deadline);
    if (st != FR_READY) {
      if (tid == 0) {
        frame_unpin(g, f);
        if (st == FR_ERROR) stat_add(g, ST_EIO, 1);
      }
      err = st < 0 ? st : -kEIO;
      __syncthreads();
      break;
    }
    if (tid < 32) check_mark(g, stream, (uint32_t)fid, fi, f, seq0, deadline, s_frames);
    __syncthreads();
    block_self_serve(g, fi, s_frames);  // the asynchronous window check_mark requested, if any
    const unsigned long long base = p << g.page_shift;
    const unsigned long long lo = (off > base ? off : base) - base;
    const unsigned long long hi = (end < base + g.page_size ? end : base + g.page_size) - base;
    copy_out<FUSED>(g.frames + ((size_t)f << g.page_shift) + lo, buf + (base + lo - off), (uint32_t)(hi - lo),
                    base + lo, acc);
    __syncthreads();
    if (tid == 0) release_page(g, f, (uint32_t)(hi - lo), deadline);
    ++p;
  }
  if (tid == 0 && stream >= 0 && (uint32_t)stream < g.max_streams)
    st_rlx64(&g.last_end[(size_t)stream * g.max_files + fid], p1 + 2);  // end page + 1
  if (tid == 0 && g.lat_cap) {
    const unsigned long long i = atomicAdd(&g.ctrl->lat_n.v, 1ull);
    if (i < g.lat_cap) g.lat[i] = now_ns() - (deadline - g.timeout_ns);
  }
  __syncthreads();
  return err ? err : (long long)(end - off);
}

__device__ __forceinline__ long long gread(const DevHandle& g, int stream, int fid, unsigned long long off,
                                           unsigned long long len, void* buf) {
  Sums unused{0, 0};
  return gread_impl<false>(g, stream, fid, off, len, (uint8_t*)buf, unused);
}

// File size of an open fid, or -EBADF.  Any thread.
__device__ __forceinline__ long long gfstat_size(const DevHandle& g, int fid) {
  if (fid < 0 || (uint32_t)fid >= g.max_files) return -kEBADF;
  const FileDev fi = load_file(g, fid);
  return fi.open ? (long long)fi.size : -kEBADF;
}

// ---------------------------------------------------------------- open / close / stat / hint
// Section 2.2: GPUfs gives GPU threads the POSIX-like calls open, read, close
// and fstat; open and close go to the host over the same queue as reads.  The
// access hint of Section 4.4 travels the same way.

// One control request over the ring (one warp).  The host answers in the
// slot's CtlMsg; the warp waits for the answer (helping with served pages in
// the GPU copy transfers) and then frees the slot itself.  Returns 0 with
// *status / *last set, or -ETIMEDOUT.
static __device__ int rpc_control(const DevHandle& g, uint32_t op, uint32_t fid, uint32_t arg, const char* path,
                                  uint32_t path_len, int* status, uint32_t* last, unsigned long long deadline) {
  const int lane = lane_id();
  unsigned long long t = 0;
  uint32_t si = 0;
  const int arc = ring_acquire(g, &t, &si, deadline);
  if (arc) return arc;
  RingSlot* s = ring_slot(g, si);
  CtlMsg* m = reinterpret_cast<CtlMsg*>(s->frames);
  if (op == OP_OPEN) {
    char* dst = g.paths + (size_t)si * GFS_PATH_MAX;
    for (uint32_t i = lane; i <= path_len; i += 32) dst[i] = i < path_len ? path[i] : '\0';
  }
  if (lane == 0) {
    if (g.xfer != GFS_XFER_DMA) {  // no pages: helpers skip the slot
      st_rlx64(&g.dticket[si], t);
      st_rlx(&g.dnpages[si], 0u);
      st_rlx(&g.dcopied[si], 0u);
    }
    st_sys32(&m->done, 0u);
    st_sys32(&m->arg, arg);
    st_sys32(&s->fid, fid);
    st_sys32(&s->npages, 0u);
    st_sys64(&s->page_lo, 0ull);
    st_sys32(&s->kind, 0u);
    st_sys32(&s->op, op);
    st_sys64(&s->issue_ns, now_ns());
  }
  __syncwarp();
  __threadfence_system();
  __syncwarp();
  if (lane == 0) st_rel_sys64(&s->seq, t + 1);
  __syncwarp();
  for (unsigned ns = 256;;) {
    int done = 0, late = 0;
    if (lane == 0) {
      done = ld_acq_sys32(&m->done) == 1u;
      late = now_ns() > deadline;
    }
    if (bcast(done)) break;
    if (bcast(late)) {  // the slot stays taken: the ring reports the loss through later timeouts
      if (lane == 0) stat_add(g, ST_TIMEOUTS, 1);
      return -kETIMEDOUT;
    }
    if (g.xfer != GFS_XFER_DMA && warp_help(g, si)) continue;
    if (lane == 0) __nanosleep(ns);
    __syncwarp();
    if (ns < 4096) ns <<= 1;
  }
  int st = 0;
  uint32_t ls = 0;
  if (lane == 0) {
    const volatile CtlMsg* vm = m;
    st = vm->status;
    ls = vm->last;
    __threadfence_system();
    st_rel_sys64(&s->seq, t + g.rpc_slots);  // the slot is free for the next lap
    if (g.xfer != GFS_XFER_DMA) st_rel64(&g.slot_free[si], t + g.rpc_slots);
    atomicAdd(&g.ctrl->freed.v, 1ull);
  }
  *status = bcast(st);
  *last = (uint32_t)bcast((int)ls);
  return 0;
}

// Threadblock-collective control call: warp 0 runs it, every thread gets the result.
static __device__ int block_control(const DevHandle& g, uint32_t op, uint32_t fid, uint32_t arg, const char* path,
                                    uint32_t path_len) {
  __shared__ int s_ret;
  if (threadIdx.x < 32) {
    int st = 0;
    uint32_t last = 0;
    int rc = rpc_control(g, op, fid, arg, path, path_len, &st, &last, now_ns() + g.timeout_ns);
    if (threadIdx.x == 0) s_ret = rc ? rc : st;
  }
  __syncthreads();
  const int ret = s_ret;
  __syncthreads();
  return ret;
}

// Threadblock-collective open (every thread, same arguments).  `path` is a
// NUL-terminated string the device can read, shorter than GFS_PATH_MAX.
// Opening a path that blocks already hold open on the device (same flags)
// returns the same fid and adds a reference; so does opening a path whose id
// the last gclose retired, until the host drops its pages.  Returns the fid or -errno
// (-EINVAL, -ENAMETOOLONG, -EMFILE, -ENOTSUP in GFS_MODE_PAPER, host open
// errors, -ETIMEDOUT).
static __device__ int gopen(const DevHandle& g, const char* path, int flags) {
  if (g.mode == GFS_MODE_PAPER) return -kENOTSUP;
  if (!path || (flags != GFS_RDONLY && flags != GFS_RDWR)) return -kEINVAL;
  __shared__ uint32_t s_len;
  if (threadIdx.x == 0) {  // one reader: the string's allocation may end at its terminator
    uint32_t len = 0;
    while (len < GFS_PATH_MAX && path[len] != '\0') ++len;
    s_len = len;
  }
  __syncthreads();
  const uint32_t len = s_len;
  __syncthreads();
  if (len == 0) return -kEINVAL;
  if (len >= GFS_PATH_MAX) return -kENAMETOOLONG;
  return block_control(g, OP_OPEN, 0u, (uint32_t)flags, path, len);
}

// Threadblock-collective close of a fid opened with gopen.  After the last
// reference the fid reads as closed; its pages stay cached, unreachable, until
// the host drops them (gfs_reset_cache, or reuse of the fid) or a gopen of the
// same path opens the fid again.  Returns 0 or
// -errno (-EBADF for a fid not opened on the device).
static __device__ int gclose(const DevHandle& g, int fid) {
  if (fid < 0 || (uint32_t)fid >= g.max_files) return -kEBADF;
  return block_control(g, OP_CLOSE, (uint32_t)fid, 0u, nullptr, 0u);
}

// Threadblock-collective access hint (Section 4.4): GFS_ADV_RANDOM turns
// readahead off for the fid, NORMAL and SEQUENTIAL turn it back on for
// read-only opens.  Applies to greads that start after the call returns, in
// every block.  Returns 0 or -errno.
static __device__ int gfadvise(const DevHandle& g, int fid, int advice) {
  if (fid < 0 || (uint32_t)fid >= g.max_files) return -kEBADF;
  if (advice < GFS_ADV_NORMAL || advice > GFS_ADV_RANDOM) return -kEINVAL;
  return block_control(g, OP_ADVISE, (uint32_t)fid, (uint32_t)advice, nullptr, 0u);
}

// fstat of an open fid (any thread).  Returns 0 or -EBADF.
__device__ __forceinline__ int gfstat(const DevHandle& g, int fid, gfs_stat* st) {
  if (fid < 0 || (uint32_t)fid >= g.max_files) return -kEBADF;
  const FileDev fi = load_file(g, fid);
  if (!fi.open) return -kEBADF;
  st->size = fi.size;
  st->page_size = g.page_size;
  st->flags = fi.flags;
  st->advice = fi.advice;
  st->mapped = fi.mapped;
  return 0;
}

// Drop every cached page of `fid` (host close).  Runs only while no other
// kernel of the context runs and no request is in flight: nothing is pinned or
// filling, and a READY frame is in the consumed FIFO exactly when it is fully
// consumed.  Warp `w` of `nw` takes frames w, w + nw, ...  Dropped frames
// become keyless EMPTY frames in the consumed FIFO (victim class 2).
static __device__ void purge_fid(const DevHandle& g, uint32_t fid, uint32_t w, uint32_t nw,
                                 unsigned long long deadline) {
  const int lane = lane_id();
  for (uint32_t f = w; f < g.n_frames; f += nw) {
    unsigned long long key = 0;
    if (lane == 0) key = ld_rlx64(&g.fkey[f]);
    key = bcast64(key);
    if (key == KEY_NONE || key_fid(key) != fid) continue;
    tab_remove(g, key, f, deadline);
    if (lane == 0) {
      const uint32_t st = ld_rlx(&g.fstate[f]);
      const uint32_t valid = ld_rlx(&g.fvalid[f]);
      const bool queued = g.repl == GFS_REPL_FIFO && st == FR_READY && valid > 0 && ld_rlx(&g.fconsumed[f]) >= valid;
      st_rlx64(&g.fkey[f], KEY_NONE);
      st_rlx(&g.fconsumed[f], 0u);
      st_rlx(&g.fvalid[f], 0u);
      st_rlx(&g.fwindow[f], 0u);
      st_rlx(&g.fmark[f], 0u);
      st_rlx64(&g.faseq[f], ~0ull);
      if (g.fsrc) st_rlx(&g.fsrc[f], SRC_NONE);
      st_rel(&g.fstate[f], FR_EMPTY);
      if (!queued) fifo_push(g, f, deadline);
    }
    __syncwarp();
  }
}

}  // namespace dev
}  // namespace gfs
