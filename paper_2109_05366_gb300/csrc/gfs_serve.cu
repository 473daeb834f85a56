// Serving: a persistent kernel that runs many sequential-scan requests at once
// through the shared GPU page cache (continuous batching).
//
//   host                          device (k_serve, all CTAs alike)
//   gfs_submit_scan -> submission ring (mapped) -> admission: one CTA at a time
//                                                  admits requests in arrival
//                                                  order while their frame
//                                                  reservation fits the cache
//                                                  budget
//                                                  work: CTAs pick active
//                                                  requests round-robin and
//                                                  claim one unit (a stride of
//                                                  unit_bytes) at a time; gread
//                                                  + checksum; per-request sums
//                                                  add up (mod 2^64)
//   gfs_poll        <- completion ring (mapped) <- the CTA finishing a
//                                                  request's last unit
//
// Requests that arrive while others run are admitted as soon as frames free
// up; their units interleave with the running ones on the same CTAs.
#include <cuda_runtime.h>
#include <errno.h>
#include <unistd.h>

#include <chrono>
#include <cstring>
#include <new>

#include "gfs_device.cuh"
#include "gfs_host.h"
#include "gfs_serve.h"

namespace gfs {
namespace serve {

struct SubSlot {  // host writes, device reads (mapped pinned)
  unsigned long long seq;
  uint32_t fid, pad;
  unsigned long long off, len, tag, t_submit;
};

struct ComplSlot {  // device writes, host reads (mapped pinned)
  unsigned long long seq;
  long long status;
  unsigned long long tag, sum, hash, bytes, t_admit, t_done;
};

struct Req {  // device memory
  unsigned long long claim;  // (generation << 32) | next unit
  uint32_t state;            // 0 free, 1 active
  uint32_t fid;
  unsigned long long off, len, tag, t_admit;
  uint32_t n_units, done_units, frames, gen;
  unsigned long long sum, hash, bytes;
  long long status;
};

struct Ctl {  // device memory
  Line sub_head;
  Line compl_tail;
  Line rr;
  Line frames_reserved;
  Line active;
  Line adm_lock;
  Line last_work;
  Line lost;  // completions dropped because the host left the completion ring full past the deadline
};

struct Handle {
  SubSlot* sub;
  ComplSlot* compl_;
  Req* req;
  Ctl* ctl;
  const uint32_t* stop;  // mapped host flag
  uint8_t* bufs;
  unsigned long long unit_bytes, buf_stride, idle_exit_ns;
  uint32_t sub_slots, compl_slots, max_req, units_cap, pages_per_unit, frame_budget;
};

__device__ __forceinline__ uint32_t ld_sys32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Write a completion record and free the request slot (one thread).  A
// completion slot is claimed (compare-and-swap) only once the host has freed it,
// so a record is never written over one the host has not read; if the host
// leaves the ring full past the deadline the completion is dropped and counted.
__device__ void complete(const DevHandle& g, const Handle& h, uint32_t r) {
  Req& q = h.req[r];
  const unsigned long long dl = dev::now_ns() + g.timeout_ns;
  unsigned long long c = 0;
  bool claimed = false;
  for (;;) {
    c = dev::ld_rlx64(&h.ctl->compl_tail.v);
    if (dev::ld_acq_sys64(&h.compl_[c % h.compl_slots].seq) == c) {
      if (atomicCAS(&h.ctl->compl_tail.v, c, c + 1) == c) {
        claimed = true;
        break;
      }
      continue;
    }
    if (dev::now_ns() > dl) break;
    __nanosleep(256);
  }
  if (!claimed) {
    atomicAdd(&h.ctl->lost.v, 1ull);
    atomicAdd(&h.ctl->frames_reserved.v, (unsigned long long)(0ull - q.frames));
    atomicAdd(&h.ctl->active.v, ~0ull);
    dev::st_rel(&q.state, 0u);
    return;
  }
  ComplSlot* cs = &h.compl_[c % h.compl_slots];
  dev::st_sys64((unsigned long long*)&cs->status, (unsigned long long)dev::ld_rlx64((unsigned long long*)&q.status));
  dev::st_sys64(&cs->tag, q.tag);
  dev::st_sys64(&cs->sum, dev::ld_rlx64(&q.sum));
  dev::st_sys64(&cs->hash, dev::ld_rlx64(&q.hash));
  dev::st_sys64(&cs->bytes, dev::ld_rlx64(&q.bytes));
  dev::st_sys64(&cs->t_admit, q.t_admit);
  dev::st_sys64(&cs->t_done, dev::now_ns());
  __threadfence_system();
  dev::st_rel_sys64(&cs->seq, c + 1);
  atomicAdd(&h.ctl->frames_reserved.v, (unsigned long long)(0ull - q.frames));
  atomicAdd(&h.ctl->active.v, ~0ull);
  dev::st_rel(&q.state, 0u);
}

// Admit waiting requests in arrival order while their frames fit (one thread,
// holding the admission lock).
__device__ void admit(const DevHandle& g, const Handle& h) {
  for (;;) {
    const unsigned long long t = dev::ld_rlx64(&h.ctl->sub_head.v);
    SubSlot* ss = &h.sub[t % h.sub_slots];
    if (dev::ld_acq_sys64(&ss->seq) != t + 1) return;  // nothing waiting
    const unsigned long long len = ss->len;
    const uint32_t n_units = (uint32_t)((len + h.unit_bytes - 1) / h.unit_bytes);
    const uint32_t cap = n_units < h.units_cap ? n_units : h.units_cap;
    const uint32_t frames = cap * h.pages_per_unit;
    const unsigned long long reserved = dev::ld_rlx64(&h.ctl->frames_reserved.v);
    const unsigned long long active = dev::ld_rlx64(&h.ctl->active.v);
    if (active > 0 && reserved + frames > h.frame_budget) return;  // admission by free cache frames
    int r = -1;
    for (uint32_t i = 0; i < h.max_req && r < 0; ++i)
      if (dev::ld_acq(&h.req[i].state) == 0) r = (int)i;
    if (r < 0) return;
    Req& q = h.req[r];
    q.fid = ss->fid;
    q.off = ss->off;
    q.len = len;
    q.tag = ss->tag;
    q.t_admit = dev::now_ns();
    q.n_units = n_units;
    q.done_units = 0;
    q.frames = frames;
    q.sum = q.hash = q.bytes = 0;
    q.status = 0;
    q.gen += 1;
    __threadfence();
    dev::st_rel64(&q.claim, ((unsigned long long)q.gen << 32) | 0ull);
    atomicAdd(&h.ctl->frames_reserved.v, (unsigned long long)frames);
    atomicAdd(&h.ctl->active.v, 1ull);
    dev::st_rel(&q.state, 1u);
    dev::st_rel_sys64(&ss->seq, t + h.sub_slots);  // submission slot free for the host
    dev::st_rlx64(&h.ctl->sub_head.v, t + 1);
    if (n_units == 0) complete(g, h, (uint32_t)r);
  }
}

// Claim one unit of an active request, round-robin over requests (one thread).
__device__ bool pick(const Handle& h, uint32_t* rr_out, uint32_t* unit_out) {
  for (uint32_t k = 0; k < h.max_req; ++k) {
    const uint32_t r = (uint32_t)(atomicAdd(&h.ctl->rr.v, 1ull) % h.max_req);
    Req& q = h.req[r];
    if (dev::ld_acq(&q.state) != 1) continue;
    unsigned long long w = dev::ld_acq64(&q.claim);
    for (;;) {
      if ((w >> 32) != dev::ld_rlx(&q.gen)) break;
      const uint32_t u = (uint32_t)w;
      if (u >= dev::ld_rlx(&q.n_units)) break;
      const unsigned long long seen = atomicCAS(&q.claim, w, w + 1);
      if (seen == w) {
        *rr_out = r;
        *unit_out = u;
        return true;
      }
      w = seen;
    }
  }
  return false;
}

__global__ void __launch_bounds__(512) k_serve(DevHandle g, Handle h) {
  __shared__ int s_r;
  __shared__ uint32_t s_u;
  __shared__ int s_exit;
  __shared__ unsigned long long s_off, s_len;
  __shared__ uint32_t s_fid;
  const uint32_t tid = threadIdx.x;
  uint8_t* buf = h.bufs + (size_t)blockIdx.x * h.buf_stride;
  unsigned idle_ns = 256;
  for (;;) {
    if (tid == 0) {
      s_exit = 0;
      s_r = -1;
      if (atomicCAS((uint32_t*)&h.ctl->adm_lock.v, 0u, 1u) == 0u) {
        admit(g, h);
        __threadfence();
        atomicExch((uint32_t*)&h.ctl->adm_lock.v, 0u);
      }
      uint32_t r, u;
      if (pick(h, &r, &u)) {
        const Req& q = h.req[r];
        s_r = (int)r;
        s_u = u;
        s_fid = q.fid;
        s_off = q.off + (unsigned long long)u * h.unit_bytes;
        const unsigned long long end = q.off + q.len;
        s_len = end - s_off < h.unit_bytes ? end - s_off : h.unit_bytes;
        dev::st_rlx64(&h.ctl->last_work.v, dev::now_ns());
      } else {
        const bool stopping = ld_sys32(h.stop) != 0;
        const bool idle = dev::ld_rlx64(&h.ctl->active.v) == 0 &&
                          dev::ld_acq_sys64(&h.sub[dev::ld_rlx64(&h.ctl->sub_head.v) % h.sub_slots].seq) !=
                              dev::ld_rlx64(&h.ctl->sub_head.v) + 1;
        unsigned long long lw = dev::ld_rlx64(&h.ctl->last_work.v);
        if (lw == 0) {  // the idle clock starts with the first look
          atomicCAS(&h.ctl->last_work.v, 0ull, dev::now_ns());
          lw = dev::ld_rlx64(&h.ctl->last_work.v);
        }
        const bool stale = dev::now_ns() - lw > h.idle_exit_ns;
        s_exit = (stopping && idle) || stale;
      }
    }
    __syncthreads();
    const int r = s_r;
    if (s_exit) break;
    if (r < 0) {
      if (tid == 0) __nanosleep(idle_ns);
      if (idle_ns < 8192) idle_ns <<= 1;
      __syncthreads();
      continue;
    }
    idle_ns = 256;
    dev::Sums acc{0ull, 0ull};
    const long long n = dev::gread_impl<true>(g, (int)blockIdx.x, (int)s_fid, s_off, s_len, buf, acc);
    dev::block_sum2(acc.sum, acc.hash);
    if (tid == 0) {
      Req& q = h.req[r];
      if (n > 0) {
        atomicAdd(&q.sum, acc.sum);
        atomicAdd(&q.hash, acc.hash);
        atomicAdd(&q.bytes, (unsigned long long)n);
      } else if (n < 0) {
        atomicCAS((unsigned long long*)&q.status, 0ull, (unsigned long long)n);
      }
      __threadfence();
      if (atomicAdd(&q.done_units, 1u) + 1 == q.n_units) complete(g, h, (uint32_t)r);
    }
    __syncthreads();
  }
  if (g.xfer != GFS_XFER_DMA)
    for (int i = 0; i < 4096; ++i)
      if (!dev::block_help(g, -1, true)) break;
}

}  // namespace serve
}  // namespace gfs

// ---------------------------------------------------------------- host side
using namespace gfs;
using namespace gfs::serve;

struct gfs_server {
  Handle h{};
  SubSlot* h_sub = nullptr;
  ComplSlot* h_compl = nullptr;
  uint32_t* h_stop = nullptr;
  uint8_t* d_mem = nullptr;
  cudaStream_t stream = nullptr;
  unsigned long long sub_tail = 0, compl_head = 0;
};

namespace {
int cerr(cudaError_t e) { return e == cudaSuccess ? 0 : (e == cudaErrorMemoryAllocation ? -ENOMEM : -EINVAL); }

void free_server(gfs_server* s) {
  if (!s) return;
  if (s->d_mem) cudaFree(s->d_mem);
  if (s->h_sub) cudaFreeHost(s->h_sub);
  if (s->h_compl) cudaFreeHost(s->h_compl);
  if (s->h_stop) cudaFreeHost(s->h_stop);
  delete s;
}
}  // namespace

extern "C" int gfs_serve_start(gfs_ctx* ctx, const gfs_serve_config* sc, void* stream) {
  if (!ctx || !sc) return -EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->server) return -EBUSY;
  if (sc->ctas == 0 || (sc->threads != 128 && sc->threads != 256 && sc->threads != 512) || sc->unit_bytes == 0 ||
      sc->max_requests == 0 || sc->queue_slots < 2)  // ring sequence rule: 2 slots at least
    return -EINVAL;
  if (cudaSetDevice(ctx->cfg.device) != cudaSuccess) return -ENODEV;
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve, (int)sc->threads, 0) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->cfg.device) != cudaSuccess)
    return -EINVAL;
  if ((int)sc->ctas > per_sm * sms) return -EINVAL;  // a persistent kernel must fit at once
  int rc = 0;
  rc = ensure_paper_state(ctx, sc->ctas);
  if (rc) return rc;
  gfs_server* s = new (std::nothrow) gfs_server();
  if (!s) return -ENOMEM;
  Handle& h = s->h;
  h.sub_slots = sc->queue_slots;
  h.compl_slots = sc->queue_slots;
  h.max_req = sc->max_requests;
  h.unit_bytes = sc->unit_bytes;
  h.buf_stride = (sc->unit_bytes + 255) / 256 * 256;
  h.units_cap = sc->units_in_flight ? sc->units_in_flight : 16;
  h.pages_per_unit = (uint32_t)((sc->unit_bytes + ctx->cfg.page_size - 1) / ctx->cfg.page_size) + 1;
  const uint32_t F = ctx->dev.n_frames;
  const uint64_t in_use = (uint64_t)sc->ctas * h.pages_per_unit;
  h.frame_budget = sc->frame_budget ? sc->frame_budget : (uint32_t)(F > in_use ? F - in_use : F / 2);
  h.idle_exit_ns = sc->idle_exit_ms ? (unsigned long long)sc->idle_exit_ms * 1000000ull : 60ull * 1000000000ull;
  const size_t req_bytes = sizeof(Req) * h.max_req;
  const size_t ctl_off = (req_bytes + 255) / 256 * 256;
  const size_t buf_off = ctl_off + (sizeof(Ctl) + 255) / 256 * 256;
  const size_t total = buf_off + (size_t)sc->ctas * h.buf_stride;
  rc = cerr(cudaMalloc((void**)&s->d_mem, total));
  if (!rc) rc = cerr(cudaMemset(s->d_mem, 0, total));
  if (!rc) rc = cerr(cudaHostAlloc((void**)&s->h_sub, sizeof(SubSlot) * h.sub_slots, cudaHostAllocMapped));
  if (!rc) rc = cerr(cudaHostAlloc((void**)&s->h_compl, sizeof(ComplSlot) * h.compl_slots, cudaHostAllocMapped));
  if (!rc) rc = cerr(cudaHostAlloc((void**)&s->h_stop, 64, cudaHostAllocMapped));
  if (rc) {
    free_server(s);
    return rc;
  }
  memset(s->h_sub, 0, sizeof(SubSlot) * h.sub_slots);
  memset(s->h_compl, 0, sizeof(ComplSlot) * h.compl_slots);
  for (uint32_t i = 0; i < h.sub_slots; ++i) s->h_sub[i].seq = i;
  for (uint32_t i = 0; i < h.compl_slots; ++i) s->h_compl[i].seq = i;
  *s->h_stop = 0;
  void* p = nullptr;
  rc = cerr(cudaHostGetDevicePointer(&p, s->h_sub, 0));
  h.sub = (SubSlot*)p;
  if (!rc) rc = cerr(cudaHostGetDevicePointer(&p, s->h_compl, 0));
  h.compl_ = (ComplSlot*)p;
  if (!rc) rc = cerr(cudaHostGetDevicePointer(&p, s->h_stop, 0));
  h.stop = (const uint32_t*)p;
  h.req = (Req*)s->d_mem;
  h.ctl = (Ctl*)(s->d_mem + ctl_off);
  h.bufs = s->d_mem + buf_off;
  if (rc) {
    free_server(s);
    return rc;
  }
  s->stream = (cudaStream_t)stream;
  DevHandle g = ctx->dev;
  g.reserve = ctx->cfg.reserve_frames ? ctx->cfg.reserve_frames : (uint32_t)(in_use + 1);
  k_serve<<<sc->ctas, sc->threads, 0, s->stream>>>(g, h);
  rc = cerr(cudaGetLastError());
  if (rc) {
    free_server(s);
    return rc;
  }
  ctx->server = s;
  return 0;
}

extern "C" int gfs_submit_scan(gfs_ctx* ctx, int fid, uint64_t off, uint64_t len, uint64_t tag) {
  if (!ctx || !ctx->server) return -EINVAL;
  if (fid < 0 || (size_t)fid >= ctx->files.size() || !ctx->files[fid].open) return -EBADF;
  gfs_server* s = ctx->server;
  const unsigned long long t = s->sub_tail;
  SubSlot* ss = &s->h_sub[t % s->h.sub_slots];
  if (__atomic_load_n(&ss->seq, __ATOMIC_ACQUIRE) != t) return -EAGAIN;  // ring full
  ss->fid = (uint32_t)fid;
  ss->off = off;
  ss->len = len;
  ss->tag = tag;
  ss->t_submit = (unsigned long long)std::chrono::duration_cast<std::chrono::nanoseconds>(
                     std::chrono::steady_clock::now().time_since_epoch())
                     .count();
  __atomic_store_n(&ss->seq, t + 1, __ATOMIC_RELEASE);
  s->sub_tail = t + 1;
  return 0;
}

extern "C" int gfs_poll(gfs_ctx* ctx, gfs_completion* out, int max) {
  if (!ctx || !ctx->server || (!out && max > 0)) return -EINVAL;
  gfs_server* s = ctx->server;
  int n = 0;
  while (n < max) {
    const unsigned long long c = s->compl_head;
    ComplSlot* cs = &s->h_compl[c % s->h.compl_slots];
    if (__atomic_load_n(&cs->seq, __ATOMIC_ACQUIRE) != c + 1) break;
    gfs_completion& o = out[n++];
    o.tag = cs->tag;
    o.status = cs->status;
    o.sum = cs->sum;
    o.hash = cs->hash;
    o.bytes = cs->bytes;
    o.t_admit_ns = cs->t_admit;
    o.t_done_ns = cs->t_done;
    __atomic_store_n(&cs->seq, c + s->h.compl_slots, __ATOMIC_RELEASE);
    s->compl_head = c + 1;
  }
  return n;
}

extern "C" int gfs_serve_stop(gfs_ctx* ctx) {
  if (!ctx) return -EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  gfs_server* s = ctx->server;
  if (!s) return 0;
  __atomic_store_n(s->h_stop, 1u, __ATOMIC_RELEASE);
  // completions not polled by now are discarded: keep the ring drained so no CTA
  // waits for a slot while the kernel finishes its last requests
  cudaError_t q;
  while ((q = cudaStreamQuery(s->stream)) == cudaErrorNotReady) {
    for (;;) {
      const unsigned long long c = s->compl_head;
      ComplSlot* cs = &s->h_compl[c % s->h.compl_slots];
      if (__atomic_load_n(&cs->seq, __ATOMIC_ACQUIRE) != c + 1) break;
      __atomic_store_n(&cs->seq, c + s->h.compl_slots, __ATOMIC_RELEASE);
      s->compl_head = c + 1;
    }
    usleep(100);
  }
  int rc = cerr(q);
  unsigned long long lost = 0;
  if (!rc) rc = cerr(cudaMemcpy(&lost, &s->h.ctl->lost.v, 8, cudaMemcpyDeviceToHost));
  free_server(s);
  ctx->server = nullptr;
  return rc ? rc : (lost ? -ENOBUFS : 0);
}
