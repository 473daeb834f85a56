/*
 * Seeded synthetic input files for the GPU file-read path and its oracle.
 *
 * This module holds no arithmetic of the method: it only produces the bytes of
 * the files that both the CUDA path and the CPU oracle read.
 *
 * Byte stream: xorshift64 (G. Marsaglia, "Xorshift RNGs", J. Stat. Softw. 8(14),
 * 2003), the 64-bit generator with shift triple (13, 7, 17):
 *     x ^= x << 13;  x ^= x >> 7;  x ^= x << 17;
 * starting from x = seed (non-zero).  Output word j (j = 0, 1, ...) is the state
 * after j + 1 steps, written as 8 little-endian bytes; a file of `size` bytes is
 * the first `size` bytes of that stream.
 *
 * The step is linear over GF(2)^64, so the state after k steps is M^k * seed
 * for the 64x64 bit matrix M of one step.  Threads use that jump-ahead to start
 * generating in the middle of the stream; the result does not depend on the
 * thread count.
 */
#define _GNU_SOURCE
#include <errno.h>
#include <fcntl.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

static inline uint64_t xs_step(uint64_t x) {
  x ^= x << 13;
  x ^= x >> 7;
  x ^= x << 17;
  return x;
}

/* A linear map on GF(2)^64, stored by columns: col[i] is the image of e_i. */
typedef struct { uint64_t col[64]; } gf2_map;

static uint64_t map_apply(const gf2_map* m, uint64_t v) {
  uint64_t r = 0;
  for (int i = 0; i < 64; ++i)
    if ((v >> i) & 1u) r ^= m->col[i];
  return r;
}

/* out = a o b (apply b first). `out` may not alias a or b. */
static void map_compose(gf2_map* out, const gf2_map* a, const gf2_map* b) {
  for (int i = 0; i < 64; ++i) out->col[i] = map_apply(a, b->col[i]);
}

/* State after k steps from `seed`. */
uint64_t xs_state_after(uint64_t seed, uint64_t k) {
  gf2_map base, acc, tmp;
  for (int i = 0; i < 64; ++i) {
    base.col[i] = xs_step(1ull << i);
    acc.col[i] = 1ull << i; /* identity */
  }
  while (k) {
    if (k & 1u) { map_compose(&tmp, &base, &acc); acc = tmp; }
    k >>= 1;
    if (k) { map_compose(&tmp, &base, &base); base = tmp; }
  }
  return map_apply(&acc, seed);
}

/* Fill buf with stream bytes [byte_off, byte_off + n). */
int xs_fill(uint8_t* buf, uint64_t seed, uint64_t byte_off, uint64_t n) {
  if (seed == 0) return -EINVAL;
  uint64_t word = byte_off / 8;
  unsigned skip = (unsigned)(byte_off % 8);
  uint64_t x = xs_state_after(seed, word); /* state after `word` steps */
  uint64_t done = 0;
  while (done < n) {
    x = xs_step(x);
    for (unsigned b = skip; b < 8 && done < n; ++b) buf[done++] = (uint8_t)(x >> (8 * b));
    skip = 0;
  }
  return 0;
}

typedef struct {
  int fd;
  uint64_t seed, begin, end; /* byte range, begin multiple of 8 */
  int err;
} gen_job;

static void* gen_worker(void* arg) {
  gen_job* j = (gen_job*)arg;
  const uint64_t CH = 4ull << 20;
  uint8_t* buf = (uint8_t*)malloc(CH);
  if (!buf) { j->err = ENOMEM; return NULL; }
  uint64_t x = xs_state_after(j->seed, j->begin / 8);
  for (uint64_t off = j->begin; off < j->end; off += CH) {
    uint64_t n = j->end - off < CH ? j->end - off : CH;
    uint64_t w = 0;
    for (; w + 8 <= n; w += 8) {
      x = xs_step(x);
      for (unsigned b = 0; b < 8; ++b) buf[w + b] = (uint8_t)(x >> (8 * b));
    }
    if (w < n) { /* ragged tail: only at the very end of the file */
      x = xs_step(x);
      for (unsigned b = 0; w < n; ++b, ++w) buf[w] = (uint8_t)(x >> (8 * b));
    }
    uint64_t put = 0;
    while (put < n) {
      ssize_t r = pwrite(j->fd, buf + put, n - put, (off_t)(off + put));
      if (r <= 0) { j->err = r < 0 ? errno : EIO; free(buf); return NULL; }
      put += (uint64_t)r;
    }
  }
  free(buf);
  return NULL;
}

/* Write a file of `size` bytes of the stream for `seed`.  Returns 0 or -errno. */
int xs_write_file(const char* path, uint64_t seed, uint64_t size, int threads) {
  if (seed == 0) return -EINVAL;
  if (threads < 1) threads = 1;
  if (threads > 64) threads = 64;
  int fd = open(path, O_CREAT | O_TRUNC | O_WRONLY, 0644);
  if (fd < 0) return -errno;
  if (size && ftruncate(fd, (off_t)size) != 0) { int e = errno; close(fd); return -e; }
  pthread_t tid[64];
  gen_job jobs[64];
  /* each thread's range: the ceiling of size / threads, rounded up to whole MiB,
     so that the ranges cover every byte */
  uint64_t per = ((size + (uint64_t)threads - 1) / (uint64_t)threads + (1ull << 20) - 1) & ~((1ull << 20) - 1);
  if (per == 0) per = 1ull << 20;
  int started = 0, spawn_err = 0;
  for (int t = 0; t < threads; ++t) {
    uint64_t b = per * (uint64_t)t;
    if (b >= size) break;
    uint64_t e = b + per < size ? b + per : size;
    jobs[t] = (gen_job){fd, seed, b, e, 0};
    if (pthread_create(&tid[t], NULL, gen_worker, &jobs[t]) != 0) { spawn_err = EAGAIN; break; }
    ++started;
  }
  int err = spawn_err;
  for (int t = 0; t < started; ++t) {
    pthread_join(tid[t], NULL);
    if (jobs[t].err && !err) err = jobs[t].err;
  }
  if (close(fd) != 0 && !err) err = errno;
  return -err;
}

/* ---------------------------------------------------------------- typed streams
 * Element j of a typed stream uses output word j of the xorshift64 stream
 * (the state after j + 1 steps).
 *   f32:  v = ((x >> 40) * 2^-24) * 2 - 1, uniform in [-1, 1), exact in float.
 *   zipf: u = (x >> 11) * 2^-53; v = the first k with cdf[k] > u, where
 *         cdf[k] = sum_{i<=k} (i+1)^-s / sum_{i<nbins} (i+1)^-s (computed in double).
 */
#include <math.h>

float xs_f32_of(uint64_t x) { return (float)((double)(x >> 40) * (1.0 / 16777216.0) * 2.0 - 1.0); }

typedef struct {
  int fd;
  uint64_t seed, begin, end; /* element range */
  int kind;                  /* 0 f32, 1 zipf */
  const double* cdf;
  uint32_t nbins;
  int err;
} typed_job;

static uint32_t zipf_pick(const double* cdf, uint32_t nbins, uint64_t x) {
  const double u = (double)(x >> 11) * (1.0 / 9007199254740992.0);
  uint32_t lo = 0, hi = nbins - 1; /* first k with cdf[k] > u; cdf[nbins-1] == 1 > u */
  while (lo < hi) {
    uint32_t mid = lo + (hi - lo) / 2;
    if (cdf[mid] > u) hi = mid; else lo = mid + 1;
  }
  return lo;
}

static void* typed_worker(void* arg) {
  typed_job* j = (typed_job*)arg;
  const uint64_t CH = 1u << 20; /* elements per write */
  uint32_t* buf = (uint32_t*)malloc(CH * 4);
  if (!buf) { j->err = ENOMEM; return NULL; }
  uint64_t x = xs_state_after(j->seed, j->begin);
  for (uint64_t e = j->begin; e < j->end; e += CH) {
    uint64_t n = j->end - e < CH ? j->end - e : CH;
    for (uint64_t i = 0; i < n; ++i) {
      x = xs_step(x);
      if (j->kind == 0) {
        float f = xs_f32_of(x);
        memcpy(&buf[i], &f, 4);
      } else {
        buf[i] = zipf_pick(j->cdf, j->nbins, x);
      }
    }
    uint64_t put = 0, bytes = n * 4;
    while (put < bytes) {
      ssize_t r = pwrite(j->fd, (uint8_t*)buf + put, bytes - put, (off_t)(e * 4 + put));
      if (r <= 0) { j->err = r < 0 ? errno : EIO; free(buf); return NULL; }
      put += (uint64_t)r;
    }
  }
  free(buf);
  return NULL;
}

/* cdf of Zipf(s) over nbins values (double), written to out[nbins]. */
int xs_zipf_cdf(double* out, uint32_t nbins, double s) {
  if (!out || nbins == 0) return -EINVAL;
  double acc = 0.0;
  for (uint32_t k = 0; k < nbins; ++k) { acc += pow((double)k + 1.0, -s); out[k] = acc; }
  for (uint32_t k = 0; k < nbins; ++k) out[k] /= acc;
  out[nbins - 1] = 1.0;
  return 0;
}

static int write_typed(const char* path, uint64_t seed, uint64_t n, int threads, int kind, uint32_t nbins, double s) {
  if (seed == 0) return -EINVAL;
  if (threads < 1) threads = 1;
  if (threads > 64) threads = 64;
  double* cdf = NULL;
  if (kind == 1) {
    if (nbins == 0) return -EINVAL;
    cdf = (double*)malloc(sizeof(double) * nbins);
    if (!cdf) return -ENOMEM;
    xs_zipf_cdf(cdf, nbins, s);
  }
  int fd = open(path, O_CREAT | O_TRUNC | O_WRONLY, 0644);
  if (fd < 0) { free(cdf); return -errno; }
  if (n && ftruncate(fd, (off_t)(n * 4)) != 0) { int e = errno; close(fd); free(cdf); return -e; }
  pthread_t tid[64];
  typed_job jobs[64];
  /* each thread's range of values: the ceiling of n / threads, rounded up to whole
     Mi values, so that the ranges cover every value */
  uint64_t per = ((n + (uint64_t)threads - 1) / (uint64_t)threads + (1u << 20) - 1) & ~(uint64_t)((1u << 20) - 1);
  if (per == 0) per = 1u << 20;
  int started = 0, err = 0;
  for (int t = 0; t < threads; ++t) {
    uint64_t b = per * (uint64_t)t;
    if (b >= n) break;
    uint64_t e = b + per < n ? b + per : n;
    jobs[t] = (typed_job){fd, seed, b, e, kind, cdf, nbins, 0};
    if (pthread_create(&tid[t], NULL, typed_worker, &jobs[t]) != 0) { err = EAGAIN; break; }
    ++started;
  }
  for (int t = 0; t < started; ++t) {
    pthread_join(tid[t], NULL);
    if (jobs[t].err && !err) err = jobs[t].err;
  }
  if (close(fd) != 0 && !err) err = errno;
  free(cdf);
  return -err;
}

/* n float32 elements (4n bytes). */
int xs_write_f32(const char* path, uint64_t seed, uint64_t n, int threads) {
  return write_typed(path, seed, n, threads, 0, 0, 0.0);
}

/* n int32 Zipf(s) values over [0, nbins) (4n bytes). */
int xs_write_zipf(const char* path, uint64_t seed, uint64_t n, uint32_t nbins, double s, int threads) {
  return write_typed(path, seed, n, threads, 1, nbins, s);
}
