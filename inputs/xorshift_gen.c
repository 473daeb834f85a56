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
  uint64_t per = (size / (uint64_t)threads + (1ull << 20) - 1) & ~((1ull << 20) - 1);
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
