/*
 * Seeded synthetic record generator, CPU side.
 *
 * This module only makes inputs: it holds none of the sort's arithmetic
 * (no key encoding, no model, no partitioning, no ordering).  The same
 * byte-for-byte definition is implemented for the GPU in recgen_cuda.cu;
 * both take the Zipf and permutation tables as data built once on the host
 * (recgen/__init__.py), so integer results are identical by construction.
 *
 * Record i (100 bytes), the shape of the paper's benchmark data (Sec. 7.1:
 * 10-byte key, 90-byte payload, printable ASCII):
 *   [0,10)   key: each byte uniform over 0x20..0x7E, or Zipf(s) over the 95
 *            printable characters with a per-position permutation, or (prefix
 *            skew, the shape of the paper's skewed data, Sec. 7.1) uniform bytes
 *            whose first 6 are replaced by entry floor(log2 i) mod 128 of a table
 *            of 128 printable 6-byte prefixes (entry t, byte p: uniform from
 *            h(t,p,4); record 0 takes entry 0), or (variable length, Sec. 4) a key
 *            of L = 1 + mulhi32(h(i,12,5) >> 32, 10) uniform bytes padded with
 *            0x00 to 10 bytes; with probability d the whole key is a copy of
 *            another record's base key
 *   [10,42)  32 upper-case hex digits of i (128-bit, big-endian, zero padded)
 *   [42,98)  filler 'A' + ((i + j) mod 26), j = 0..55
 *   [98,100) "\r\n"
 *
 * Counter-based randomness: h(i,pos,stream) =
 *   splitmix64(seed * 0x9E3779B97F4A7C15 ^ (i*16 + pos) ^ (stream << 60)),
 * splitmix64 as published by Steele, Lea and Flood (2014) / Vigna.
 */
#include <stdint.h>
#include <pthread.h>
#include <string.h>

#define RG_RECORD 100

static inline uint64_t rg_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static inline uint64_t rg_h(uint64_t seed, uint64_t i, uint64_t pos, uint64_t stream) {
  return rg_splitmix64((seed * 0x9E3779B97F4A7C15ull) ^ (i * 16u + pos) ^ (stream << 60));
}

static inline uint64_t rg_mulhi64(uint64_t a, uint64_t b) {
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
}

typedef struct {
  uint64_t seed;
  uint64_t n_total;     /* size of the record set (duplicate sources are drawn from it) */
  int kind;             /* 0 uniform, 1 zipf, 2 prefix skew, 3 variable length */
  uint64_t dup_thr;     /* duplicate if h(i,10,1) < dup_thr (0 = none) */
  const uint64_t* cum;  /* 94 cumulative Zipf thresholds (fixed point, 2^64 scale) */
  const uint8_t* perm;  /* 10 x 95 per-position permutation of ranks */
} rg_spec;

static inline uint8_t rg_uniform_byte(uint64_t h) { return (uint8_t)(0x20 + (((h >> 32) * 95u) >> 32)); }

static inline uint8_t rg_key_byte(const rg_spec* s, uint64_t i, int pos) {
  if (s->kind == 2 && pos < 6) {
    const uint64_t t = i ? (uint64_t)(63 - __builtin_clzll(i)) & 127u : 0;
    return rg_uniform_byte(rg_h(s->seed, t, (uint64_t)pos, 4));
  }
  if (s->kind == 3) {
    const uint64_t len = 1 + (((rg_h(s->seed, i, 12, 5) >> 32) * 10u) >> 32);
    if ((uint64_t)pos >= len) return 0;
  }
  if (s->kind == 0 || s->kind == 2 || s->kind == 3) {
    uint64_t u = rg_h(s->seed, i, (uint64_t)pos, 0) >> 32;
    return (uint8_t)(0x20 + ((u * 95u) >> 32));
  }
  uint64_t u = rg_h(s->seed, i, (uint64_t)pos, 2);
  /* rank = #{k : cum[k] <= u}, cum ascending */
  int lo = 0, hi = 94;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (s->cum[mid] <= u) lo = mid + 1; else hi = mid;
  }
  return (uint8_t)(0x20 + s->perm[pos * 95 + lo]);
}

static void rg_record(const rg_spec* s, uint64_t i, uint8_t* r) {
  uint64_t src = i;
  if (s->dup_thr && rg_h(s->seed, i, 10, 1) < s->dup_thr)
    src = rg_mulhi64(rg_h(s->seed, i, 11, 1), s->n_total);
  for (int p = 0; p < 10; ++p) r[p] = rg_key_byte(s, src, p);
  static const char hex[] = "0123456789ABCDEF";
  for (int j = 0; j < 16; ++j) r[10 + j] = '0';
  for (int j = 0; j < 16; ++j) r[26 + j] = (uint8_t)hex[(i >> (60 - 4 * j)) & 15];
  for (int j = 0; j < 56; ++j) r[42 + j] = (uint8_t)('A' + (i + (uint64_t)j) % 26);
  r[98] = '\r';
  r[99] = '\n';
}

typedef struct {
  const rg_spec* s;
  uint8_t* out;
  uint64_t i0, i1, base;
} rg_job;

static void* rg_worker(void* arg) {
  rg_job* j = (rg_job*)arg;
  for (uint64_t i = j->i0; i < j->i1; ++i) rg_record(j->s, i, j->out + (i - j->base) * RG_RECORD);
  return 0;
}

/* Records [i0, i0+count) of a set of n_total records into out (count*100 bytes). */
int recgen_cpu(uint8_t* out, uint64_t n_total, uint64_t i0, uint64_t count, uint64_t seed, int kind,
               const uint64_t* cum, const uint8_t* perm, uint64_t dup_thr, int nthreads) {
  rg_spec s = {seed, n_total, kind, dup_thr, cum, perm};
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (count < 65536) nthreads = 1;
  pthread_t th[256];
  rg_job jobs[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].s = &s;
    jobs[t].out = out;
    jobs[t].base = i0;
    jobs[t].i0 = i0 + count * (uint64_t)t / (uint64_t)nthreads;
    jobs[t].i1 = i0 + count * (uint64_t)(t + 1) / (uint64_t)nthreads;
  }
  if (nthreads == 1) {
    rg_worker(&jobs[0]);
    return 0;
  }
  for (int t = 0; t < nthreads; ++t)
    if (pthread_create(&th[t], 0, rg_worker, &jobs[t])) return -1;
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], 0);
  return 0;
}

uint64_t recgen_splitmix64(uint64_t x) { return rg_splitmix64(x); }
