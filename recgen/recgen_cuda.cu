// Seeded synthetic record generator, GPU side: the same byte-for-byte
// definition as recgen.c (record layout, counter-based splitmix64 streams,
// Zipf thresholds and per-position permutations passed in as data).  It holds
// none of the sort's arithmetic; it only fills input buffers quickly so that
// 10-100 GB workloads need not cross the host link.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr int kRec = 100;
constexpr int kThreads = 128;

struct Spec {
  uint64_t seed, n_total, dup_thr, i0, count;
  int kind;
  uint64_t cum[94];
  uint8_t perm[10 * 95];
};

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t hrand(uint64_t seed, uint64_t i, uint64_t pos, uint64_t stream) {
  return splitmix64((seed * 0x9E3779B97F4A7C15ull) ^ (i * 16u + pos) ^ (stream << 60));
}

__device__ __forceinline__ uint8_t key_byte(const Spec& s, const uint64_t* cum, const uint8_t* perm,
                                            uint64_t i, int pos) {
  if (s.kind == 2 && pos < 6) {  // prefix skew: entry floor(log2 i) mod 128 of the 6-byte prefix table
    const uint64_t t = i ? (uint64_t)(63 - __clzll((long long)i)) & 127u : 0;
    const uint64_t u = hrand(s.seed, t, (uint64_t)pos, 4) >> 32;
    return (uint8_t)(0x20 + ((u * 95u) >> 32));
  }
  if (s.kind == 3) {  // variable length: 1..10 uniform bytes, then 0x00
    const uint64_t len = 1 + (((hrand(s.seed, i, 12, 5) >> 32) * 10u) >> 32);
    if ((uint64_t)pos >= len) return 0;
  }
  if (s.kind == 0 || s.kind == 2 || s.kind == 3) {
    uint64_t u = hrand(s.seed, i, (uint64_t)pos, 0) >> 32;
    return (uint8_t)(0x20 + ((u * 95u) >> 32));
  }
  uint64_t u = hrand(s.seed, i, (uint64_t)pos, 2);
  int lo = 0, hi = 94;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (cum[mid] <= u) lo = mid + 1; else hi = mid;
  }
  return (uint8_t)(0x20 + perm[pos * 95 + lo]);
}

__global__ void __launch_bounds__(kThreads) gen_kernel(const __grid_constant__ Spec s, uint8_t* out) {
  __shared__ uint64_t cum[94];
  __shared__ uint8_t perm[10 * 95];
  __shared__ __align__(16) uint8_t stage[kThreads * kRec];
  for (int k = threadIdx.x; k < 94; k += kThreads) cum[k] = s.cum[k];
  for (int k = threadIdx.x; k < 950; k += kThreads) perm[k] = s.perm[k];
  __syncthreads();
  const uint64_t tile0 = (uint64_t)blockIdx.x * kThreads;
  const uint64_t local = tile0 + threadIdx.x;
  if (local < s.count) {
    const uint64_t i = s.i0 + local;
    uint8_t* r = stage + threadIdx.x * kRec;
    uint64_t src = i;
    if (s.dup_thr && hrand(s.seed, i, 10, 1) < s.dup_thr) src = __umul64hi(hrand(s.seed, i, 11, 1), s.n_total);
    for (int p = 0; p < 10; ++p) r[p] = key_byte(s, cum, perm, src, p);
    const char* hex = "0123456789ABCDEF";
    for (int j = 0; j < 16; ++j) r[10 + j] = '0';
    for (int j = 0; j < 16; ++j) r[26 + j] = (uint8_t)hex[(i >> (60 - 4 * j)) & 15];
    for (int j = 0; j < 56; ++j) r[42 + j] = (uint8_t)('A' + (i + (uint64_t)j) % 26);
    r[98] = '\r';
    r[99] = '\n';
  }
  __syncthreads();
  // cooperative, coalesced copy of the tile (4-byte words; records are 4-byte aligned)
  uint64_t nrec = s.count - tile0;
  if (nrec > (uint64_t)kThreads) nrec = kThreads;
  const uint32_t words = (uint32_t)nrec * (kRec / 4);
  const uint32_t* src = reinterpret_cast<const uint32_t*>(stage);
  uint32_t* dst = reinterpret_cast<uint32_t*>(out + tile0 * kRec);
  for (uint32_t w = threadIdx.x; w < words; w += kThreads) dst[w] = src[w];
}

}  // namespace

extern "C" int recgen_gpu(void* d_out, uint64_t n_total, uint64_t i0, uint64_t count, uint64_t seed, int kind,
                          const uint64_t* h_cum, const uint8_t* h_perm, uint64_t dup_thr, void* stream) {
  if (count == 0) return 0;
  if (!d_out || (reinterpret_cast<uintptr_t>(d_out) & 3)) return 1;
  Spec s;
  s.seed = seed;
  s.n_total = n_total;
  s.dup_thr = dup_thr;
  s.i0 = i0;
  s.count = count;
  s.kind = kind;
  for (int k = 0; k < 94; ++k) s.cum[k] = h_cum ? h_cum[k] : ~0ull;
  for (int k = 0; k < 950; ++k) s.perm[k] = h_perm ? h_perm[k] : (uint8_t)(k % 95);
  const uint64_t blocks = (count + kThreads - 1) / kThreads;
  gen_kernel<<<(unsigned)blocks, kThreads, 0, (cudaStream_t)stream>>>(s, (uint8_t*)d_out);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
