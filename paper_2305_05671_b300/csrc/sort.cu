// Sorting every partition and concatenating (Sec. 3.4, Sec. 3.5, and the
// touch-up of Sec. 4) on the GPU.  A work item is a run of consecutive fine
// bins (model sub-buckets) of one partition holding at most `cap` pairs.  One
// CTA sorts an item in shared memory -- a counting sort on the leading bits
// of the key below the item's common prefix (the model-style placement),
// then a per-run touch-up by insertion sort (bitonic for long runs) -- and
// gathers the 100-byte records of the item, in order, straight into their
// final place in the output, so the partitions come out concatenated with no
// merge.  Items above `cap` pairs (heavy duplicate keys) take a multi-pass
// path: chunk sorts plus merge passes through global memory.
//
// Schedules: PERSISTENT = one launch, CTAs pull items from a global queue
// (oversize items first) -- the GPU form of the paper's dynamic scheduling of
// uneven partitions; PER_PARTITION = one launch per partition.
#include "common.cuh"

namespace elsar {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr int kLongMax = 64;
constexpr uint32_t kSent = 0xFFFFFFFFu;

struct Misc {
  uint64_t red[2][kWarps];
  uint64_t kmin, kmax;
  uint32_t use_lo;
  uint32_t nlong;
  uint32_t long_start[kLongMax], long_len[kLongMax];
  uint32_t item;
  uint64_t split[2];
  uint32_t wsum[33];
};

struct KArgs {
  const uint8_t* in;
  uint8_t* out;
  Pair* pairs;
  Pair* temp;
  const uint32_t* bin_off;
  const uint32_t* items;
  const uint32_t* oversize;
  const uint32_t* part_items;  // per-partition schedule: item range of partition `part`
  uint32_t* ctrl;
  uint32_t cap, part;
  int persistent;
};

__device__ __forceinline__ uint64_t key_of(const Pair& p, bool use_lo) { return use_lo ? p.lo : p.hi; }

__device__ __forceinline__ uint32_t block_scan_excl(uint32_t v, uint32_t* wsum) {
  uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= (uint32_t)d) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < (uint32_t)kWarps ? wsum[lane] : 0;
    uint32_t wi = w;
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= (uint32_t)d) wi += y;
    }
    if (lane < (uint32_t)kWarps) wsum[lane] = wi - w;
  }
  __syncthreads();
  uint32_t r = wsum[warp] + incl - v;
  __syncthreads();
  return r;
}

// min and max of one key field over A[0, m)
__device__ void block_minmax(const Pair* A, uint32_t m, bool use_lo, Misc& ms) {
  uint64_t mn = ~0ull, mx = 0;
  for (uint32_t j = threadIdx.x; j < m; j += kThreads) {
    uint64_t k = key_of(A[j], use_lo);
    mn = min(mn, k);
    mx = max(mx, k);
  }
  for (int d = 16; d; d >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, d));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, d));
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    ms.red[0][warp] = mn;
    ms.red[1][warp] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    uint64_t a = ~0ull, b = 0;
    for (int w = 0; w < kWarps; ++w) {
      a = min(a, ms.red[0][w]);
      b = max(b, ms.red[1][w]);
    }
    ms.kmin = a;
    ms.kmax = b;
  }
  __syncthreads();
}

__device__ __forceinline__ bool idx_less(const Pair* A, uint32_t a, uint32_t b) {
  if (a == kSent) return false;
  if (b == kSent) return true;
  return pair_less(A[a], A[b]);
}

// Bitonic sort of `len` indices perm[start, start+len) by A[.], through scratch (pow2 >= len entries).
__device__ void bitonic_run(const Pair* A, uint16_t* perm, uint32_t start, uint32_t len, uint32_t* scratch) {
  uint32_t m2 = 1;
  while (m2 < len) m2 <<= 1;
  for (uint32_t i = threadIdx.x; i < m2; i += kThreads) scratch[i] = i < len ? perm[start + i] : kSent;
  __syncthreads();
  for (uint32_t k = 2; k <= m2; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < m2; i += kThreads) {
        uint32_t ixj = i ^ j;
        if (ixj > i) {
          uint32_t a = scratch[i], b = scratch[ixj];
          bool up = (i & k) == 0;
          if (idx_less(A, b, a) == up) {
            scratch[i] = b;
            scratch[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (uint32_t i = threadIdx.x; i < len; i += kThreads) perm[start + i] = (uint16_t)scratch[i];
  __syncthreads();
}

// Sort A[0, m) (m <= cap) in shared memory: on return perm[0, m) lists A in
// (hi, lo) order.  cnt has room for cap counters.
__device__ void tile_sort(const Pair* A, uint32_t m, uint32_t* cnt, uint16_t* perm, Misc& ms) {
  if (m <= 1) {
    if (threadIdx.x == 0 && m == 1) perm[0] = 0;
    __syncthreads();
    return;
  }
  block_minmax(A, m, false, ms);
  bool use_lo = ms.kmin == ms.kmax;
  if (use_lo) block_minmax(A, m, true, ms);
  const uint64_t kmin = ms.kmin, span = ms.kmax - ms.kmin;
  uint32_t logD = 0;
  while ((1u << logD) < m) ++logD;
  const uint32_t D = 1u << logD;
  const uint32_t bits = span ? 64 - __clzll((long long)span) : 0;
  const uint32_t shift = bits > logD ? bits - logD : 0;
  for (uint32_t d = threadIdx.x; d < D; d += kThreads) cnt[d] = 0;
  if (threadIdx.x == 0) ms.nlong = 0;
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < m; j += kThreads)
    atomicAdd(cnt + ((key_of(A[j], use_lo) - kmin) >> shift), 1u);
  __syncthreads();
  // exclusive scan of the D digit counters, D/kThreads per thread
  {
    const uint32_t per = (D + kThreads - 1) / kThreads;
    const uint32_t b = min(D, threadIdx.x * per), e = min(D, b + per);
    uint32_t local = 0;
    for (uint32_t d = b; d < e; ++d) local += cnt[d];
    uint32_t run = block_scan_excl(local, ms.wsum);
    for (uint32_t d = b; d < e; ++d) {
      uint32_t c = cnt[d];
      cnt[d] = run;
      run += c;
    }
  }
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < m; j += kThreads) {
    uint32_t pos = atomicAdd(cnt + ((key_of(A[j], use_lo) - kmin) >> shift), 1u);
    perm[pos] = (uint16_t)j;
  }
  __syncthreads();
  // touch-up: cnt[d] is now the end of run d
  for (uint32_t d = threadIdx.x; d < D; d += kThreads) {
    const uint32_t s = d ? cnt[d - 1] : 0, e = cnt[d];
    const uint32_t len = e - s;
    if (len < 2) continue;
    if (len <= 32) {
      for (uint32_t i = s + 1; i < e; ++i) {
        uint16_t v = perm[i];
        const Pair pv = A[v];
        uint32_t k = i;
        while (k > s && pair_less(pv, A[perm[k - 1]])) {
          perm[k] = perm[k - 1];
          --k;
        }
        perm[k] = v;
      }
    } else {
      uint32_t slot = atomicAdd(&ms.nlong, 1u);
      if (slot < (uint32_t)kLongMax) {
        ms.long_start[slot] = s;
        ms.long_len[slot] = len;
      }
    }
  }
  __syncthreads();
  const uint32_t nlong = ms.nlong;
  if (nlong > (uint32_t)kLongMax) {
    bitonic_run(A, perm, 0, m, cnt);  // too many long runs: one network over the whole tile
  } else {
    for (uint32_t r = 0; r < nlong; ++r) bitonic_run(A, perm, ms.long_start[r], ms.long_len[r], cnt);
  }
}

// Gather m records in sorted order into out[o0, o0 + m): warp-cooperative,
// 32 records (800 words) per step, loads and stores both coalesced.
template <typename IdxFn>
__device__ __forceinline__ void gather(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, uint64_t o0,
                                       uint32_t m, IdxFn idx_of) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t* __restrict__ in32 = reinterpret_cast<const uint32_t*>(in);
  uint32_t* __restrict__ out32 = reinterpret_cast<uint32_t*>(out);
  for (uint32_t j0 = warp * 32; j0 < m; j0 += kThreads) {
    const uint32_t nrec = min(32u, m - j0);
    const uint32_t my = lane < nrec ? idx_of(j0 + lane) : 0;
    uint32_t v[25];
#pragma unroll
    for (int it = 0; it < 25; ++it) {
      const uint32_t w = lane + 32u * it;
      const uint32_t r = w / 25u, k = w - 25u * r;
      const uint32_t src = __shfl_sync(0xffffffffu, my, r);
      v[it] = r < nrec ? __ldg(in32 + (uint64_t)src * 25u + k) : 0u;
    }
    uint32_t* dst = out32 + (o0 + j0) * 25u;
#pragma unroll
    for (int it = 0; it < 25; ++it) {
      const uint32_t w = lane + 32u * it;
      if (w < nrec * 25u) dst[w] = v[it];
    }
  }
}

// number of elements of a among the first diag outputs of merge(a, b)
__device__ __forceinline__ uint32_t merge_split(const Pair* a, uint32_t na, const Pair* b, uint32_t nb,
                                                uint32_t diag) {
  uint32_t lo = diag > nb ? diag - nb : 0, hi = diag < na ? diag : na;
  while (lo < hi) {
    uint32_t mid = (lo + hi) >> 1;
    if (!pair_less(b[diag - 1 - mid], a[mid])) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// items above cap: sort cap-sized chunks in place, then merge passes between
// pairs and temp; returns the array holding the sorted run
__device__ const Pair* sort_oversize(const KArgs& k, uint64_t o0, uint32_t m, Pair* A, uint32_t* cnt, uint16_t* perm,
                                     Misc& ms) {
  const uint32_t cap = k.cap;
  Pair* src = k.pairs;
  Pair* dst = k.temp;
  for (uint32_t c0 = 0; c0 < m; c0 += cap) {
    const uint32_t mc = min(cap, m - c0);
    for (uint32_t j = threadIdx.x; j < mc; j += kThreads) A[j] = src[o0 + c0 + j];
    __syncthreads();
    tile_sort(A, mc, cnt, perm, ms);
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < mc; j += kThreads) src[o0 + c0 + j] = A[perm[j]];
    __syncthreads();
  }
  for (uint32_t w = cap; w < m; w *= 2) {
    for (uint32_t t0 = 0; t0 < m; t0 += cap) {
      const uint32_t p0 = (t0 / (2 * w)) * (2 * w);
      const uint32_t a1 = min(m, p0 + w), b1 = min(m, p0 + 2 * w);
      const uint32_t t1 = min(b1, t0 + cap);
      const Pair* ga = src + o0 + p0;
      const Pair* gb = src + o0 + a1;
      if (threadIdx.x < 2) ms.split[threadIdx.x] = merge_split(ga, a1 - p0, gb, b1 - a1, (threadIdx.x ? t1 : t0) - p0);
      __syncthreads();
      const uint32_t ka0 = (uint32_t)ms.split[0], ka1 = (uint32_t)ms.split[1];
      const uint32_t kb0 = (t0 - p0) - ka0, kb1 = (t1 - p0) - ka1;
      const uint32_t na = ka1 - ka0, nb = kb1 - kb0;
      for (uint32_t j = threadIdx.x; j < na; j += kThreads) A[j] = ga[ka0 + j];
      for (uint32_t j = threadIdx.x; j < nb; j += kThreads) A[na + j] = gb[kb0 + j];
      __syncthreads();
      const uint32_t tot = na + nb;
      const uint32_t per = (tot + kThreads - 1) / kThreads;
      const uint32_t d = threadIdx.x * per;
      if (d < tot) {
        uint32_t lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
        while (lo < hi) {
          uint32_t mid = (lo + hi) >> 1;
          if (!pair_less(A[na + d - 1 - mid], A[mid])) lo = mid + 1;
          else hi = mid;
        }
        uint32_t ia = lo, ib = d - lo;
        for (uint32_t t = 0; t < per && d + t < tot; ++t) {
          bool takeA = ib >= nb || (ia < na && !pair_less(A[na + ib], A[ia]));
          dst[o0 + t0 + d + t] = takeA ? A[ia++] : A[na + ib++];
        }
      }
      __syncthreads();
    }
    Pair* tmp = src;
    src = dst;
    dst = tmp;
    __syncthreads();
  }
  return src;
}

__device__ void process_item(const KArgs& k, uint32_t it, Pair* A, uint32_t* cnt, uint16_t* perm, Misc& ms) {
  const uint64_t o0 = k.bin_off[k.items[it]];
  const uint32_t m = k.bin_off[k.items[it + 1]] - (uint32_t)o0;
  if (m == 0) return;
  if (m <= k.cap) {
    for (uint32_t j = threadIdx.x; j < m; j += kThreads) A[j] = k.pairs[o0 + j];
    __syncthreads();
    tile_sort(A, m, cnt, perm, ms);
    __syncthreads();
    gather(k.in, k.out, o0, m, [&](uint32_t j) { return (uint32_t)A[perm[j]].lo; });
  } else {
    const Pair* sorted = sort_oversize(k, o0, m, A, cnt, perm, ms);
    gather(k.in, k.out, o0, m, [&](uint32_t j) { return (uint32_t)sorted[o0 + j].lo; });
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kThreads) sort_gather_kernel(KArgs k) {
  extern __shared__ __align__(16) uint8_t smem[];
  Pair* A = reinterpret_cast<Pair*>(smem);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(smem + (size_t)k.cap * sizeof(Pair));
  uint16_t* perm = reinterpret_cast<uint16_t*>(smem + (size_t)k.cap * (sizeof(Pair) + 4));
  Misc& ms = *reinterpret_cast<Misc*>(smem + (size_t)k.cap * (sizeof(Pair) + 6));
  const uint32_t num_items = k.ctrl[kNumItems];
  if (k.persistent) {
    const uint32_t num_over = k.ctrl[kNumOversize];
    for (;;) {
      if (threadIdx.x == 0) ms.item = atomicAdd(k.ctrl + kQueueHead, 1u);
      __syncthreads();
      const uint32_t j = ms.item;
      __syncthreads();
      if (j >= num_over + num_items) break;
      uint32_t it;
      if (j < num_over) {
        it = k.oversize[j];
      } else {
        it = j - num_over;
        if (k.bin_off[k.items[it + 1]] - k.bin_off[k.items[it]] > k.cap) continue;  // done in the oversize phase
      }
      process_item(k, it, A, cnt, perm, ms);
    }
  } else {
    const uint32_t i0 = k.part_items[k.part], i1 = k.part_items[k.part + 1];
    for (uint32_t it = i0 + blockIdx.x; it < i1; it += gridDim.x) process_item(k, it, A, cnt, perm, ms);
  }
}

// item range of each partition (per-partition schedule): item id of the partition's first bin
__global__ void part_items_kernel(const uint32_t* cuts, const uint32_t* item_of_bin, uint32_t P, uint32_t log2B,
                                  const uint32_t* ctrl, uint32_t* part_items) {
  const uint32_t B = 1u << log2B;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p <= P; p += gridDim.x * blockDim.x)
    part_items[p] = cuts[p] < B ? item_of_bin[cuts[p]] : ctrl[kNumItems];
}

}  // namespace

size_t sort_smem_bytes(uint32_t cap) { return (size_t)cap * (sizeof(Pair) + 6) + sizeof(Misc) + 16; }

cudaError_t sort_items(const SortArgs& a) {
  KArgs k = {};
  k.in = a.records;
  k.out = a.out;
  k.pairs = a.pairs;
  k.temp = a.temp;
  k.bin_off = a.bin_off;
  k.items = a.items;
  k.oversize = a.oversize;
  k.ctrl = a.ctrl;
  k.cap = a.tile_pairs;
  const size_t smem = sort_smem_bytes(a.tile_pairs);
  cudaError_t err = cudaFuncSetAttribute(sort_gather_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sort_gather_kernel, kThreads, smem);
  if (per_sm < 1) per_sm = 1;
  const int sms = sm_count();
  if (a.schedule == 1) {
    k.persistent = 1;
    sort_gather_kernel<<<sms * per_sm, kThreads, smem, a.stream>>>(k);
    *a.launches += 1;
  } else {
    // one launch per partition; part_items computed on the device from the cuts
    uint32_t* part_items = a.ctrl + 64;  // P+1 words reserved after the control block
    part_items_kernel<<<(a.P + 1 + 255) / 256, 256, 0, a.stream>>>(a.cuts, a.item_of_bin, a.P, a.log2B, a.ctrl,
                                                                    part_items);
    k.persistent = 0;
    k.part_items = part_items;
    const int grid = sms * per_sm < 64 ? sms * per_sm : 64;
    for (uint32_t p = 0; p < a.P; ++p) {
      k.part = p;
      sort_gather_kernel<<<grid, kThreads, smem, a.stream>>>(k);
    }
    *a.launches += 1 + a.P;
  }
  return cudaGetLastError();
}

}  // namespace elsar
