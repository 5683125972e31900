// Model-based partitioning (Sec. 3.3, Algorithm 1 reader loop, Eq. 1) on the
// GPU: pack + classify + histogram, scan of the fine bins, partition cuts,
// scatter of 16-byte pairs into bin order, and the work items of the sort.
#include "common.cuh"

namespace elsar {
namespace {

inline uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
inline uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

constexpr int kThreads = 256;
constexpr int kUnroll = 8;
constexpr int kTileRecs = kThreads;  // records staged per bulk copy (25,600 bytes)
constexpr int kStages = 2;
constexpr uint32_t kTileBytes = kTileRecs * kRecord;

__device__ __forceinline__ void classify_one(const Pair& key, uint64_t i, const uint64_t* __restrict__ t,
                                             const uint32_t* __restrict__ lut, Pair* __restrict__ pairs,
                                             uint32_t* __restrict__ hist) {
  Pair p = key;
  const uint32_t q = splitter_search(t, lut, enc9_pair(p));
  p.lo |= q;
  pairs[i] = p;
  atomicAdd(hist + q, 1u);
}

__device__ __forceinline__ Pair pair_from_words(uint32_t a, uint32_t b, uint32_t c) {
  Pair p;
  p.hi = ((uint64_t)__byte_perm(a, 0, 0x0123) << 32) | __byte_perm(b, 0, 0x0123);
  p.lo = (uint64_t)__byte_perm(c, 0, 0x4401) << 32;
  return p;
}

// Pass A, TMA form: tiles of 256 records (25,600 bytes, 16-byte aligned when
// the record buffer is) are bulk-copied into shared memory, double buffered
// on mbarriers; each thread packs one key from shared memory, classifies it
// and counts it.  The input-order pair carries {hi, (key bytes 8-9) << 32 | q}.
// Every wait is bounded: on timeout the CTA raises the status word, waits
// (bounded) for its own copies in flight and leaves.
__global__ void __launch_bounds__(kThreads) classify_tma_kernel(const uint8_t* __restrict__ rec, uint64_t n,
                                                                const uint64_t* __restrict__ t,
                                                                const uint32_t* __restrict__ lut,
                                                                Pair* __restrict__ pairs, uint32_t* __restrict__ hist,
                                                                uint32_t* ctrl) {
  extern __shared__ __align__(128) uint8_t buf[];  // kStages x kTileBytes
  __shared__ uint64_t bar[kStages];
  const uint64_t ntiles = n / kTileRecs;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t issued[kStages] = {};  // copies issued per stage (thread 0)
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      const uint64_t k = blockIdx.x + (uint64_t)s * gridDim.x;
      if (k < ntiles) {
        mbar_expect_tx(&bar[s], kTileBytes);
        bulk_g2s(buf + s * kTileBytes, rec + k * kTileBytes, kTileBytes, &bar[s]);
        issued[s] = 1;
      }
    }
  }
  bool failed = false;
  uint32_t j = 0;
  for (uint64_t k = blockIdx.x; k < ntiles; k += gridDim.x, ++j) {
    const int s = j % kStages;
    const uint32_t parity = (j / kStages) & 1;
    const bool ok = mbar_wait(&bar[s], parity, kWaitLimitCycles);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    const uint32_t* w = reinterpret_cast<const uint32_t*>(buf + s * kTileBytes + threadIdx.x * kRecord);
    const uint64_t i = k * kTileRecs + threadIdx.x;
    classify_one(pair_from_words(w[0], w[1], w[2]), i, t, lut, pairs, hist);
    __syncthreads();  // every thread is done with this stage
    if (threadIdx.x == 0) {
      const uint64_t k2 = k + (uint64_t)kStages * gridDim.x;
      if (k2 < ntiles) {
        fence_proxy_async();
        mbar_expect_tx(&bar[s], kTileBytes);
        bulk_g2s(buf + s * kTileBytes, rec + k2 * kTileBytes, kTileBytes, &bar[s]);
        ++issued[s];
      }
    }
  }
  if (failed) {
    if (threadIdx.x == 0) {
      atomicOr(ctrl + kStatusWord, 1u);
      // copies still in flight target this CTA's shared memory: wait for them, bounded
      for (int s = 0; s < kStages; ++s) {
        // stage s completed (j_s) phases so far; its last issued copy ends phase issued[s]-1
        if (issued[s]) mbar_wait(&bar[s], (issued[s] - 1) & 1, kWaitLimitCycles);
      }
    }
    return;
  }
  // ragged tail (n mod 256 records): plain loads
  for (uint64_t i = ntiles * kTileRecs + blockIdx.x * (uint64_t)kThreads + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * kThreads)
    classify_one(load_pair(rec + i * kRecord, 0), i, t, lut, pairs, hist);
}

// Pass A, plain form (record buffers that are not 16-byte aligned).
__global__ void __launch_bounds__(kThreads) classify_kernel(const uint8_t* __restrict__ rec, uint64_t n,
                                                            const uint64_t* __restrict__ t,
                                                            const uint32_t* __restrict__ lut,
                                                            Pair* __restrict__ pairs, uint32_t* __restrict__ hist) {
  const uint64_t stride = (uint64_t)gridDim.x * kThreads * kUnroll;
  for (uint64_t i0 = (uint64_t)blockIdx.x * kThreads * kUnroll + threadIdx.x; i0 < n; i0 += stride) {
    Pair p[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint64_t i = i0 + (uint64_t)u * kThreads;
      if (i < n) p[u] = load_pair(rec + i * kRecord, 0);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint64_t i = i0 + (uint64_t)u * kThreads;
      if (i < n) classify_one(p[u], i, t, lut, pairs, hist);
    }
  }
}

constexpr int kScanThreads = 1024;

// block-wide exclusive scan of one value per thread; returns the total
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* excl, uint32_t* wsum) {
  uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= (uint32_t)d) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t nw = blockDim.x >> 5;
    uint32_t w = lane < nw ? wsum[lane] : 0;
    uint32_t wi = w;
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= (uint32_t)d) wi += y;
    }
    if (lane < nw) wsum[lane] = wi - w;
    if (lane == 31) wsum[32] = wi;
  }
  __syncthreads();
  *excl = wsum[warp] + incl - v;
  uint32_t total = wsum[32];
  __syncthreads();
  return total;
}

// Single CTA: bin offsets (exclusive scan of the histogram), scatter cursors,
// max bin.  Coalesced tiles of kScanThreads bins with a running carry.
__global__ void __launch_bounds__(kScanThreads) scan_bins(const uint32_t* hist, uint32_t B,
                                                          uint32_t* __restrict__ bin_off, uint32_t* cursor,
                                                          uint32_t* ctrl) {
  __shared__ uint32_t wsum[33];
  __shared__ uint32_t carry_sh;
  if (threadIdx.x == 0) carry_sh = 0;
  uint32_t mx = 0;
  __syncthreads();
  for (uint32_t base = 0; base < B; base += kScanThreads) {
    const uint32_t q = base + threadIdx.x;
    const uint32_t h = q < B ? hist[q] : 0;  // hist and cursor may be the same array
    mx = max(mx, h);
    uint32_t excl;
    const uint32_t tot = block_exclusive_scan(h, &excl, wsum);
    const uint32_t carry = carry_sh;
    if (q < B) {
      bin_off[q] = carry + excl;
      cursor[q] = carry + excl;
    }
    __syncthreads();
    if (threadIdx.x == 0) carry_sh = carry + tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) bin_off[B] = carry_sh;
  for (int d = 16; d; d >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, d));
  if ((threadIdx.x & 31) == 0) atomicMax(ctrl + kMaxBin, mx);
}

// Partition cuts.  Paper rule: c_p = p * B / P.  Refined rule: the boundary t
// whose cumulative count C(t) is closest to p*N/P, ties to the smaller t.
__global__ void cuts_kernel(const uint32_t* __restrict__ bin_off, uint32_t log2B, uint32_t P, int balance,
                            uint32_t* __restrict__ cuts, uint64_t* __restrict__ part_off, uint32_t* item_flag) {
  const uint32_t B = 1u << log2B;
  const uint64_t N = bin_off[B];
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p <= P; p += gridDim.x * blockDim.x) {
    uint32_t c;
    if (p == 0) c = 0;
    else if (p == P) c = B;
    else if (!balance) c = p * (B / P);
    else {
      const int64_t target = (int64_t)p * (int64_t)N;
      // t1 = first t with P*C(t) >= target
      uint32_t lo = 0, hi = B;
      while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if ((int64_t)P * bin_off[mid] >= target) hi = mid;
        else lo = mid + 1;
      }
      const uint32_t t1 = lo;
      if (t1 == 0) c = 0;
      else {
        const int64_t dA = target - (int64_t)P * bin_off[t1 - 1];
        const int64_t dB = (int64_t)P * bin_off[t1] - target;
        if (dB < dA) c = t1;
        else {  // smallest t with C(t) == C(t1 - 1)
          const uint32_t v = bin_off[t1 - 1];
          uint32_t l2 = 0, h2 = t1 - 1;
          while (l2 < h2) {
            uint32_t mid = (l2 + h2) >> 1;
            if (bin_off[mid] >= v) h2 = mid;
            else l2 = mid + 1;
          }
          c = l2;
        }
      }
    }
    cuts[p] = c;
    part_off[p] = bin_off[c];
    if (item_flag && p > 0 && p < P && c < B) item_flag[c] = 1u;
  }
}

// Single CTA: work items = runs of consecutive fine bins.  A bin starts a new
// item if it starts a partition, is not "small" (> W = cap/2 pairs), follows a
// bin that is not small, or its start offset enters a new W-window; a run of
// small bins inside one window holds < 2W = cap pairs.  Oversize bins
// (> cap pairs) are listed separately.  item_flag becomes the item id of
// every bin.  Coalesced tiles with a running carry.
__global__ void __launch_bounds__(kScanThreads) items_kernel(const uint32_t* __restrict__ bin_off, uint32_t B,
                                                             uint32_t cap, uint32_t* item_flag, uint32_t* items,
                                                             uint32_t* oversize, uint32_t* ctrl) {
  __shared__ uint32_t wsum[33];
  __shared__ uint32_t carry_sh;
  const uint32_t W = cap / 2;
  if (threadIdx.x == 0) carry_sh = 0;
  __syncthreads();
  for (uint32_t base = 0; base < B; base += kScanThreads) {
    const uint32_t q = base + threadIdx.x;
    uint32_t f = 0;
    if (q < B) {
      const uint32_t o = bin_off[q], cnt = bin_off[q + 1] - o;
      f = item_flag[q] != 0 || q == 0 || cnt > W;
      if (!f) {
        const uint32_t po = bin_off[q - 1];
        f = (o - po) > W || (o / W) != (po / W);
      }
    }
    uint32_t excl;
    const uint32_t tot = block_exclusive_scan(f, &excl, wsum);
    const uint32_t id = carry_sh + excl;
    if (q < B) {
      if (f) {
        items[id] = q;
        if (bin_off[q + 1] - bin_off[q] > cap) oversize[atomicAdd(ctrl + kNumOversize, 1u)] = id;
        item_flag[q] = id;
      } else {
        item_flag[q] = id - 1;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) carry_sh += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    items[carry_sh] = B;
    ctrl[kNumItems] = carry_sh;
  }
}

// Pass B: pairs (input order) -> bin order; slot from an atomic cursor per
// bin; the fine bin rides in the pair, the record index replaces it.
__global__ void __launch_bounds__(kThreads) scatter_kernel(const Pair* __restrict__ in, uint64_t n,
                                                           uint32_t* __restrict__ cursor, Pair* __restrict__ out) {
  const uint64_t stride = (uint64_t)gridDim.x * kThreads * kUnroll;
  for (uint64_t i0 = (uint64_t)blockIdx.x * kThreads * kUnroll + threadIdx.x; i0 < n; i0 += stride) {
    Pair p[kUnroll];
    uint32_t slot[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint64_t i = i0 + (uint64_t)u * kThreads;
      if (i < n) p[u] = in[i];
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint64_t i = i0 + (uint64_t)u * kThreads;
      if (i < n) slot[u] = atomicAdd(cursor + (uint32_t)p[u].lo, 1u);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint64_t i = i0 + (uint64_t)u * kThreads;
      if (i < n) {
        Pair o;
        o.hi = p[u].hi;
        o.lo = (p[u].lo & 0xFFFFFFFF00000000ull) | (uint32_t)i;
        out[slot[u]] = o;
      }
    }
  }
}

// ---------------------------------------------------------------- many record sets at once
__device__ __forceinline__ uint32_t upper_set(const uint64_t* __restrict__ off, uint32_t K, uint64_t g) {
  uint32_t lo = 0, hi = K - 1;  // largest k with off[k] <= g
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Pass A over K record sets: record i of set k goes to global pair slot
// poff[k] + i with the set's fine bin tbase[k] + q (binary search over the
// set's own splitters).
__global__ void __launch_bounds__(kThreads) classify_batch_kernel(const uint8_t* const* __restrict__ ins,
                                                                  const uint64_t* __restrict__ poff, uint32_t K,
                                                                  const uint64_t* __restrict__ t,
                                                                  const uint64_t* __restrict__ tbase,
                                                                  const uint32_t* __restrict__ log2B,
                                                                  Pair* __restrict__ pairs, uint32_t* __restrict__ hist) {
  const uint64_t N = poff[K];
  for (uint64_t g = blockIdx.x * (uint64_t)kThreads + threadIdx.x; g < N; g += (uint64_t)gridDim.x * kThreads) {
    const uint32_t k = upper_set(poff, K, g);
    const uint64_t i = g - poff[k];
    Pair p = load_pair(ins[k] + i * kRecord, 0);
    const uint64_t x = enc9_pair(p);
    const uint64_t* tk = t + tbase[k];
    uint32_t lo = 0, hi = (1u << log2B[k]) - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (__ldg(tk + mid) <= x) lo = mid;
      else hi = mid - 1;
    }
    const uint32_t q = (uint32_t)tbase[k] + lo;
    p.lo |= q;
    pairs[g] = p;
    atomicAdd(hist + q, 1u);
  }
}

// Pass B over K record sets: the pair's index becomes the index within its set.
__global__ void __launch_bounds__(kThreads) scatter_batch_kernel(const Pair* __restrict__ in,
                                                                 const uint64_t* __restrict__ poff, uint32_t K,
                                                                 uint32_t* __restrict__ cursor, Pair* __restrict__ out) {
  const uint64_t N = poff[K];
  for (uint64_t g = blockIdx.x * (uint64_t)kThreads + threadIdx.x; g < N; g += (uint64_t)gridDim.x * kThreads) {
    const Pair p = in[g];
    const uint32_t slot = atomicAdd(cursor + (uint32_t)p.lo, 1u);
    const uint32_t k = upper_set(poff, K, g);
    Pair o;
    o.hi = p.hi;
    o.lo = (p.lo & 0xFFFFFFFF00000000ull) | (uint32_t)(g - poff[k]);
    out[slot] = o;
  }
}

// every set's first bin starts a work item (items never span two sets)
__global__ void mark_set_starts(const uint64_t* __restrict__ tbase, uint32_t K, uint32_t* item_flag) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x)
    item_flag[tbase[k]] = 1u;
}

}  // namespace

cudaError_t partition_batch(const BatchPartArgs& a) {
  cudaStream_t st = a.stream;
  const int sms = sm_count();
  cudaMemsetAsync(a.cursor, 0, (size_t)a.B * 4, st);
  cudaMemsetAsync(a.ctrl, 0, 32 * sizeof(uint32_t), st);
  cudaMemsetAsync(a.item_flag, 0, (size_t)a.B * 4, st);
  const unsigned grid = (unsigned)sms * 8;
  classify_batch_kernel<<<grid, kThreads, 0, st>>>(a.ins, a.poff, a.K, a.splitters, a.tbase, a.log2B, a.pairs_in_order,
                                                  a.cursor);
  scan_bins<<<1, kScanThreads, 0, st>>>(a.cursor, a.B, a.bin_off, a.cursor, a.ctrl);
  scatter_batch_kernel<<<grid, kThreads, 0, st>>>(a.pairs_in_order, a.poff, a.K, a.cursor, a.pairs);
  mark_set_starts<<<(a.K + 255) / 256, 256, 0, st>>>(a.tbase, a.K, a.item_flag);
  items_kernel<<<1, kScanThreads, 0, st>>>(a.bin_off, a.B, a.tile_pairs, a.item_flag, a.items, a.oversize, a.ctrl);
  *a.launches += 5;
  return cudaGetLastError();
}

cudaError_t partition_records(const PartArgs& a) {
  const uint32_t B = 1u << a.log2B;
  cudaStream_t st = a.stream;
  const int sms = sm_count();
  cudaMemsetAsync(a.cursor, 0, (size_t)B * 4, st);  // the histogram lives in `cursor` until the scan
  cudaMemsetAsync(a.ctrl, 0, 32 * sizeof(uint32_t), st);
  const uint64_t per_block = (uint64_t)kThreads * kUnroll;
  const uint64_t blocks = (a.n + per_block - 1) / per_block;
  int occ_s = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_s, scatter_kernel, kThreads, 0);
  const unsigned grid_s = (unsigned)umax64(1, umin64(blocks, (uint64_t)sms * (occ_s > 0 ? occ_s : 1)));
  Pair* pin = static_cast<Pair*>(a.pairs_in_order);
  if ((reinterpret_cast<uintptr_t>(a.records) & 15) == 0) {
    const size_t smem = (size_t)kStages * kTileBytes;
    cudaFuncSetAttribute(classify_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, classify_tma_kernel, kThreads, smem);
    const uint64_t tiles = a.n / kTileRecs;
    const unsigned grid = (unsigned)umax64(1, umin64(tiles, (uint64_t)sms * (occ > 0 ? occ : 1)));
    classify_tma_kernel<<<grid, kThreads, smem, st>>>(a.records, a.n, a.splitters, a.lut, pin, a.cursor, a.ctrl);
  } else {
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, classify_kernel, kThreads, 0);
    const unsigned grid = (unsigned)umax64(1, umin64(blocks, (uint64_t)sms * (occ > 0 ? occ : 1)));
    classify_kernel<<<grid, kThreads, 0, st>>>(a.records, a.n, a.splitters, a.lut, pin, a.cursor);
  }
  if (a.ev[0]) cudaEventRecord(a.ev[0], st);
  scan_bins<<<1, kScanThreads, 0, st>>>(a.cursor, B, a.bin_off, a.cursor, a.ctrl);
  cuts_kernel<<<(a.P + 1 + 255) / 256, 256, 0, st>>>(a.bin_off, a.log2B, a.P, (int)a.balance, a.cuts, a.part_off,
                                                      nullptr);
  if (a.ev[1]) cudaEventRecord(a.ev[1], st);
  scatter_kernel<<<grid_s, kThreads, 0, st>>>(static_cast<const Pair*>(a.pairs_in_order), a.n, a.cursor,
                                            static_cast<Pair*>(a.pairs));
  if (a.ev[2]) cudaEventRecord(a.ev[2], st);
  *a.launches += 4;
  return cudaGetLastError();
}

cudaError_t classify_accumulate(const PartArgs& a) {
  cudaStream_t st = a.stream;
  const int sms = sm_count();
  Pair* pin = static_cast<Pair*>(a.pairs_in_order);
  if ((reinterpret_cast<uintptr_t>(a.records) & 15) == 0) {
    const size_t smem = (size_t)kStages * kTileBytes;
    cudaFuncSetAttribute(classify_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, classify_tma_kernel, kThreads, smem);
    const uint64_t tiles = a.n / kTileRecs;
    const unsigned grid = (unsigned)umax64(1, umin64(tiles, (uint64_t)sms * (occ > 0 ? occ : 1)));
    classify_tma_kernel<<<grid, kThreads, smem, st>>>(a.records, a.n, a.splitters, a.lut, pin, a.cursor, a.ctrl);
  } else {
    const uint64_t per_block = (uint64_t)kThreads * kUnroll;
    const unsigned grid = (unsigned)umax64(1, umin64((a.n + per_block - 1) / per_block, (uint64_t)sms * 4));
    classify_kernel<<<grid, kThreads, 0, st>>>(a.records, a.n, a.splitters, a.lut, pin, a.cursor);
  }
  *a.launches += 1;
  return cudaGetLastError();
}

cudaError_t scan_and_cut(const PartArgs& a) {
  const uint32_t B = 1u << a.log2B;
  scan_bins<<<1, kScanThreads, 0, a.stream>>>(a.cursor, B, a.bin_off, a.cursor, a.ctrl);
  cuts_kernel<<<(a.P + 1 + 255) / 256, 256, 0, a.stream>>>(a.bin_off, a.log2B, a.P, (int)a.balance, a.cuts,
                                                           a.part_off, nullptr);
  *a.launches += 2;
  return cudaGetLastError();
}

cudaError_t build_items(const PartArgs& a) {
  cudaStream_t st = a.stream;
  const uint32_t B = 1u << a.log2B;
  cudaMemsetAsync(a.item_flag, 0, (size_t)B * 4, st);
  cudaMemsetAsync(a.ctrl, 0, 3 * sizeof(uint32_t), st);  // item count, oversize count, queue head
  cuts_kernel<<<(a.P + 1 + 255) / 256, 256, 0, st>>>(a.bin_off, a.log2B, a.P, (int)a.balance, a.cuts, a.part_off,
                                                      a.item_flag);
  items_kernel<<<1, kScanThreads, 0, st>>>(a.bin_off, B, a.tile_pairs, a.item_flag, a.items, a.oversize,
                                           a.ctrl);
  *a.launches += 2;
  return cudaGetLastError();
}

}  // namespace elsar
