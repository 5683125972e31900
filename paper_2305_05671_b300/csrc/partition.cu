// Model-based partitioning (Sec. 3.3, Algorithm 1 reader loop, Eq. 1) on the
// GPU: pack + classify + histogram, scan of the fine bins, partition cuts,
// scatter of 16-byte pairs into bin order, and the work items of the sort.
#include "common.cuh"

namespace elsar {
namespace {

inline uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
inline uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }

constexpr int kThreads = 256;
constexpr int kUnroll = 4;

// splitter table -> shared coarse table (every G-th splitter)
__device__ __forceinline__ void load_coarse(const uint64_t* __restrict__ t, uint32_t log2B, uint64_t* ct,
                                            uint32_t* ncoarse, uint32_t* G) {
  const uint32_t B = 1u << log2B;
  const uint32_t nc = B < (uint32_t)kCoarse ? B : (uint32_t)kCoarse;
  const uint32_t g = B / nc;
  for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) ct[i] = t[(uint64_t)i * g];
  *ncoarse = nc;
  *G = g;
  __syncthreads();
}

// Pass A: every record -> (pair in input order, fine bin histogram).
__global__ void __launch_bounds__(kThreads) classify_kernel(const uint8_t* __restrict__ rec, uint64_t n,
                                                            const uint64_t* __restrict__ t, uint32_t log2B,
                                                            Pair* __restrict__ pairs, uint32_t* __restrict__ hist) {
  __shared__ uint64_t ct[kCoarse];
  uint32_t nc, G;
  load_coarse(t, log2B, ct, &nc, &G);
  const uint64_t stride = (uint64_t)gridDim.x * kThreads * kUnroll;
  for (uint64_t i0 = (uint64_t)blockIdx.x * kThreads * kUnroll + threadIdx.x; i0 < n; i0 += stride) {
    Pair p[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      uint64_t i = i0 + (uint64_t)u * kThreads;
      if (i < n) p[u] = load_pair(rec + i * kRecord, (uint32_t)i);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      uint64_t i = i0 + (uint64_t)u * kThreads;
      if (i < n) {
        uint32_t q = fine_bin(t, ct, nc, G, enc9_pair(p[u]));
        pairs[i] = p[u];
        atomicAdd(hist + q, 1u);
      }
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

// Single CTA: bin offsets (exclusive scan of the histogram), scatter cursors, max bin.
__global__ void __launch_bounds__(kScanThreads) scan_bins(const uint32_t* hist, uint32_t log2B,
                                                          uint32_t* __restrict__ bin_off, uint32_t* cursor,
                                                          uint32_t* ctrl) {
  __shared__ uint32_t wsum[33];
  const uint32_t B = 1u << log2B;
  const uint32_t per = (B + kScanThreads - 1) / kScanThreads;
  const uint32_t b = min(B, threadIdx.x * per), e = min(B, b + per);
  uint32_t local = 0, mx = 0;
  for (uint32_t q = b; q < e; ++q) {
    uint32_t h = hist[q];
    local += h;
    mx = max(mx, h);
  }
  uint32_t run;
  uint32_t total = block_exclusive_scan(local, &run, wsum);
  for (uint32_t q = b; q < e; ++q) {
    const uint32_t h = hist[q];  // hist and cursor may be the same array
    bin_off[q] = run;
    cursor[q] = run;
    run += h;
  }
  if (threadIdx.x == 0) bin_off[B] = total;
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
// (> cap pairs) are listed separately.
__global__ void __launch_bounds__(kScanThreads) items_kernel(const uint32_t* __restrict__ bin_off, uint32_t log2B,
                                                             uint32_t cap, uint32_t* item_flag, uint32_t* items,
                                                             uint32_t* oversize, uint32_t* ctrl) {
  __shared__ uint32_t wsum[33];
  const uint32_t B = 1u << log2B;
  const uint32_t W = cap / 2;
  const uint32_t per = (B + kScanThreads - 1) / kScanThreads;
  const uint32_t b = min(B, threadIdx.x * per), e = min(B, b + per);
  uint32_t local = 0;
  for (uint32_t q = b; q < e; ++q) {
    const uint32_t cnt = bin_off[q + 1] - bin_off[q];
    bool f = item_flag[q] != 0 || q == 0 || cnt > W;
    if (!f) {
      const uint32_t pc = bin_off[q] - bin_off[q - 1];
      f = pc > W || (bin_off[q] / W) != (bin_off[q - 1] / W);
    }
    item_flag[q] = f;
    local += f;
  }
  uint32_t run;
  uint32_t total = block_exclusive_scan(local, &run, wsum);
  for (uint32_t q = b; q < e; ++q) {
    if (item_flag[q]) {
      items[run] = q;
      if (bin_off[q + 1] - bin_off[q] > cap) oversize[atomicAdd(ctrl + kNumOversize, 1u)] = run;
      item_flag[q] = run;
      ++run;
    } else {
      item_flag[q] = run - 1;  // item id of every bin
    }
  }
  if (threadIdx.x == 0) {
    items[total] = B;
    ctrl[kNumItems] = total;
  }
}

// Pass B: pairs (input order) -> bin order; slot from an atomic cursor per bin.
__global__ void __launch_bounds__(kThreads) scatter_kernel(const Pair* __restrict__ in, uint64_t n,
                                                           const uint64_t* __restrict__ t, uint32_t log2B,
                                                           uint32_t* __restrict__ cursor, Pair* __restrict__ out) {
  __shared__ uint64_t ct[kCoarse];
  uint32_t nc, G;
  load_coarse(t, log2B, ct, &nc, &G);
  const uint64_t stride = (uint64_t)gridDim.x * kThreads * kUnroll;
  for (uint64_t i0 = (uint64_t)blockIdx.x * kThreads * kUnroll + threadIdx.x; i0 < n; i0 += stride) {
    Pair p[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      uint64_t i = i0 + (uint64_t)u * kThreads;
      if (i < n) p[u] = in[i];
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      uint64_t i = i0 + (uint64_t)u * kThreads;
      if (i < n) {
        uint32_t q = fine_bin(t, ct, nc, G, enc9_pair(p[u]));
        uint32_t slot = atomicAdd(cursor + q, 1u);
        out[slot] = p[u];
      }
    }
  }
}

}  // namespace

cudaError_t partition_records(const PartArgs& a) {
  const uint32_t B = 1u << a.log2B;
  cudaStream_t st = a.stream;
  const int sms = sm_count();
  cudaMemsetAsync(a.cursor, 0, (size_t)B * 4, st);  // the histogram lives in `cursor` until the scan
  cudaMemsetAsync(a.ctrl, 0, 64, st);
  const uint64_t per_block = (uint64_t)kThreads * kUnroll;
  const unsigned grid = (unsigned)umax64(1, umin64((a.n + per_block - 1) / per_block, (uint64_t)sms * 8));
  classify_kernel<<<grid, kThreads, 0, st>>>(a.records, a.n, a.splitters, a.log2B,
                                             static_cast<Pair*>(a.pairs_in_order), a.cursor);
  if (a.ev[0]) cudaEventRecord(a.ev[0], st);
  scan_bins<<<1, kScanThreads, 0, st>>>(a.cursor, a.log2B, a.bin_off, a.cursor, a.ctrl);
  cuts_kernel<<<(a.P + 1 + 255) / 256, 256, 0, st>>>(a.bin_off, a.log2B, a.P, (int)a.balance, a.cuts, a.part_off,
                                                      nullptr);
  if (a.ev[1]) cudaEventRecord(a.ev[1], st);
  scatter_kernel<<<grid, kThreads, 0, st>>>(static_cast<const Pair*>(a.pairs_in_order), a.n, a.splitters, a.log2B,
                                            a.cursor, static_cast<Pair*>(a.pairs));
  if (a.ev[2]) cudaEventRecord(a.ev[2], st);
  *a.launches += 4;
  return cudaGetLastError();
}

cudaError_t build_items(const PartArgs& a) {
  cudaStream_t st = a.stream;
  const uint32_t B = 1u << a.log2B;
  cudaMemsetAsync(a.item_flag, 0, (size_t)B * 4, st);
  cudaMemsetAsync(a.ctrl, 0, 3 * sizeof(uint32_t), st);  // item count, oversize count, queue head
  cuts_kernel<<<(a.P + 1 + 255) / 256, 256, 0, st>>>(a.bin_off, a.log2B, a.P, (int)a.balance, a.cuts, a.part_off,
                                                      a.item_flag);
  items_kernel<<<1, kScanThreads, 0, st>>>(a.bin_off, a.log2B, a.tile_pairs, a.item_flag, a.items, a.oversize,
                                           a.ctrl);
  *a.launches += 2;
  return cudaGetLastError();
}

}  // namespace elsar
