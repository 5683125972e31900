// Model-based partitioning (Sec. 3.3, Algorithm 1 reader loop, Eq. 1) on the
// GPU: pack + classify + histogram, scan of the fine bins, partition cuts,
// scatter of 16-byte pairs into bin order (two passes with their cursors in
// shared memory: coarse bins, then the fine bins inside each), and the work
// items of the sort.
#include "common.cuh"

namespace elsar {
namespace {

inline uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
inline uint64_t umax64(uint64_t a, uint64_t b) { return a > b ? a : b; }
// log2 of a power of two
inline uint32_t ilog2(uint64_t v) { return 63 - __builtin_clzll(v); }

constexpr int kThreads = 256;
constexpr int kUnroll = 8;
constexpr int kTileRecs = kThreads;  // records staged per bulk copy (25,600 bytes)
constexpr uint32_t kTileBytes = kTileRecs * kRecord;

__device__ __forceinline__ uint32_t classify_one(const Pair& key, uint64_t i, const uint64_t* __restrict__ t,
                                                 const uint32_t* __restrict__ lut, Pair* __restrict__ pairs,
                                                 uint32_t* __restrict__ hist) {
  Pair p = key;
  const uint32_t q = splitter_search(t, lut, enc9_pair(p));
  p.lo |= q;
  pairs[i] = p;
  atomicAdd(hist + q, 1u);
  return q;
}

__device__ __forceinline__ Pair pair_from_words(uint32_t a, uint32_t b, uint32_t c, const KeyMask& km) {
  Pair p;
  p.hi = (((uint64_t)__byte_perm(a, 0, 0x0123) << 32) | __byte_perm(b, 0, 0x0123)) & km.hi;
  p.lo = ((uint64_t)__byte_perm(c, 0, 0x4401) << 32) & km.lo;
  return p;
}

// Pass A, TMA form: tiles of 256 records (25,600 bytes, 16-byte aligned when
// the record buffer is) are bulk-copied into shared memory, NS tiles in
// flight on their own mbarriers.  A round takes the CTA's next NS tiles:
// every thread copies the key words of its KPT = NS*256/NT records out of the
// stages, the stages are refilled with the following round's tiles at once,
// and the thread then packs, classifies and counts its keys -- the splitter
// searches run in lockstep, so their loads overlap one another and the
// refill.  The input-order pair carries {hi, (key bytes 8-9) << 32 | q}.
// Every wait is bounded: on timeout the CTA raises the status word, waits
// (bounded) for its own copies in flight and leaves.
template <int NT, int NS>
__global__ void __launch_bounds__(NT) classify_tma_kernel(const uint8_t* __restrict__ rec, KeyMask km, uint64_t n,
                                                          const uint64_t* __restrict__ t,
                                                          const uint32_t* __restrict__ lut, Pair* __restrict__ pairs,
                                                          uint32_t* __restrict__ hist, uint32_t* ctrl, uint32_t cshift,
                                                          uint32_t* __restrict__ seg_hist, uint32_t seg_stride,
                                                          long long wait_limit) {
  constexpr int KPT = NS * kTileRecs / NT;
  extern __shared__ __align__(128) uint8_t buf[];  // NS x kTileBytes
  __shared__ uint64_t bar[NS];
  __shared__ uint32_t hc[kMaxCoarse];  // this CTA's counts per coarse bin
  const uint64_t ntiles = n / kTileRecs;
  const uint64_t G = gridDim.x;
  for (uint32_t c = threadIdx.x; c < kMaxCoarse; c += NT) hc[c] = 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t issued[NS] = {};  // copies issued per stage (thread 0)
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      const uint64_t k = blockIdx.x + (uint64_t)s * G;
      if (k < ntiles) {
        mbar_expect_tx(&bar[s], kTileBytes);
        bulk_g2s(buf + s * kTileBytes, rec + k * kTileBytes, kTileBytes, &bar[s]);
        issued[s] = 1;
      }
    }
  }
  bool failed = false;
  uint32_t round = 0;
  for (uint64_t k0 = blockIdx.x; k0 < ntiles; k0 += NS * G, ++round) {
    uint32_t w[KPT][3];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
      const int slot = threadIdx.x + j * NT, s = slot / kTileRecs, r = slot % kTileRecs;
      w[j][0] = w[j][1] = w[j][2] = 0x20202020u;  // a key of spaces where the round has no tile
      if (k0 + s * G < ntiles) {
        ok = ok && mbar_wait(&bar[s], round & 1, wait_limit);
        const uint32_t* ws = reinterpret_cast<const uint32_t*>(buf + s * kTileBytes + r * kRecord);
        w[j][0] = ws[0];
        w[j][1] = ws[1];
        w[j][2] = ws[2];
      }
    }
    if (__syncthreads_or(!ok)) {  // every thread is also done reading the stages
      failed = true;
      break;
    }
    if (threadIdx.x == 0) {
      fence_proxy_async();
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        const uint64_t k2 = k0 + (uint64_t)(s + NS) * G;
        if (k2 < ntiles) {
          mbar_expect_tx(&bar[s], kTileBytes);
          bulk_g2s(buf + s * kTileBytes, rec + k2 * kTileBytes, kTileBytes, &bar[s]);
          ++issued[s];
        }
      }
    }
    Pair pr[KPT];
    uint64_t x[KPT];
    uint32_t lo[KPT], hi[KPT];
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
      const int slot = threadIdx.x + j * NT, s = slot / kTileRecs;
      pr[j] = pair_from_words(w[j][0], w[j][1], w[j][2], km);
      x[j] = enc9_pair(pr[j]);
      lo[j] = hi[j] = 0;
      if (k0 + s * G < ntiles) lut_range(lut, x[j], lo[j], hi[j]);
    }
    for (;;) {
      bool more = false;
#pragma unroll
      for (int j = 0; j < KPT; ++j) {
        if (lo[j] < hi[j]) {
          const uint32_t mid = (lo[j] + hi[j] + 1) >> 1;
          if (__ldg(t + mid) <= x[j]) lo[j] = mid;
          else hi[j] = mid - 1;
          more = true;
        }
      }
      if (!more) break;
    }
#pragma unroll
    for (int j = 0; j < KPT; ++j) {
      const int slot = threadIdx.x + j * NT, s = slot / kTileRecs, r = slot % kTileRecs;
      const uint64_t k = k0 + s * G;
      if (k < ntiles) {
        const uint32_t q = lo[j];
        Pair p = pr[j];
        p.lo |= q;
        pairs[k * kTileRecs + r] = p;
        atomicAdd(hist + q, 1u);
        if (seg_hist) atomicAdd(&hc[q >> cshift], 1u);
      }
    }
  }
  if (failed) {
    if (threadIdx.x == 0) {
      atomicOr(ctrl + kStatusWord, 1u);
      // copies still in flight target this CTA's shared memory: wait for them, bounded
      for (int s = 0; s < NS; ++s) {
        // the last copy issued on stage s completes that stage's phase issued[s]-1
        if (issued[s]) mbar_wait(&bar[s], (issued[s] - 1) & 1, kWaitLimitCycles);
      }
    }
    return;
  }
  // ragged tail (n mod 256 records, so CTA 0 alone): plain loads
  for (uint64_t i = ntiles * kTileRecs + blockIdx.x * (uint64_t)NT + threadIdx.x; i < n && blockIdx.x == 0;
       i += (uint64_t)NT) {
    const uint32_t q = classify_one(load_pair(rec + i * kRecord, 0, km), i, t, lut, pairs, hist);
    if (seg_hist) atomicAdd(&hc[q >> cshift], 1u);
  }
  if (seg_hist) {
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < kMaxCoarse; c += NT) seg_hist[c * seg_stride + blockIdx.x] = hc[c];
  }
}

#ifndef ELSAR_CLASSIFY_NT
#define ELSAR_CLASSIFY_NT 256
#endif
#ifndef ELSAR_CLASSIFY_NS
#define ELSAR_CLASSIFY_NS 2
#endif
constexpr int kClassifyThreads = ELSAR_CLASSIFY_NT;
constexpr int kClassifyStages = ELSAR_CLASSIFY_NS;
#define CLASSIFY_TMA classify_tma_kernel<kClassifyThreads, kClassifyStages>

// Pass A, plain form (record buffers that are not 16-byte aligned).
__global__ void __launch_bounds__(kThreads) classify_kernel(const uint8_t* __restrict__ rec, KeyMask km, uint64_t n,
                                                            const uint64_t* __restrict__ t,
                                                            const uint32_t* __restrict__ lut,
                                                            Pair* __restrict__ pairs, uint32_t* __restrict__ hist,
                                                            uint32_t cshift, uint32_t* __restrict__ seg_hist,
                                                            uint32_t seg_stride) {
  __shared__ uint32_t hc[kMaxCoarse];
  for (uint32_t c = threadIdx.x; c < kMaxCoarse; c += kThreads) hc[c] = 0;
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * kThreads * kUnroll;
  for (uint64_t i0 = (uint64_t)blockIdx.x * kThreads * kUnroll + threadIdx.x; i0 < n; i0 += stride) {
    Pair p[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint64_t i = i0 + (uint64_t)u * kThreads;
      if (i < n) p[u] = load_pair(rec + i * kRecord, 0, km);
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint64_t i = i0 + (uint64_t)u * kThreads;
      if (i < n) {
        const uint32_t q = classify_one(p[u], i, t, lut, pairs, hist);
        if (seg_hist) atomicAdd(&hc[q >> cshift], 1u);
      }
    }
  }
  if (seg_hist) {
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < kMaxCoarse; c += kThreads) seg_hist[c * seg_stride + blockIdx.x] = hc[c];
  }
}


constexpr int kTileChunks = 16;  // 32-element chunks per warp and tile of the single-CTA scans

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
  const uint32_t lane = threadIdx.x & 31;
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= (uint32_t)d) v += y;
  }
  return v;
}

// exclusive scan of the warps' totals: wsum[w] in, wsum[w] = the warps
// before w out, wsum[32] = the tile's total (two barriers)
__device__ __forceinline__ void scan_warp_totals(uint32_t* wsum) {
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31;
  if (threadIdx.x < 32) {
    const uint32_t nw = blockDim.x >> 5;
    const uint32_t w = lane < nw ? wsum[lane] : 0;
    const uint32_t wi = warp_incl_scan(w);
    if (lane < nw) wsum[lane] = wi - w;
    if (lane == 31) wsum[32] = wi;
  }
  __syncthreads();
}

// Bin offsets (exclusive scan of the histogram), scatter cursors, max bin,
// in two launches over tiles of kTsTile bins (one CTA each): tile sums, then
// every CTA adds the sums of the tiles before its own and scans its tile.
// Warp w of a tile scans chunks of 32 consecutive bins (coalesced) across its
// 32 * kTileChunks bins, then the warps' totals are scanned.  Each bin is read
// and written by one thread (hist and cursor may be the same array); no CTA
// waits for another.
constexpr int kTsThreads = 256;
constexpr uint32_t kTsTile = kTsThreads * kTileChunks;  // 4096 bins

// sum of one value per thread over the CTA, returned to every thread
// (red: 33 words; three barriers, so it may be called again at once)
__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t* red) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = 16; d; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    uint32_t x = lane < (blockDim.x >> 5) ? red[lane] : 0;
    for (int d = 16; d; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
    if (lane == 0) red[32] = x;
  }
  __syncthreads();
  return red[32];
}

__global__ void __launch_bounds__(kTsThreads) bin_tile_sums(const uint32_t* __restrict__ hist, uint32_t B,
                                                            uint32_t* __restrict__ tsum, uint32_t* ctrl) {
  __shared__ uint32_t red[33];
  if (ctrl[kStatusWord]) return;  // classify gave up: nothing downstream runs
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t w0 = blockIdx.x * kTsTile + warp * 32 * kTileChunks;
  uint32_t sum = 0, mx = 0;
#pragma unroll
  for (int j = 0; j < kTileChunks; ++j) {
    const uint32_t q = w0 + j * 32 + lane;
    const uint32_t h = q < B ? hist[q] : 0;
    sum += h;
    mx = max(mx, h);
  }
  for (int d = 16; d; d >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, d));
  if (lane == 0) atomicMax(ctrl + kMaxBin, mx);
  sum = block_sum(sum, red);
  if (threadIdx.x == 0) tsum[blockIdx.x] = sum;
}

__global__ void __launch_bounds__(kTsThreads) bin_tile_scan(const uint32_t* hist, uint32_t B,
                                                            const uint32_t* __restrict__ tsum,
                                                            uint32_t* __restrict__ bin_off, uint32_t* cursor,
                                                            const uint32_t* ctrl) {
  __shared__ uint32_t wsum[33];
  if (ctrl[kStatusWord]) return;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t before = 0;  // the bins of the tiles before this one
  for (uint32_t i = threadIdx.x; i < blockIdx.x; i += kTsThreads) before += tsum[i];
  before = block_sum(before, wsum);
  const uint32_t w0 = blockIdx.x * kTsTile + warp * 32 * kTileChunks;
  uint32_t ex[kTileChunks], run = 0;
#pragma unroll
  for (int j = 0; j < kTileChunks; ++j) {
    const uint32_t q = w0 + j * 32 + lane;
    const uint32_t h = q < B ? hist[q] : 0;
    const uint32_t incl = warp_incl_scan(h);
    ex[j] = run + incl - h;
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) wsum[warp] = run;
  scan_warp_totals(wsum);
  const uint32_t off = before + wsum[warp];
#pragma unroll
  for (int j = 0; j < kTileChunks; ++j) {
    const uint32_t q = w0 + j * 32 + lane;
    if (q < B) {
      bin_off[q] = off + ex[j];
      cursor[q] = off + ex[j];
    }
  }
  if (threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) bin_off[B] = before + wsum[32];
}

// hist -> bin_off, cursor (may be hist), max bin; tsum: one word per tile
// (scratch).  Returns the number of launches.
uint32_t scan_bins(const uint32_t* hist, uint32_t B, uint32_t* bin_off, uint32_t* cursor, uint32_t* ctrl,
                   uint32_t* tsum, cudaStream_t st) {
  const uint32_t T = (B + kTsTile - 1) / kTsTile;
  bin_tile_sums<<<T, kTsThreads, 0, st>>>(hist, B, tsum, ctrl);
  bin_tile_scan<<<T, kTsThreads, 0, st>>>(hist, B, tsum, bin_off, cursor, ctrl);
  return 2;
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

// Work items = runs of consecutive fine bins.  A bin starts a new item if it
// starts a partition, is not "small" (> W = cap/2 pairs), follows a bin that
// is not small, or its start offset enters a new W-window; a run of small
// bins inside one window holds < 2W = cap pairs.  Oversize bins (> cap pairs)
// are listed separately.  item_flag becomes the item id of every bin.  The
// rule looks at a bin and its neighbour only, so the items are found in two
// launches over tiles of kTsTile bins laid out as in the bin scan: the count
// of item starts per tile, then every CTA adds the counts of the tiles before
// its own and numbers its tile's items.
__device__ __forceinline__ uint32_t starts_item(const uint32_t* __restrict__ bin_off, const uint32_t* item_flag,
                                                uint32_t q, uint32_t W) {
  const uint32_t o = bin_off[q], cnt = bin_off[q + 1] - o;
  if (item_flag[q] != 0 || q == 0 || cnt > W) return 1;
  const uint32_t po = bin_off[q - 1];
  return (o - po) > W || (o / W) != (po / W);
}

__global__ void __launch_bounds__(kTsThreads) item_tile_counts(const uint32_t* __restrict__ bin_off, uint32_t B,
                                                               uint32_t cap, const uint32_t* __restrict__ item_flag,
                                                               uint32_t* __restrict__ tcnt, const uint32_t* ctrl) {
  __shared__ uint32_t red[33];
  if (ctrl[kStatusWord]) return;
  const uint32_t W = cap / 2;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t w0 = blockIdx.x * kTsTile + warp * 32 * kTileChunks;
  uint32_t n = 0;
#pragma unroll
  for (int j = 0; j < kTileChunks; ++j) {
    const uint32_t q = w0 + j * 32 + lane;
    if (q < B) n += starts_item(bin_off, item_flag, q, W);
  }
  n = block_sum(n, red);
  if (threadIdx.x == 0) tcnt[blockIdx.x] = n;
}

__global__ void __launch_bounds__(kTsThreads) item_tile_write(const uint32_t* __restrict__ bin_off, uint32_t B,
                                                              uint32_t cap, uint32_t* item_flag, uint32_t* items,
                                                              uint32_t* oversize, const uint32_t* __restrict__ tcnt,
                                                              uint32_t* ctrl) {
  __shared__ uint32_t wsum[33];
  if (ctrl[kStatusWord]) return;
  const uint32_t W = cap / 2;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t before = 0;  // the items of the tiles before this one
  for (uint32_t i = threadIdx.x; i < blockIdx.x; i += kTsThreads) before += tcnt[i];
  before = block_sum(before, wsum);
  const uint32_t w0 = blockIdx.x * kTsTile + warp * 32 * kTileChunks;
  uint32_t ex[kTileChunks], run = 0, fl = 0;  // fl bit j: bin of chunk j starts an item
#pragma unroll
  for (int j = 0; j < kTileChunks; ++j) {
    const uint32_t q = w0 + j * 32 + lane;
    const uint32_t f = q < B ? starts_item(bin_off, item_flag, q, W) : 0;
    fl |= f << j;
    const uint32_t incl = warp_incl_scan(f);
    ex[j] = run + incl - f;
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) wsum[warp] = run;
  scan_warp_totals(wsum);
  const uint32_t off = before + wsum[warp];
#pragma unroll
  for (int j = 0; j < kTileChunks; ++j) {
    const uint32_t q = w0 + j * 32 + lane;
    if (q < B) {
      const uint32_t id = off + ex[j];
      if ((fl >> j) & 1) {
        items[id] = q;
        if (bin_off[q + 1] - bin_off[q] > cap) oversize[atomicAdd(ctrl + kNumOversize, 1u)] = id;
        item_flag[q] = id;
      } else {
        item_flag[q] = id - 1;
      }
    }
  }
  if (threadIdx.x == 0 && blockIdx.x == gridDim.x - 1) {
    const uint32_t total = before + wsum[32];
    items[total] = B;
    ctrl[kNumItems] = total;
  }
}

// items, item_flag (partition starts in, item ids out), oversize list, item
// count; tcnt: one word per tile (scratch).  Returns the number of launches.
uint32_t find_items(const uint32_t* bin_off, uint32_t B, uint32_t cap, uint32_t* item_flag, uint32_t* items,
                    uint32_t* oversize, uint32_t* ctrl, uint32_t* tcnt, cudaStream_t st) {
  const uint32_t T = (B + kTsTile - 1) / kTsTile;
  item_tile_counts<<<T, kTsThreads, 0, st>>>(bin_off, B, cap, item_flag, tcnt, ctrl);
  item_tile_write<<<T, kTsThreads, 0, st>>>(bin_off, B, cap, item_flag, items, oversize, tcnt, ctrl);
  return 2;
}

// Coarse offsets: seg[c][b] (counts of classify CTA b in coarse bin c) becomes
// the start of CTA b's slots in coarse bin c: the coarse bin's start
// bin_off[c << cshift] plus the counts of the CTAs before b.  A warp per c.
__global__ void coarse_offsets_kernel(uint32_t* __restrict__ seg, uint32_t seg_stride, uint32_t G, uint32_t C,
                                      uint32_t cshift, const uint32_t* __restrict__ bin_off, const uint32_t* ctrl) {
  if (ctrl[kStatusWord]) return;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= C) return;
  uint32_t* col = seg + (size_t)c * seg_stride;
  uint32_t carry = bin_off[c << cshift];
  for (uint32_t b0 = 0; b0 < G; b0 += 32) {
    const uint32_t b = b0 + lane;
    const uint32_t h = b < G ? col[b] : 0;
    uint32_t incl = h;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= (uint32_t)d) incl += y;
    }
    if (b < G) col[b] = carry + incl - h;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
}

__device__ __forceinline__ uint32_t upper_set(const uint64_t* __restrict__ off, uint32_t K, uint64_t g) {
  uint32_t lo = 0, hi = K - 1;  // largest k with off[k] <= g
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Scatter through shared memory.  A CTA's input pairs arrive by bulk copy
// (TMA) into one of two input buffers while the previous batch is worked on;
// a batch is put in bin order in shared memory (rank inside the batch from a
// shared counter, offsets from a block scan), then written out slot by slot,
// so the pairs of one bin leave as one contiguous run (whole lines rather
// than 16-byte pieces scattered over the device).  cur[] holds every bin's
// next output slot.  Four block barriers per batch: the counts are complete
// (the input buffer is free again), two in the scan, the offsets are set,
// the batch is placed; the owner of a bin turns its offset into the bin's
// output base (base = cur - off), advances cur and clears the count while
// setting the offset, so no barrier follows the write-out.  Waits on the
// copies are bounded like classify's.
constexpr int kStageThreads = 512;
constexpr int kStagePer = 4;
constexpr uint32_t kStagePairs = kStageThreads * kStagePer;  // 2048 pairs = 32 KB
// the classify units the coarse pass takes are powers of two that divide a batch
static_assert((kTileRecs & (kTileRecs - 1)) == 0 && kStagePairs % kTileRecs == 0, "classify tile");
static_assert(((kThreads * kUnroll) & (kThreads * kUnroll - 1)) == 0 && kStagePairs % (kThreads * kUnroll) == 0,
              "plain classify unit");

struct Stage {
  Pair* in[2];      // kStagePairs each: input batches (bulk-copy targets)
  Pair* pairs;      // kStagePairs: the batch in bin order
  uint16_t* binof;  // kStagePairs
  uint32_t* cnt;    // nb: counts of the batch
  uint32_t* off;    // nb: exclusive offsets in the batch
  uint32_t* base;   // nb: output slot of the batch's slot 0 of each bin (cur - off)
  uint32_t* cur;    // nb: next output slot
  uint32_t* wsum;   // 33: the scan's warp sums, then [32] = the batch's pair count
  uint64_t* bar;    // 2
};

// block-wide exclusive scan of one value per thread (two barriers; wsum is
// next written by the following batch's scan, after its own barriers)
__device__ __forceinline__ uint32_t stage_scan(uint32_t v, uint32_t* wsum) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= (uint32_t)d) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < kStageThreads / 32 ? wsum[lane] : 0;
    uint32_t wi = w;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= (uint32_t)d) wi += y;
    }
    if (lane < kStageThreads / 32) wsum[lane] = wi - w;
  }
  __syncthreads();
  return wsum[warp] + incl - v;
}

// rank of the batch's pairs inside their bins (p[k] valid when bin[k] < nb);
// before the barrier that ends the count
__device__ __forceinline__ void stage_count(const Stage& S, uint32_t nb, const uint32_t (&bin)[kStagePer],
                                            uint32_t (&r)[kStagePer]) {
#pragma unroll
  for (int k = 0; k < kStagePer; ++k)
    if (bin[k] < nb) r[k] = atomicAdd(&S.cnt[bin[k]], 1u);
}

// the rest of a counted batch; out slots checked against `bound`
__device__ void stage_scatter(const Stage& S, uint32_t nb, const Pair (&p)[kStagePer], const uint32_t (&bin)[kStagePer],
                              const uint32_t (&r)[kStagePer], Pair* __restrict__ out, uint64_t bound) {
  // exclusive offsets of the nb counts: each thread owns a contiguous group of bins
  const uint32_t per = (nb + kStageThreads - 1) / kStageThreads;
  const uint32_t g0 = min(nb, threadIdx.x * per), g1 = min(nb, g0 + per);
  uint32_t local = 0;
  for (uint32_t c = g0; c < g1; ++c) local += S.cnt[c];
  uint32_t run = stage_scan(local, S.wsum);
  for (uint32_t c = g0; c < g1; ++c) {
    const uint32_t k = S.cnt[c];
    S.off[c] = run;
    S.base[c] = S.cur[c] - run;
    S.cur[c] += k;
    S.cnt[c] = 0;
    run += k;
  }
  if (g1 == nb && g0 < g1) S.wsum[32] = run;  // the batch's pair count
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kStagePer; ++k)
    if (bin[k] < nb) {
      const uint32_t sl = S.off[bin[k]] + r[k];
      S.pairs[sl] = p[k];
      S.binof[sl] = (uint16_t)bin[k];
    }
  __syncthreads();
  const uint32_t total = S.wsum[32];
  for (uint32_t sl = threadIdx.x; sl < total; sl += kStageThreads) {
    const uint64_t dst = (uint64_t)S.base[S.binof[sl]] + sl;
    if (dst < bound) out[dst] = S.pairs[sl];
  }
}

__device__ __forceinline__ Stage carve_stage(uint8_t* smem, uint32_t nb) {
  Stage S;
  S.in[0] = reinterpret_cast<Pair*>(smem);
  S.in[1] = S.in[0] + kStagePairs;
  S.pairs = S.in[1] + kStagePairs;
  S.binof = reinterpret_cast<uint16_t*>(S.pairs + kStagePairs);
  uint32_t* w = reinterpret_cast<uint32_t*>(S.binof + kStagePairs);
  S.cnt = w;
  S.off = w + nb;
  S.base = w + 2 * nb;
  S.cur = w + 3 * nb;
  S.wsum = w + 4 * nb;
  S.bar = reinterpret_cast<uint64_t*>(reinterpret_cast<uintptr_t>(w + 4 * nb + 33 + 1) & ~(uintptr_t)7);
  return S;
}

size_t stage_smem_bytes(uint32_t nb) {
  return (size_t)kStagePairs * (3 * sizeof(Pair) + 2) + (4 * (size_t)nb + 33 + 1) * 4 + 2 * 8 + 8;
}

// Pass B1: pairs (input order) -> coarse-bin order.  With K record sets
// (poff non-null) the index written is the one inside the record's set.
// CTA b takes the same
// records as classify's CTA b -- units of U records, unit u to CTA u mod G;
// the ragged last unit to CTA 0 (TMA classify) or to its own CTA (plain
// classify) -- so its counts per coarse bin are the ones classify wrote, and
// its slots in coarse bin c start at seg[c][b].  The record index replaces
// the fine bin in lo; the fine bin's place inside its coarse bin rides in
// bits 48.. of lo for pass B2.
__global__ void __launch_bounds__(kStageThreads, 2) coarse_scatter_kernel(const Pair* __restrict__ in, uint64_t n,
                                                                       uint32_t log2U, int tail_to_first,
                                                                       const uint32_t* __restrict__ seg,
                                                                       uint32_t seg_stride, uint32_t cshift,
                                                                       uint32_t C, Pair* __restrict__ out,
                                                                       uint32_t* ctrl, const uint64_t* __restrict__ poff,
                                                                       uint32_t K, long long wait_limit) {
  extern __shared__ __align__(128) uint8_t smem[];
  if (ctrl[kStatusWord]) return;
  const Stage S = carve_stage(smem, C);
  for (uint32_t c = threadIdx.x; c < C; c += kStageThreads) {
    S.cnt[c] = 0;
    S.cur[c] = seg[(size_t)c * seg_stride + blockIdx.x];
  }
  if (threadIdx.x == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint32_t fmask = (1u << cshift) - 1;
  const uint32_t U = 1u << log2U, umask = U - 1;
  const uint64_t G = gridDim.x, b = blockIdx.x;
  const uint64_t nfull = n >> log2U;
  const uint32_t rag = (uint32_t)(n & umask);
  const uint64_t mine_full = b < nfull ? (nfull - b + G - 1) / G : 0;
  const bool tail = rag && b == (tail_to_first ? 0 : nfull % G);
  const uint64_t mine = mine_full + (tail ? 1 : 0);  // units of this CTA: b, b+G, ..., then the ragged one
  const uint32_t upb = kStagePairs >> log2U;           // units per batch (U divides kStagePairs)
  const uint64_t nbatch = (mine + upb - 1) / upb;
  // unit k of this CTA: its first record and its size
  auto unit_of = [&](uint64_t k, uint64_t* first) -> uint32_t {
    if (k < mine_full) {
      *first = (b + k * G) << log2U;
      return U;
    }
    if (k < mine) {
      *first = nfull << log2U;
      return rag;
    }
    *first = 0;
    return 0;
  };
  // thread 0: the bulk copies of batch j into input buffer buf (a batch
  // below nbatch always holds at least one record)
  auto issue = [&](uint64_t j, int buf) {
    uint32_t bytes = 0;
    for (uint32_t u = 0; u < upb; ++u) {
      uint64_t first;
      bytes += unit_of(j * upb + u, &first) * (uint32_t)sizeof(Pair);
    }
    mbar_expect_tx(&S.bar[buf], bytes);
    for (uint32_t u = 0; u < upb; ++u) {
      uint64_t first;
      const uint32_t c = unit_of(j * upb + u, &first);
      if (c) bulk_g2s(S.in[buf] + u * U, in + first, c * (uint32_t)sizeof(Pair), &S.bar[buf]);
    }
  };
  uint32_t issued[2] = {0, 0};
  if (threadIdx.x == 0)
    for (int q = 0; q < 2; ++q)
      if ((uint64_t)q < nbatch) {
        issue(q, q);
        issued[q] = 1;
      }
  for (uint64_t j = 0; j < nbatch; ++j) {
    const int buf = (int)(j & 1);
    const bool ok = mbar_wait(&S.bar[buf], (uint32_t)((j >> 1) & 1), wait_limit);
    Pair p[kStagePer];
    uint32_t bin[kStagePer];
#pragma unroll
    for (int k = 0; k < kStagePer; ++k) {
      const uint32_t slot = threadIdx.x + k * kStageThreads;
      uint64_t first;
      const uint32_t c = unit_of(j * upb + (slot >> log2U), &first);
      bin[k] = ~0u;
      if (ok && (slot & umask) < c) {
        const Pair q = S.in[buf][slot];
        const uint32_t f = (uint32_t)q.lo;
        bin[k] = min(f >> cshift, C - 1);
        p[k].hi = q.hi;
        const uint64_t g = first + (slot & umask);  // the record's place in the input (all sets together)
        const uint64_t i = poff ? g - poff[upper_set(poff, K, g)] : g;
        p[k].lo = (q.lo & 0x0000FFFF00000000ull) | ((uint64_t)(f & fmask) << 48) | (uint32_t)i;
      }
    }
    uint32_t r[kStagePer];
    stage_count(S, C, bin, r);
    if (__syncthreads_or(!ok)) {  // the counts are complete, and input buffer `buf` is read
      if (threadIdx.x == 0) {
        atomicOr(ctrl + kStatusWord, 1u);
        for (int q = 0; q < 2; ++q)  // copies in flight target this CTA's shared memory: wait, bounded
          if (issued[q]) mbar_wait(&S.bar[q], (issued[q] - 1) & 1, kWaitLimitCycles);
      }
      return;
    }
    if (threadIdx.x == 0 && j + 2 < nbatch) {
      fence_proxy_async();
      issue(j + 2, buf);
      ++issued[buf];
    }
    stage_scatter(S, C, p, bin, r, out, n);
  }
}

// Pass B2: one CTA per coarse bin: its pairs to their fine bins (2^cshift of
// them), through the same staging.
__global__ void __launch_bounds__(kStageThreads, 2) fine_scatter_kernel(const Pair* __restrict__ in,
                                                                     const uint32_t* __restrict__ bin_off, uint32_t B,
                                                                     uint32_t cshift, Pair* __restrict__ out,
                                                                     uint32_t* ctrl, long long wait_limit) {
  extern __shared__ __align__(128) uint8_t smem[];
  if (ctrl[kStatusWord]) return;
  const uint32_t nf = 1u << cshift;
  const Stage S = carve_stage(smem, nf);
  const uint32_t f0 = blockIdx.x << cshift;
  for (uint32_t f = threadIdx.x; f < nf; f += kStageThreads) {
    S.cnt[f] = 0;
    S.cur[f] = bin_off[min(B, f0 + f)];
  }
  if (threadIdx.x == 0) {
    mbar_init(&S.bar[0], 1);
    mbar_init(&S.bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const uint32_t s = bin_off[f0], e = bin_off[min(B, f0 + nf)];
  const uint32_t nbatch = (e - s + kStagePairs - 1) / kStagePairs;
  auto issue = [&](uint32_t j, int buf) {  // thread 0; a batch below nbatch is never empty
    const uint32_t i0 = s + j * kStagePairs;
    const uint32_t bytes = min(kStagePairs, e - i0) * (uint32_t)sizeof(Pair);
    mbar_expect_tx(&S.bar[buf], bytes);
    bulk_g2s(S.in[buf], in + i0, bytes, &S.bar[buf]);
  };
  uint32_t issued[2] = {0, 0};
  if (threadIdx.x == 0)
    for (int q = 0; q < 2; ++q)
      if ((uint32_t)q < nbatch) {
        issue(q, q);
        issued[q] = 1;
      }
  for (uint32_t j = 0; j < nbatch; ++j) {
    const int buf = (int)(j & 1);
    const bool ok = mbar_wait(&S.bar[buf], (j >> 1) & 1, wait_limit);
    const uint32_t i0 = s + j * kStagePairs;
    Pair p[kStagePer];
    uint32_t bin[kStagePer];
#pragma unroll
    for (int k = 0; k < kStagePer; ++k) {
      const uint32_t slot = threadIdx.x + k * kStageThreads;
      bin[k] = ~0u;
      if (ok && i0 + slot < e) {
        const Pair q = S.in[buf][slot];
        bin[k] = (uint32_t)(q.lo >> 48) & (nf - 1);
        p[k].hi = q.hi;
        p[k].lo = q.lo & 0x0000FFFFFFFFFFFFull;
      }
    }
    uint32_t r[kStagePer];
    stage_count(S, nf, bin, r);
    if (__syncthreads_or(!ok)) {  // the counts are complete, and input buffer `buf` is read
      if (threadIdx.x == 0) {
        atomicOr(ctrl + kStatusWord, 1u);
        for (int q = 0; q < 2; ++q)
          if (issued[q]) mbar_wait(&S.bar[q], (issued[q] - 1) & 1, kWaitLimitCycles);
      }
      return;
    }
    if (threadIdx.x == 0 && j + 2 < nbatch) {
      fence_proxy_async();
      issue(j + 2, buf);
      ++issued[buf];
    }
    stage_scatter(S, nf, p, bin, r, out, e);
  }
}

// ---------------------------------------------------------------- many record sets at once

// Pass A over K record sets: record i of set k goes to global pair slot
// poff[k] + i with the set's fine bin tbase[k] + q (binary search over the
// set's own splitters).
__global__ void __launch_bounds__(kThreads) classify_batch_kernel(const uint8_t* const* __restrict__ ins, KeyMask km,
                                                                  const uint64_t* __restrict__ poff, uint32_t K,
                                                                  const uint64_t* __restrict__ t,
                                                                  const uint64_t* __restrict__ tbase,
                                                                  const uint32_t* __restrict__ log2B,
                                                                  Pair* __restrict__ pairs, uint32_t* __restrict__ hist,
                                                                  uint32_t cshift, uint32_t* __restrict__ seg_hist,
                                                                  uint32_t seg_stride) {
  __shared__ uint32_t hc[kMaxCoarse];  // this CTA's counts per coarse bin (units of 256 records)
  for (uint32_t c = threadIdx.x; c < kMaxCoarse; c += kThreads) hc[c] = 0;
  __syncthreads();
  const uint64_t N = poff[K];
  for (uint64_t g = blockIdx.x * (uint64_t)kThreads + threadIdx.x; g < N; g += (uint64_t)gridDim.x * kThreads) {
    const uint32_t k = upper_set(poff, K, g);
    const uint64_t i = g - poff[k];
    Pair p = load_pair(ins[k] + i * kRecord, 0, km);
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
    if (seg_hist) atomicAdd(&hc[min(q >> cshift, kMaxCoarse - 1)], 1u);
  }
  if (seg_hist) {
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < kMaxCoarse; c += kThreads) seg_hist[c * seg_stride + blockIdx.x] = hc[c];
  }
}

// Pass B in one step, for fine-bin spaces too large for the two staged
// passes (more than 2^kStagedMaxShift fine bins per coarse bin: the fine
// pass's cursors would not fit in shared memory): slot from an atomic cursor
// per bin; the record index (inside its set when poff is given) replaces the
// fine bin.
__global__ void __launch_bounds__(kThreads) scatter_atomic_kernel(const Pair* __restrict__ in, uint64_t N,
                                                                  const uint64_t* __restrict__ poff, uint32_t K,
                                                                  uint32_t* __restrict__ cursor, Pair* __restrict__ out,
                                                                  const uint32_t* ctrl) {
  if (ctrl[kStatusWord]) return;
  for (uint64_t g = blockIdx.x * (uint64_t)kThreads + threadIdx.x; g < N; g += (uint64_t)gridDim.x * kThreads) {
    const Pair p = in[g];
    const uint32_t slot = atomicAdd(cursor + (uint32_t)p.lo, 1u);
    const uint64_t i = poff ? g - poff[upper_set(poff, K, g)] : g;
    Pair o;
    o.hi = p.hi;
    o.lo = (p.lo & 0xFFFFFFFF00000000ull) | (uint32_t)i;
    if (slot < N) out[slot] = o;
  }
}

// every set's first bin starts a work item (items never span two sets)
__global__ void mark_set_starts(const uint64_t* __restrict__ tbase, uint32_t K, uint32_t* item_flag) {
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x)
    item_flag[tbase[k]] = 1u;
}

}  // namespace

cudaError_t prepare_scatter_kernels() {
  const int smem = (int)stage_smem_bytes(1u << kMaxFineShift);  // the largest bin count a pass takes
  cudaError_t e = cudaFuncSetAttribute(coarse_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fine_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  return e;
}

// coarse bins over a fine-bin space of B bins: 2^cshift fine bins each, at most kMaxCoarse
static void coarse_of(uint64_t B, uint32_t* cshift, uint32_t* C) {
  uint32_t s = 0;
  while (((B + (1ull << s) - 1) >> s) > kMaxCoarse) ++s;
  *cshift = s;
  *C = (uint32_t)((B + (1ull << s) - 1) >> s);
}

// Many record sets: one atomic pass above 2^9 fine bins per coarse bin (the
// batched workload measured faster that way than with the staged passes up
// to kStagedMaxShift, which a single large set prefers).
constexpr uint32_t kBatchStagedMaxShift = 9;

cudaError_t partition_batch(const BatchPartArgs& a) {
  cudaStream_t st = a.stream;
  const int sms = sm_count();
  cudaMemsetAsync(a.cursor, 0, (size_t)a.B * 4, st);
  cudaMemsetAsync(a.ctrl, 0, 32 * sizeof(uint32_t), st);
  cudaMemsetAsync(a.item_flag, 0, (size_t)a.B * 4, st);
  uint32_t cshift, C;
  coarse_of(a.B, &cshift, &C);
  const uint64_t segs = coarse_segments(a.N);
  const unsigned G = (unsigned)umin64(segs, (uint64_t)sms * 8);
  if (cshift > kBatchStagedMaxShift) {  // many sets: one atomic pass
    classify_batch_kernel<<<G, kThreads, 0, st>>>(a.ins, a.km, a.poff, a.K, a.splitters, a.tbase, a.log2B,
                                                 a.pairs_in_order, a.cursor, 0, nullptr, 0);
    *a.launches += scan_bins(a.cursor, a.B, a.bin_off, a.cursor, a.ctrl, a.items, st);
    scatter_atomic_kernel<<<G, kThreads, 0, st>>>(a.pairs_in_order, a.N, a.poff, a.K, a.cursor, a.pairs, a.ctrl);
    mark_set_starts<<<(a.K + 255) / 256, 256, 0, st>>>(a.tbase, a.K, a.item_flag);
    // the cursors are spent: they hold the item scan's tile counts
    *a.launches += find_items(a.bin_off, a.B, a.tile_pairs, a.item_flag, a.items, a.oversize, a.ctrl, a.cursor, st);
    *a.launches += 3;
    return cudaGetLastError();
  }
  // roles: input-order pairs and the final bin order share `pairs`; the
  // coarse order between the two passes lives in `pairs_in_order`
  classify_batch_kernel<<<G, kThreads, 0, st>>>(a.ins, a.km, a.poff, a.K, a.splitters, a.tbase, a.log2B, a.pairs,
                                               a.cursor, cshift, a.seg_hist, (uint32_t)segs);
  *a.launches += scan_bins(a.cursor, a.B, a.bin_off, a.cursor, a.ctrl, a.items, st);
  coarse_offsets_kernel<<<(C + 7) / 8, 256, 0, st>>>(a.seg_hist, (uint32_t)segs, G, C, cshift, a.bin_off, a.ctrl);
  coarse_scatter_kernel<<<G, kStageThreads, stage_smem_bytes(C), st>>>(a.pairs, a.N, ilog2(kThreads), 0, a.seg_hist,
                                                                        (uint32_t)segs, cshift, C, a.pairs_in_order,
                                                                        a.ctrl, a.poff, a.K, kWaitLimitCycles);
  fine_scatter_kernel<<<C, kStageThreads, stage_smem_bytes(1u << cshift), st>>>(a.pairs_in_order, a.bin_off, a.B,
                                                                                 cshift, a.pairs, a.ctrl,
                                                                                 kWaitLimitCycles);
  mark_set_starts<<<(a.K + 255) / 256, 256, 0, st>>>(a.tbase, a.K, a.item_flag);
  *a.launches += find_items(a.bin_off, a.B, a.tile_pairs, a.item_flag, a.items, a.oversize, a.ctrl, a.cursor, st);
  *a.launches += 5;
  return cudaGetLastError();
}

cudaError_t partition_records(const PartArgs& a) {
  const uint32_t B = 1u << a.log2B;
  cudaStream_t st = a.stream;
  const int sms = sm_count();
  const uint32_t cshift = coarse_shift(a.log2B);
  const uint32_t C = B >> cshift;
  cudaMemsetAsync(a.cursor, 0, (size_t)B * 4, st);  // the histogram lives in `cursor` until the scan
  cudaMemsetAsync(a.ctrl, 0, 32 * sizeof(uint32_t), st);
  Pair* pin = static_cast<Pair*>(a.pairs_in_order);
  const uint64_t segs = coarse_segments(a.n);
  unsigned G;
  uint32_t U;
  int tail_to_first;
  if ((reinterpret_cast<uintptr_t>(a.records) & 15) == 0) {
    const size_t smem = (size_t)kClassifyStages * kTileBytes;
    cudaFuncSetAttribute(CLASSIFY_TMA, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, CLASSIFY_TMA, kClassifyThreads, smem);
    const uint64_t tiles = a.n / kTileRecs;
    G = (unsigned)umin64(segs, umax64(1, umin64(tiles, (uint64_t)sms * (occ > 0 ? occ : 1))));
    U = kTileRecs;
    tail_to_first = 1;
    CLASSIFY_TMA<<<G, kClassifyThreads, smem, st>>>(a.records, a.km, a.n, a.splitters, a.lut, pin, a.cursor, a.ctrl, cshift,
                                                    a.seg_hist, (uint32_t)segs, a.wait_limit);
  } else {
    const uint64_t per_block = (uint64_t)kThreads * kUnroll;
    const uint64_t blocks = (a.n + per_block - 1) / per_block;
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, classify_kernel, kThreads, 0);
    G = (unsigned)umin64(segs, umax64(1, umin64(blocks, (uint64_t)sms * (occ > 0 ? occ : 1))));
    U = (uint32_t)per_block;
    tail_to_first = 0;
    classify_kernel<<<G, kThreads, 0, st>>>(a.records, a.km, a.n, a.splitters, a.lut, pin, a.cursor, cshift,
                                            a.seg_hist, (uint32_t)segs);
  }
  if (a.ev[0]) cudaEventRecord(a.ev[0], st);
  *a.launches += scan_bins(a.cursor, B, a.bin_off, a.cursor, a.ctrl, a.items, st);
  cuts_kernel<<<(a.P + 1 + 255) / 256, 256, 0, st>>>(a.bin_off, a.log2B, a.P, (int)a.balance, a.cuts, a.part_off,
                                                      nullptr);
  if (a.ev[1]) cudaEventRecord(a.ev[1], st);
  if (cshift > kStagedMaxShift) {  // more fine bins per coarse bin than the fine pass holds: one atomic pass
    scatter_atomic_kernel<<<(unsigned)sms * 8, kThreads, 0, st>>>(pin, a.n, nullptr, 0, a.cursor,
                                                                static_cast<Pair*>(a.pairs), a.ctrl);
    if (a.ev[2]) cudaEventRecord(a.ev[2], st);
    *a.launches += 3;
    return cudaGetLastError();
  }
  // two scatter passes through shared memory: coarse bins, then fine bins inside each
  const uint32_t seg_stride = (uint32_t)segs;
  coarse_offsets_kernel<<<(C + 7) / 8, 256, 0, st>>>(a.seg_hist, seg_stride, G, C, cshift, a.bin_off, a.ctrl);
  const size_t smem1 = stage_smem_bytes(C), smem2 = stage_smem_bytes(1u << cshift);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  if (cs == cudaStreamCaptureStatusNone) prepare_scatter_kernels();
  coarse_scatter_kernel<<<G, kStageThreads, smem1, st>>>(pin, a.n, ilog2(U), tail_to_first, a.seg_hist, seg_stride, cshift,
                                                          C, static_cast<Pair*>(a.mid), a.ctrl, nullptr, 0,
                                                          a.wait_limit);
  fine_scatter_kernel<<<C, kStageThreads, smem2, st>>>(static_cast<const Pair*>(a.mid), a.bin_off, B, cshift,
                                                        static_cast<Pair*>(a.pairs), a.ctrl, a.wait_limit);
  if (a.ev[2]) cudaEventRecord(a.ev[2], st);
  *a.launches += 5;
  return cudaGetLastError();
}

cudaError_t classify_accumulate(const PartArgs& a) {
  cudaStream_t st = a.stream;
  const int sms = sm_count();
  Pair* pin = static_cast<Pair*>(a.pairs_in_order);
  if ((reinterpret_cast<uintptr_t>(a.records) & 15) == 0) {
    const size_t smem = (size_t)kClassifyStages * kTileBytes;
    cudaFuncSetAttribute(CLASSIFY_TMA, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int occ = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, CLASSIFY_TMA, kClassifyThreads, smem);
    const uint64_t tiles = a.n / kTileRecs;
    const unsigned grid = (unsigned)umax64(1, umin64(tiles, (uint64_t)sms * (occ > 0 ? occ : 1)));
    CLASSIFY_TMA<<<grid, kClassifyThreads, smem, st>>>(a.records, a.km, a.n, a.splitters, a.lut, pin, a.cursor, a.ctrl, 0,
                                                       nullptr, 0, a.wait_limit);
  } else {
    const uint64_t per_block = (uint64_t)kThreads * kUnroll;
    const unsigned grid = (unsigned)umax64(1, umin64((a.n + per_block - 1) / per_block, (uint64_t)sms * 4));
    classify_kernel<<<grid, kThreads, 0, st>>>(a.records, a.km, a.n, a.splitters, a.lut, pin, a.cursor, 0, nullptr, 0);
  }
  *a.launches += 1;
  return cudaGetLastError();
}

cudaError_t scan_and_cut(const PartArgs& a) {
  const uint32_t B = 1u << a.log2B;
  *a.launches += scan_bins(a.cursor, B, a.bin_off, a.cursor, a.ctrl, a.items, a.stream);
  cuts_kernel<<<(a.P + 1 + 255) / 256, 256, 0, a.stream>>>(a.bin_off, a.log2B, a.P, (int)a.balance, a.cuts,
                                                           a.part_off, nullptr);
  *a.launches += 1;
  return cudaGetLastError();
}

cudaError_t build_items(const PartArgs& a) {
  cudaStream_t st = a.stream;
  const uint32_t B = 1u << a.log2B;
  cudaMemsetAsync(a.item_flag, 0, (size_t)B * 4, st);
  cudaMemsetAsync(a.ctrl, 0, 3 * sizeof(uint32_t), st);  // item count, oversize count, queue head
  cuts_kernel<<<(a.P + 1 + 255) / 256, 256, 0, st>>>(a.bin_off, a.log2B, a.P, (int)a.balance, a.cuts, a.part_off,
                                                      a.item_flag);
  // the scatter cursors are spent: they hold the item scan's tile counts
  *a.launches += find_items(a.bin_off, B, a.tile_pairs, a.item_flag, a.items, a.oversize, a.ctrl, a.cursor, st);
  *a.launches += 1;
  return cudaGetLastError();
}

}  // namespace elsar
