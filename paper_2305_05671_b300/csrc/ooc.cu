// Out-of-core support kernels: records that live in host memory are
// partitioned on the device chunk by chunk (Sec. 3.3's reader loop over
// batches) and each chunk's records are split stably by partition before
// they go back to their partition's range of the host output (the paper's
// fragment files, appended in input order).
#include "common.cuh"

namespace elsar {
namespace {

constexpr int kTile = 8192;       // records per stable-split tile
constexpr int kTileThreads = 1024;

// bin -> partition id from the cuts: the last p < P with cuts[p] <= q
// (cuts[0] = 0, cuts[P] = B and the cuts do not decrease)
__global__ void bin_to_part_kernel(const uint32_t* __restrict__ cuts, uint32_t P, uint32_t B, uint16_t* __restrict__ lut) {
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < B; q += gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = P - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (cuts[mid] <= q) lo = mid;
      else hi = mid - 1;
    }
    lut[q] = (uint16_t)lo;
  }
}

// Per tile: stable ranks of the tile's records within their partitions
// (a bitonic sort of (partition << 13 | position) in shared memory) and the
// tile's partition counts.
__global__ void __launch_bounds__(kTileThreads) tile_split_kernel(const Pair* __restrict__ pairs, uint64_t n,
                                                                  const uint16_t* __restrict__ lut, uint32_t P,
                                                                  uint32_t* __restrict__ tile_hist,
                                                                  uint16_t* __restrict__ rank,
                                                                  const uint32_t* ctrl) {
  __shared__ uint32_t key[kTile];
  if (ctrl[kStatusWord]) return;  // classify gave up: its fine bins are not valid
  const uint64_t t0 = (uint64_t)blockIdx.x * kTile;
  const uint32_t m = (uint32_t)min((uint64_t)kTile, n - t0);
  for (uint32_t i = threadIdx.x; i < kTile; i += kTileThreads)
    key[i] = i < m ? ((uint32_t)lut[(uint32_t)pairs[t0 + i].lo] << 13) | i : 0xFFFFFFFFu;
  uint32_t* h = tile_hist + (uint64_t)blockIdx.x * P;
  for (uint32_t p = threadIdx.x; p < P; p += kTileThreads) h[p] = 0;
  __syncthreads();
  for (uint32_t k = 2; k <= kTile; k <<= 1) {
    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
      for (uint32_t i = threadIdx.x; i < kTile; i += kTileThreads) {
        const uint32_t ixj = i ^ j;
        if (ixj > i) {
          const uint32_t a = key[i], b = key[ixj];
          if ((a > b) == ((i & k) == 0)) {
            key[i] = b;
            key[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  // rank = position - first position of the same partition (the run start)
  for (uint32_t j = threadIdx.x; j < m; j += kTileThreads) {
    const uint32_t p = key[j] >> 13;
    uint32_t lo = 0, hi = j;  // first position with partition p
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      if ((key[mid] >> 13) < p) lo = mid + 1;
      else hi = mid;
    }
    rank[t0 + (key[j] & 0x1FFFu)] = (uint16_t)(j - lo);
    if (j + 1 == m || (key[j + 1] >> 13) != p) h[p] = j - lo + 1;
  }
}

// column scan over tiles for every partition: tile_hist[t][p] becomes the
// tile's start inside the chunk's piece of partition p; totals per partition
__global__ void column_scan_kernel(uint32_t* __restrict__ tile_hist, uint32_t tiles, uint32_t P,
                                   uint32_t* __restrict__ part_count) {
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    uint32_t run = 0;
    for (uint32_t t = 0; t < tiles; ++t) {
      const uint32_t c = tile_hist[(uint64_t)t * P + p];
      tile_hist[(uint64_t)t * P + p] = run;
      run += c;
    }
    part_count[p] = run;
  }
}

// single CTA: exclusive scan of the chunk's partition counts; every
// partition's destination for this chunk (dst_cur) is where the previous
// chunks left off (dst_next), which then advances by the chunk's count
__global__ void __launch_bounds__(1024) part_scan_kernel(const uint32_t* __restrict__ cnt, uint32_t P,
                                                         uint32_t* __restrict__ off, uint64_t* __restrict__ dst_next,
                                                         uint64_t* __restrict__ dst_cur) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < P; base += 1024) {
    const uint32_t p = base + threadIdx.x;
    const uint32_t v = p < P ? cnt[p] : 0;
    uint32_t incl = v;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= (uint32_t)d) incl += y;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      const uint32_t w = wsum[lane];
      uint32_t wi = w;
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, wi, d);
        if (lane >= (uint32_t)d) wi += y;
      }
      wsum[lane] = wi - w;
    }
    __syncthreads();
    const uint32_t c = carry;
    if (p < P) {
      off[p] = c + wsum[warp] + incl - v;
      const uint64_t d = dst_next[p];
      dst_cur[p] = d;
      dst_next[p] = d + v;
    }
    __syncthreads();
    if (threadIdx.x == 1023) carry = c + wsum[warp] + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) off[P] = carry;
}

// every record of the chunk to its slot in partition order (warp per 32 records, 4-byte words)
__global__ void split_records_kernel(const uint8_t* __restrict__ in, uint64_t n, const Pair* __restrict__ pairs,
                                     const uint16_t* __restrict__ lut, const uint32_t* __restrict__ tile_hist,
                                     const uint32_t* __restrict__ part_off, const uint16_t* __restrict__ rank,
                                     uint32_t P, uint8_t* __restrict__ out, const uint32_t* ctrl) {
  if (ctrl[kStatusWord]) return;
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint32_t* in32 = reinterpret_cast<const uint32_t*>(in);
  uint32_t* out32 = reinterpret_cast<uint32_t*>(out);
  for (uint64_t g = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); g * 32 < n; g += warps) {
    const uint64_t i = g * 32 + lane;
    uint32_t dst = 0;
    if (i < n) {
      const uint32_t p = lut[(uint32_t)pairs[i].lo];
      const uint64_t t = i / kTile;
      dst = part_off[p] + tile_hist[t * P + p] + rank[i];
    }
    const uint32_t nrec = (uint32_t)min((uint64_t)32, n - g * 32);
    // 32 records x 25 words: every lane runs the same 25 steps so the
    // shuffle sees the whole warp; word w belongs to record w / 25 (< 32)
#pragma unroll 5
    for (uint32_t j = 0; j < 25u; ++j) {
      const uint32_t w = j * 32u + lane;
      const uint32_t r = w / 25u, k = w - 25u * r;
      const uint32_t d = __shfl_sync(0xffffffffu, dst, r);
      if (r < nrec) out32[(uint64_t)d * 25u + k] = in32[(g * 32 + r) * 25u + k];
    }
  }
}

// the partition-ordered chunk to its partitions' ranges of the output (host
// memory mapped into the device's address space): record j of the chunk
// belongs to the last q with off[q] <= j and goes to dst_cur[q] + j - off[q];
// consecutive records of a partition land next to each other, so a warp's
// stores form long contiguous runs.  A destination at or past the
// partition's end (part_end[q]) is not written; the caller checks the counts.
__global__ void copy_out_kernel(const uint8_t* __restrict__ stage, uint64_t n, const uint32_t* __restrict__ off,
                                uint32_t P, const uint64_t* __restrict__ dst_cur, const uint64_t* __restrict__ part_end,
                                uint8_t* __restrict__ out) {
  const uint32_t lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint32_t* in32 = reinterpret_cast<const uint32_t*>(stage);
  uint32_t* out32 = reinterpret_cast<uint32_t*>(out);
  for (uint64_t g = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); g * 32 < n; g += warps) {
    const uint64_t j = g * 32 + lane;
    uint64_t dst = 0;
    uint32_t ok = 0;
    if (j < n) {
      uint32_t lo = 0, hi = P - 1;
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (off[mid] <= j) lo = mid;
        else hi = mid - 1;
      }
      dst = dst_cur[lo] + (j - off[lo]);
      ok = dst < part_end[lo];
    }
    const uint32_t nrec = (uint32_t)min((uint64_t)32, n - g * 32);
#pragma unroll 5
    for (uint32_t k0 = 0; k0 < 25u; ++k0) {
      const uint32_t w = k0 * 32u + lane;
      const uint32_t r = w / 25u, k = w - 25u * r;
      const uint64_t d = __shfl_sync(0xffffffffu, dst, r);
      const uint32_t okr = __shfl_sync(0xffffffffu, ok, r);
      if (r < nrec && okr) out32[d * 25u + k] = in32[(g * 32 + r) * 25u + k];
    }
  }
}

}  // namespace

uint64_t ooc_tiles(uint64_t n) { return (n + kTile - 1) / kTile; }

cudaError_t ooc_bin_to_part(const uint32_t* cuts, uint32_t P, uint32_t B, uint16_t* lut, cudaStream_t st) {
  if (P == 0 || P > 65536) return cudaErrorInvalidValue;
  bin_to_part_kernel<<<(B + 255) / 256, 256, 0, st>>>(cuts, P, B, lut);
  return cudaGetLastError();
}

cudaError_t ooc_split_chunk(const OocSplitArgs& a, cudaStream_t st) {
  if (!a.n) return cudaSuccess;
  const uint64_t tiles = ooc_tiles(a.n);
  tile_split_kernel<<<(unsigned)tiles, kTileThreads, 0, st>>>(a.pairs, a.n, a.lut, a.P, a.tile_hist, a.rank, a.ctrl);
  column_scan_kernel<<<(a.P + 255) / 256, 256, 0, st>>>(a.tile_hist, (uint32_t)tiles, a.P, a.part_count);
  part_scan_kernel<<<1, 1024, 0, st>>>(a.part_count, a.P, a.chunk_off, a.dst_next, a.dst_cur);
  const unsigned grid = (unsigned)min((uint64_t)sm_count() * 16, (a.n + 255) / 256 + 1);
  split_records_kernel<<<grid, 256, 0, st>>>(a.chunk, a.n, a.pairs, a.lut, a.tile_hist, a.chunk_off, a.rank, a.P,
                                             a.stage, a.ctrl);
  return cudaGetLastError();
}

cudaError_t ooc_copy_out(const OocSplitArgs& a, cudaStream_t st) {
  if (!a.n) return cudaSuccess;
  // stores to host memory need few warps to keep the link busy; leave the
  // rest of the GPU to the next chunk's kernels on the other stream
  const unsigned grid = (unsigned)min((uint64_t)sm_count() * 2, (a.n + 255) / 256 + 1);
  copy_out_kernel<<<grid, 256, 0, st>>>(a.stage, a.n, a.chunk_off, a.P, a.dst_cur, a.part_end, a.out);
  return cudaGetLastError();
}

}  // namespace elsar
