// Sorting every partition and concatenating (Sec. 3.4, Sec. 3.5, and the
// touch-up of Sec. 4) on the GPU.  A work item is a run of consecutive fine
// bins (model sub-buckets) of one partition holding at most `cap` pairs.  One
// CTA sorts an item in shared memory -- a counting sort on the leading bits of
// the keys' base-95 encoding over the item's key range (a placement by value,
// like the model's); when that leaves many keys in buckets of kSplitMin or
// more (skewed keys), a second counting pass splits those buckets on their
// next bits; every bucket of up to kRankMax pairs is then finished by ranking
// each pair against its bucket (the touch-up, one thread per pair), longer
// buckets split again the same way by warps on their own key range --
// and gathers the 100-byte records of the item, in order, straight into their
// final place in the output, so the partitions come out concatenated with no
// merge.  Items above `cap` pairs (heavy duplicate keys) take a multi-pass
// path: chunk sorts plus merge passes through global memory.
//
// Schedules: PERSISTENT = one launch, CTAs pull items from a global queue
// (oversize items first) -- the GPU form of the paper's dynamic scheduling of
// uneven partitions; PER_PARTITION = one launch per partition.
//
// Each CTA is warp-specialised: 8 sorter warps sort the next item in shared
// memory while kGatherWarps gatherer warps move the records of earlier ones,
// so that the sort's shared-memory work overlaps the gather's DRAM traffic.
// The sorters hand each sorted item over as a list of record indices in a
// ring of kSlots shared-memory slots (item s in slot s mod kSlots); named
// barriers FULL[b] (sorters arrive, gatherers wait) and EMPTY[b] (gatherers
// arrive, sorters wait before refilling slot b) order the two groups, every
// phase of each barrier taking exactly the 256 sorter and the gatherer
// threads once.  A last, producer warp finds the next item one ahead of the
// sorters (the queue claim or the partition's next item, its bounds, an L2
// prefetch of its pairs) and hands it over through two mbarrier-guarded
// slots, so that those dependent loads stay off the sorters' path.
#include "common.cuh"

namespace elsar {
namespace {

constexpr int kThreads = 256;  // sorter threads (warps 0-7)
constexpr int kWarps = kThreads / 32;
#ifndef ELSAR_GATHER_WARPS
#define ELSAR_GATHER_WARPS 5
#endif
constexpr int kGatherWarps = ELSAR_GATHER_WARPS;  // gatherer warps (after the sorters)
constexpr int kHandThreads = kThreads + 32 * kGatherWarps;  // the sorters and the gatherers
constexpr int kBlockThreads = kHandThreads + 32;           // and the producer warp (last)
constexpr uint32_t kSlots = 2;      // hand-over ring between the sorters and the gatherers
constexpr uint32_t kRankMax = 128;  // buckets up to this length are ranked inside the digit pass (the touch-up)

// named barriers: 1 = the sorter group; FULL[b] = 2 + b and EMPTY[b] = 2 + kSlots + b over the
// sorters and the gatherers (immediate ids, so that the kernel reserves only the barriers it uses)
__device__ __forceinline__ void sorter_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory"); }
#define ELSAR_BAR(op, id) asm volatile("bar." op " " #id ", %0;" ::"n"(kHandThreads) : "memory")
__device__ __forceinline__ void full_arrive(uint32_t b) {
  if (b == 0) ELSAR_BAR("arrive", 2);
  else if (b == 1) ELSAR_BAR("arrive", 3);
  else ELSAR_BAR("arrive", 4);
}
__device__ __forceinline__ void full_wait(uint32_t b) {
  if (b == 0) ELSAR_BAR("sync", 2);
  else if (b == 1) ELSAR_BAR("sync", 3);
  else ELSAR_BAR("sync", 4);
}
__device__ __forceinline__ void empty_arrive(uint32_t b) {
  if (b == 0) ELSAR_BAR("arrive", 5);
  else if (b == 1) ELSAR_BAR("arrive", 6);
  else ELSAR_BAR("arrive", 7);
}
__device__ __forceinline__ void empty_wait(uint32_t b) {
  if (b == 0) ELSAR_BAR("sync", 5);
  else if (b == 1) ELSAR_BAR("sync", 6);
  else ELSAR_BAR("sync", 7);
}
static_assert(kSlots <= 3, "the barrier helpers above name up to three slots");

// A sorted item handed from the sorters to the gatherers.
struct Handoff {
  uint64_t o0;            // first output record of the item (inside its record set)
  const uint8_t* in;      // the set's input records
  uint8_t* out;           // the set's output records
  const Pair* gsorted;    // mode 1: the item's sorted pairs in global memory
  uint32_t m;             // records
  uint32_t mode;          // 0: record indices in the slot's index list, 1: gsorted, 2: no more items
};

// The next work item, found by the producer warp: its id, first pair, pairs
// and record set, or the end of the work.
struct Meta {
  uint64_t o0;
  uint32_t it, m, set;
  uint32_t kind;  // 0: an item to sort, 1: no more items
};
constexpr uint32_t kMetaSlots = 2;

struct Misc {
  Handoff ho[kSlots];
  Meta meta[kMetaSlots];
  uint64_t meta_full[kMetaSlots];   // the producer posted meta[b] (one arrival)
  uint64_t meta_empty[kMetaSlots];  // the sorters are done with the item of meta[b] (one arrival)
  uint32_t meta_ok;                 // sorter thread 0's wait for the next meta succeeded
  volatile uint32_t heartbeat;      // advanced by the sorters inside long (oversize) items
  uint64_t red[2][kWarps];
  uint64_t kmin, kmax;
  uint32_t nlong, next_long, nsplit;
  uint32_t stk_top[kWarps];
  uint32_t item;
  uint64_t split[2];
  uint32_t wsum[33];
};

// Shared-memory tile of one work item.  Runs are packed as (start << 16) | length.
struct Tile {
  Pair* A;         // cap pairs
  uint32_t* cnt;   // cap digit counters
  uint16_t* perm;  // cap: sorted order being built
  uint16_t* perm2; // cap: scatter target
  uint32_t* longs; // cap/kRankMax + 1 long runs of the first digit pass
  uint32_t* stk;   // kWarps x (cap/kRankMax + 1) refinement stacks
  uint32_t* idx;   // kSlots x cap: record indices of the items handed to the gatherers
  uint16_t* dig2;  // cap: second-pass slot of each position
  uint16_t* sb;    // cap: second-pass slot of each placed element
  uint64_t* enc;   // cap: base-95 encodings of the tile's keys (computed once per item)
  uint32_t stk_cap, cap;
  Misc* ms;
};

struct KArgs {
  const uint8_t* in;
  uint8_t* out;
  const uint8_t* const* ins;  // batched path (null for one record set)
  uint8_t* const* outs;
  const uint64_t* tbase;
  const uint64_t* poff;
  uint32_t K;
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

// key used by a digit pass: 0 = base-95 encoding (dense for printable keys;
// cached in shared memory when the tile is loaded), 1 = raw key bytes 0-7,
// 2 = key bytes 8-9 and index.  Encoding order agrees with byte order; equal
// encodings are split by the raw bytes, then by lo.
__device__ __forceinline__ uint64_t sel_key(const Tile& t, uint32_t j, int sel) {
  return sel == 0 ? t.enc[j] : (sel == 1 ? t.A[j].hi : t.A[j].lo);
}

__device__ __forceinline__ uint32_t block_scan_excl(uint32_t v, uint32_t* wsum) {
  uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= (uint32_t)d) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  sorter_sync();
  if (warp == 0) {
    uint32_t w = lane < (uint32_t)kWarps ? wsum[lane] : 0;
    uint32_t wi = w;
    for (int d = 1; d < 32; d <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, wi, d);
      if (lane >= (uint32_t)d) wi += y;
    }
    if (lane < (uint32_t)kWarps) wsum[lane] = wi - w;
  }
  sorter_sync();
  uint32_t r = wsum[warp] + incl - v;
  sorter_sync();
  return r;
}

// block-wide min and max of one key field over the tile
__device__ void block_minmax(const Tile& t, uint32_t m, int sel) {
  uint64_t mn = ~0ull, mx = 0;
  for (uint32_t j = threadIdx.x; j < m; j += kThreads) {
    const uint64_t k = sel_key(t, j, sel);
    mn = min(mn, k);
    mx = max(mx, k);
  }
  for (int d = 16; d; d >>= 1) {
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, d));
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, d));
  }
  const int warp = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    t.ms->red[0][warp] = mn;
    t.ms->red[1][warp] = mx;
  }
  sorter_sync();
  if (threadIdx.x == 0) {
    uint64_t a = ~0ull, b = 0;
    for (int w = 0; w < kWarps; ++w) {
      a = min(a, t.ms->red[0][w]);
      b = max(b, t.ms->red[1][w]);
    }
    t.ms->kmin = a;
    t.ms->kmax = b;
  }
  sorter_sync();
}

// After a digit pass: position pos of perm holds record j of the bucket
// [rs, re).  A bucket of 2..kRankMax elements is finished here: every element
// is placed at its rank by the full key among the bucket (the touch-up: a
// comparison sort of what the model and the digit left unordered, each
// element ranked by its own thread, so long buckets of skewed keys spread over
// all threads); other elements keep their place.  The order is total (the
// record index breaks ties), so ranks are distinct.
__device__ __forceinline__ void place_ranked(const Tile& t, uint32_t pos, uint32_t rs, uint32_t re) {
  const uint16_t j = t.perm[pos];
  uint32_t dst = pos;
  if (re - rs >= 2 && re - rs <= kRankMax) {
    const Pair pj = t.A[j];
    uint32_t c = 0, q = rs;
    for (; q + 4 <= re; q += 4) {
      const uint16_t a0 = t.perm[q], a1 = t.perm[q + 1], a2 = t.perm[q + 2], a3 = t.perm[q + 3];
      c += (pair_less(t.A[a0], pj) ? 1u : 0u) + (pair_less(t.A[a1], pj) ? 1u : 0u) +
           (pair_less(t.A[a2], pj) ? 1u : 0u) + (pair_less(t.A[a3], pj) ? 1u : 0u);
    }
    for (; q < re; ++q) c += pair_less(t.A[t.perm[q]], pj) ? 1u : 0u;
    dst = rs + c;
  }
  t.perm2[dst] = j;
}

__device__ __forceinline__ uint64_t warp_min(uint64_t v) {
  for (int d = 16; d; d >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, d));
  return v;
}
__device__ __forceinline__ uint64_t warp_max(uint64_t v) {
  for (int d = 16; d; d >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, d));
  return v;
}

// One warp sorts perm[s0, s0+len0) (len0 > kRankMax) completely: a counting
// pass on a digit of the run's own key range, its buckets of up to kRankMax
// ranked in place and longer ones refined the same way (explicit stack).
// Every pass splits a run into at least two non-empty parts, so it
// terminates.
__device__ void warp_refine(const Tile& t, uint32_t s0, uint32_t len0) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t* stk = t.stk + warp * t.stk_cap;
  uint32_t* top = &t.ms->stk_top[warp];
  if (lane == 0) {
    stk[0] = (s0 << 16) | len0;
    *top = 1;
  }
  __syncwarp();
  for (;;) {
    const uint32_t n_top = *top;
    __syncwarp();
    if (n_top == 0) break;
    const uint32_t ent = stk[n_top - 1];
    __syncwarp();
    if (lane == 0) *top = n_top - 1;
    __syncwarp();
    const uint32_t s = ent >> 16, len = ent & 0xFFFFu;
    int sel = 0;
    uint64_t mn = ~0ull, mx = 0;
    for (;;) {
      mn = ~0ull;
      mx = 0;
      for (uint32_t i = lane; i < len; i += 32) {
        const uint64_t k = sel_key(t, t.perm[s + i], sel);
        mn = min(mn, k);
        mx = max(mx, k);
      }
      mn = warp_min(mn);
      mx = warp_max(mx);
      if (mn < mx || sel == 2) break;
      ++sel;
    }
    const uint32_t logD = 31 - __clz(len);  // len > kRankMax, so D >= 128
    const uint32_t D = 1u << logD;
    const uint64_t span = mx - mn;
    const uint32_t bits = 64 - __clzll((long long)span);
    const uint32_t shift = bits > logD ? bits - logD : 0;
    for (uint32_t d = lane; d < D; d += 32) t.cnt[s + d] = 0;
    __syncwarp();
    for (uint32_t i = lane; i < len; i += 32)
      atomicAdd(t.cnt + s + (uint32_t)((sel_key(t, t.perm[s + i], sel) - mn) >> shift), 1u);
    __syncwarp();
    {
      const uint32_t per = (D + 31) / 32;
      const uint32_t b = min(D, lane * per), e = min(D, b + per);
      uint32_t local = 0;
      for (uint32_t d = b; d < e; ++d) local += t.cnt[s + d];
      uint32_t incl = local;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += y;
      }
      uint32_t run = s + incl - local;
      for (uint32_t d = b; d < e; ++d) {
        const uint32_t c = t.cnt[s + d];
        t.cnt[s + d] = run;
        run += c;
      }
    }
    __syncwarp();
    for (uint32_t i = lane; i < len; i += 32) {
      const uint16_t j = t.perm[s + i];
      const uint32_t pos = atomicAdd(t.cnt + s + (uint32_t)((sel_key(t, j, sel) - mn) >> shift), 1u);
      t.perm2[pos] = j;
    }
    __syncwarp();
    for (uint32_t i = lane; i < len; i += 32) t.perm[s + i] = t.perm2[s + i];
    __syncwarp();
    // buckets up to kRankMax ranked in place; longer ones go on the stack
    for (uint32_t i = lane; i < len; i += 32) {
      const uint32_t d = (uint32_t)((sel_key(t, t.perm[s + i], sel) - mn) >> shift);
      place_ranked(t, s + i, d ? t.cnt[s + d - 1] : s, t.cnt[s + d]);
    }
    __syncwarp();
    for (uint32_t i = lane; i < len; i += 32) t.perm[s + i] = t.perm2[s + i];
    __syncwarp();
    for (uint32_t d = lane; d < D; d += 32) {
      const uint32_t ss = d ? t.cnt[s + d - 1] : s, ee = t.cnt[s + d];
      const uint32_t l = ee - ss;
      if (l > kRankMax) stk[atomicAdd(top, 1u)] = (ss << 16) | l;
    }
    __syncwarp();
  }
}

// Sort the tile A[0, m) (m <= cap): on return perm[0, m) lists A in
// (hi, lo) order.  First digit pass block-wide over the whole tile, its short
// buckets ranked in place by all threads, then the long runs are finished by
// warps in parallel.
// buckets of the first digit pass with this many elements or more are split
// by a second counting pass when they hold at least 1/8 of the tile
constexpr uint32_t kSplitMin = 8;

__device__ void tile_sort(const Tile& t, uint32_t m) {
  Misc& ms = *t.ms;
  if (m <= 1) {
    if (threadIdx.x == 0 && m == 1) t.perm[0] = 0;
    sorter_sync();
    return;
  }
  int sel = 0;
  block_minmax(t, m, 0);
  if (ms.kmin == ms.kmax) {
    sel = 1;
    block_minmax(t, m, 1);
    if (ms.kmin == ms.kmax) {
      sel = 2;
      block_minmax(t, m, 2);
    }
  }
  const uint64_t kmin = ms.kmin, span = ms.kmax - ms.kmin;
  uint32_t logD = 0;
  while ((1u << logD) < m) ++logD;
  const uint32_t D = 1u << logD;
  const uint32_t bits = span ? 64 - __clzll((long long)span) : 0;
  const uint32_t shift = bits > logD ? bits - logD : 0;
  for (uint32_t d = threadIdx.x; d < D; d += kThreads) t.cnt[d] = 0;
  if (threadIdx.x == 0) {
    ms.nlong = 0;
    ms.next_long = 0;
    ms.nsplit = 0;
  }
  sorter_sync();
  for (uint32_t j = threadIdx.x; j < m; j += kThreads)
    atomicAdd(t.cnt + (uint32_t)((sel_key(t, j, sel) - kmin) >> shift), 1u);
  sorter_sync();
  {
    const uint32_t per = (D + kThreads - 1) / kThreads;
    const uint32_t b = min(D, threadIdx.x * per), e = min(D, b + per);
    uint32_t local = 0, big = 0;
    for (uint32_t d = b; d < e; ++d) {
      const uint32_t c = t.cnt[d];
      local += c;
      big += c >= kSplitMin ? c : 0u;
    }
    if (big) atomicAdd(&ms.nsplit, big);  // elements in buckets of kSplitMin or more
    uint32_t run = block_scan_excl(local, ms.wsum);
    for (uint32_t d = b; d < e; ++d) {
      const uint32_t c = t.cnt[d];
      t.cnt[d] = run;
      run += c;
    }
  }
  sorter_sync();
  if (ms.nsplit * 8 >= m) {
    // second counting pass, straight from the first pass's bucket starts (no
    // placement by the first digit): an element of a bucket [rs, rs + len) of
    // kSplitMin or more goes to slot rs + sub, sub the next lb = floor(log2 len)
    // bits of its key below the bucket's digit (2^lb <= len, so the slots stay
    // inside the bucket); an element of a smaller bucket goes to slot rs.  Slots
    // of different buckets never mix, so one plain exclusive scan over the tile
    // gives every slot its final start, and a bucket's slots start at rs.
    for (uint32_t j = threadIdx.x; j < m; j += kThreads) {
      const uint64_t key = sel_key(t, j, sel);
      const uint32_t d = (uint32_t)((key - kmin) >> shift);
      const uint32_t rs = t.cnt[d], len = (d + 1 < D ? t.cnt[d + 1] : m) - rs;
      uint32_t x = rs;
      if (len >= kSplitMin) {
        const uint32_t lb = 31 - __clz(len);
        const uint64_t local = (key - kmin) - ((uint64_t)d << shift);
        x = rs + (uint32_t)(shift >= lb ? local >> (shift - lb) : local);
      }
      t.dig2[j] = (uint16_t)x;
    }
    sorter_sync();
    for (uint32_t x = threadIdx.x; x < m; x += kThreads) t.cnt[x] = 0;
    sorter_sync();
    for (uint32_t j = threadIdx.x; j < m; j += kThreads) atomicAdd(t.cnt + t.dig2[j], 1u);
    sorter_sync();
    {
      const uint32_t per = (m + kThreads - 1) / kThreads;
      const uint32_t b = min(m, threadIdx.x * per), e = min(m, b + per);
      uint32_t local = 0;
      for (uint32_t x = b; x < e; ++x) local += t.cnt[x];
      uint32_t run = block_scan_excl(local, ms.wsum);
      for (uint32_t x = b; x < e; ++x) {
        const uint32_t c = t.cnt[x];
        t.cnt[x] = run;
        run += c;
      }
    }
    sorter_sync();
    for (uint32_t j = threadIdx.x; j < m; j += kThreads) {
      const uint32_t x = t.dig2[j];
      const uint32_t np = atomicAdd(t.cnt + x, 1u);
      t.perm[np] = (uint16_t)j;
      t.sb[np] = (uint16_t)x;
    }
    sorter_sync();
    // slot x now holds [cnt[x-1], cnt[x]); rank inside slots of up to kRankMax
    for (uint32_t pos = threadIdx.x; pos < m; pos += kThreads) {
      const uint32_t x = t.sb[pos];
      place_ranked(t, pos, x ? t.cnt[x - 1] : 0, t.cnt[x]);
    }
    sorter_sync();
    for (uint32_t pos = threadIdx.x; pos < m; pos += kThreads) t.perm[pos] = t.perm2[pos];
    for (uint32_t x = threadIdx.x; x < m; x += kThreads) {
      const uint32_t s0 = x ? t.cnt[x - 1] : 0, len = t.cnt[x] - s0;
      if (len > kRankMax) t.longs[atomicAdd(&ms.nlong, 1u)] = (s0 << 16) | len;
    }
    sorter_sync();
  } else {
    for (uint32_t j = threadIdx.x; j < m; j += kThreads) {
      const uint32_t pos = atomicAdd(t.cnt + (uint32_t)((sel_key(t, j, sel) - kmin) >> shift), 1u);
      t.perm[pos] = (uint16_t)j;
    }
    sorter_sync();
    // buckets up to kRankMax ranked in place (every element by its own thread)
    for (uint32_t pos = threadIdx.x; pos < m; pos += kThreads) {
      const uint32_t d = (uint32_t)((sel_key(t, t.perm[pos], sel) - kmin) >> shift);
      place_ranked(t, pos, d ? t.cnt[d - 1] : 0, t.cnt[d]);
    }
    sorter_sync();
    for (uint32_t pos = threadIdx.x; pos < m; pos += kThreads) t.perm[pos] = t.perm2[pos];
    for (uint32_t d = threadIdx.x; d < D; d += kThreads) {
      const uint32_t s = d ? t.cnt[d - 1] : 0, e = t.cnt[d];
      const uint32_t len = e - s;
      if (len > kRankMax) t.longs[atomicAdd(&ms.nlong, 1u)] = (s << 16) | len;
    }
    sorter_sync();
  }
  const uint32_t lane = threadIdx.x & 31;
  for (;;) {
    uint32_t r = 0;
    if (lane == 0) r = atomicAdd(&ms.next_long, 1u);
    r = __shfl_sync(0xffffffffu, r, 0);
    if (r >= ms.nlong) break;
    const uint32_t ent = t.longs[r];
    warp_refine(t, ent >> 16, ent & 0xFFFFu);
  }
  sorter_sync();
}

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Gather m records in sorted order into out[o0, o0 + m) by the gatherer
// warps, 32 records per warp step: lanes 0-24 each move word `lane` of every
// record of the group (one broadcast shuffle, one load and one store per
// word: a record's 25 words are one coalesced 100-byte access).  While a warp
// moves one group it asks L2 for the lines of its next group, so twice as
// many records are in flight without holding more registers.
template <typename IdxFn>
__device__ __forceinline__ void gather(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, uint64_t o0,
                                       uint32_t m, IdxFn idx_of) {
  constexpr uint32_t kStride = 32 * kGatherWarps;
  const uint32_t lane = threadIdx.x & 31, warp = (threadIdx.x - kThreads) >> 5;
  const uint32_t* __restrict__ in32 = reinterpret_cast<const uint32_t*>(in);
  uint32_t* __restrict__ out32 = reinterpret_cast<uint32_t*>(out);
  for (uint32_t j0 = warp * 32; j0 < m; j0 += kStride) {
    const uint32_t nrec = min(32u, m - j0);
    const uint32_t my = lane < nrec ? idx_of(j0 + lane) : 0;
    const uint32_t jn = j0 + kStride + lane;
    if (jn < m) {
      const uint8_t* r = in + (uint64_t)idx_of(jn) * kRecord;
      prefetch_l2(r);
      prefetch_l2(r + kRecord - 1);
    }
    uint32_t v[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
      const uint32_t src = __shfl_sync(0xffffffffu, my, r);
      v[r] = (lane < 25u && (uint32_t)r < nrec) ? __ldg(in32 + (uint64_t)src * 25u + lane) : 0u;
    }
    uint32_t* dst = out32 + (o0 + j0) * 25u + lane;
#pragma unroll
    for (int r = 0; r < 32; ++r)
      if (lane < 25u && (uint32_t)r < nrec) dst[r * 25] = v[r];
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

__device__ __forceinline__ void load_tile(const Tile& t, const Pair* src, uint32_t m) {
  for (uint32_t j = threadIdx.x; j < m; j += kThreads) {
    const Pair p = src[j];
    t.A[j] = p;
    t.enc[j] = enc9_pair(p);
  }
  sorter_sync();
}

// items above cap: sort cap-sized chunks in place, then merge passes between
// pairs and temp; returns the array holding the sorted run
__device__ const Pair* sort_oversize(const KArgs& k, const Tile& t, uint64_t o0, uint32_t m) {
  const uint32_t cap = k.cap;
  Pair* src = k.pairs;
  Pair* dst = k.temp;
  Misc& ms = *t.ms;
  for (uint32_t c0 = 0; c0 < m; c0 += cap) {
    const uint32_t mc = min(cap, m - c0);
    load_tile(t, src + o0 + c0, mc);
    tile_sort(t, mc);
    for (uint32_t j = threadIdx.x; j < mc; j += kThreads) src[o0 + c0 + j] = t.A[t.perm[j]];
    if (threadIdx.x == 0) ms.heartbeat = ms.heartbeat + 1;  // progress, for the producer's bounded wait
    sorter_sync();
  }
  Pair* A = t.A;
  for (uint32_t w = cap; w < m; w *= 2) {
    for (uint32_t t0 = 0; t0 < m; t0 += cap) {
      const uint32_t p0 = (t0 / (2 * w)) * (2 * w);
      const uint32_t a1 = min(m, p0 + w), b1 = min(m, p0 + 2 * w);
      const uint32_t t1 = min(b1, t0 + cap);
      const Pair* ga = src + o0 + p0;
      const Pair* gb = src + o0 + a1;
      if (threadIdx.x < 2) ms.split[threadIdx.x] = merge_split(ga, a1 - p0, gb, b1 - a1, (threadIdx.x ? t1 : t0) - p0);
      if (threadIdx.x == 0) ms.heartbeat = ms.heartbeat + 1;
      sorter_sync();
      const uint32_t ka0 = (uint32_t)ms.split[0], ka1 = (uint32_t)ms.split[1];
      const uint32_t kb0 = (t0 - p0) - ka0, kb1 = (t1 - p0) - ka1;
      const uint32_t na = ka1 - ka0, nb = kb1 - kb0;
      for (uint32_t j = threadIdx.x; j < na; j += kThreads) A[j] = ga[ka0 + j];
      for (uint32_t j = threadIdx.x; j < nb; j += kThreads) A[na + j] = gb[kb0 + j];
      sorter_sync();
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
        for (uint32_t q = 0; q < per && d + q < tot; ++q) {
          bool takeA = ib >= nb || (ia < na && !pair_less(A[na + ib], A[ia]));
          dst[o0 + t0 + d + q] = takeA ? A[ia++] : A[na + ib++];
        }
      }
      sorter_sync();
    }
    Pair* tmp = src;
    src = dst;
    dst = tmp;
    sorter_sync();
  }
  return src;
}

__device__ __forceinline__ uint32_t set_of_bin(const uint64_t* __restrict__ tbase, uint32_t K, uint64_t b) {
  uint32_t lo = 0, hi = K - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (tbase[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Sorter side of one work item (found by the producer): sort it and hand it
// to the gatherers in slot (slot mod kSlots).
__device__ void sort_item(const KArgs& k, const Tile& t, const Meta& me, uint32_t slot) {
  const uint64_t o0 = me.o0;
  const uint32_t m = me.m;
  // records of this item: one set's buffers (batched path) or the only set
  const uint8_t* in = k.in;
  uint8_t* out = k.out;
  uint64_t base = 0;
  if (k.ins) {
    in = k.ins[me.set];
    out = k.outs[me.set];
    base = k.poff[me.set];
  }
  const uint32_t b = slot % kSlots;
  Handoff h;
  h.o0 = o0 - base;
  h.in = in;
  h.out = out;
  h.m = m;
  if (m <= k.cap) {
    load_tile(t, k.pairs + o0, m);
    tile_sort(t, m);
    if (slot >= kSlots) empty_wait(b);  // the gatherers are done with this slot's previous item
    uint32_t* idx = t.idx + b * t.cap;
    for (uint32_t j = threadIdx.x; j < m; j += kThreads) idx[j] = (uint32_t)t.A[t.perm[j]].lo;
    h.gsorted = nullptr;
    h.mode = 0;
  } else {
    const Pair* sorted = sort_oversize(k, t, o0, m);
    if (slot >= kSlots) empty_wait(b);
    h.gsorted = sorted + o0;
    h.mode = 1;
  }
  if (threadIdx.x == 0) t.ms->ho[b] = h;
  __threadfence_block();  // global (oversize) and shared writes before the hand-over
  full_arrive(b);
}

// Sorter side: no more items.  Slot n (the number handed over) says so; then
// the gatherers' releases of the last items still unclaimed are taken, so
// that every phase of every EMPTY barrier has completed when the sorters leave.
__device__ void sorters_done(const Tile& t, uint32_t n) {
  const uint32_t b = n % kSlots;
  if (n >= kSlots) empty_wait(b);  // releases item n - kSlots
  if (threadIdx.x == 0) t.ms->ho[b].mode = 2;
  __threadfence_block();
  full_arrive(b);
  for (uint32_t s = n >= kSlots ? n - kSlots + 1 : 0; s < n; ++s) empty_wait(s % kSlots);
}

// Gatherer side: items in slot order until the sorters say there are no more.
__device__ void gatherer_loop(const Tile& t) {
  for (uint32_t slot = 0;; ++slot) {
    const uint32_t b = slot % kSlots;
    full_wait(b);
    const Handoff h = t.ms->ho[b];
    if (h.mode == 2) break;
    if (h.mode == 0) {
      const uint32_t* idx = t.idx + b * t.cap;
      gather(h.in, h.out, h.o0, h.m, [&](uint32_t j) { return idx[j]; });
    } else {
      const Pair* g = h.gsorted;
      gather(h.in, h.out, h.o0, h.m, [&](uint32_t j) { return (uint32_t)g[j].lo; });
    }
    empty_arrive(b);
  }
}

__device__ __forceinline__ Tile carve(uint8_t* smem, uint32_t cap) {
  Tile t;
  uint8_t* p = smem;
  t.A = reinterpret_cast<Pair*>(p);
  p += (size_t)cap * sizeof(Pair);
  t.cnt = reinterpret_cast<uint32_t*>(p);
  p += (size_t)cap * 4;
  t.perm = reinterpret_cast<uint16_t*>(p);
  p += (size_t)cap * 2;
  t.perm2 = reinterpret_cast<uint16_t*>(p);
  p += (size_t)cap * 2;
  t.stk_cap = cap / kRankMax + 1;  // disjoint runs longer than kRankMax
  t.longs = reinterpret_cast<uint32_t*>(p);
  p += (size_t)t.stk_cap * 4;
  t.stk = reinterpret_cast<uint32_t*>(p);
  p += (size_t)kWarps * t.stk_cap * 4;
  t.idx = reinterpret_cast<uint32_t*>(p);
  p += (size_t)kSlots * cap * 4;
  t.dig2 = reinterpret_cast<uint16_t*>(p);
  p += (size_t)cap * 2;
  t.sb = reinterpret_cast<uint16_t*>(p);
  p += (size_t)cap * 2;
  p = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15);
  t.enc = reinterpret_cast<uint64_t*>(p);
  p += (size_t)cap * 8;
  t.cap = cap;
  p = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 15) & ~(uintptr_t)15);
  t.ms = reinterpret_cast<Misc*>(p);
  return t;
}

// Bounded wait of the producer for the sorters to finish an item: the clock
// restarts whenever the sorters advance the heartbeat, so a long oversize
// item does not run it out while a stall still ends it.
__device__ bool producer_wait(Misc& ms, uint64_t* bar, uint32_t parity) {
  long long t0 = clock64();
  uint32_t hb = ms.heartbeat;
  while (!mbar_test_wait(bar, parity)) {
    const uint32_t now = ms.heartbeat;
    if (now != hb) {
      hb = now;
      t0 = clock64();
    } else if (clock64() - t0 > kWaitLimitCycles) {
      return false;
    }
  }
  return true;
}

// Producer warp: finds the CTA's next work item (claimed from the global
// queue, or the next of its partition), reads where its pairs lie and asks
// L2 for them, one item ahead of the sorters, so that the claim and the
// dependent index loads leave the sorters' path.  Item n goes through
// meta[n mod 2]: meta_full[b] completes when it is posted, meta_empty[b] when
// the sorters have finished it.
__device__ void producer_loop(const KArgs& k, Misc& ms) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t num_items = k.ctrl[kNumItems];
  const uint32_t num_over = k.persistent ? k.ctrl[kNumOversize] : 0;
  uint32_t next = k.persistent ? 0 : k.part_items[k.part] + blockIdx.x;  // per-partition: the next item id
  const uint32_t last = k.persistent ? 0 : k.part_items[k.part + 1];
  for (uint32_t n = 0;; ++n) {
    const uint32_t b = n % kMetaSlots;
    uint32_t ok = 1;
    if (lane == 0 && n >= kMetaSlots) ok = producer_wait(ms, &ms.meta_empty[b], ((n - kMetaSlots) / kMetaSlots) & 1);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) {  // the sorters stopped advancing: report it and stop (their own wait for meta gives up too)
      if (lane == 0) atomicOr(k.ctrl + kStatusWord, 1u);
      return;
    }
    Meta me = {};
    me.kind = 1;
    if (lane == 0) {
      for (;;) {
        uint32_t it;
        if (k.persistent) {
          const uint32_t j = atomicAdd(k.ctrl + kQueueHead, 1u);
          if (j >= num_over + num_items) break;
          it = j < num_over ? k.oversize[j] : j - num_over;
          const uint64_t a = k.bin_off[k.items[it]], e = k.bin_off[k.items[it + 1]];
          if (j >= num_over && e - a > k.cap) continue;  // done in the oversize phase
          if (e == a) continue;
          me.o0 = a;
          me.m = (uint32_t)(e - a);
        } else {
          if (next >= last) break;
          it = next;
          next += gridDim.x;
          const uint64_t a = k.bin_off[k.items[it]], e = k.bin_off[k.items[it + 1]];
          if (e == a) continue;
          me.o0 = a;
          me.m = (uint32_t)(e - a);
        }
        me.it = it;
        me.set = k.ins ? set_of_bin(k.tbase, k.K, k.items[it]) : 0;
        me.kind = 0;
        // the item's pairs into L2 now (16-byte aligned, whole pairs)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(k.pairs + me.o0),
                     "r"(min(me.m, k.cap) * (uint32_t)sizeof(Pair))
                     : "memory");
        break;
      }
      ms.meta[b] = me;
      asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&ms.meta_full[b]))
                   : "memory");
    }
    if (__shfl_sync(0xffffffffu, me.kind, 0) == 1) return;
  }
}

__global__ void __launch_bounds__(kBlockThreads, 2) sort_gather_kernel(KArgs k) {
  extern __shared__ __align__(16) uint8_t smem[];
  if (k.ctrl[kStatusWord]) return;  // partitioning gave up: no item is valid (uniform over the CTA)
  const Tile t = carve(smem, k.cap);
  Misc& ms = *t.ms;
  if (threadIdx.x == 0) {
    for (uint32_t b = 0; b < kMetaSlots; ++b) {
      mbar_init(&ms.meta_full[b], 1);
      mbar_init(&ms.meta_empty[b], 1);
    }
    ms.heartbeat = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x >= kHandThreads) {
    producer_loop(k, ms);
    return;
  }
  if (threadIdx.x >= kThreads) {
    gatherer_loop(t);
    return;
  }
  uint32_t slot = 0;
  for (uint32_t n = 0;; ++n) {
    const uint32_t b = n % kMetaSlots;
    if (threadIdx.x == 0) ms.meta_ok = mbar_wait(&ms.meta_full[b], (n / kMetaSlots) & 1, kWaitLimitCycles) ? 1u : 0u;
    sorter_sync();
    if (!ms.meta_ok) {  // the producer stopped: the status word says why (or is set here)
      if (threadIdx.x == 0) atomicOr(k.ctrl + kStatusWord, 1u);
      break;
    }
    const Meta me = ms.meta[b];
    if (me.kind == 1) break;
    sort_item(k, t, me, slot);
    ++slot;
    sorter_sync();  // every sorter thread is done with the item (and with meta[b])
    if (threadIdx.x == 0)
      asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&ms.meta_empty[b]))
                   : "memory");
  }
  sorters_done(t, slot);
}

// item range of each partition (per-partition schedule): item id of the partition's first bin
__global__ void part_items_kernel(const uint32_t* cuts, const uint32_t* item_of_bin, uint32_t P, uint32_t log2B,
                                  const uint32_t* ctrl, uint32_t* part_items) {
  const uint32_t B = 1u << log2B;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p <= P; p += gridDim.x * blockDim.x)
    part_items[p] = cuts[p] < B ? item_of_bin[cuts[p]] : ctrl[kNumItems];
}

}  // namespace

size_t sort_smem_bytes(uint32_t cap) {
  const size_t stk = (size_t)(cap / kRankMax + 1) * 4;
  return (size_t)cap * (sizeof(Pair) + 4 + 2 + 2 + kSlots * 4 + 8 + 4) + stk * (1 + kWarps) + 32 + sizeof(Misc);
}

cudaError_t prepare_sort_kernel(uint32_t cap) {
  return cudaFuncSetAttribute(sort_gather_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sort_smem_bytes(cap));
}

cudaError_t sort_items(const SortArgs& a) {
  KArgs k = {};
  k.in = a.records;
  k.out = a.out;
  k.ins = a.ins;
  k.outs = a.outs;
  k.tbase = a.tbase;
  k.poff = a.poff;
  k.K = a.K;
  k.pairs = a.pairs;
  k.temp = a.temp;
  k.bin_off = a.bin_off;
  k.items = a.items;
  k.oversize = a.oversize;
  k.ctrl = a.ctrl;
  k.cap = a.tile_pairs;
  const size_t smem = sort_smem_bytes(a.tile_pairs);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(a.stream, &cs);
  if (cs == cudaStreamCaptureStatusNone) {
    cudaError_t err = prepare_sort_kernel(a.tile_pairs);
    if (err != cudaSuccess) return err;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sort_gather_kernel, kBlockThreads, smem);
  if (per_sm < 1) per_sm = 1;
  const int sms = sm_count();
  if (a.schedule == 1) {
    k.persistent = 1;
    sort_gather_kernel<<<sms * per_sm, kBlockThreads, smem, a.stream>>>(k);
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
      sort_gather_kernel<<<grid, kBlockThreads, smem, a.stream>>>(k);
    }
    *a.launches += 1 + a.P;
  }
  return cudaGetLastError();
}

}  // namespace elsar
