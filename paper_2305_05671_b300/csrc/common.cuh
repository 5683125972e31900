// Internal declarations shared by the libelsar CUDA sources (not part of the ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace elsar {

constexpr int kRecord = 100;
constexpr uint64_t kEncTop = 630249409724609375ull;  // 95^9: one past the largest 9-character encoding
constexpr uint32_t kModelMagic = 0x52534C45u;        // "ELSR"
constexpr uint32_t kSettled = 0xFFFFFFFFu;           // sample point whose RMI node is already a leaf
constexpr uint32_t kSettledBit = 0x80000000u;        // settled point: this bit | the index of its leaf
constexpr int kCoarse = 4096;                        // splitters kept in shared memory for classification

// 16-byte sort pair (the paper's pointer-only record, Sec. 3.3): ordering by
// (hi, lo) is memcmp order of the 10-byte key, then input order.
//   hi = key bytes 0-7 big-endian
//   lo = (key bytes 8-9 big-endian) << 32 | record index
struct __align__(16) Pair {
  uint64_t hi;
  uint64_t lo;
};

__device__ __forceinline__ bool pair_less(const Pair& a, const Pair& b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}

// One RMI node (64 bytes).  Internal: a = gamma, b = delta, c = scale.
// Leaf: a = g, b = d, c = lo, h = hi (output constants of Sec. 3.1's model).
// depth_set = depth (low 8 bits) | record set << 8 (batched fits hold one
// tree per set; s, e are positions in the concatenated sorted samples).
struct __align__(64) DNode {
  uint32_t s, e;  // sample positions covered
  uint64_t base;
  uint32_t child0, fanout;  // fanout 0 = leaf
  uint32_t shift, depth_set;
  double a, b, c, h;
};

// Sample segment of one record set: sorted sample positions [soff, soff + S).
struct SetInfo {
  uint64_t soff, S;
};

struct ModelHeader {
  uint32_t magic, kind, log2B, num_nodes;
  uint64_t S, node_cap;
  uint64_t nodes_off, splitters_off, bytes;
  uint32_t T, Dmax, levels, fallback;
  uint64_t lut_off, knots_off, weights_off;  // radix index, the network's knots and weights
};

// The k-th output of the SplitMix64 generator seeded with `seed` (Steele,
// Lea, Flood 2014): the sample positions are mulhi64(SplitMix64_k(seed), n).
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Key encoding (Sec. 4): 9 base-95 digits (ASCII - 32) of printable bytes.
// w0 = bytes 0-3, w1 = bytes 4-7 as big-endian words; b8 = byte 8.  A byte
// outside 32..126 saturates that digit and every later one to 0 (below) or
// 94 (above), which keeps the encoding monotone in byte order for any key.
__device__ __forceinline__ uint32_t digits4(uint32_t w) {
  w = __vsub4(w, 0x20202020u);
  return (((w >> 24) * 95u + ((w >> 16) & 0xFFu)) * 95u + ((w >> 8) & 0xFFu)) * 95u + (w & 0xFFu);
}

static __device__ __noinline__ uint64_t enc9_saturating(uint32_t w0, uint32_t w1, uint32_t b8) {
  uint64_t e = 0;
  int sat = 0;
  for (int i = 0; i < 9; ++i) {
    uint32_t c = i < 4 ? (w0 >> (24 - 8 * i)) & 0xFFu : (i < 8 ? (w1 >> (56 - 8 * i)) & 0xFFu : b8);
    if (sat == 0 && c < 32u) sat = 1;
    if (sat == 0 && c > 126u) sat = 2;
    e = e * 95u + (sat == 1 ? 0u : (sat == 2 ? 94u : c - 32u));
  }
  return e;
}

__device__ __forceinline__ uint64_t enc9_words(uint32_t w0, uint32_t w1, uint32_t b8) {
  const uint32_t out = __vcmpltu4(w0, 0x20202020u) | __vcmpgtu4(w0, 0x7E7E7E7Eu) | __vcmpltu4(w1, 0x20202020u) |
                       __vcmpgtu4(w1, 0x7E7E7E7Eu);
  if (out | (b8 < 32u) | (b8 > 126u)) return enc9_saturating(w0, w1, b8);
  return ((uint64_t)digits4(w0) * 81450625ull + digits4(w1)) * 95ull + (b8 - 32u);  // 95^4 = 81450625
}

__device__ __forceinline__ uint64_t enc9_pair(const Pair& p) {
  return enc9_words((uint32_t)(p.hi >> 32), (uint32_t)p.hi, (uint32_t)(p.lo >> 40) & 0xFFu);
}

// Keys of key_bytes = l (1..10) bytes (Sec. 4's variable-length keys, l the
// longest): the bytes of the key field after the key count as 0 -- in the
// pair they are masked to 0, so the encoding saturates to 0 there and byte
// order compares the padded keys.  hi keeps key bytes 0-7, lo bits 32-47
// bytes 8-9 (and the record index below).
struct KeyMask {
  uint64_t hi, lo;
};
inline KeyMask key_mask(uint32_t key_bytes) {
  KeyMask m;
  m.hi = key_bytes >= 8 ? ~0ull : (key_bytes ? ~0ull << (64 - 8 * key_bytes) : 0ull);
  const uint64_t lo16 = key_bytes >= 10 ? 0xFFFFull : (key_bytes == 9 ? 0xFF00ull : 0ull);
  m.lo = (lo16 << 32) | 0xFFFFFFFFull;
  return m;
}

// Load the key of a 4-byte-aligned record and pack it.
__device__ __forceinline__ Pair load_pair(const uint8_t* rec, uint32_t idx, const KeyMask& km) {
  const uint32_t* w = reinterpret_cast<const uint32_t*>(rec);
  uint32_t a = __ldg(w), b = __ldg(w + 1), c = __ldg(w + 2);
  uint32_t be0 = __byte_perm(a, 0, 0x0123), be1 = __byte_perm(b, 0, 0x0123);
  uint32_t be16 = __byte_perm(c, 0, 0x4401);
  Pair p;
  p.hi = (((uint64_t)be0 << 32) | be1) & km.hi;
  p.lo = (((uint64_t)be16 << 32) | idx) & km.lo;
  return p;
}

// ---------------------------------------------------------------- radix index of the splitters
// Cell c covers encodings [c << kFineLutShift, (c + 1) << kFineLutShift).
// Level 1 (uint4 per cell): .x = q, the largest index with t[q] <= c <<
// kFineLutShift; .z/.w = the low and high words of t[q + 1] (95^9 past the
// last splitter), so a cell holding one splitter is resolved by its own
// entry; .y = (the cell's splitter count << 5) for a cell of up to kLutDense
// splitters, or, for a cell holding more, (offset << 5) | nb (nb > 0): the
// cell is split into 2^nb sub-cells whose level-2
// entries lut2[offset + k] (k = 0..2^nb) hold the largest q with t[q] <= the
// sub-cell's start.  Either way the answer for x lies in [lo, hi] of x's cell
// or sub-cell, and a short binary search finishes it.  The level-2 table
// lives right after level 1 (kFineLutCells uint4 entries).
constexpr int kFineLutShift = 42;
constexpr uint32_t kFineLutCells = (uint32_t)((kEncTop - 1) >> kFineLutShift) + 2;
constexpr uint32_t kLutL1Words = 4;    // words of a level-1 entry
constexpr uint32_t kLutDense = 4;      // cells with more splitters get a level-2 split
constexpr uint32_t kLutMaxBits = 14;   // at most 2^14 sub-cells per cell
constexpr uint32_t kLutOversplit = 2;  // sub-cells = 4 x the cell's splitters rounded up to a power of two
constexpr uint32_t kLutWarpBits = 10;  // cells of up to 2^10 sub-cells are filled by a warp, larger ones by a block
// Level-2 capacity for 2^log2B splitters: a dense cell with cnt splitters
// takes 2^nb + 1 < 8 cnt + 1 words and at most B/5 cells are dense, so
// 8B + B/4 words hold every split.  While the index is built, the words
// after those hold the list of cells with more than 2^kLutWarpBits sub-cells
// (more than 256 splitters each, so at most B/256 of them; a count, then
// the cells) and, in the last 256, the scan's block totals.
inline size_t lut_big_words(uint32_t log2B) { return ((size_t)1 << log2B) / 256 + 2; }
inline size_t lut_level2_words(uint32_t log2B) {
  const size_t B = (size_t)1 << log2B;
  return 8 * B + B / 4 + lut_big_words(log2B) + 256;
}
// words of the whole index (level 1 and level 2)
inline size_t lut_words_for(uint32_t log2B) {
  return kLutL1Words * (size_t)kFineLutCells + lut_level2_words(log2B);
}

// [lo, hi]: the search range of splitter indices for x (lo == hi: resolved)
__device__ __forceinline__ void lut_range(const uint32_t* __restrict__ lut, uint64_t x, uint32_t& lo, uint32_t& hi) {
  const uint4* l1 = reinterpret_cast<const uint4*>(lut);
  const uint32_t c = (uint32_t)(x >> kFineLutShift);
  const uint4 a = __ldg(l1 + c);
  lo = a.x;
  const uint32_t nb = a.y & 31;
  if (nb) {
    const uint32_t off = a.y >> 5;
    const uint32_t k = (uint32_t)(x >> (kFineLutShift - nb)) & ((1u << nb) - 1);
    const uint32_t* l2 = lut + kLutL1Words * kFineLutCells + off;
    lo = __ldg(l2 + k);
    hi = __ldg(l2 + k + 1);
  } else {
    hi = lo + (a.y >> 5);  // the cell's splitter count is in the entry
    if (hi == lo + 1) {    // one splitter in the cell: its value is in the entry
      const uint64_t next = ((uint64_t)a.w << 32) | a.z;
      lo = next <= x ? hi : lo;
      hi = lo;
    }
  }
}

// q = largest j with t[j] <= x, via the radix index then a binary search
__device__ __forceinline__ uint32_t splitter_search(const uint64_t* __restrict__ t, const uint32_t* __restrict__ lut,
                                                    uint64_t x) {
  uint32_t lo, hi;
  lut_range(lut, x, lo, hi);
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(t + mid) <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------- bulk copies (TMA) and mbarriers
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Non-blocking test of an mbarrier phase (mbarrier.test_wait returns at once).
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

constexpr long long kWaitLimitCycles = 2000000000ll;  // about one second at B300 clocks
constexpr long long kShortWaitCycles = 1000000ll;     // limits below this poll without suspending

// Bounded wait on an mbarrier phase: false after `limit` clock cycles.  A
// try_wait may suspend the thread until the phase completes, so a short limit
// (below kShortWaitCycles, about half a millisecond) polls with the
// non-blocking test_wait instead, which lets it run out while a copy is
// still in flight.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  if (limit < kShortWaitCycles) {
    while (!mbar_test_wait(bar, parity))
      if (clock64() - t0 > limit) return false;
    return true;
  }
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// ---------------------------------------------------------------- launchers
struct FitArgs {
  const uint8_t* records;
  KeyMask km;
  uint64_t n, S, seed;
  uint32_t log2B, T, Dmax;
  void* model;
  size_t model_bytes;
  // scratch
  uint64_t* samp;   // 2*S
  uint32_t* pnode;  // S
  uint64_t* sums;   // node_cap * 6
  uint32_t* fc;     // 2 * node_cap: split fanouts, child offsets
  uint32_t* ctrl;   // 64 words
  SetInfo* sets;    // one entry (single record set)
  cudaStream_t stream;
  uint32_t* launches;
};

// Level-by-level RMI construction over K trees at once (K record sets whose
// sorted samples are concatenated; sets[k] gives each segment).  `device_loop`
// runs the levels in a graph whose while-node repeats them until a level has
// no children (single-set path; no host round trip) unless the stream is
// being captured; otherwise a fixed number of levels is launched and empty
// levels exit at once (capturable in a caller's graph).  The level count ends in ctrl[kLevelNodes + 5], the node
// count in ctrl[kLevelNodes + 3].
struct RmiLevelsArgs {
  const uint64_t* x;  // concatenated sorted samples
  uint64_t S_total;
  const SetInfo* sets;
  uint32_t K, T, Dmax;
  uint64_t node_cap;
  DNode* nodes;
  uint32_t* pnode;
  uint64_t* sums;
  uint32_t* fc;
  uint32_t* ctrl;
  bool device_loop;
  cudaStream_t stream;
  uint32_t* launches;
};
cudaError_t build_rmi_levels(const RmiLevelsArgs& a);
// Splitters of every set: set k's B_k = 1 << log2B[k] splitters at t + tbase[k], tree k rooted at node k,
// from the settled sample points (build_rmi_levels' x and pnode); pbin: S_total words of scratch.  Two launches.
cudaError_t splitters_batch(const DNode* nodes, uint32_t K, const SetInfo* sets, const uint32_t* log2B,
                            const uint64_t* tbase, uint64_t total_bins, const uint64_t* x, uint64_t S_total,
                            const uint32_t* pnode, uint32_t* pbin, uint64_t* t, cudaStream_t st);

uint64_t node_cap_for(uint64_t S, uint32_t T);

// Byte offsets inside the device model buffer.
struct ModelLayout {
  size_t nodes, splitters, lut, mlp_knots, mlp_w, alt_splitters, bytes;
};
ModelLayout model_layout(uint64_t S, uint32_t log2B, uint32_t T);
inline size_t model_bytes_for(uint64_t S, uint32_t log2B, uint32_t T) { return model_layout(S, log2B, T).bytes; }

// fits the RMI without a host round trip (the node and level counts are in
// the model header); *sorted_out = the buffer holding the sorted sample
// (a.samp or a.samp + S)
cudaError_t fit_rmi(const FitArgs& a, const uint64_t** sorted_out);
cudaError_t sample_keys(const uint8_t* records, uint64_t n, uint64_t S, uint64_t seed, const KeyMask& km, uint64_t* out,
                        cudaStream_t st);
// builds both levels of the radix index (kFineLutLaunches kernels)
constexpr uint32_t kFineLutLaunches = 5;
cudaError_t build_fine_lut(const uint64_t* splitters, uint32_t log2B, uint32_t* lut, cudaStream_t st);
cudaError_t set_model_kind(void* model, uint32_t kind, uint32_t fallback, cudaStream_t st);
// no model: the equal-width (radix) splitters t_q = ceil(q 95^9 / B), their index and the header
cudaError_t fit_radix(const FitArgs& a);

struct PartArgs {
  const uint8_t* records;
  KeyMask km;
  uint64_t n;
  const uint64_t* splitters;  // B fine-bin splitters of the fitted model
  const uint32_t* lut;        // radix index of the splitters
  uint32_t log2B, P, balance, tile_pairs;
  void* pairs_in_order;  // n pairs (scratch)
  void* pairs;           // n pairs, bin-ordered (output)
  uint32_t* bin_off;     // B+1
  uint64_t* part_off;    // P+1
  uint32_t* cuts;        // P+1
  uint32_t* cursor;      // B
  uint32_t* items;       // B+1 : first bin of each item
  uint32_t* item_flag;   // B   scratch (becomes the item id of every bin)
  uint32_t* oversize;    // B   item ids of oversize items
  uint32_t* ctrl;        // control words
  void* mid;             // n pairs (scratch, 16-byte aligned): coarse-bin order between the two scatter passes
  uint32_t* seg_hist;    // coarse_segments(n) x kMaxCoarse counts of every classify CTA
  long long wait_limit;  // limit of the bounded mbarrier waits (SM clock cycles)
  cudaStream_t stream;
  uint32_t* launches;
  cudaEvent_t ev[4];  // optional: after classify, after scan/cuts/items, after scatter
};

// Two-pass scatter: coarse bins of 2^coarse_shift(log2B) fine bins, at most
// kMaxCoarse of them; classify CTAs (at most kMaxSegments) count per coarse bin.
constexpr uint32_t kMaxCoarse = 512;
constexpr uint32_t kMaxFineShift = 11;    // at most 2^11 fine bins per coarse bin (shared-memory cursors)
constexpr uint32_t kStagedMaxShift = kMaxFineShift;  // beyond it the fine pass's cursors do not fit: one atomic pass
constexpr uint32_t kMaxSegments = 2048;
inline uint32_t coarse_shift(uint32_t log2B) { return log2B > 9 ? log2B - 9 : 0; }
inline uint64_t coarse_segments(uint64_t n) {
  const uint64_t t = (n + 255) / 256 + 1;
  return t < kMaxSegments ? t : kMaxSegments;
}

cudaError_t partition_records(const PartArgs& a);
cudaError_t build_items(const PartArgs& a);

// many record sets (batched path): all sets share one fine-bin space, set k
// owning bins [tbase[k], tbase[k] + 2^log2B[k]) and pair slots [poff[k], poff[k+1])
struct BatchPartArgs {
  const uint8_t* const* ins;  // device array of K record buffers
  KeyMask km;
  const uint64_t* poff;       // K+1
  uint32_t K, B, tile_pairs;  // B = total bins
  const uint64_t* splitters;  // B
  const uint64_t* tbase;      // K+1
  const uint32_t* log2B;      // K
  uint64_t N;               // records of all sets
  Pair* pairs_in_order;     // N pairs scratch
  Pair* pairs;              // N pairs: bin-ordered output
  uint32_t* seg_hist;       // coarse_segments(N) x kMaxCoarse
  uint32_t* bin_off;  // B+1
  uint32_t* cursor;   // B
  uint32_t* items;    // B+1
  uint32_t* item_flag;
  uint32_t* oversize;
  uint32_t* ctrl;
  cudaStream_t stream;
  uint32_t* launches;
};
cudaError_t partition_batch(const BatchPartArgs& a);
// the scatter passes' shared-memory limit (call before graph capture)
cudaError_t prepare_scatter_kernels();

struct SortArgs {
  const uint8_t* records;
  uint8_t* out;
  // batched path: per-set record buffers; items map to sets through tbase/poff
  const uint8_t* const* ins;
  uint8_t* const* outs;
  const uint64_t* tbase;
  const uint64_t* poff;
  uint32_t K;
  uint64_t n;
  uint32_t log2B, P, schedule, tile_pairs;
  Pair* pairs;  // bin-ordered
  Pair* temp;   // n pairs scratch (oversize merges)
  const uint32_t* bin_off;
  const uint32_t* items;
  const uint32_t* oversize;
  const uint32_t* cuts;
  const uint32_t* item_of_bin;
  uint32_t* ctrl;  // control words; words [64, 64+P+1) hold per-partition item ranges
  cudaStream_t stream;
  uint32_t* launches;
};

cudaError_t sort_items(const SortArgs& a);

// out-of-core helpers (ooc.cu)
uint64_t ooc_tiles(uint64_t n);
cudaError_t ooc_bin_to_part(const uint32_t* cuts, uint32_t P, uint32_t B, uint16_t* lut, cudaStream_t st);
struct OocSplitArgs {
  const uint8_t* chunk;      // the chunk's records (device)
  uint64_t n;                // records in the chunk
  const Pair* pairs;         // the chunk's pairs in input order, fine bin in lo
  const uint16_t* lut;       // fine bin -> partition
  uint32_t P;
  uint32_t* tile_hist;       // ooc_tiles(n) x P
  uint16_t* rank;            // n
  uint32_t* part_count;      // P
  uint32_t* chunk_off;       // P + 1: partition starts inside the chunk
  uint8_t* stage;            // n records, the chunk in partition order
  uint64_t* dst_next;        // P: next free output record of every partition
  uint64_t* dst_cur;         // P: this chunk's destination of every partition
  const uint64_t* part_end;  // P: end of every partition's output range (records)
  uint8_t* out;              // the output records (host memory mapped into the device)
  const uint32_t* ctrl;      // control words (status word: classify gave up)
};
// stable split of a chunk by partition into `stage`
cudaError_t ooc_split_chunk(const OocSplitArgs& a, cudaStream_t st);
// every partition's piece of `stage` appended to its output range
cudaError_t ooc_copy_out(const OocSplitArgs& a, cudaStream_t st);
// classify a chunk into input-order pairs (fine bin in the pair) and add to hist
cudaError_t classify_accumulate(const PartArgs& a);
// scan of the histogram and partition cuts
cudaError_t scan_and_cut(const PartArgs& a);
cudaError_t prepare_sort_kernel(uint32_t cap);  // kernel attributes, before any stream capture
int sm_count();

// control word indices
enum Ctrl : int {
  kNumItems = 0,
  kNumOversize = 1,
  kQueueHead = 2,
  kMaxBin = 3,
  kStatus = 4,
  kLevelNodes = 8,  // fit: [8] level begin, [9] level end, [10] next level count, [11] total nodes, [12] overflow,
                    // [13] levels done
  kStatusWord = 16,
  // words 0-31 are cleared at the start of every partition; these are not:
  kStickyTag = 32,     // [32], [33]: kStickyMagic once the sticky word below is valid
  kStickyStatus = 34,  // OR of the status words of the calls that did not read theirs back
};
constexpr uint64_t kStickyMagic = 0x53544b59454c5352ull;

}  // namespace elsar
