// Model training on the GPU (Sec. 3.1 of the paper): key sample, sample sort,
// the RMI of linear models, and the fine-bin splitters classification uses.
//
// Every floating-point step uses explicit round-to-nearest intrinsics in the
// order the model definition fixes (this file is also built with
// -fmad=false), so the fitted model is bit-identical wherever it is computed
// in that order.  Least-squares sums are exact integers (order independent).
#include <mutex>
#include <vector>

#include "common.cuh"
#include "mlp.cuh"

namespace elsar {
namespace {

inline uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

typedef unsigned __int128 u128;
typedef __int128 i128;

// ------------------------------------------------------------------ helpers
// Correctly rounded (to nearest even) unsigned 128-bit -> double: keep the
// top 64 bits with the discarded bits ORed into bit 0 (a sticky bit below
// the rounding position), let the hardware round 64 -> 53 bits, then scale
// by the exact power of two.
__device__ __forceinline__ double u128_to_double(u128 v) {
  uint64_t hi = (uint64_t)(v >> 64), lo = (uint64_t)v;
  if (hi == 0) return __ull2double_rn(lo);
  int s = 64 - __clzll((long long)hi);  // bits beyond the top 64: 1..64
  uint64_t top = (uint64_t)(v >> s);
  uint64_t sticky = (s == 64) ? (lo != 0) : ((lo & ((1ull << s) - 1)) != 0);
  double d = __ull2double_rn(top | sticky);
  return __dmul_rn(d, __longlong_as_double((long long)(1023 + s) << 52));
}

__device__ __forceinline__ double i128_to_double(i128 v) {
  return v < 0 ? -u128_to_double((u128)(-v)) : u128_to_double((u128)v);
}

__device__ __forceinline__ double pos_or_zero(double v) { return v > 0.0 ? v : 0.0; }

__device__ __forceinline__ uint64_t local_u(const DNode& v, uint64_t x) {
  return x > v.base ? (x - v.base) >> v.shift : 0;
}

// router of an internal node: clamp(floor(fma(gamma, u, delta) * scale), 0, f-1),
// a monotone function of the local coordinate u (gamma >= 0, scale > 0)
__device__ __forceinline__ uint32_t route_u(const DNode& v, uint64_t u) {
  double t = __dmul_rn(__fma_rn(v.a, __ull2double_rn(u), v.b), v.c);
  if (!(t > 0.0)) return 0;
  if (t >= __uint2double_rn(v.fanout)) return v.fanout - 1;
  return __double2uint_rz(t);
}

__device__ __forceinline__ uint32_t route(const DNode& v, uint64_t x) { return route_u(v, local_u(v, x)); }

// The router of a finished internal node, decided in FP32 where that is
// safe.  The node keeps A = a c and B = b c rounded to FP32 in h (which only
// leaves use otherwise), and t32 = fma(A, u, B) in FP32.  With A, B and u
// each rounded once to FP32 and one rounded fma, |t32 - t64| <=
// (|A u| + |B|) 2^-21, t64 being route_u's FP64 value (whose own rounding is
// below 2^-50 of the same terms).  The screen keeps twice that margin plus
// 2^-30 and answers only when the whole interval around t32 takes the same
// branch of route_u (0, fanout - 1, or one floor); otherwise, and for any
// inf or NaN, it returns route_u's FP64 result, so every decision is route_u's.
__device__ __forceinline__ void set_route_screen(DNode& v) {
  const float A = __double2float_rn(__dmul_rn(v.a, v.c)), B = __double2float_rn(__dmul_rn(v.b, v.c));
  v.h = __hiloint2double(__float_as_int(B), __float_as_int(A));
}

__device__ __forceinline__ uint32_t route_screened(const DNode& v, uint64_t x) {
  const uint64_t u = local_u(v, x);
  const float A = __int_as_float(__double2loint(v.h)), B = __int_as_float(__double2hiint(v.h));
  const float uf = __ull2float_rn(u);
  const float t = __fmaf_rn(A, uf, B);
  const float err = __fmaf_rn(__fadd_rn(fabsf(__fmul_rn(A, uf)), fabsf(B)), 0x1p-20f, 0x1p-30f);
  const float lo = __fsub_rn(t, err), hi = __fadd_rn(t, err);
  const float F = __uint2float_rn(v.fanout);  // exact: fanouts are far below 2^24
  if (hi <= 0.0f) return 0;
  if (lo >= F) return v.fanout - 1;
  if (lo > 0.0f && hi < F) {
    const float fl = floorf(lo);
    if (fl == floorf(hi)) return (uint32_t)fl;
  }
  return route_u(v, u);
}

// Smallest u in (a, b] with f(u) >= q for a monotone f with f(a) < q <=
// f(b): a gallop from the guess m (it only sets the start; m > b: none, the
// middle is taken), then a bisection.  Every decision evaluates f exactly.
template <class F>
__device__ __forceinline__ uint64_t first_at_least(const F& f, uint64_t a, uint64_t b, uint32_t q, uint64_t m) {
  if (m > b) m = a + ((b - a + 1) >> 1);
  else if (m <= a) m = a + 1;
  if (f(m) >= q) {  // gallop down from m
    b = m;
    for (uint64_t step = 1; b - a > 1; step <<= 1) {
      const uint64_t t = b - a > step ? b - step : a + 1;
      if (f(t) >= q) {
        b = t;
      } else {
        a = t;
        break;
      }
    }
  } else {  // gallop up from m
    a = m;
    for (uint64_t step = 1; b - a > 1; step <<= 1) {
      const uint64_t t = b - a > step ? a + step : b - 1;
      if (f(t) >= q) {
        b = t;
        break;
      }
      a = t;
    }
  }
  while (b - a > 1) {
    const uint64_t mid = a + ((b - a) >> 1);
    if (f(mid) >= q) b = mid;
    else a = mid;
  }
  return b;
}

// first index i in [lo, hi) with at(i) >= key (hi if none) of a
// non-decreasing sequence: a gallop from the guess g, then a bisection
template <class A, class T>
__device__ __forceinline__ uint64_t gallop_first(const A& arr, uint64_t lo, uint64_t hi, T key, uint64_t g) {
  uint64_t a = lo, b = hi;  // the answer lies in [a, b]
  if (lo < hi) {
    if (g < lo) g = lo;
    if (g > hi - 1) g = hi - 1;
    if (arr(g) >= key) {
      b = g;
      for (uint64_t step = 1; b > lo; step <<= 1) {
        const uint64_t i = b - lo > step ? b - step : lo;
        if (arr(i) >= key) {
          b = i;
        } else {
          a = i + 1;
          break;
        }
      }
    } else {
      a = g + 1;
      for (uint64_t step = 1; a < hi; step <<= 1) {
        const uint64_t i = a + step - 1 < hi - 1 ? a + step - 1 : hi - 1;
        if (arr(i) >= key) {
          b = i;
          break;
        }
        a = i + 1;
      }
    }
  }
  while (a < b) {
    const uint64_t mid = (a + b) >> 1;
    if (arr(mid) >= key) b = mid;
    else a = mid + 1;
  }
  return a;
}

template <class T>
__device__ __forceinline__ uint64_t gallop_lower_bound(const T* __restrict__ arr, uint64_t lo, uint64_t hi, T key,
                                                       uint64_t g) {
  return gallop_first([&](uint64_t i) { return arr[i]; }, lo, hi, key, g);
}

__device__ __forceinline__ void atomic_add_u128(uint64_t* p, u128 v) {
  uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
  unsigned long long old = atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)lo);
  if (old + lo < old) hi += 1;
  if (hi) atomicAdd(reinterpret_cast<unsigned long long*>(p + 1), (unsigned long long)hi);
}

// ------------------------------------------------------------------ sample
__global__ void sample_kernel(const uint8_t* __restrict__ rec, uint64_t n, uint64_t S, uint64_t seed, KeyMask km,
                              uint64_t* __restrict__ out) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < S; k += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t i = __umul64hi(splitmix64_at(seed, k), n);
    out[k] = enc9_pair(load_pair(rec + i * kRecord, 0, km));
  }
}

// ------------------------------------------------------------------ u64 sort: chunk bitonic + merge path
constexpr int kChunk = 4096;
constexpr int kChunkThreads = 1024;

// Bitonic sort of one chunk of kChunk keys (padding ~0 past S), 4 keys per
// thread in registers (element e = 4 * thread + r): compare-exchange stages
// with partners 1 or 2 apart stay in the thread, 4 to 64 apart go through warp
// shuffles, 128 and more through shared memory, so only those take barriers.
__global__ void __launch_bounds__(kChunkThreads) chunk_sort_u64(uint64_t* data, uint64_t S) {
  static_assert(kChunk == 4 * kChunkThreads, "four keys per thread");
  __shared__ uint64_t s[kChunk];
  const uint64_t base = (uint64_t)blockIdx.x * kChunk;
  const uint32_t t = threadIdx.x;
  uint64_t v[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const uint64_t g = base + 4 * t + r;
    v[r] = g < S ? data[g] : ~0ull;
  }
  for (uint32_t k = 2; k <= (uint32_t)kChunk; k <<= 1) {
    uint32_t j = k >> 1;
    if (j >= 128) {  // partners in other warps: through shared memory
      __syncthreads();  // the previous read-back is done
#pragma unroll
      for (int r = 0; r < 4; ++r) s[4 * t + r] = v[r];
      __syncthreads();
      for (; j >= 128; j >>= 1) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {  // kChunk / 2 pairs, two per thread
          const uint32_t p = t + q * kChunkThreads;
          const uint32_t e = ((p & ~(j - 1)) << 1) | (p & (j - 1)), f = e | j;
          const uint64_t x = s[e], y = s[f];
          if ((x > y) == ((e & k) == 0)) {
            s[e] = y;
            s[f] = x;
          }
        }
        __syncthreads();
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) v[r] = s[4 * t + r];
    }
    for (; j >= 4; j >>= 1) {  // partners in this warp, j / 4 lanes away
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const uint32_t e = 4 * t + r;
        const uint64_t w = __shfl_xor_sync(0xffffffffu, v[r], j >> 2);
        const bool keep_min = ((e & j) == 0) == ((e & k) == 0);
        v[r] = keep_min ? min(v[r], w) : max(v[r], w);
      }
    }
    // partners in this thread: j = 2 (when k >= 4), then j = 1
    auto cx = [&](uint64_t& x, uint64_t& y, uint32_t e) {  // e: the lower element
      if ((x > y) == ((e & k) == 0)) {
        const uint64_t z = x;
        x = y;
        y = z;
      }
    };
    if (j == 2) {
      cx(v[0], v[2], 4 * t);
      cx(v[1], v[3], 4 * t + 1);
    }
    cx(v[0], v[1], 4 * t);
    cx(v[2], v[3], 4 * t + 2);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const uint64_t g = base + 4 * t + r;
    if (g < S) data[g] = v[r];
  }
}

constexpr int kMergeTile = 2048;
constexpr int kMergeThreads = 256;
constexpr int kMergeItems = kMergeTile / kMergeThreads;

// Number of elements taken from a among the first diag outputs of merge(a, b)
// (the largest i with a[i - 1] <= b[diag - i], ties to a), found by one warp:
// each round tests 32 evenly spaced candidates at once (one load per lane)
// and keeps the segment where the predicate a[mid] <= b[diag - 1 - mid] turns
// false, so the dependent loads fall from log2 of the range to about log32 of
// it.  Returned to every lane.
__device__ __forceinline__ uint64_t warp_merge_split(const uint64_t* a, uint64_t na, const uint64_t* b, uint64_t nb,
                                                     uint64_t diag) {
  const uint32_t lane = threadIdx.x & 31;
  uint64_t lo = diag > nb ? diag - nb : 0, hi = diag < na ? diag : na;  // the answer lies in [lo, hi]
  while (hi - lo > 32) {
    const uint64_t step = (hi - lo + 31) / 32;
    const uint64_t mid = lo + lane * step;  // lane 0 tests lo itself
    const bool t = mid < hi && a[mid] <= b[diag - 1 - mid];
    const uint32_t m = __ballot_sync(0xffffffffu, t);  // candidates below the answer
    const uint32_t k = 32 - __clz(m);                   // the first candidate that fails (or 32)
    // the predicate is true before the answer and false from it on
    const uint64_t nlo = k ? lo + (uint64_t)(k - 1) * step + 1 : lo;
    const uint64_t nhi = k < 32 ? min(hi, lo + (uint64_t)k * step) : hi;
    lo = nlo;
    hi = nhi;
  }
  const uint64_t mid = lo + lane;
  const bool t = mid < hi && a[mid] <= b[diag - 1 - mid];
  return lo + __popc(__ballot_sync(0xffffffffu, t));
}

__global__ void __launch_bounds__(kMergeThreads) merge_pass_u64(const uint64_t* __restrict__ src,
                                                                uint64_t* __restrict__ dst, uint64_t S, uint64_t w) {
  __shared__ uint64_t s[kMergeTile];
  const uint64_t o0 = (uint64_t)blockIdx.x * kMergeTile;
  if (o0 >= S) return;
  const uint64_t o1 = min(S, o0 + kMergeTile);
  const uint64_t p0 = (o0 / (2 * w)) * (2 * w);
  const uint64_t a0 = p0, a1 = min(S, p0 + w), b0 = a1, b1 = min(S, p0 + 2 * w);
  __shared__ uint64_t split[2];
  if (threadIdx.x < 64) {  // warp 0: the window's start, warp 1: its end
    const uint32_t w = threadIdx.x >> 5;
    const uint64_t r = warp_merge_split(src + a0, a1 - a0, src + b0, b1 - b0, (w ? o1 : o0) - p0);
    if ((threadIdx.x & 31) == 0) split[w] = r;
  }
  __syncthreads();
  const uint64_t ka0 = split[0], ka1 = split[1];
  const uint64_t kb0 = (o0 - p0) - ka0, kb1 = (o1 - p0) - ka1;
  const int na = (int)(ka1 - ka0), nb = (int)(kb1 - kb0);
  for (int i = threadIdx.x; i < na; i += kMergeThreads) s[i] = src[a0 + ka0 + i];
  for (int i = threadIdx.x; i < nb; i += kMergeThreads) s[na + i] = src[b0 + kb0 + i];
  __syncthreads();
  const int tot = na + nb;
  int d = threadIdx.x * kMergeItems;
  if (d >= tot) return;
  // split of this thread's diagonal inside the tile
  int lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (s[mid] <= s[na + d - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  int ia = lo, ib = d - lo;
  for (int t = 0; t < kMergeItems && d + t < tot; ++t) {
    bool takeA = ib >= nb || (ia < na && s[ia] <= s[na + ib]);
    dst[o0 + d + t] = takeA ? s[ia++] : s[na + ib++];
  }
}

// ------------------------------------------------------------------ RMI, level by level
// K trees at once: tree k (record set k) has its root at node k and covers the
// sorted-sample segment sets[k].  A single record set is K = 1.

__device__ __forceinline__ uint32_t set_of_point(const SetInfo* sets, uint32_t K, uint64_t j) {
  uint32_t lo = 0, hi = K - 1;  // largest k with soff_k <= j
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (sets[mid].soff <= j) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// per-node base and shift, read by every point of the node
__device__ __forceinline__ void node_frame(const uint64_t* x, uint32_t s, uint32_t e, uint64_t* base, uint32_t* sh) {
  uint64_t b = x[s];
  uint64_t span = x[e - 1] - b;
  uint32_t bits = span ? 64 - __clzll((long long)span) : 0;
  *base = b;
  *sh = bits > 32 ? bits - 32 : 0;
}

// the roots (with their frames) and every point in its set's root
__global__ void init_roots(const uint64_t* __restrict__ x, DNode* nodes, uint32_t* pnode,
                           const SetInfo* __restrict__ sets, uint32_t K, uint64_t S_total, uint32_t* ctrl) {
  const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = t0; k < K; k += stride) {
    DNode r = {};
    r.s = (uint32_t)sets[k].soff;
    r.e = (uint32_t)(sets[k].soff + sets[k].S);
    r.depth_set = (uint32_t)k << 8;
    if (r.e > r.s) node_frame(x, r.s, r.e, &r.base, &r.shift);
    nodes[k] = r;
  }
  if (t0 == 0) {
    ctrl[kLevelNodes + 0] = 0;
    ctrl[kLevelNodes + 1] = K;
    ctrl[kLevelNodes + 2] = 0;
    ctrl[kLevelNodes + 3] = K;
    ctrl[kLevelNodes + 4] = 0;
    ctrl[kLevelNodes + 5] = 0;
  }
  for (uint64_t j = t0; j < S_total; j += stride) pnode[j] = set_of_point(sets, K, j);
}

__device__ __forceinline__ u128 shfl_u128(u128 v, int src) {
  uint64_t lo = __shfl_sync(0xffffffffu, (uint64_t)v, src);
  uint64_t hi = __shfl_sync(0xffffffffu, (uint64_t)(v >> 64), src);
  return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ u128 shfl_up_u128(u128 v, int d) {
  uint64_t lo = __shfl_up_sync(0xffffffffu, (uint64_t)v, d);
  uint64_t hi = __shfl_up_sync(0xffffffffu, (uint64_t)(v >> 64), d);
  return ((u128)hi << 64) | lo;
}

__device__ __forceinline__ void add_node_sums(uint64_t* sums, uint32_t lv0, uint32_t v, uint64_t u, u128 uu, u128 ur) {
  uint64_t* sm = sums + (uint64_t)(v - lv0) * 6;
  atomicAdd(reinterpret_cast<unsigned long long*>(sm), (unsigned long long)u);
  atomic_add_u128(sm + 2, uu);
  atomic_add_u128(sm + 4, ur);
}

constexpr int kSumsWarpPoints = 256;                   // consecutive points per warp
constexpr int kSumsBlockPoints = 8 * kSumsWarpPoints;  // per 256-thread block

// sum over the warp, every lane gets the totals
__device__ __forceinline__ void warp_sum3(uint64_t& u, u128& uu, u128& ur) {
  for (int d = 16; d; d >>= 1) {
    u += __shfl_xor_sync(0xffffffffu, u, d);
    uu += ((u128)__shfl_xor_sync(0xffffffffu, (uint64_t)(uu >> 64), d) << 64) |
          __shfl_xor_sync(0xffffffffu, (uint64_t)uu, d);
    ur += ((u128)__shfl_xor_sync(0xffffffffu, (uint64_t)(ur >> 64), d) << 64) |
          __shfl_xor_sync(0xffffffffu, (uint64_t)ur, d);
  }
}

// Exact sums Su, Suu, Sur per node (u = the node's local coordinate, r = the
// local rank), over the points of the level's nodes [lv0, lv1).  kRoute =
// false: the sums of those nodes (the roots, before the first level).  kRoute
// = true: every point of an internal node first moves to its child (a point
// of a leaf settles: kSettledBit | the leaf), and the sums are the children's
// (the next level, numbered from lv1, ranges and frames set by
// level_init_next).
// A node holds a contiguous range of the sorted points, so a warp walks a
// run of consecutive points 32 at a time.  A step whose 32 points share the
// run's node only adds into per-lane sums; any other step gathers the run
// (a warp sum), sums the step per node segment (segmented shuffle scan),
// adds the segments that end and carries the last one on.  The warps of a
// block then merge their final carries, so a node that spans the block is
// added once per block.  Integer sums: the order of the additions does not
// matter.
template <bool kRoute>
__global__ void __launch_bounds__(256) level_sums(const uint64_t* __restrict__ x, uint64_t S, const DNode* nodes,
                                                  uint32_t* pnode, uint64_t* sums, const uint32_t* ctrl) {
  __shared__ uint32_t cv_sh[8];
  __shared__ uint64_t cu_sh[8];
  __shared__ u128 cuu_sh[8], cur_sh[8];
  const uint32_t lv0 = ctrl[kLevelNodes + 0], lv1 = ctrl[kLevelNodes + 1];
  if (lv0 >= lv1) return;
  const uint32_t ofs = kRoute ? lv1 : lv0;  // sums of node v at (v - ofs) * 6
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (uint64_t b0 = blockIdx.x * (uint64_t)kSumsBlockPoints; b0 < S; b0 += (uint64_t)gridDim.x * kSumsBlockPoints) {
    const uint64_t c0 = b0 + (uint64_t)warp * kSumsWarpPoints;
    const uint64_t c1 = c0 + kSumsWarpPoints < S ? c0 + kSumsWarpPoints : S;
    uint32_t cv = kSettled;  // the run's node (warp-uniform)
    bool spread = false;     // the run's sums: per lane (spread) or warp-uniform (cu, cuu, cur)
    uint64_t cu = 0, lu = 0;
    u128 cuu = 0, cur = 0, luu = 0, lur = 0;
    for (uint64_t k0 = c0; k0 < c1; k0 += 32) {
      const uint64_t k = k0 + lane;
      uint32_t v = k < c1 ? pnode[k] : kSettled;
      if (v < lv0 || v >= lv1) v = kSettled;  // settled in a leaf of an earlier level
      if (kRoute && v != kSettled) {
        const DNode& nd = nodes[v];
        if (nd.fanout) {
          const uint32_t ch = nd.child0 + route_screened(nd, x[k]);
          pnode[k] = ch;
          v = ch;
        } else {
          pnode[k] = kSettledBit | v;
          v = kSettled;
        }
      }
      uint64_t u = 0;
      u128 uu = 0, ur = 0;
      if (v != kSettled) {
        const DNode& c = nodes[v];
        const uint64_t uv = (x[k] - c.base) >> c.shift;
        u = uv;
        uu = (u128)uv * uv;
        ur = (u128)uv * (uint64_t)(k - c.s);
      }
      const uint32_t v0 = __shfl_sync(0xffffffffu, v, 0);
      const bool same = __all_sync(0xffffffffu, v == v0);
      if (same && v0 == cv && cv != kSettled) {  // the run goes on
        if (!spread) {
          lu = lane == 0 ? cu : 0;
          luu = lane == 0 ? cuu : 0;
          lur = lane == 0 ? cur : 0;
          spread = true;
        }
        lu += u;
        luu += uu;
        lur += ur;
        continue;
      }
      if (spread) {  // gather the run
        warp_sum3(lu, luu, lur);
        cu = lu;
        cuu = luu;
        cur = lur;
        spread = false;
      }
      if (cv != kSettled && cv != v0) {  // the run ends before this step
        if (lane == 0) add_node_sums(sums, ofs, cv, cu, cuu, cur);
        cv = kSettled;
      }
      if (same) {  // all settled, or one node that starts a run
        if (v0 != kSettled) {
          cv = v0;
          spread = true;
          lu = u;
          luu = uu;
          lur = ur;
        }
        continue;
      }
      if (cv != kSettled && lane == 0) {  // lane 0 holds node cv: the scan takes the carry from there
        u += cu;
        uu += cuu;
        ur += cur;
      }
      for (int d = 1; d < 32; d <<= 1) {  // inclusive scan inside each run of equal v
        const uint32_t vp = __shfl_up_sync(0xffffffffu, v, d);
        const uint64_t up = __shfl_up_sync(0xffffffffu, u, d);
        const u128 uup = shfl_up_u128(uu, d), urp = shfl_up_u128(ur, d);
        if (lane >= (uint32_t)d && vp == v) {
          u += up;
          uu += uup;
          ur += urp;
        }
      }
      const uint32_t vn = __shfl_down_sync(0xffffffffu, v, 1);
      if (lane != 31 && vn != v && v != kSettled) add_node_sums(sums, ofs, v, u, uu, ur);
      cv = __shfl_sync(0xffffffffu, v, 31);
      cu = __shfl_sync(0xffffffffu, u, 31);
      cuu = shfl_u128(uu, 31);
      cur = shfl_u128(ur, 31);
    }
    if (spread) {
      warp_sum3(lu, luu, lur);
      cu = lu;
      cuu = luu;
      cur = lur;
    }
    if (lane == 0) {
      cv_sh[warp] = cv;
      cu_sh[warp] = cu;
      cuu_sh[warp] = cuu;
      cur_sh[warp] = cur;
    }
    __syncthreads();
    if (threadIdx.x == 0) {  // merge the warps' carries, a node once per run of equal carries
      uint32_t mv = kSettled;
      uint64_t mu = 0;
      u128 muu = 0, mur = 0;
      for (int w = 0; w < 8; ++w) {
        if (cv_sh[w] != mv) {
          if (mv != kSettled) add_node_sums(sums, ofs, mv, mu, muu, mur);
          mv = cv_sh[w];
          mu = 0;
          muu = mur = 0;
        }
        mu += cu_sh[w];
        muu += cuu_sh[w];
        mur += cur_sh[w];
      }
      if (mv != kSettled) add_node_sums(sums, ofs, mv, mu, muu, mur);
    }
    __syncthreads();
  }
}

// least-squares fit of every node of the level and its split decision
__global__ void level_fit(const uint64_t* __restrict__ x, DNode* nodes, const uint64_t* sums, uint32_t* fc, uint32_t T,
                          uint32_t Dmax, const uint32_t* ctrl) {
  const uint32_t lv0 = ctrl[kLevelNodes + 0], lv1 = ctrl[kLevelNodes + 1];
  for (uint32_t v = lv0 + blockIdx.x * blockDim.x + threadIdx.x; v < lv1; v += gridDim.x * blockDim.x) {
    DNode nd = nodes[v];
    uint32_t n = nd.e - nd.s;
    fc[v - lv0] = 0;
    if (n == 0) {
      nd.base = 0;
      nd.shift = 0;
      nd.a = 0.0;
      nd.b = 0.0;
      nodes[v] = nd;
      continue;
    }
    node_frame(x, nd.s, nd.e, &nd.base, &nd.shift);
    const uint64_t* sm = sums + (uint64_t)(v - lv0) * 6;
    u128 Su = sm[0];
    u128 Suu = ((u128)sm[3] << 64) | sm[2];
    u128 Sur = ((u128)sm[5] << 64) | sm[4];
    i128 nn = (i128)n;
    i128 Sr = nn * (nn - 1) / 2;
    i128 Duu = nn * (i128)Suu - (i128)Su * (i128)Su;
    i128 Dur = nn * (i128)Sur - (i128)Su * Sr;
    double gamma = (n >= 2 && Duu > 0) ? pos_or_zero(__ddiv_rn(i128_to_double(Dur), i128_to_double(Duu))) : 0.0;
    double delta = __ddiv_rn(__dsub_rn(i128_to_double(Sr), __dmul_rn(gamma, u128_to_double(Su))), __uint2double_rn(n));
    nd.a = gamma;
    nd.b = delta;
    nd.c = 0.0;
    bool split = n > 2u * T && (nd.depth_set & 0xFFu) < Dmax && x[nd.s] < x[nd.e - 1];
    if (split) {
      uint32_t f = (n + T - 1) / T;
      nd.fanout = f;
      nd.c = __ddiv_rn(__uint2double_rn(f), __uint2double_rn(n));
      if (route(nd, x[nd.s]) == route(nd, x[nd.e - 1])) split = false;
      nd.fanout = 0;
      if (split) fc[v - lv0] = f;
    }
    nodes[v] = nd;
  }
}

constexpr int kScanThreads = 1024;

constexpr int kScanChunks = 16;  // 32-fanout chunks per warp and tile

// Single CTA: child numbering = exclusive scan of the split fanouts of the
// level and the node budget check.  A tile is kScanThreads x kScanChunks
// fanouts; warp w scans chunks of 32 consecutive ones (coalesced) across its
// 512-fanout part, then the warps' totals are scanned and a running carry
// joins the tiles.  ctrl[kLevelNodes+2] = next level size (0 on overflow),
// ctrl[kLevelNodes+4] = 1 when the budget forbids splitting this level.
__global__ void __launch_bounds__(kScanThreads) level_scan(const uint32_t* __restrict__ fc, uint32_t* __restrict__ childoff,
                                                           uint64_t node_cap, uint32_t* ctrl) {
  __shared__ uint32_t wsum[kScanThreads / 32];
  __shared__ uint32_t carry_sh;
  const uint32_t lv0 = ctrl[kLevelNodes + 0], lv1 = ctrl[kLevelNodes + 1];
  const uint32_t cnt = lv1 - lv0;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry_sh = 0;
  __syncthreads();
  for (uint32_t base = 0; base < cnt; base += kScanThreads * kScanChunks) {
    const uint32_t w0 = base + warp * 32 * kScanChunks;
    uint32_t ex[kScanChunks], run = 0;  // exclusive offset inside the warp's part
#pragma unroll
    for (int j = 0; j < kScanChunks; ++j) {
      const uint32_t i = w0 + j * 32 + lane;
      const uint32_t v = i < cnt ? fc[i] : 0;
      uint32_t incl = v;
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= (uint32_t)d) incl += y;
      }
      ex[j] = run + incl - v;
      run += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) wsum[warp] = run;
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
    const uint32_t carry = carry_sh, off = carry + wsum[warp];
#pragma unroll
    for (int j = 0; j < kScanChunks; ++j) {
      const uint32_t i = w0 + j * 32 + lane;
      if (i < cnt) childoff[i] = off + ex[j];
    }
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry_sh = off + run;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const uint32_t total = carry_sh;
    const uint32_t total_nodes = ctrl[kLevelNodes + 3];
    const bool overflow = (uint64_t)total_nodes + total > node_cap;
    const uint32_t next = overflow ? 0 : total;
    ctrl[kLevelNodes + 2] = next;
    ctrl[kLevelNodes + 3] = total_nodes + next;
    ctrl[kLevelNodes + 4] = overflow ? 1u : 0u;
  }
}

// Every node of the level: internal nodes get their children, the rest
// become leaves with their output constants (Sec. 3.1 reading: F clamped to
// the leaf's sample-rank range, ranks counted within its record set).
__global__ void level_finalize(DNode* nodes, const uint32_t* __restrict__ fc, const uint32_t* __restrict__ childoff,
                               const SetInfo* __restrict__ sets, const uint32_t* ctrl) {
  const uint32_t lv0 = ctrl[kLevelNodes + 0], lv1 = ctrl[kLevelNodes + 1];
  const bool overflow = ctrl[kLevelNodes + 4] != 0;
  for (uint32_t v = lv0 + blockIdx.x * blockDim.x + threadIdx.x; v < lv1; v += gridDim.x * blockDim.x) {
    const uint32_t i = v - lv0;
    DNode nd = nodes[v];
    if (fc[i] && !overflow) {
      nd.fanout = fc[i];
      nd.child0 = lv1 + childoff[i];
      nd.c = __ddiv_rn(__uint2double_rn(nd.fanout), __uint2double_rn(nd.e - nd.s));
      set_route_screen(nd);
    } else {
      const SetInfo si = sets[nd.depth_set >> 8];
      const double dS = __ull2double_rn(si.S);
      const uint32_t rs = nd.s - (uint32_t)si.soff, re = nd.e - (uint32_t)si.soff;
      nd.fanout = 0;
      nd.child0 = 0;
      const double lo = __ddiv_rn(__uint2double_rn(rs), dS), hi = __ddiv_rn(__uint2double_rn(re), dS);
      if (nd.e == nd.s) {
        nd.a = 0.0;
        nd.b = lo;
      } else {
        const double g = __ddiv_rn(nd.a, dS);
        const double d = __ddiv_rn(__dadd_rn(__uint2double_rn(rs), nd.b), dS);
        nd.a = g;
        nd.b = d;
      }
      nd.c = lo;
      nd.h = hi;
    }
    nodes[v] = nd;
  }
}

// first point k of internal node nd (nd.e if none) with route(nd, x[k]) >= cc:
// routing is monotone in the sorted points
__device__ __forceinline__ uint32_t first_routed(const uint64_t* __restrict__ x, const DNode& nd, uint32_t cc) {
  uint32_t lo = nd.s, hi = nd.e;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (route_screened(nd, x[mid]) >= cc) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// The nodes of the next level, each by one thread, with their sums zeroed:
// child w finds its parent (the last node of the level whose first child is
// <= w), its point range (the first point its parent routes to it, up to
// the next child's first) and its frame.
__global__ void level_init_next(DNode* nodes, uint64_t* sums, const uint32_t* __restrict__ childoff,
                                const uint64_t* __restrict__ x, const uint32_t* ctrl) {
  const uint32_t lv0 = ctrl[kLevelNodes + 0], lv1 = ctrl[kLevelNodes + 1], next = ctrl[kLevelNodes + 2];
  const uint32_t cnt = lv1 - lv0;
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  // a warp owns 31 consecutive children; lane 31 finds the start of the
  // next one, which ends lane 30's child, so every lane searches once
  for (uint32_t w0 = gw * 31; w0 < next; w0 += nw * 31) {
    const uint32_t w = w0 + lane;
    const bool act = w < next;
    DNode nd = {};
    uint32_t cc = 0, s = 0;
    if (act) {
      uint32_t lo = 0, hi = cnt - 1;
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (childoff[mid] <= w) lo = mid;
        else hi = mid - 1;
      }
      nd = nodes[lv0 + lo];
      cc = w - childoff[lo];
      s = first_routed(x, nd, cc);
    }
    const uint32_t s_next = __shfl_down_sync(0xffffffffu, s, 1);
    if (!act || lane == 31) continue;
    DNode c = {};
    c.s = s;
    // the end is the next child's start (child w + 1 of the same parent, on
    // the next lane), or the parent's end for its last child
    c.e = cc + 1 == nd.fanout ? nd.e : s_next;
    c.depth_set = nd.depth_set + 1;  // same set, one level deeper
    if (c.e > c.s) node_frame(x, c.s, c.e, &c.base, &c.shift);
    nodes[lv1 + w] = c;
    uint64_t* sm = sums + (uint64_t)w * 6;
    for (int t = 0; t < 6; ++t) sm[t] = 0;
  }
}

__device__ __forceinline__ bool advance_level(uint32_t* ctrl) {
  uint32_t lv1 = ctrl[kLevelNodes + 1];
  ctrl[kLevelNodes + 0] = lv1;
  ctrl[kLevelNodes + 1] = lv1 + ctrl[kLevelNodes + 2];
  const bool more = ctrl[kLevelNodes + 2] != 0;
  ctrl[kLevelNodes + 2] = 0;
  ++ctrl[kLevelNodes + 5];
  return more;
}

__global__ void level_advance(uint32_t* ctrl) { advance_level(ctrl); }

// the last kernel of the device loop's body: repeat while the new level has
// nodes and the depth limit allows another
__global__ void level_advance_loop(uint32_t* ctrl, cudaGraphConditionalHandle h, uint32_t max_levels) {
  const bool more = advance_level(ctrl);
  cudaGraphSetConditional(h, (more && ctrl[kLevelNodes + 5] < max_levels) ? 1u : 0u);
}

// bin of x at leaf v: F clamped to the leaf's rank range, min(B-1, floor(B F))
__device__ __forceinline__ uint32_t leaf_bin(const DNode& v, uint64_t x, uint32_t log2B) {
  const uint32_t B = 1u << log2B;
  double y = __fma_rn(v.a, __ull2double_rn(local_u(v, x)), v.b);
  if (y < v.c) y = v.c;
  else if (y > v.h) y = v.h;
  const uint32_t q = __double2uint_rz(__dmul_rn(y, __uint2double_rn(B)));
  return q < B ? q : B - 1;
}

// bin at leaf v as a function of the local coordinate u (monotone in u)
__device__ __forceinline__ uint32_t leaf_bin_u(const DNode& v, uint64_t u, uint32_t log2B) {
  const uint32_t B = 1u << log2B;
  double y = __fma_rn(v.a, __ull2double_rn(u), v.b);
  if (y < v.c) y = v.c;
  else if (y > v.h) y = v.h;
  const uint32_t q = __double2uint_rz(__dmul_rn(y, __uint2double_rn(B)));
  return q < B ? q : B - 1;
}

// Smallest x in [lo, hi) whose bin at leaf v is >= q, hi if none; every key
// of [lo, hi) routes to v.  Keys with the same local coordinate u = (x -
// base) >> shift share a bin, so the search runs over u: the first u of the
// range whose bin is >= q, started from the line's inverse (first_at_least),
// and the key is then the first one with that u.
__device__ __forceinline__ uint64_t leaf_lower_bound(const DNode& v, uint64_t lo, uint64_t hi, uint32_t q,
                                                     uint32_t log2B) {
  if (lo >= hi) return hi;
  const uint64_t u0 = local_u(v, lo), u1 = local_u(v, hi - 1);
  if (leaf_bin_u(v, u0, log2B) >= q) return lo;
  if (leaf_bin_u(v, u1, log2B) < q) return hi;
  const double g = (v.a > 0.0) ? __ddiv_rn(__dsub_rn(__ddiv_rn(__uint2double_rn(q), __uint2double_rn(1u << log2B)), v.b), v.a)
                               : -1.0;
  const uint64_t m = (g > (double)u0 && g < (double)u1) ? (uint64_t)g : ~0ull;
  const uint64_t ub = first_at_least([&](uint64_t u) { return leaf_bin_u(v, u, log2B); }, u0, u1, q, m);
  return v.base + (ub << v.shift);  // > lo, as ub > u0
}

// Smallest x in [lo, hi] whose bin is >= q, given that the answer lies in
// [lo, hi] (hi itself is never evaluated).  Routers are monotone in x, so
// when lo and hi take the same child of a node, so does every key between
// them: the search descends to the deepest node that holds the whole
// bracket, bisects (full descents from there) while the bracket spans
// several of its children, and finishes inside one leaf by leaf_lower_bound.
__device__ __forceinline__ uint64_t bin_lower_bound(const DNode* __restrict__ nodes, uint32_t root, uint64_t lo,
                                                    uint64_t hi, uint32_t q, uint32_t log2B) {
  DNode v = nodes[root];
  while (lo < hi) {
    while (v.fanout) {
      const uint32_t c = route_screened(v, lo);
      if (c != route_screened(v, hi)) break;
      v = nodes[v.child0 + c];
    }
    if (!v.fanout) return leaf_lower_bound(v, lo, hi, q, log2B);
    const uint64_t mid = lo + ((hi - lo) >> 1);
    DNode w = nodes[v.child0 + route_screened(v, mid)];
    while (w.fanout) w = nodes[w.child0 + route_screened(w, mid)];
    if (leaf_bin(w, mid, log2B) >= q) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// bin of every sorted sample point, at the leaf it settled in (set k's
// points with set k's bin count; lb == nullptr: one set of 2^log2B bins)
__global__ void point_bins_kernel(const uint64_t* __restrict__ x, uint64_t S, const DNode* __restrict__ nodes,
                                  const uint32_t* __restrict__ pnode, const SetInfo* __restrict__ sets, uint32_t K,
                                  const uint32_t* __restrict__ lb, uint32_t log2B, uint32_t* __restrict__ pbin) {
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < S; j += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t l = lb ? lb[set_of_point(sets, K, j)] : log2B;
    pbin[j] = leaf_bin(nodes[pnode[j] & ~kSettledBit], x[j], l);
  }
}

// The sample bracket of bin q in one record set (sorted points xs[0, S),
// their bins pb and leaves pl): k = the first point whose bin is >= q (S if
// none), found by a gallop from the guess g (the model was fitted to the
// ranks, so the bin of xs[k] is near B k / S) and a bisection; the answer
// lies in [xs[k-1] + 1, xs[k]] (0 and 95^9 past the ends).  Returns the leaf
// when both ends settled in the same leaf (then every key of the bracket
// routes there), else kSettled.
__device__ __forceinline__ uint32_t sample_bracket(uint32_t q, uint64_t g, const uint64_t* __restrict__ xs,
                                                   const uint32_t* __restrict__ pb, const uint32_t* __restrict__ pl,
                                                   uint64_t S, uint64_t* lo, uint64_t* hi) {
  const uint64_t a = gallop_lower_bound(pb, 0, S, q, g);
  *lo = a ? xs[a - 1] + 1 : 0;
  *hi = a < S ? xs[a] : kEncTop;
  return (a && a < S && pl[a - 1] == pl[a]) ? pl[a] & ~kSettledBit : kSettled;
}

constexpr int kSplitThreads = 256;
constexpr uint32_t kSplitChunk = kSplitThreads;  // bins per block round

// Fine-bin splitters: t[q] = smallest encoding whose bin is >= q (t[0] = 0;
// 95^9 when no key reaches bin q).  The bin is a monotone function of the
// encoding, so any bracket holding the answer gives the same t[q]; the
// bracket comes from the sorted sample and its bins.  A block takes a chunk
// of bins: those whose bracket lies in one leaf are inverted there at once
// (leaf_lower_bound); the rest (about one in T, where a leaf boundary falls
// between two sample points) are queued in shared memory and searched
// afterwards by the whole block, so the FP64 descents of bin_lower_bound run
// in full warps.  Set k (k < K) has its tree at node k, its points at
// sets[k], its bins at tbase[k] .. tbase[k+1]; K == 1 with tbase == nullptr
// is one set of 2^log2B bins.
__global__ void __launch_bounds__(kSplitThreads) splitter_kernel(const DNode* __restrict__ nodes, uint32_t K,
                                                                const SetInfo* __restrict__ sets,
                                                                const uint32_t* __restrict__ lb, uint32_t log2B,
                                                                const uint64_t* __restrict__ tbase, uint64_t total,
                                                                const uint64_t* __restrict__ xs,
                                                                const uint32_t* __restrict__ pnode,
                                                                const uint32_t* __restrict__ pbin, uint64_t* t) {
  __shared__ uint32_t queue[kSplitChunk];
  __shared__ uint32_t qn;
  auto set_of_bin = [&](uint64_t g) -> uint32_t {
    if (!tbase) return 0;
    uint32_t lo = 0, hi = K - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (tbase[mid] <= g) lo = mid;
      else hi = mid - 1;
    }
    return lo;
  };
  for (uint64_t c0 = blockIdx.x * (uint64_t)kSplitChunk; c0 < total; c0 += (uint64_t)gridDim.x * kSplitChunk) {
    const uint32_t cn = (uint32_t)(total - c0 < kSplitChunk ? total - c0 : kSplitChunk);
    if (threadIdx.x == 0) qn = 0;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < cn; i += kSplitThreads) {
      const uint64_t g = c0 + i;
      const uint32_t k = set_of_bin(g);
      const uint32_t q = (uint32_t)(g - (tbase ? tbase[k] : 0));
      if (q == 0) {
        t[g] = 0;
        continue;
      }
      const uint64_t so = sets[k].soff, Sk = sets[k].S;
      const uint32_t l2 = lb ? lb[k] : log2B;
      uint64_t lo, hi;
      const uint32_t leaf = sample_bracket(q, ((uint64_t)q * Sk) >> l2, xs + so, pbin + so, pnode + so, Sk, &lo, &hi);
      if (leaf != kSettled) t[g] = leaf_lower_bound(nodes[leaf], lo, hi, q, l2);
      else queue[atomicAdd(&qn, 1u)] = i;
    }
    __syncthreads();
    for (uint32_t j = threadIdx.x; j < qn; j += kSplitThreads) {
      const uint64_t g = c0 + queue[j];
      const uint32_t k = set_of_bin(g);
      const uint32_t q = (uint32_t)(g - (tbase ? tbase[k] : 0));
      const uint64_t so = sets[k].soff, Sk = sets[k].S;
      const uint32_t l2 = lb ? lb[k] : log2B;
      uint64_t lo, hi;
      sample_bracket(q, ((uint64_t)q * Sk) >> l2, xs + so, pbin + so, pnode + so, Sk, &lo, &hi);
      t[g] = bin_lower_bound(nodes, k, lo, hi, q, l2);
    }
    __syncthreads();
  }
}


// radix index of the splitters, level 1: cells c with t[q] <= c << 42 < t[q+1] hold q
__global__ void fine_lut_kernel(const uint64_t* __restrict__ t, uint32_t log2B, uint4* __restrict__ lut) {
  const uint32_t B = 1u << log2B;
  const uint64_t cell = 1ull << kFineLutShift;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < B; q += gridDim.x * blockDim.x) {
    const uint64_t c0 = (t[q] + cell - 1) >> kFineLutShift;
    const uint64_t c1 = q + 1 < B ? (t[q + 1] + cell - 1) >> kFineLutShift : (uint64_t)kFineLutCells;
    const uint64_t next = q + 1 < B ? t[q + 1] : kEncTop;  // above every key past the last splitter
    for (uint64_t c = c0; c < c1 && c < kFineLutCells; ++c)
      lut[c] = make_uint4(q, 0u, (uint32_t)next, (uint32_t)(next >> 32));
  }
}

// level-2 sub-cells of a cell holding cnt splitters (0 = no split)
__device__ __forceinline__ uint32_t lut_split_bits(uint32_t cnt) {
  if (cnt <= kLutDense) return 0;
  const uint32_t b = (32 - __clz(cnt - 1)) + kLutOversplit;  // ceil(log2 cnt) + oversplit
  return b < kLutMaxBits ? b : kLutMaxBits;
}

// level-2 sizes (2^nb + 1 per dense cell): per block of 1024 cells, their total
__device__ __forceinline__ uint32_t lut_cell_bits(const uint4* lut, uint32_t c) {
  return c + 1 < kFineLutCells ? lut_split_bits(lut[c + 1].x - lut[c].x) : 0u;
}
__device__ __forceinline__ uint32_t block_sum_1024(uint32_t v, uint32_t* wsum) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = 16; d; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
  if (lane == 0) wsum[warp] = v;
  __syncthreads();
  uint32_t t = 0;
  for (int w = 0; w < 32; ++w) t += wsum[w];
  return t;
}
__global__ void __launch_bounds__(1024) lut_block_sizes_kernel(const uint4* __restrict__ lut, uint32_t* __restrict__ part,
                                                               uint32_t* __restrict__ big) {
  __shared__ uint32_t wsum[32];
  if (blockIdx.x == 0 && threadIdx.x == 0) big[0] = 0;
  const uint32_t c = blockIdx.x * 1024 + threadIdx.x;
  const uint32_t nb = c < kFineLutCells ? lut_cell_bits(lut, c) : 0;
  const uint32_t t = block_sum_1024(nb ? (1u << nb) + 1 : 0, wsum);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// level-2 offsets: exclusive scan of the sizes (block carry from the block
// totals before it), written into the cells' .y as (offset << 5) | nb
__global__ void __launch_bounds__(1024) lut_offsets_kernel(uint4* __restrict__ lut, const uint32_t* __restrict__ part,
                                                           uint32_t* __restrict__ big) {
  __shared__ uint32_t wsum[33];
  __shared__ uint32_t carry_sh;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x < 32) {
    uint32_t s = 0;
    for (uint32_t b = lane; b < blockIdx.x; b += 32) s += part[b];
    for (int d = 16; d; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (lane == 0) carry_sh = s;
  }
  const uint32_t c = blockIdx.x * 1024 + threadIdx.x;
  const uint32_t nb = c < kFineLutCells ? lut_cell_bits(lut, c) : 0;
  const uint32_t v = nb ? (1u << nb) + 1 : 0;
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
  // every block reads its cells' .x before any block writes .y: the two are
  // separate words, so the reads of the neighbours' .x stay valid
  // (a cell of few splitters keeps its count instead, sparing a lookup the next cell's entry)
  if (c < kFineLutCells)
    lut[c].y = nb ? ((carry_sh + wsum[warp] + incl - v) << 5) | nb : (c + 1 < kFineLutCells ? lut[c + 1].x - lut[c].x : 0u) << 5;
  if (nb > kLutWarpBits) big[1 + atomicAdd(big, 1u)] = c;  // filled by a block
}

// Level-2 entries [k0, k1) of dense cell c: entry k = the largest q in the
// cell's range [q0, q1] with t[q] <= the start of sub-cell k.  A bisection
// for the first, then a walk (entries are non-decreasing in k).
__device__ __forceinline__ void lut_fill_run(const uint64_t* __restrict__ t, uint32_t q0, uint32_t q1, uint32_t c,
                                             uint32_t nb, uint32_t k0, uint32_t k1, uint32_t* __restrict__ l2) {
  const uint64_t start = (uint64_t)c << kFineLutShift;
  uint64_t v = start + ((uint64_t)k0 << (kFineLutShift - nb));
  uint32_t lo = q0, hi = q1;  // t[q0] <= v, answer <= q1
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (t[mid] <= v) lo = mid;
    else hi = mid - 1;
  }
  uint64_t next = lo < q1 ? t[lo + 1] : ~0ull;
  for (uint32_t k = k0;;) {
    l2[k] = lo;
    if (++k == k1) break;
    v = start + ((uint64_t)k << (kFineLutShift - nb));
    while (next <= v) {  // then lo < q1
      ++lo;
      next = lo < q1 ? t[lo + 1] : ~0ull;
    }
  }
}

// level-2 entries of the cells of up to 2^kLutWarpBits sub-cells: a warp per
// cell, each lane a run of consecutive entries
__global__ void lut_fill_kernel(const uint64_t* __restrict__ t, const uint4* __restrict__ lut, uint32_t* __restrict__ l2) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c + 1 < kFineLutCells; c += warps) {
    const uint4 a = lut[c];
    const uint32_t nb = a.y & 31;
    if (!nb || nb > kLutWarpBits) continue;
    const uint32_t m = (1u << nb) + 1, per = (m + 31) / 32;
    const uint32_t k0 = lane * per, k1 = min(m, k0 + per);
    if (k0 < k1) lut_fill_run(t, a.x, lut[c + 1].x, c, nb, k0, k1, l2 + (a.y >> 5));
  }
}

// The cells listed in big (more than 2^kLutWarpBits sub-cells, more than 256
// splitters): a block per cell, its threads over the cell's splitters q0 ..
// q1 (t[q0] <= the cell's start < t[q0 + 1], t[q1] <= the next cell's start
// < t[q1 + 1]).  Splitter q owns the entries whose sub-cell start lies in
// [t[q], t[q + 1]): the first is the start's ceiling in sub-cell units (0
// for q0), the last ends where q + 1's begin (the table's end for q1).  No
// dependent loads, so a dense cell costs two loads per splitter.
__global__ void lut_fill_big_kernel(const uint64_t* __restrict__ t, const uint4* __restrict__ lut,
                                    const uint32_t* __restrict__ big, uint32_t* __restrict__ l2) {
  const uint32_t count = big[0];
  for (uint32_t i = blockIdx.x; i < count; i += gridDim.x) {
    const uint32_t c = big[1 + i];
    const uint4 a = lut[c];
    const uint32_t nb = a.y & 31, m = (1u << nb) + 1, sh = kFineLutShift - nb;
    const uint32_t q0 = a.x, q1 = lut[c + 1].x;
    const uint64_t start = (uint64_t)c << kFineLutShift;
    uint32_t* e = l2 + (a.y >> 5);
    auto first_entry = [&](uint32_t q) -> uint32_t {  // q0 < q <= q1: start < t[q] <= start + 2^42
      return (uint32_t)((t[q] - start + (1ull << sh) - 1) >> sh);
    };
    for (uint32_t q = q0 + threadIdx.x; q <= q1; q += blockDim.x) {
      const uint32_t k0 = q == q0 ? 0u : first_entry(q);
      const uint32_t k1 = q == q1 ? m : first_entry(q + 1);
      for (uint32_t k = k0; k < k1; ++k) e[k] = q;
    }
  }
}

// equal-width slices of the printable key domain: t_q = ceil(q * 95^9 / B)
__global__ void radix_splitter_kernel(uint32_t log2B, uint64_t* __restrict__ t) {
  const uint32_t B = 1u << log2B;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < B; q += gridDim.x * blockDim.x)
    t[q] = (uint64_t)(((unsigned __int128)q * kEncTop + (B - 1)) >> log2B);
}

__global__ void set_single_kernel(SetInfo* sets, uint64_t S) {
  sets[0].soff = 0;
  sets[0].S = S;
}

__global__ void write_header(ModelHeader h, ModelHeader* dst, const uint32_t* ctrl) {
  h.num_nodes = ctrl[kLevelNodes + 3];
  h.levels = ctrl[kLevelNodes + 5];
  *dst = h;
}

}  // namespace

uint64_t node_cap_for(uint64_t S, uint32_t T) { return 4 * ((S + T - 1) / T) + 1024; }

ModelLayout model_layout(uint64_t S, uint32_t log2B, uint32_t T) {
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  ModelLayout L;
  size_t o = 256;
  L.nodes = o;
  o += up(node_cap_for(S, T) * sizeof(DNode));
  L.splitters = o;
  o += up((size_t)8 << log2B);
  L.lut = o;
  o += up(lut_words_for(log2B) * 4);
  L.mlp_knots = o;
  o += 256;
  L.mlp_w = o;
  o += up(kMlpParamCount * 4);
  L.alt_splitters = o;
  o += up((size_t)8 << log2B);
  L.bytes = o;
  return L;
}

__global__ void write_kind_kernel(ModelHeader* h, uint32_t kind, uint32_t fallback) {
  h->kind = kind;
  h->fallback = fallback;
}

cudaError_t set_model_kind(void* model, uint32_t kind, uint32_t fallback, cudaStream_t st) {
  write_kind_kernel<<<1, 1, 0, st>>>(reinterpret_cast<ModelHeader*>(model), kind, fallback);
  return cudaGetLastError();
}

cudaError_t fit_radix(const FitArgs& a) {
  ModelHeader h = {};
  h.magic = kModelMagic;
  h.kind = 2;  // ELSAR_MODEL_RADIX
  h.log2B = a.log2B;
  h.S = a.S;
  h.node_cap = node_cap_for(a.S, a.T);
  const ModelLayout ml = model_layout(a.S, a.log2B, a.T);
  h.nodes_off = ml.nodes;
  h.splitters_off = ml.splitters;
  h.bytes = ml.bytes;
  h.lut_off = ml.lut;
  h.knots_off = ml.mlp_knots;
  h.weights_off = ml.mlp_w;
  h.T = a.T;
  h.Dmax = a.Dmax;
  uint8_t* mb = static_cast<uint8_t*>(a.model);
  uint64_t* t = reinterpret_cast<uint64_t*>(mb + ml.splitters);
  const uint32_t B = 1u << a.log2B;
  radix_splitter_kernel<<<(B + 255) / 256, 256, 0, a.stream>>>(a.log2B, t);
  build_fine_lut(t, a.log2B, reinterpret_cast<uint32_t*>(mb + ml.lut), a.stream);
  cudaMemsetAsync(a.ctrl + kLevelNodes + 3, 0, 3 * 4, a.stream);  // no RMI nodes, no levels
  write_header<<<1, 1, 0, a.stream>>>(h, reinterpret_cast<ModelHeader*>(mb), a.ctrl);
  *a.launches += 2 + kFineLutLaunches;
  return cudaGetLastError();
}

cudaError_t sample_keys(const uint8_t* records, uint64_t n, uint64_t S, uint64_t seed, const KeyMask& km, uint64_t* out,
                        cudaStream_t st) {
  const unsigned grid = (unsigned)umin64((S + 255) / 256, (uint64_t)sm_count() * 8);
  sample_kernel<<<grid ? grid : 1, 256, 0, st>>>(records, n, S, seed, km, out);
  return cudaGetLastError();
}

cudaError_t build_fine_lut(const uint64_t* splitters, uint32_t log2B, uint32_t* lut, cudaStream_t st) {
  const uint32_t B = 1u << log2B;
  uint4* l1 = reinterpret_cast<uint4*>(lut);
  uint32_t* l2 = lut + kLutL1Words * kFineLutCells;
  fine_lut_kernel<<<(B + 255) / 256, 256, 0, st>>>(splitters, log2B, l1);
  const uint32_t blocks = (kFineLutCells + 1023) / 1024;
  // block totals go to the last 256 words of level 2 and the list of large
  // cells before them: the entries never reach either
  uint32_t* part = l2 + lut_level2_words(log2B) - 256;
  uint32_t* big = part - lut_big_words(log2B);
  lut_block_sizes_kernel<<<blocks, 1024, 0, st>>>(l1, part, big);
  lut_offsets_kernel<<<blocks, 1024, 0, st>>>(l1, part, big);
  lut_fill_kernel<<<(kFineLutCells + 7) / 8, 256, 0, st>>>(splitters, l1, l2);
  lut_fill_big_kernel<<<(unsigned)sm_count() * 2, 256, 0, st>>>(splitters, l1, big, l2);
  return cudaGetLastError();
}

int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev);
    if (cached <= 0) cached = 148;
  }
  return cached;
}

namespace {

// Executable graphs of the device level loop, one per argument set (a graph
// with a conditional node has one instantiation); kept for reuse, as
// successive calls on one workspace pass the same pointers.
struct LevelLoop {
  int dev;
  RmiLevelsArgs a;
  unsigned ngrid, sgrid;
  cudaGraph_t g;
  cudaGraphExec_t exec;
};
std::mutex g_loop_mu;
std::vector<LevelLoop> g_loops;
constexpr size_t kMaxLoops = 32;

bool same_loop(const LevelLoop& l, int dev, const RmiLevelsArgs& a, unsigned ngrid, unsigned sgrid) {
  return l.dev == dev && l.a.x == a.x && l.a.S_total == a.S_total && l.a.sets == a.sets && l.a.K == a.K &&
         l.a.T == a.T && l.a.Dmax == a.Dmax && l.a.node_cap == a.node_cap && l.a.nodes == a.nodes &&
         l.a.pnode == a.pnode && l.a.sums == a.sums && l.a.fc == a.fc && l.a.ctrl == a.ctrl && l.ngrid == ngrid &&
         l.sgrid == sgrid;
}

// the loop: a while-node whose body is one level (fit, child numbering,
// finalisation, the next level's nodes, routing with the children's sums,
// advance); the handle starts at 1 on every launch and the body's last
// kernel sets it
cudaError_t make_level_loop(const RmiLevelsArgs& a, unsigned ngrid, unsigned sgrid, cudaGraph_t* g_out,
                            cudaGraphExec_t* exec_out) {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  cudaGraphConditionalHandle h = 0;
  if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cond = nullptr;
  if (e == cudaSuccess) e = cudaGraphAddNode(&cond, g, nullptr, nullptr, 0, &cp);
  cudaGraph_t body = e == cudaSuccess ? cp.conditional.phGraph_out[0] : nullptr;
  cudaGraphNode_t prev = nullptr;
  auto add = [&](const void* fn, unsigned grid, unsigned block, void** args) {
    if (e != cudaSuccess) return;
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void*>(fn);
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(block);
    kp.kernelParams = args;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddKernelNode(&node, body, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
    prev = node;
  };
  const uint64_t* x = a.x;
  uint64_t S = a.S_total, cap = a.node_cap;
  DNode* nodes = a.nodes;
  uint32_t* pnode = a.pnode;
  uint64_t* sums = a.sums;
  uint32_t* fc = a.fc;
  uint32_t* childoff = a.fc + a.node_cap;
  uint32_t* ctrl = a.ctrl;
  const SetInfo* sets = a.sets;
  uint32_t T = a.T, Dmax = a.Dmax, max_levels = a.Dmax + 1;
  void* fit_args[] = {&x, &nodes, &sums, &fc, &T, &Dmax, &ctrl};
  add((const void*)level_fit, ngrid, 256, fit_args);
  void* scan_args[] = {&fc, &childoff, &cap, &ctrl};
  add((const void*)level_scan, 1, kScanThreads, scan_args);
  void* fin_args[] = {&nodes, &fc, &childoff, &sets, &ctrl};
  add((const void*)level_finalize, ngrid, 256, fin_args);
  void* init_args[] = {&nodes, &sums, &childoff, &x, &ctrl};
  add((const void*)level_init_next, ngrid, 256, init_args);
  void* sums_args[] = {&x, &S, &nodes, &pnode, &sums, &ctrl};
  add((const void*)level_sums<true>, sgrid, 256, sums_args);
  void* adv_args[] = {&ctrl, &h, &max_levels};
  add((const void*)level_advance_loop, 1, 1, adv_args);
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
  if (e != cudaSuccess) {
    if (exec) cudaGraphExecDestroy(exec);
    if (g) cudaGraphDestroy(g);
    return e;
  }
  *g_out = g;
  *exec_out = exec;
  return cudaSuccess;
}

// launch the device loop for a on its stream (building or reusing its graph)
cudaError_t launch_level_loop(const RmiLevelsArgs& a, unsigned ngrid, unsigned sgrid) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_loop_mu);
  for (auto& l : g_loops)
    if (same_loop(l, dev, a, ngrid, sgrid)) return cudaGraphLaunch(l.exec, a.stream);
  if (g_loops.size() >= kMaxLoops) {  // retire the oldest, once no launch of it can be in flight
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
    for (auto& l : g_loops) {
      cudaGraphExecDestroy(l.exec);
      cudaGraphDestroy(l.g);
    }
    g_loops.clear();
  }
  LevelLoop l = {};
  l.dev = dev;
  l.a = a;
  l.ngrid = ngrid;
  l.sgrid = sgrid;
  if ((e = make_level_loop(a, ngrid, sgrid, &l.g, &l.exec)) != cudaSuccess) return e;
  g_loops.push_back(l);
  return cudaGraphLaunch(l.exec, a.stream);
}

}  // namespace

cudaError_t build_rmi_levels(const RmiLevelsArgs& a) {
  cudaStream_t st = a.stream;
  const int sms = sm_count();
  const unsigned pgrid = (unsigned)umin64((a.S_total + 255) / 256 + 1, (uint64_t)sms * 8);
  const unsigned ngrid = (unsigned)sms * 8;
  const unsigned sgrid = (unsigned)umin64((a.S_total + kSumsBlockPoints - 1) / kSumsBlockPoints + 1, (uint64_t)sms * 8);
  cudaMemsetAsync(a.sums, 0, (size_t)a.K * 6 * sizeof(uint64_t), st);
  init_roots<<<pgrid, 256, 0, st>>>(a.x, a.nodes, a.pnode, a.sets, a.K, a.S_total, a.ctrl);
  level_sums<false><<<sgrid, 256, 0, st>>>(a.x, a.S_total, a.nodes, a.pnode, a.sums, a.ctrl);
  *a.launches += 2;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (a.device_loop && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
    *a.launches += 1;  // one graph launch (six kernels per level)
    return launch_level_loop(a, ngrid, sgrid);
  }
  // a fixed number of levels (inside a caller's stream capture too, where a
  // graph with a while-node cannot be embedded); empty levels exit at once
  const uint32_t max_levels = a.Dmax + 1;
  for (uint32_t lv = 0; lv < max_levels; ++lv) {
    level_fit<<<ngrid, 256, 0, st>>>(a.x, a.nodes, a.sums, a.fc, a.T, a.Dmax, a.ctrl);
    level_scan<<<1, kScanThreads, 0, st>>>(a.fc, a.fc + a.node_cap, a.node_cap, a.ctrl);
    level_finalize<<<ngrid, 256, 0, st>>>(a.nodes, a.fc, a.fc + a.node_cap, a.sets, a.ctrl);
    level_init_next<<<ngrid, 256, 0, st>>>(a.nodes, a.sums, a.fc + a.node_cap, a.x, a.ctrl);
    level_sums<true><<<sgrid, 256, 0, st>>>(a.x, a.S_total, a.nodes, a.pnode, a.sums, a.ctrl);
    level_advance<<<1, 1, 0, st>>>(a.ctrl);
    *a.launches += 6;
  }
  return cudaGetLastError();
}

cudaError_t splitters_batch(const DNode* nodes, uint32_t K, const SetInfo* sets, const uint32_t* log2B,
                            const uint64_t* tbase, uint64_t total_bins, const uint64_t* x, uint64_t S_total,
                            const uint32_t* pnode, uint32_t* pbin, uint64_t* t, cudaStream_t st) {
  const unsigned pgrid = (unsigned)umin64((S_total + 255) / 256 + 1, (uint64_t)sm_count() * 8);
  point_bins_kernel<<<pgrid, 256, 0, st>>>(x, S_total, nodes, pnode, sets, K, log2B, 0, pbin);
  const unsigned grid = (unsigned)umin64((total_bins + kSplitChunk - 1) / kSplitChunk, (uint64_t)sm_count() * 16);
  splitter_kernel<<<grid ? grid : 1, kSplitThreads, 0, st>>>(nodes, K, sets, log2B, 0, tbase, total_bins, x, pnode,
                                                             pbin, t);
  return cudaGetLastError();
}

cudaError_t fit_rmi(const FitArgs& a, const uint64_t** sorted_out) {
  const uint64_t S = a.S;
  const uint64_t cap = node_cap_for(S, a.T);
  uint8_t* mb = static_cast<uint8_t*>(a.model);
  ModelHeader h = {};
  h.magic = kModelMagic;
  h.kind = 0;
  h.log2B = a.log2B;
  h.S = S;
  h.node_cap = cap;
  const ModelLayout ml = model_layout(S, a.log2B, a.T);
  h.nodes_off = ml.nodes;
  h.splitters_off = ml.splitters;
  h.bytes = ml.bytes;
  h.lut_off = ml.lut;
  h.knots_off = ml.mlp_knots;
  h.weights_off = ml.mlp_w;
  h.T = a.T;
  h.Dmax = a.Dmax;
  DNode* nodes = reinterpret_cast<DNode*>(mb + h.nodes_off);
  uint64_t* splitters = reinterpret_cast<uint64_t*>(mb + h.splitters_off);
  const int sms = sm_count();
  cudaStream_t st = a.stream;
  uint32_t& L = *a.launches;
  // 1. sample (Sec. 3.1)
  const unsigned sgrid = (unsigned)umin64((S + 255) / 256, (uint64_t)sms * 8);
  sample_kernel<<<sgrid, 256, 0, st>>>(a.records, a.n, S, a.seed, a.km, a.samp);
  ++L;
  // 2. sort the sample
  chunk_sort_u64<<<(unsigned)((S + kChunk - 1) / kChunk), kChunkThreads, 0, st>>>(a.samp, S);
  ++L;
  uint64_t* src = a.samp;
  uint64_t* dst = a.samp + S;
  for (uint64_t w = kChunk; w < S; w *= 2) {
    merge_pass_u64<<<(unsigned)((S + kMergeTile - 1) / kMergeTile), kMergeThreads, 0, st>>>(src, dst, S, w);
    ++L;
    uint64_t* tmp = src;
    src = dst;
    dst = tmp;
  }
  const uint64_t* x = src;
  if (sorted_out) *sorted_out = src;
  // 3. RMI, breadth first, one level per round
  set_single_kernel<<<1, 1, 0, st>>>(a.sets, S);
  ++L;
  RmiLevelsArgs la = {};
  la.x = x;
  la.S_total = S;
  la.sets = a.sets;
  la.K = 1;
  la.T = a.T;
  la.Dmax = a.Dmax;
  la.node_cap = cap;
  la.nodes = nodes;
  la.pnode = a.pnode;
  la.sums = a.sums;
  la.fc = a.fc;
  la.ctrl = a.ctrl;
  la.device_loop = true;
  la.stream = st;
  la.launches = a.launches;
  cudaError_t err = build_rmi_levels(la);
  if (err != cudaSuccess) return err;
  // 4. splitters of the fine bins (the bins of the sample points in the sums' place)
  const uint32_t B = 1u << a.log2B;
  uint32_t* pbin = reinterpret_cast<uint32_t*>(a.sums);
  const unsigned pgrid = (unsigned)umin64((S + 255) / 256 + 1, (uint64_t)sms * 8);
  point_bins_kernel<<<pgrid, 256, 0, st>>>(x, S, nodes, a.pnode, a.sets, 1, nullptr, a.log2B, pbin);
  splitter_kernel<<<(B + kSplitChunk - 1) / kSplitChunk, kSplitThreads, 0, st>>>(nodes, 1, a.sets, nullptr, a.log2B,
                                                                                nullptr, B, x, a.pnode, pbin, splitters);
  build_fine_lut(splitters, a.log2B, reinterpret_cast<uint32_t*>(mb + ml.lut), st);
  write_header<<<1, 1, 0, st>>>(h, reinterpret_cast<ModelHeader*>(mb), a.ctrl);
  L += 3 + kFineLutLaunches;
  return cudaGetLastError();
}

}  // namespace elsar
