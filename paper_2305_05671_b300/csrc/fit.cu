// Model training on the GPU (Sec. 3.1 of the paper): key sample, sample sort,
// the RMI of linear models, and the fine-bin splitters classification uses.
//
// Every floating-point step uses explicit round-to-nearest intrinsics in the
// order the model definition fixes (this file is also built with
// -fmad=false), so the fitted model is bit-identical wherever it is computed
// in that order.  Least-squares sums are exact integers (order independent).
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

// router of an internal node: clamp(floor(fma(gamma, u, delta) * scale), 0, f-1)
__device__ __forceinline__ uint32_t route(const DNode& v, uint64_t x) {
  double t = __dmul_rn(__fma_rn(v.a, __ull2double_rn(local_u(v, x)), v.b), v.c);
  if (!(t > 0.0)) return 0;
  if (t >= __uint2double_rn(v.fanout)) return v.fanout - 1;
  return __double2uint_rz(t);
}

__device__ __forceinline__ void atomic_add_u128(uint64_t* p, u128 v) {
  uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
  unsigned long long old = atomicAdd(reinterpret_cast<unsigned long long*>(p), (unsigned long long)lo);
  if (old + lo < old) hi += 1;
  if (hi) atomicAdd(reinterpret_cast<unsigned long long*>(p + 1), (unsigned long long)hi);
}

__device__ __forceinline__ u128 shfl_down_u128(u128 v, int d) {
  uint64_t lo = __shfl_down_sync(0xffffffffu, (uint64_t)v, d);
  uint64_t hi = __shfl_down_sync(0xffffffffu, (uint64_t)(v >> 64), d);
  return ((u128)hi << 64) | lo;
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

__global__ void __launch_bounds__(kChunkThreads) chunk_sort_u64(uint64_t* data, uint64_t S) {
  __shared__ uint64_t s[kChunk];
  const uint64_t base = (uint64_t)blockIdx.x * kChunk;
  for (int i = threadIdx.x; i < kChunk; i += kChunkThreads) s[i] = base + i < S ? data[base + i] : ~0ull;
  __syncthreads();
  for (int k = 2; k <= kChunk; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < kChunk; i += kChunkThreads) {
        int ixj = i ^ j;
        if (ixj > i) {
          uint64_t a = s[i], b = s[ixj];
          bool up = (i & k) == 0;
          if ((a > b) == up) {
            s[i] = b;
            s[ixj] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < kChunk; i += kChunkThreads)
    if (base + i < S) data[base + i] = s[i];
}

constexpr int kMergeTile = 2048;
constexpr int kMergeThreads = 256;
constexpr int kMergeItems = kMergeTile / kMergeThreads;

// number of elements taken from a among the first diag outputs of merge(a, b)
__device__ __forceinline__ uint64_t merge_split(const uint64_t* a, uint64_t na, const uint64_t* b, uint64_t nb,
                                                uint64_t diag) {
  uint64_t lo = diag > nb ? diag - nb : 0, hi = diag < na ? diag : na;
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if (a[mid] <= b[diag - 1 - mid]) lo = mid + 1;
    else hi = mid;
  }
  return lo;
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
  if (threadIdx.x < 2) {
    uint64_t diag = (threadIdx.x ? o1 : o0) - p0;
    split[threadIdx.x] = merge_split(src + a0, a1 - a0, src + b0, b1 - b0, diag);
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

__global__ void init_roots(DNode* nodes, uint32_t* pnode, const SetInfo* __restrict__ sets, uint32_t K,
                           uint64_t S_total, uint32_t* ctrl) {
  const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x, stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t k = t0; k < K; k += stride) {
    DNode r = {};
    r.s = (uint32_t)sets[k].soff;
    r.e = (uint32_t)(sets[k].soff + sets[k].S);
    r.depth_set = (uint32_t)k << 8;
    nodes[k] = r;
  }
  if (t0 == 0) {
    ctrl[kLevelNodes + 0] = 0;
    ctrl[kLevelNodes + 1] = K;
    ctrl[kLevelNodes + 2] = 0;
    ctrl[kLevelNodes + 3] = K;
    ctrl[kLevelNodes + 4] = 0;
  }
  for (uint64_t j = t0; j < S_total; j += stride) pnode[j] = set_of_point(sets, K, j);
}

// per-node base and shift, read by every point of the node
__device__ __forceinline__ void node_frame(const uint64_t* x, uint32_t s, uint32_t e, uint64_t* base, uint32_t* sh) {
  uint64_t b = x[s];
  uint64_t span = x[e - 1] - b;
  uint32_t bits = span ? 64 - __clzll((long long)span) : 0;
  *base = b;
  *sh = bits > 32 ? bits - 32 : 0;
}

// exact sums Su, Suu, Sur of each node of the level (u = local coordinate, r = local rank)
__global__ void level_sums(const uint64_t* __restrict__ x, uint64_t S, const DNode* __restrict__ nodes,
                           const uint32_t* __restrict__ pnode, uint64_t* sums, const uint32_t* ctrl) {
  const uint32_t lv0 = ctrl[kLevelNodes + 0], lv1 = ctrl[kLevelNodes + 1];
  if (lv0 >= lv1) return;
  for (uint64_t k0 = blockIdx.x * (uint64_t)blockDim.x; k0 < S; k0 += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t k = k0 + threadIdx.x;
    uint32_t v = k < S ? pnode[k] : kSettled;
    u128 u = 0, uu = 0, ur = 0;
    if (v != kSettled) {
      uint32_t s = nodes[v].s, e = nodes[v].e;
      uint64_t base;
      uint32_t sh;
      node_frame(x, s, e, &base, &sh);
      uint64_t uv = (x[k] - base) >> sh;
      u = uv;
      uu = (u128)uv * uv;
      ur = (u128)uv * (uint64_t)(k - s);
    }
    uint32_t v0 = __shfl_sync(0xffffffffu, v, 0);
    if (__all_sync(0xffffffffu, v == v0) && v0 != kSettled) {
      for (int d = 16; d; d >>= 1) {
        u += shfl_down_u128(u, d);
        uu += shfl_down_u128(uu, d);
        ur += shfl_down_u128(ur, d);
      }
      if ((threadIdx.x & 31) == 0) {
        uint64_t* sm = sums + (uint64_t)(v0 - lv0) * 6;
        atomicAdd(reinterpret_cast<unsigned long long*>(sm), (unsigned long long)(uint64_t)u);
        atomic_add_u128(sm + 2, uu);
        atomic_add_u128(sm + 4, ur);
      }
    } else if (v != kSettled) {
      uint64_t* sm = sums + (uint64_t)(v - lv0) * 6;
      atomicAdd(reinterpret_cast<unsigned long long*>(sm), (unsigned long long)(uint64_t)u);
      atomic_add_u128(sm + 2, uu);
      atomic_add_u128(sm + 4, ur);
    }
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

// Single CTA: child numbering = exclusive scan of the split fanouts of the
// level (coalesced tiles of kScanThreads with a running carry) and the node
// budget check.  ctrl[kLevelNodes+2] = next level size (0 on overflow),
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
  for (uint32_t base = 0; base < cnt; base += kScanThreads) {
    const uint32_t i = base + threadIdx.x;
    const uint32_t v = i < cnt ? fc[i] : 0;
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
    const uint32_t carry = carry_sh;
    if (i < cnt) childoff[i] = carry + wsum[warp] + incl - v;
    __syncthreads();
    if (threadIdx.x == kScanThreads - 1) carry_sh = carry + wsum[warp] + incl;
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

// Records of the next level zeroed with their sums (level_route sets ranges,
// depth and set).
__global__ void level_init_next(DNode* nodes, uint64_t* sums, const uint32_t* ctrl) {
  const uint32_t lv1 = ctrl[kLevelNodes + 1], next = ctrl[kLevelNodes + 2];
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < next; w += gridDim.x * blockDim.x) {
    DNode c = {};
    nodes[lv1 + w] = c;
    uint64_t* sm = sums + (uint64_t)w * 6;
    for (int t = 0; t < 6; ++t) sm[t] = 0;
  }
}

// route every point of an internal node to its child; children's rank ranges
__global__ void level_route(const uint64_t* __restrict__ x, uint64_t S, DNode* nodes, uint32_t* pnode,
                            const uint32_t* ctrl) {
  const uint32_t lv0 = ctrl[kLevelNodes + 0], lv1 = ctrl[kLevelNodes + 1];
  if (lv0 >= lv1) return;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < S; k += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t v = pnode[k];
    if (v == kSettled || v < lv0 || v >= lv1) continue;
    const DNode nd = nodes[v];
    if (!nd.fanout) {
      pnode[k] = kSettled;
      continue;
    }
    const uint32_t cds = nd.depth_set + 1;  // same set, one level deeper
    uint32_t c = route(nd, x[k]);
    pnode[k] = nd.child0 + c;
    int pc = (k == nd.s) ? -1 : (int)route(nd, x[k - 1]);
    for (int cc = pc + 1; cc <= (int)c; ++cc) {
      nodes[nd.child0 + cc].s = (uint32_t)k;
      nodes[nd.child0 + cc].depth_set = cds;
      if (cc >= 1) nodes[nd.child0 + cc - 1].e = (uint32_t)k;
    }
    if (k == nd.e - 1) {
      for (uint32_t cc = c + 1; cc < nd.fanout; ++cc) {
        nodes[nd.child0 + cc].s = nd.e;
        nodes[nd.child0 + cc].depth_set = cds;
        nodes[nd.child0 + cc - 1].e = nd.e;
      }
      nodes[nd.child0 + nd.fanout - 1].e = nd.e;
    }
  }
}

__global__ void level_advance(uint32_t* ctrl) {
  uint32_t lv1 = ctrl[kLevelNodes + 1];
  ctrl[kLevelNodes + 0] = lv1;
  ctrl[kLevelNodes + 1] = lv1 + ctrl[kLevelNodes + 2];
  ctrl[kLevelNodes + 2] = 0;
}

__device__ __forceinline__ double tree_cdf(const DNode* __restrict__ nodes, uint32_t root, uint64_t x) {
  DNode v = nodes[root];
  while (v.fanout) v = nodes[v.child0 + route(v, x)];
  double y = __fma_rn(v.a, __ull2double_rn(local_u(v, x)), v.b);
  if (y < v.c) return v.c;
  if (y > v.h) return v.h;
  return y;
}

__device__ __forceinline__ uint32_t tree_bin(const DNode* __restrict__ nodes, uint32_t root, uint64_t x,
                                             uint32_t log2B) {
  const uint32_t B = 1u << log2B;
  const uint32_t q = __double2uint_rz(__dmul_rn(tree_cdf(nodes, root, x), __uint2double_rn(B)));
  return q < B ? q : B - 1;
}

// fine-bin splitters: t[q] = smallest encoding whose bin is >= q (t[0] = 0);
// 95^9 when no key reaches bin q.  The bin is a monotone function of the
// encoding, so a bisection over any bracket [lo, hi] holding the answer gives
// the same t[q] as one over the whole range; the bracket comes from the
// sorted sample xs (the model was fitted to its ranks, so the bin of xs[k] is
// near B k / S): start at k = q S / B and gallop outwards to a sample key on
// each side of the answer, then bisect between them.
__global__ void splitter_kernel(const DNode* __restrict__ nodes, uint32_t log2B, uint64_t* t,
                                const uint64_t* __restrict__ xs, uint64_t S) {
  const uint32_t B = 1u << log2B;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < B; q += gridDim.x * blockDim.x) {
    if (q == 0) {
      t[0] = 0;
      continue;
    }
    uint64_t lo = 0, hi = kEncTop;  // the answer lies in [lo, hi]
    if (S) {
      uint64_t k = ((uint64_t)q * S) >> log2B;  // q < 2^20, S < 2^24: no overflow
      if (k > S - 1) k = S - 1;
      if (tree_bin(nodes, 0, xs[k], log2B) >= q) {  // answer <= xs[k]: walk down to a key below it
        hi = xs[k];
        for (uint64_t step = 1;; step <<= 1) {
          if (k == 0) break;  // lo stays 0
          const uint64_t i = k > step ? k - step : 0;
          if (tree_bin(nodes, 0, xs[i], log2B) >= q) {
            hi = xs[i];
            k = i;
          } else {
            lo = xs[i] + 1;
            break;
          }
        }
      } else {  // answer > xs[k]: walk up to a key at or above it
        lo = xs[k] + 1;
        for (uint64_t step = 1;; step <<= 1) {
          if (k == S - 1) break;  // hi stays 95^9
          const uint64_t i = k + step < S - 1 ? k + step : S - 1;
          if (tree_bin(nodes, 0, xs[i], log2B) >= q) {
            hi = xs[i];
            break;
          }
          lo = xs[i] + 1;
          k = i;
        }
      }
    }
    while (lo < hi) {
      uint64_t mid = lo + ((hi - lo) >> 1);
      if (tree_bin(nodes, 0, mid, log2B) >= q) hi = mid;
      else lo = mid + 1;
    }
    t[q] = lo;
  }
}

// the same for K trees: global bin g belongs to set k with tbase[k] <= g < tbase[k+1]
__global__ void splitter_batch_kernel(const DNode* __restrict__ nodes, uint32_t K, const uint32_t* __restrict__ log2B,
                                      const uint64_t* __restrict__ tbase, uint64_t total, uint64_t* t) {
  for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < total; g += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = K - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (tbase[mid] <= g) lo = mid;
      else hi = mid - 1;
    }
    const uint32_t k = lo, lb = log2B[k];
    const uint32_t q = (uint32_t)(g - tbase[k]);
    if (q == 0) {
      t[g] = 0;
      continue;
    }
    uint64_t a = 0, b = kEncTop;
    while (a < b) {
      const uint64_t mid = a + ((b - a) >> 1);
      if (tree_bin(nodes, k, mid, lb) >= q) b = mid;
      else a = mid + 1;
    }
    t[g] = a;
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
__global__ void __launch_bounds__(1024) lut_block_sizes_kernel(const uint4* __restrict__ lut, uint32_t* __restrict__ part) {
  __shared__ uint32_t wsum[32];
  const uint32_t c = blockIdx.x * 1024 + threadIdx.x;
  const uint32_t nb = c < kFineLutCells ? lut_cell_bits(lut, c) : 0;
  const uint32_t t = block_sum_1024(nb ? (1u << nb) + 1 : 0, wsum);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// level-2 offsets: exclusive scan of the sizes (block carry from the block
// totals before it), written into the cells' .y as (offset << 5) | nb
__global__ void __launch_bounds__(1024) lut_offsets_kernel(uint4* __restrict__ lut, const uint32_t* __restrict__ part) {
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
  if (c < kFineLutCells) lut[c].y = nb ? ((carry_sh + wsum[warp] + incl - v) << 5) | nb : 0u;
}

// level-2 entries: a warp per dense cell, lanes over its sub-cell starts;
// entry k = largest q in the cell's range with t[q] <= the sub-cell's start
__global__ void lut_fill_kernel(const uint64_t* __restrict__ t, const uint4* __restrict__ lut, uint32_t* __restrict__ l2) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); c + 1 < kFineLutCells; c += warps) {
    const uint4 a = lut[c];
    if (!a.y) continue;
    const uint32_t nb = a.y & 31, off = a.y >> 5;
    const uint32_t q0 = a.x, q1 = lut[c + 1].x;
    const uint64_t start = (uint64_t)c << kFineLutShift;
    for (uint32_t k = lane; k <= (1u << nb); k += 32) {
      const uint64_t v = start + ((uint64_t)k << (kFineLutShift - nb));
      uint32_t lo = q0, hi = q1;  // t[q0] <= v, answer <= q1
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (t[mid] <= v) lo = mid;
        else hi = mid - 1;
      }
      l2[off + k] = lo;
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
  cudaMemsetAsync(a.ctrl + kLevelNodes + 3, 0, 4, a.stream);  // no RMI nodes
  write_header<<<1, 1, 0, a.stream>>>(h, reinterpret_cast<ModelHeader*>(mb), a.ctrl);
  *a.launches += 6;
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
  // block totals go to the last 256 words of level 2, which the entries never reach
  uint32_t* part = l2 + lut_level2_words(log2B) - 256;
  lut_block_sizes_kernel<<<blocks, 1024, 0, st>>>(l1, part);
  lut_offsets_kernel<<<blocks, 1024, 0, st>>>(l1, part);
  lut_fill_kernel<<<(kFineLutCells + 7) / 8, 256, 0, st>>>(splitters, l1, l2);
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

cudaError_t build_rmi_levels(const RmiLevelsArgs& a, uint32_t* nodes_out, uint32_t* levels_out) {
  cudaStream_t st = a.stream;
  const int sms = sm_count();
  const unsigned pgrid = (unsigned)umin64((a.S_total + 255) / 256 + 1, (uint64_t)sms * 8);
  const unsigned ngrid = (unsigned)sms * 8;
  cudaMemsetAsync(a.sums, 0, (size_t)a.K * 6 * sizeof(uint64_t), st);
  init_roots<<<pgrid, 256, 0, st>>>(a.nodes, a.pnode, a.sets, a.K, a.S_total, a.ctrl);
  *a.launches += 1;
  uint32_t host_ctrl[4] = {0, a.K, 0, a.K};
  uint32_t levels = 0;
  const uint32_t max_levels = a.Dmax + 1;
  for (uint32_t lv = 0; lv < max_levels; ++lv) {
    level_sums<<<pgrid, 256, 0, st>>>(a.x, a.S_total, a.nodes, a.pnode, a.sums, a.ctrl);
    level_fit<<<ngrid, 256, 0, st>>>(a.x, a.nodes, a.sums, a.fc, a.T, a.Dmax, a.ctrl);
    level_scan<<<1, kScanThreads, 0, st>>>(a.fc, a.fc + a.node_cap, a.node_cap, a.ctrl);
    level_finalize<<<ngrid, 256, 0, st>>>(a.nodes, a.fc, a.fc + a.node_cap, a.sets, a.ctrl);
    level_init_next<<<ngrid, 256, 0, st>>>(a.nodes, a.sums, a.ctrl);
    level_route<<<pgrid, 256, 0, st>>>(a.x, a.S_total, a.nodes, a.pnode, a.ctrl);
    level_advance<<<1, 1, 0, st>>>(a.ctrl);
    *a.launches += 7;
    ++levels;
    if (a.host_sync) {
      cudaError_t err = cudaMemcpyAsync(host_ctrl, a.ctrl + kLevelNodes, sizeof(host_ctrl), cudaMemcpyDeviceToHost, st);
      if (err != cudaSuccess) return err;
      if ((err = cudaStreamSynchronize(st)) != cudaSuccess) return err;
      if (host_ctrl[0] == host_ctrl[1]) break;
    }
  }
  *nodes_out = host_ctrl[3];
  *levels_out = levels;
  return cudaGetLastError();
}

cudaError_t splitters_batch(const DNode* nodes, uint32_t K, const uint32_t* log2B, const uint64_t* tbase,
                            uint64_t total_bins, uint64_t* t, cudaStream_t st) {
  const unsigned grid = (unsigned)umin64((total_bins + 127) / 128 + 1, (uint64_t)sm_count() * 16);
  splitter_batch_kernel<<<grid, 128, 0, st>>>(nodes, K, log2B, tbase, total_bins, t);
  return cudaGetLastError();
}

cudaError_t fit_rmi(const FitArgs& a, uint32_t* nodes_out, const uint64_t** sorted_out) {
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
  la.host_sync = true;
  la.stream = st;
  la.launches = a.launches;
  uint32_t nodes_total = 0, levels = 0;
  cudaError_t err = build_rmi_levels(la, &nodes_total, &levels);
  if (err != cudaSuccess) return err;
  h.levels = levels;
  // 4. splitters of the fine bins
  const uint32_t B = 1u << a.log2B;
  splitter_kernel<<<(B + 127) / 128, 128, 0, st>>>(nodes, a.log2B, splitters, x, S);
  build_fine_lut(splitters, a.log2B, reinterpret_cast<uint32_t*>(mb + ml.lut), st);
  write_header<<<1, 1, 0, st>>>(h, reinterpret_cast<ModelHeader*>(mb), a.ctrl);
  L += 3;
  *nodes_out = nodes_total;
  return cudaGetLastError();
}

}  // namespace elsar
