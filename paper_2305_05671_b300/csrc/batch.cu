// Many independent record sets sorted by one CUDA-graph-captured launch
// sequence (the batched form of the method).  Every set keeps its own model
// (a sample of 1 % of its records, its own RMI, its own fine bins), but all
// sets share the passes: one batched sample and sample sort, one level-wise
// build of all the sets' trees at once, one classify / scan / scatter over a
// common fine-bin space in which set k owns its own range, and one persistent
// sort+gather whose work items never span two sets.  Nothing in the sequence
// reads back to the host, so it is captured once per plan and replayed with a
// single cudaGraphLaunch.  An autotuner picks the tile size and, per size
// class of sets, the fine-bin density, by timing candidate graphs.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/elsar.h"
#include "common.cuh"

namespace elsar {
void set_last_error(const char* msg);
}

using namespace elsar;

namespace {

inline uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

// ------------------------------------------------------------------ kernels
__device__ __forceinline__ uint32_t seg_of(const SetInfo* __restrict__ sets, uint32_t K, uint64_t j) {
  uint32_t lo = 0, hi = K - 1;
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (sets[mid].soff <= j) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// sample j of the concatenation: set k, position mulhi64(SplitMix64_j'(seed + k), n_k)
__global__ void batch_sample_kernel(const uint8_t* const* __restrict__ ins, KeyMask km, const uint64_t* __restrict__ n,
                                    const SetInfo* __restrict__ sets, uint32_t K, uint64_t S_total, uint64_t seed,
                                    Pair* __restrict__ out) {
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < S_total; j += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t k = seg_of(sets, K, j);
    const uint64_t i = __umul64hi(splitmix64_at(seed + k, j - sets[k].soff), n[k]);
    Pair p;
    p.hi = k;
    p.lo = enc9_pair(load_pair(ins[k] + i * kRecord, 0, km));
    out[j] = p;
  }
}

constexpr int kChunk = 2048;
constexpr int kChunkThreads = 1024;

__global__ void __launch_bounds__(kChunkThreads) chunk_sort_pairs(Pair* data, uint64_t S) {
  __shared__ Pair s[kChunk];
  const uint64_t base = (uint64_t)blockIdx.x * kChunk;
  for (int i = threadIdx.x; i < kChunk; i += kChunkThreads) {
    Pair v;
    v.hi = ~0ull;
    v.lo = ~0ull;
    s[i] = base + i < S ? data[base + i] : v;
  }
  __syncthreads();
  for (int k = 2; k <= kChunk; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < kChunk; i += kChunkThreads) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const Pair a = s[i], b = s[ixj];
          const bool up = (i & k) == 0;
          if (pair_less(b, a) == up) {
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

__device__ __forceinline__ uint64_t umin_dev(uint64_t a, uint64_t b) { return a < b ? a : b; }

constexpr int kMergeTile = 1024;
constexpr int kMergeThreads = 256;
constexpr int kMergeItems = kMergeTile / kMergeThreads;

__device__ __forceinline__ uint64_t merge_split(const Pair* a, uint64_t na, const Pair* b, uint64_t nb, uint64_t diag) {
  uint64_t lo = diag > nb ? diag - nb : 0, hi = diag < na ? diag : na;
  while (lo < hi) {
    const uint64_t mid = (lo + hi) >> 1;
    if (!pair_less(b[diag - 1 - mid], a[mid])) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kMergeThreads) merge_pass_pairs(const Pair* __restrict__ src, Pair* __restrict__ dst,
                                                                  uint64_t S, uint64_t w) {
  __shared__ Pair s[kMergeTile];
  __shared__ uint64_t split[2];
  const uint64_t o0 = (uint64_t)blockIdx.x * kMergeTile;
  if (o0 >= S) return;
  const uint64_t o1 = umin_dev(S, o0 + kMergeTile);
  const uint64_t p0 = (o0 / (2 * w)) * (2 * w);
  const uint64_t a1 = umin_dev(S, p0 + w), b1 = umin_dev(S, p0 + 2 * w);
  if (threadIdx.x < 2)
    split[threadIdx.x] = merge_split(src + p0, a1 - p0, src + a1, b1 - a1, (threadIdx.x ? o1 : o0) - p0);
  __syncthreads();
  const uint64_t ka0 = split[0], ka1 = split[1];
  const uint64_t kb0 = (o0 - p0) - ka0, kb1 = (o1 - p0) - ka1;
  const int na = (int)(ka1 - ka0), nb = (int)(kb1 - kb0);
  for (int i = threadIdx.x; i < na; i += kMergeThreads) s[i] = src[p0 + ka0 + i];
  for (int i = threadIdx.x; i < nb; i += kMergeThreads) s[na + i] = src[a1 + kb0 + i];
  __syncthreads();
  const int tot = na + nb;
  const int d = threadIdx.x * kMergeItems;
  if (d >= tot) return;
  int lo = d > nb ? d - nb : 0, hi = d < na ? d : na;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (!pair_less(s[na + d - 1 - mid], s[mid])) lo = mid + 1;
    else hi = mid;
  }
  int ia = lo, ib = d - lo;
  for (int t = 0; t < kMergeItems && d + t < tot; ++t) {
    const bool takeA = ib >= nb || (ia < na && !pair_less(s[na + ib], s[ia]));
    dst[o0 + d + t] = takeA ? s[ia++] : s[na + ib++];
  }
}

__global__ void extract_keys(const Pair* __restrict__ p, uint64_t S, uint64_t* __restrict__ x) {
  for (uint64_t j = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; j < S; j += (uint64_t)gridDim.x * blockDim.x)
    x[j] = p[j].lo;
}

// ------------------------------------------------------------------ host plan
int size_class(uint64_t n) { return n < (1ull << 15) ? 0 : (n < (1ull << 18) ? 1 : 2); }

uint64_t default_sample(uint64_t n) {
  uint64_t s = (n + 99) / 100;
  if (s < 1000) s = 1000;
  if (s > 10000000) s = 10000000;
  return s;
}

uint32_t ceil_log2(uint64_t v) {
  uint32_t r = 0;
  while (r < 63 && (1ull << r) < v) ++r;
  return r;
}

// fine bins of a set: about 2^rpb records per bin, within [6, 20]
uint32_t set_log2B(uint64_t n, uint32_t rpb) {
  const uint32_t c = ceil_log2(n ? n : 1);
  uint32_t b = c > rpb ? c - rpb : 0;
  if (b < 6) b = 6;
  if (b > 20) b = 20;
  return b;
}

struct Tuning {
  uint32_t cap = 2048;
  uint32_t rpb[3] = {10, 10, 10};
};

size_t up(size_t v) { return (v + 255) & ~(size_t)255; }

struct BatchLayout {
  size_t ctrl, ins, outs, n, sets, log2B, tbase, poff, sp0, sp1, x, pnode, nodes, sums, fc, t, pairsA, pairsB, seg,
      bin_off, cursor, items, item_flag, oversize, total;
  uint64_t S_total, B_total, N_total, node_cap;
};

BatchLayout batch_layout(const uint64_t* n, uint32_t K, const Tuning& tu, uint32_t T) {
  BatchLayout L = {};
  uint64_t S = 0, B = 0, N = 0, cap = 0;
  for (uint32_t k = 0; k < K; ++k) {
    const uint64_t s = default_sample(n[k]);
    S += s;
    B += 1ull << set_log2B(n[k], tu.rpb[size_class(n[k])]);
    N += n[k];
    cap += 4 * ((s + T - 1) / T) + 1024;
  }
  L.S_total = S;
  L.B_total = B;
  L.N_total = N;
  L.node_cap = cap;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t a = o;
    o += up(bytes);
    return a;
  };
  L.ctrl = take((64 + 64) * 4);
  L.ins = take(K * 8);
  L.outs = take(K * 8);
  L.n = take(K * 8);
  L.sets = take(K * sizeof(SetInfo));
  L.log2B = take(K * 4);
  L.tbase = take((K + 1) * 8);
  L.poff = take((K + 1) * 8);
  L.sp0 = take(S * sizeof(Pair));
  L.sp1 = take(S * sizeof(Pair));
  L.x = take(S * 8);
  L.pnode = take(S * 4);
  L.nodes = take(cap * sizeof(DNode));
  L.sums = take(cap * 48);
  L.fc = take(cap * 8);
  L.t = take(B * 8);
  L.pairsA = take(N * sizeof(Pair));
  L.pairsB = take(N * sizeof(Pair));
  L.seg = take(coarse_segments(N) * kMaxCoarse * 4);
  L.bin_off = take((B + 1) * 4);
  L.cursor = take(B * 4);
  L.items = take((B + 1) * 4);
  L.item_flag = take(B * 4);
  L.oversize = take(B * 4);
  L.total = o;
  return L;
}

template <typename T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<uint8_t*>(base) + off);
}

}  // namespace

struct elsar_batch {
  uint32_t K = 0;
  std::vector<uint64_t> n;
  std::vector<const void*> ins;
  std::vector<void*> outs;
  elsar_params p = {};
  uint32_t T = 16, Dmax = 32;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  Tuning tune;
  BatchLayout L = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  uint32_t launches = 0;
  float tune_ms[16] = {};
  uint32_t tune_runs = 0;
};

namespace {

std::mutex g_tune_mu;
std::map<std::string, Tuning> g_tune_cache;

std::string tune_key(const elsar_batch& b) {
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  uint64_t cls[3] = {0, 0, 0}, rec[3] = {0, 0, 0};
  for (uint64_t v : b.n) {
    cls[size_class(v)]++;
    rec[size_class(v)] += v;
  }
  char buf[640];
  // sets and records per class, rounded to 2 significant bits, identify the workload shape
  auto r2 = [](uint64_t v) { return v ? (1ull << ceil_log2(v)) : 0ull; };
  snprintf(buf, sizeof buf, "%s|%llu,%llu,%llu|%llu,%llu,%llu", prop.name, (unsigned long long)r2(cls[0]),
           (unsigned long long)r2(cls[1]), (unsigned long long)r2(cls[2]), (unsigned long long)r2(rec[0]),
           (unsigned long long)r2(rec[1]), (unsigned long long)r2(rec[2]));
  return buf;
}

// Upload the per-set tables for a tuning (synchronous; before capture).
cudaError_t upload_tables(elsar_batch& b, cudaStream_t st) {
  const uint32_t K = b.K;
  std::vector<uint64_t> tbase(K + 1), poff(K + 1);
  std::vector<SetInfo> sets(K);
  std::vector<uint32_t> lb(K);
  uint64_t so = 0;
  tbase[0] = 0;
  poff[0] = 0;
  for (uint32_t k = 0; k < K; ++k) {
    const uint64_t s = default_sample(b.n[k]);
    sets[k].soff = so;
    sets[k].S = s;
    so += s;
    lb[k] = set_log2B(b.n[k], b.tune.rpb[size_class(b.n[k])]);
    tbase[k + 1] = tbase[k] + (1ull << lb[k]);
    poff[k + 1] = poff[k] + b.n[k];
  }
  cudaError_t e = cudaSuccess;
  auto cp = [&](size_t off, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(at<void>(b.ws, off), src, bytes, cudaMemcpyHostToDevice, st);
  };
  cp(b.L.ins, b.ins.data(), K * 8);
  cp(b.L.outs, b.outs.data(), K * 8);
  cp(b.L.n, b.n.data(), K * 8);
  cp(b.L.sets, sets.data(), K * sizeof(SetInfo));
  cp(b.L.log2B, lb.data(), K * 4);
  cp(b.L.tbase, tbase.data(), (K + 1) * 8);
  cp(b.L.poff, poff.data(), (K + 1) * 8);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

// The whole batched sequence on `st` (captured by the caller).
cudaError_t enqueue(elsar_batch& b, cudaStream_t st) {
  const BatchLayout& L = b.L;
  void* ws = b.ws;
  const uint32_t K = b.K;
  const int sms = sm_count();
  uint32_t& launches = b.launches;
  launches = 0;
  cudaMemsetAsync(at<void>(ws, L.ctrl), 0, (64 + 64) * 4, st);
  // 1. samples of every set, sorted by (set, key)
  Pair* sp0 = at<Pair>(ws, L.sp0);
  Pair* sp1 = at<Pair>(ws, L.sp1);
  const uint64_t S = L.S_total;
  batch_sample_kernel<<<(unsigned)umin64((S + 255) / 256 + 1, (uint64_t)sms * 8), 256, 0, st>>>(
      at<const uint8_t* const>(ws, L.ins), key_mask(b.p.key_bytes ? b.p.key_bytes : 10), at<uint64_t>(ws, L.n),
      at<SetInfo>(ws, L.sets), K, S, b.p.seed, sp0);
  chunk_sort_pairs<<<(unsigned)((S + kChunk - 1) / kChunk), kChunkThreads, 0, st>>>(sp0, S);
  launches += 2;
  Pair* src = sp0;
  Pair* dst = sp1;
  for (uint64_t w = kChunk; w < S; w *= 2) {
    merge_pass_pairs<<<(unsigned)((S + kMergeTile - 1) / kMergeTile), kMergeThreads, 0, st>>>(src, dst, S, w);
    ++launches;
    Pair* tmp = src;
    src = dst;
    dst = tmp;
  }
  uint64_t* x = at<uint64_t>(ws, L.x);
  extract_keys<<<(unsigned)umin64((S + 255) / 256 + 1, (uint64_t)sms * 8), 256, 0, st>>>(src, S, x);
  ++launches;
  // 2. every set's RMI, all trees level by level together (fixed level count)
  RmiLevelsArgs la = {};
  la.x = x;
  la.S_total = S;
  la.sets = at<SetInfo>(ws, L.sets);
  la.K = K;
  la.T = b.T;
  la.Dmax = b.Dmax;
  la.node_cap = L.node_cap;
  la.nodes = at<DNode>(ws, L.nodes);
  la.pnode = at<uint32_t>(ws, L.pnode);
  la.sums = at<uint64_t>(ws, L.sums);
  la.fc = at<uint32_t>(ws, L.fc);
  la.ctrl = at<uint32_t>(ws, L.ctrl);
  la.device_loop = false;
  la.stream = st;
  la.launches = &launches;
  cudaError_t e = build_rmi_levels(la);
  if (e != cudaSuccess) return e;
  // 3. each set's splitters in its own range of the common bin space
  uint64_t* t = at<uint64_t>(ws, L.t);
  // (the bins of the sample points in the sums' place)
  if ((e = splitters_batch(la.nodes, K, la.sets, at<uint32_t>(ws, L.log2B), at<uint64_t>(ws, L.tbase), L.B_total, x, S,
                           la.pnode, reinterpret_cast<uint32_t*>(la.sums), t, st)) != cudaSuccess)
    return e;
  launches += 2;
  // 4. classify, scan, scatter, work items
  BatchPartArgs pa = {};
  pa.ins = at<const uint8_t* const>(ws, L.ins);
  pa.km = key_mask(b.p.key_bytes ? b.p.key_bytes : 10);
  pa.poff = at<uint64_t>(ws, L.poff);
  pa.K = K;
  pa.B = (uint32_t)L.B_total;
  pa.tile_pairs = b.tune.cap;
  pa.splitters = t;
  pa.tbase = at<uint64_t>(ws, L.tbase);
  pa.log2B = at<uint32_t>(ws, L.log2B);
  pa.pairs_in_order = at<Pair>(ws, L.pairsA);
  pa.pairs = at<Pair>(ws, L.pairsB);
  pa.N = L.N_total;
  pa.seg_hist = at<uint32_t>(ws, L.seg);
  pa.bin_off = at<uint32_t>(ws, L.bin_off);
  pa.cursor = at<uint32_t>(ws, L.cursor);
  pa.items = at<uint32_t>(ws, L.items);
  pa.item_flag = at<uint32_t>(ws, L.item_flag);
  pa.oversize = at<uint32_t>(ws, L.oversize);
  pa.ctrl = at<uint32_t>(ws, L.ctrl);
  pa.stream = st;
  pa.launches = &launches;
  if ((e = partition_batch(pa)) != cudaSuccess) return e;
  // 5. one persistent sort + gather over the items of all sets
  SortArgs sa = {};
  sa.ins = at<const uint8_t* const>(ws, L.ins);
  sa.outs = at<uint8_t* const>(ws, L.outs);
  sa.tbase = pa.tbase;
  sa.poff = pa.poff;
  sa.K = K;
  sa.n = L.N_total;
  sa.schedule = 1;
  sa.tile_pairs = b.tune.cap;
  sa.pairs = pa.pairs;
  sa.temp = pa.pairs_in_order;
  sa.bin_off = pa.bin_off;
  sa.items = pa.items;
  sa.oversize = pa.oversize;
  sa.ctrl = pa.ctrl;
  sa.stream = st;
  sa.launches = &launches;
  return sort_items(sa);
}

cudaError_t build_graph(elsar_batch& b, cudaStream_t st) {
  if (b.exec) {
    cudaGraphExecDestroy(b.exec);
    b.exec = nullptr;
  }
  if (b.graph) {
    cudaGraphDestroy(b.graph);
    b.graph = nullptr;
  }
  b.L = batch_layout(b.n.data(), b.K, b.tune, b.T);
  cudaError_t e = upload_tables(b, st);
  if (e != cudaSuccess) return e;
  if ((e = prepare_sort_kernel(b.tune.cap)) != cudaSuccess) return e;
  if ((e = prepare_scatter_kernels()) != cudaSuccess) return e;
  if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
  cudaError_t qe = enqueue(b, st);
  e = cudaStreamEndCapture(st, &b.graph);
  if (qe != cudaSuccess) return qe;
  if (e != cudaSuccess) return e;
  return cudaGraphInstantiate(&b.exec, b.graph, 0);
}

cudaError_t time_graph(elsar_batch& b, cudaStream_t st, float* ms) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaError_t e = cudaGraphLaunch(b.exec, st);
  if (e == cudaSuccess) e = cudaEventRecord(e0, st);
  if (e == cudaSuccess) e = cudaGraphLaunch(b.exec, st);
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

void load_cache_file() {
  static bool loaded = false;
  if (loaded) return;
  loaded = true;
  const char* path = getenv("ELSAR_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char key[256];
  Tuning t;
  while (fscanf(f, "%255s %u %u %u %u", key, &t.cap, &t.rpb[0], &t.rpb[1], &t.rpb[2]) == 5) g_tune_cache[key] = t;
  fclose(f);
}

void save_cache_file(const std::string& key, const Tuning& t) {
  const char* path = getenv("ELSAR_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %u %u %u %u\n", key.c_str(), t.cap, t.rpb[0], t.rpb[1], t.rpb[2]);
  fclose(f);
}

}  // namespace

extern "C" {

size_t elsar_batch_workspace_size(const uint64_t* n, uint32_t num_sets, const elsar_params* p) {
  if (!n || num_sets == 0) return 0;
  Tuning most;  // the densest bins any tuning may pick
  most.rpb[0] = most.rpb[1] = most.rpb[2] = 9;
  const uint32_t T = p && p->leaf_target ? p->leaf_target : 16;
  return batch_layout(n, num_sets, most, T).total;
}

elsar_status elsar_batch_create(const void* const* d_in, void* const* d_out, const uint64_t* n, uint32_t num_sets,
                                const elsar_params* p, void* d_ws, size_t ws_bytes, elsar_stream_t stream,
                                elsar_batch** out) {
  if (!out) return ELSAR_EINVAL;
  *out = nullptr;
  if (!d_in || !d_out || !n || num_sets == 0 || num_sets > (1u << 24)) {
    set_last_error("elsar_batch_create: need 1..2^24 record sets and their buffers");
    return ELSAR_EINVAL;
  }
  if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255)) {
    set_last_error("elsar_batch_create: workspace must be non-null and 256-byte aligned");
    return ELSAR_EINVAL;
  }
  if (p && p->key_bytes > 10) {
    set_last_error("elsar_batch_create: key_bytes must be in [1, 10] (0 = 10)");
    return ELSAR_EINVAL;
  }
  uint64_t total = 0;
  for (uint32_t k = 0; k < num_sets; ++k) {
    if (n[k] == 0 || !d_in[k] || !d_out[k] || (reinterpret_cast<uintptr_t>(d_in[k]) & 3) ||
        (reinterpret_cast<uintptr_t>(d_out[k]) & 3)) {
      set_last_error("elsar_batch_create: every set needs n > 0 and 4-byte aligned input and output buffers");
      return ELSAR_EINVAL;
    }
    total += n[k];
  }
  if (total >= (1ull << 32)) {
    set_last_error("elsar_batch_create: the sets together must hold fewer than 2^32 records");
    return ELSAR_EUNSUPPORTED;
  }
  const size_t need = elsar_batch_workspace_size(n, num_sets, p);
  if (ws_bytes < need) {
    char msg[160];
    snprintf(msg, sizeof msg, "elsar_batch_create: workspace too small: %zu < %zu bytes", ws_bytes, need);
    set_last_error(msg);
    return ELSAR_ENOMEM;
  }
  elsar_batch* b = new elsar_batch();
  b->K = num_sets;
  b->n.assign(n, n + num_sets);
  b->ins.assign(d_in, d_in + num_sets);
  b->outs.assign(d_out, d_out + num_sets);
  elsar_default_params(&b->p);
  if (p) b->p = *p;
  b->T = b->p.leaf_target ? b->p.leaf_target : 16;
  b->Dmax = b->p.max_depth ? b->p.max_depth : 32;
  b->ws = d_ws;
  b->ws_bytes = ws_bytes;
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess && stream) {
    // order the plan's work after what the caller queued so far
    cudaEvent_t ev;
    e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
    cudaEventDestroy(ev);
  }
  const uint32_t fixed_cap = b->p.tile_pairs;
  if (e == cudaSuccess) {
    if (fixed_cap) {
      b->tune.cap = fixed_cap;
      e = build_graph(*b, st);
    } else {
      std::string key = tune_key(*b);
      bool cached = false;
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        load_cache_file();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
          b->tune = it->second;
          cached = true;
        }
      }
      if (cached) {
        e = build_graph(*b, st);
      } else {
        // autotune: tile size first, then the fine-bin density of each size class
        Tuning best;
        float best_ms = 1e30f;
        auto trial = [&](const Tuning& t) -> cudaError_t {
          b->tune = t;
          cudaError_t err = build_graph(*b, st);
          if (err != cudaSuccess) return err;
          float ms = 0;
          if ((err = time_graph(*b, st, &ms)) != cudaSuccess) return err;
          if (b->tune_runs < 16) b->tune_ms[b->tune_runs] = ms;
          ++b->tune_runs;
          if (ms < best_ms) {
            best_ms = ms;
            best = t;
          }
          return cudaSuccess;
        };
        for (uint32_t cap : {1024u, 2048u, 4096u}) {
          Tuning t = best;
          t.cap = cap;
          if (best_ms == 1e30f) t.rpb[0] = t.rpb[1] = t.rpb[2] = 10;
          if ((e = trial(t)) != cudaSuccess) break;
        }
        bool present[3] = {false, false, false};
        for (uint64_t v : b->n) present[size_class(v)] = true;
        for (int c = 0; c < 3 && e == cudaSuccess; ++c) {
          if (!present[c]) continue;
          for (uint32_t r : {9u, 11u}) {
            Tuning t = best;
            t.rpb[c] = r;
            if ((e = trial(t)) != cudaSuccess) break;
          }
        }
        if (e == cudaSuccess) {
          b->tune = best;
          e = build_graph(*b, st);
          std::lock_guard<std::mutex> lk(g_tune_mu);
          g_tune_cache[key] = best;
          save_cache_file(key, best);
        }
      }
    }
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess) {
    char msg[200];
    snprintf(msg, sizeof msg, "elsar_batch_create: %s", cudaGetErrorString(e));
    set_last_error(msg);
    elsar_batch_destroy(b);
    return ELSAR_ECUDA;
  }
  *out = b;
  return ELSAR_OK;
}

elsar_status elsar_batch_run(elsar_batch* b, elsar_stream_t stream) {
  if (!b || !b->exec) return ELSAR_EINVAL;
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return ELSAR_ECUDA;
  }
  return ELSAR_OK;
}

elsar_status elsar_batch_wait(elsar_batch* b, elsar_stream_t stream) {
  if (!b) return ELSAR_EINVAL;
  uint32_t w = 0;
  cudaError_t e = cudaMemcpyAsync(&w, at<uint32_t>(b->ws, b->L.ctrl) + kStatusWord, 4, cudaMemcpyDeviceToHost,
                                  (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) {
    set_last_error(cudaGetErrorString(e));
    return ELSAR_ECUDA;
  }
  if (w) {
    set_last_error("elsar_batch_wait: a device-side wait timed out");
    return ELSAR_ETIMEOUT;
  }
  return ELSAR_OK;
}

elsar_status elsar_batch_describe(const elsar_batch* b, elsar_batch_info* info) {
  if (!b || !info) return ELSAR_EINVAL;
  std::memset(info, 0, sizeof(*info));
  info->tile_pairs = b->tune.cap;
  for (int c = 0; c < 3; ++c) info->records_per_bin_log2[c] = b->tune.rpb[c];
  info->total_records = b->L.N_total;
  info->total_bins = b->L.B_total;
  info->sample_keys = b->L.S_total;
  info->launches = b->launches;
  info->tuning_runs = b->tune_runs;
  for (uint32_t i = 0; i < 16 && i < b->tune_runs; ++i) info->tuning_ms[i] = b->tune_ms[i];
  return ELSAR_OK;
}

void elsar_batch_destroy(elsar_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  delete b;
}

}  // extern "C"
