// C ABI of libelsar (declared in include/elsar.h): argument checks, parameter
// defaults, the workspace layout, and the order of the GPU passes.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <string>
#include <vector>

#include "../../include/elsar.h"
#include "common.cuh"
#include "mlp.cuh"

namespace elsar {
size_t sort_smem_bytes(uint32_t cap);
void set_last_error(const char* msg);
}

using namespace elsar;

namespace {

thread_local std::string g_err;

elsar_status fail(elsar_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

elsar_status cuda_fail(cudaError_t e, const char* where) {
  return fail(ELSAR_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

struct Resolved {
  uint32_t P, log2B, T, Dmax, kind, balance, schedule, cap, skip, key_bytes;
  uint64_t S, seed;
  long long wait_limit;
};

uint32_t ilog2(uint64_t v) {
  uint32_t r = 0;
  while ((1ull << (r + 1)) <= v) ++r;
  return r;
}

bool pow2(uint64_t v) { return v && !(v & (v - 1)); }

elsar_status resolve(uint64_t n, const elsar_params* p, Resolved* r) {
  elsar_params d;
  elsar_default_params(&d);
  const elsar_params& q = p ? *p : d;
  r->P = q.num_partitions ? q.num_partitions : d.num_partitions;
  if (!pow2(r->P) || r->P > 65536) return fail(ELSAR_EINVAL, "num_partitions must be a power of two <= 65536");
  const uint32_t lp = ilog2(r->P);
  if (q.fine_bins_log2) {
    r->log2B = q.fine_bins_log2;
  } else {
    uint32_t want = 0;
    while (want < 63 && (1ull << want) < (n ? n : 1)) ++want;  // ceil(log2 n)
    want = want > 10 ? want - 10 : 0;
    uint32_t b = want < 6 ? 6 : want;
    if (b > 20) b = 20;
    r->log2B = b > lp ? b : lp;
  }
  if (r->log2B < lp || r->log2B > 22) return fail(ELSAR_EINVAL, "fine_bins_log2 must be in [log2 P, 22]");
  r->T = q.leaf_target ? q.leaf_target : 16;
  r->Dmax = q.max_depth ? q.max_depth : 32;
  r->kind = q.model_kind;
  if (r->kind > 2) return fail(ELSAR_EINVAL, "unknown model_kind");
  r->skip = q.skip_checks;
  if (r->skip > 7) return fail(ELSAR_EINVAL, "skip_checks must be an OR of ELSAR_SKIP_* values");
  r->key_bytes = q.key_bytes ? q.key_bytes : 10;
  if (r->key_bytes > 10) return fail(ELSAR_EINVAL, "key_bytes must be in [1, 10] (0 = 10)");
  if (q.wait_limit_cycles > (1ull << 40)) return fail(ELSAR_EINVAL, "wait_limit_cycles must be <= 2^40");
  r->wait_limit = q.wait_limit_cycles ? (long long)q.wait_limit_cycles : kWaitLimitCycles;
  r->balance = q.balance;
  if (r->balance > 1) return fail(ELSAR_EINVAL, "unknown balance rule");
  r->schedule = q.schedule;
  if (r->schedule > 1) return fail(ELSAR_EINVAL, "unknown schedule");
  r->cap = q.tile_pairs ? q.tile_pairs : 2048;
  if (!pow2(r->cap) || r->cap < 256 || r->cap > 8192) return fail(ELSAR_EINVAL, "tile_pairs must be a power of two in [256, 8192]");
  if (q.sample_size) {
    r->S = q.sample_size;
  } else {
    uint64_t s = (n + 99) / 100;
    if (s < 1000) s = 1000;
    if (s > 10000000) s = 10000000;
    r->S = n ? s : 0;
  }
  if (r->S >= (1ull << 24)) return fail(ELSAR_EINVAL, "sample_size must be < 2^24");
  r->seed = q.seed;
  return ELSAR_OK;
}

struct Layout {
  size_t ctrl, model, pairsA, pairsB, bin_off, part_off, cuts, cursor, items, item_flag, oversize, samp, pnode, sums,
      fc, sets, seg, mlp_phi, mlp_y, mlp_partial, mlp_m, mlp_v, swap, judge, total;
};

constexpr uint64_t kMlpTrainMax = 2000000;  // keys the network trains on (every k-th of the sorted sample)
constexpr uint32_t kMlpBatch = 8192, kMlpSteps = 400, kMlpGrid = 512;
constexpr float kMlpLr = 1e-3f, kMlpLrMin = 1e-5f;

uint64_t mlp_ntrain(uint64_t S) { return S < kMlpTrainMax ? S : kMlpTrainMax; }

size_t up(size_t v) { return (v + 255) & ~(size_t)255; }

Layout layout(uint64_t n, const Resolved& r) {
  Layout L;
  const uint64_t B = 1ull << r.log2B;
  const uint64_t cap = node_cap_for(r.S, r.T);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o += up(bytes);
    return at;
  };
  L.ctrl = take((64 + 65537) * 4);
  L.model = take(model_bytes_for(r.S, r.log2B, r.T));
  L.pairsA = take(n * 16);
  L.pairsB = take(n * 16);
  L.bin_off = take((B + 1) * 4);
  L.part_off = take((r.P + 1) * 8);
  L.cuts = take((r.P + 1) * 4);
  L.cursor = take(B * 4);
  L.items = take((B + 1) * 4);
  L.item_flag = take(B * 4);
  L.oversize = take(B * 4);
  L.samp = take(2 * r.S * 8);
  L.pnode = take(r.S * 4);
  L.sums = take(cap * 48);
  L.fc = take(cap * 8);  // split fanouts + child offsets of one level
  L.sets = take(sizeof(SetInfo));
  L.seg = take(coarse_segments(n) * kMaxCoarse * 4);
  const bool mlp = r.kind == ELSAR_MODEL_MLP;
  const uint64_t nt = mlp ? mlp_ntrain(r.S) : 0;
  L.mlp_phi = take(nt * 12 * 4);
  L.mlp_y = take(nt * 4);
  L.mlp_partial = take(mlp ? (size_t)kMlpGrid * kMlpParamCount * 4 : 0);
  L.mlp_m = take(mlp ? kMlpParamCount * 4 : 0);
  L.mlp_v = take(mlp ? kMlpParamCount * 4 : 0);
  L.swap = take(mlp ? B * 8 : 0);
  L.judge = take(mlp ? (2 * B + 13) * 4 : 0);  // two J-bucket histograms (J <= B) and F at the 13 knots
  L.total = o;
  return L;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

template <typename T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<uint8_t*>(base) + off);
}

elsar_status common_checks(uint64_t n, const void* d_ws, size_t ws_bytes, const Layout& L) {
  if (n >= (1ull << 32)) return fail(ELSAR_EUNSUPPORTED, "n must be < 2^32");
  if (!d_ws || !aligned(d_ws, 256)) return fail(ELSAR_EINVAL, "workspace must be non-null and 256-byte aligned");
  if (ws_bytes < L.total) return fail(ELSAR_ENOMEM, "workspace too small: %zu < %zu bytes", ws_bytes, L.total);
  return ELSAR_OK;
}

const uint64_t* splitters_in(const void* d_model, const Resolved& r) {
  if (!d_model) return nullptr;
  return reinterpret_cast<const uint64_t*>(static_cast<const uint8_t*>(d_model) + model_layout(r.S, r.log2B, r.T).splitters);
}

const uint32_t* lut_in(const void* d_model, const Resolved& r) {
  if (!d_model) return nullptr;
  return reinterpret_cast<const uint32_t*>(static_cast<const uint8_t*>(d_model) + model_layout(r.S, r.log2B, r.T).lut);
}

struct FitResult {
  uint32_t nodes = 0, kind = ELSAR_MODEL_RMI, fallback = 0;
  uint32_t judge_J = 0, judge_rmi_max = 0, judge_mlp_max = 0;
  float F_first = 0.0f, F_last = 0.0f;
};

// largest count of a judge histogram (J buckets)
uint32_t max_bucket(const uint32_t* c, uint32_t J) {
  uint32_t mx = 0;
  for (uint32_t j = 0; j < J; ++j) mx = c[j] > mx ? c[j] : mx;
  return mx;
}

elsar_status do_fit(const void* d_records, uint64_t n, const Resolved& r, void* d_model, void* d_ws, const Layout& L,
                    cudaStream_t st, uint32_t* launches, FitResult* res) {
  FitArgs f = {};
  f.records = static_cast<const uint8_t*>(d_records);
  f.km = key_mask(r.key_bytes);
  f.n = n;
  f.S = r.S;
  f.seed = r.seed;
  f.log2B = r.log2B;
  f.T = r.T;
  f.Dmax = r.Dmax;
  f.model = d_model;
  f.model_bytes = model_bytes_for(r.S, r.log2B, r.T);
  f.samp = at<uint64_t>(d_ws, L.samp);
  f.pnode = at<uint32_t>(d_ws, L.pnode);
  f.sums = at<uint64_t>(d_ws, L.sums);
  f.fc = at<uint32_t>(d_ws, L.fc);
  f.ctrl = at<uint32_t>(d_ws, L.ctrl);
  f.sets = at<SetInfo>(d_ws, L.sets);
  f.stream = st;
  f.launches = launches;
  cudaError_t e;
  if (r.kind == ELSAR_MODEL_RADIX) {  // no model to fit: equal-width slices
    if ((e = fit_radix(f)) != cudaSuccess) return cuda_fail(e, "radix");
    res->kind = ELSAR_MODEL_RADIX;
    res->fallback = 0;
    res->nodes = 0;
    return ELSAR_OK;
  }
  const uint64_t* sorted = nullptr;
  e = fit_rmi(f, &sorted);
  if (e != cudaSuccess) return cuda_fail(e, "fit");
  res->kind = ELSAR_MODEL_RMI;
  res->fallback = 0;
  if (r.kind != ELSAR_MODEL_MLP) return ELSAR_OK;
  // ---- the learned network: train, derive its splitters, let the RMI judge it
  const ModelLayout ml = model_layout(r.S, r.log2B, r.T);
  uint8_t* mb = static_cast<uint8_t*>(d_model);
  uint64_t* T = reinterpret_cast<uint64_t*>(mb + ml.mlp_knots);
  float* w = reinterpret_cast<float*>(mb + ml.mlp_w);
  uint64_t* rmi_t = reinterpret_cast<uint64_t*>(mb + ml.splitters);
  uint64_t* mlp_t = reinterpret_cast<uint64_t*>(mb + ml.alt_splitters);
  MlpTrainArgs ta = {};
  ta.sorted = sorted;
  ta.S = r.S;
  ta.ntrain = mlp_ntrain(r.S);
  ta.batch = kMlpBatch;
  ta.steps = kMlpSteps;
  ta.lr = kMlpLr;
  ta.lr_min = kMlpLrMin;
  ta.T = T;
  ta.w = w;
  ta.m = at<float>(d_ws, L.mlp_m);
  ta.v = at<float>(d_ws, L.mlp_v);
  ta.phi = at<float>(d_ws, L.mlp_phi);
  ta.y = at<float>(d_ws, L.mlp_y);
  ta.partial = at<float>(d_ws, L.mlp_partial);
  ta.grid = kMlpGrid;
  ta.stream = st;
  ta.launches = launches;
  if ((e = mlp_train(ta)) != cudaSuccess) return cuda_fail(e, "mlp train");
  // held-out keys (seed + 1) put into J judge buckets: by the RMI's fine bins
  // (floor(q / 2^(log2B - log2J))) and by the network's J-resolution splitters
  // (its fine-bin splitters are computed only if it is kept)
  uint64_t* held = sorted == f.samp ? f.samp + r.S : f.samp;
  uint32_t log2J = 1;
  while (log2J < r.log2B && (64ull << (log2J + 1)) <= r.S) ++log2J;
  const uint32_t J = 1u << log2J;
  uint32_t* hj = at<uint32_t>(d_ws, L.judge);
  if ((e = mlp_splitters(w, T, log2J, mlp_t, st)) != cudaSuccess) return cuda_fail(e, "mlp judge splitters");
  if ((e = sample_keys(f.records, n, r.S, r.seed + 1, f.km, held, st)) != cudaSuccess) return cuda_fail(e, "held-out");
  if ((e = judge_histogram(held, r.S, rmi_t, r.log2B, log2J, hj, st)) != cudaSuccess) return cuda_fail(e, "judge");
  if ((e = judge_histogram(held, r.S, mlp_t, log2J, log2J, hj + J, st)) != cudaSuccess) return cuda_fail(e, "judge");
  // boundary check: F at the smallest and largest sample keys
  float* Fb = reinterpret_cast<float*>(hj + 2 * J);
  if ((e = mlp_eval(w, T, T, 13, Fb, st)) != cudaSuccess) return cuda_fail(e, "mlp eval");
  std::vector<uint32_t> hh((size_t)2 * J + 13);
  e = cudaMemcpyAsync(hh.data(), hj, hh.size() * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "judge readback");
  res->judge_J = J;
  res->judge_rmi_max = max_bucket(hh.data(), J);
  res->judge_mlp_max = max_bucket(hh.data() + J, J);
  float Fk[13];
  std::memcpy(Fk, hh.data() + 2 * J, sizeof Fk);
  res->F_first = Fk[0];
  res->F_last = Fk[12];
  // coarse sanity of the ends (the held-out balance below judges the rest)
  const bool boundary_ok = Fk[0] < 1.0f / 16 && Fk[12] > 1.0f - 1.0f / 16;
  if (!(r.skip & ELSAR_SKIP_BOUNDARY) && !boundary_ok) res->fallback = 1;
  else if (!(r.skip & ELSAR_SKIP_JUDGE) && res->judge_mlp_max > res->judge_rmi_max) res->fallback = 2;
  if (res->fallback == 0) {
    // the network wins: its fine-bin splitters become the active ones, the RMI's are kept as the alternate
    if ((e = mlp_splitters(w, T, r.log2B, mlp_t, st)) != cudaSuccess) return cuda_fail(e, "mlp splitters");
    uint64_t* tmp = at<uint64_t>(d_ws, L.swap);
    const size_t bytes = (size_t)8 << r.log2B;
    cudaMemcpyAsync(tmp, rmi_t, bytes, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(rmi_t, mlp_t, bytes, cudaMemcpyDeviceToDevice, st);
    cudaMemcpyAsync(mlp_t, tmp, bytes, cudaMemcpyDeviceToDevice, st);
    if ((e = build_fine_lut(rmi_t, r.log2B, reinterpret_cast<uint32_t*>(mb + ml.lut), st)) != cudaSuccess)
      return cuda_fail(e, "lut");
    res->kind = ELSAR_MODEL_MLP;
    *launches += 2 + kFineLutLaunches;
  }
  if ((e = set_model_kind(d_model, res->kind, res->fallback, st)) != cudaSuccess) return cuda_fail(e, "header");
  *launches += 7;  // judge splitters (2), held-out sample, two histograms, F at the knots, header
  return ELSAR_OK;
}

// The network's partitions failed the full-data check: restore the RMI's splitters.
elsar_status revert_to_rmi(void* d_model, const Resolved& r, void* d_ws, const Layout& L, cudaStream_t st,
                           uint32_t fallback) {
  const ModelLayout ml = model_layout(r.S, r.log2B, r.T);
  uint8_t* mb = static_cast<uint8_t*>(d_model);
  const size_t bytes = (size_t)8 << r.log2B;
  cudaError_t e = cudaMemcpyAsync(mb + ml.splitters, mb + ml.alt_splitters, bytes, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = build_fine_lut(reinterpret_cast<uint64_t*>(mb + ml.splitters), r.log2B,
                                           reinterpret_cast<uint32_t*>(mb + ml.lut), st);
  if (e == cudaSuccess) e = set_model_kind(d_model, ELSAR_MODEL_RMI, fallback, st);
  if (e != cudaSuccess) return cuda_fail(e, "revert");
  return ELSAR_OK;
}

PartArgs part_args(const void* d_model, const void* d_records, uint64_t n, const Resolved& r, void* d_pairs,
                   uint32_t* d_bin_off, uint64_t* d_part_off, void* d_ws, const Layout& L, cudaStream_t st,
                   uint32_t* launches) {
  PartArgs a = {};
  a.records = static_cast<const uint8_t*>(d_records);
  a.km = key_mask(r.key_bytes);
  a.n = n;
  a.splitters = splitters_in(d_model, r);
  a.lut = lut_in(d_model, r);
  a.log2B = r.log2B;
  a.P = r.P;
  a.balance = r.balance;
  a.tile_pairs = r.cap;
  a.pairs_in_order = at<void>(d_ws, L.pairsA);
  a.pairs = d_pairs;
  a.bin_off = d_bin_off;
  a.part_off = d_part_off;
  a.cuts = at<uint32_t>(d_ws, L.cuts);
  a.cursor = at<uint32_t>(d_ws, L.cursor);
  a.items = at<uint32_t>(d_ws, L.items);
  a.item_flag = at<uint32_t>(d_ws, L.item_flag);
  a.oversize = at<uint32_t>(d_ws, L.oversize);
  a.ctrl = at<uint32_t>(d_ws, L.ctrl);
  a.seg_hist = at<uint32_t>(d_ws, L.seg);
  a.mid = at<void>(d_ws, L.pairsB);
  a.wait_limit = r.wait_limit;
  a.stream = st;
  a.launches = launches;
  return a;
}

elsar_status do_sort_partitions(const void* d_records, uint64_t n, const Resolved& r, void* d_pairs,
                                const uint32_t* d_bin_off, void* d_out, void* d_ws, const Layout& L, cudaStream_t st,
                                uint32_t* launches, cudaEvent_t ev_items) {
  PartArgs a = part_args(nullptr, d_records, n, r, d_pairs, const_cast<uint32_t*>(d_bin_off),
                         at<uint64_t>(d_ws, L.part_off), d_ws, L, st, launches);
  cudaError_t e = build_items(a);
  if (e != cudaSuccess) return cuda_fail(e, "items");
  if (ev_items) cudaEventRecord(ev_items, st);
  SortArgs s = {};
  s.records = static_cast<const uint8_t*>(d_records);
  s.out = static_cast<uint8_t*>(d_out);
  s.n = n;
  s.log2B = r.log2B;
  s.P = r.P;
  s.schedule = r.schedule;
  s.tile_pairs = r.cap;
  s.pairs = static_cast<Pair*>(d_pairs);
  s.temp = at<Pair>(d_ws, L.pairsA);
  s.bin_off = d_bin_off;
  s.items = a.items;
  s.oversize = a.oversize;
  s.cuts = a.cuts;
  s.item_of_bin = a.item_flag;
  s.ctrl = a.ctrl;
  s.stream = st;
  s.launches = launches;
  e = sort_items(s);
  if (e != cudaSuccess) return cuda_fail(e, "sort");
  return ELSAR_OK;
}

// Device-side failures (a bounded wait that gave up) are latched in the
// workspace status word; read it back (synchronises the stream).
// A call that does not read its status word back ORs it into the sticky
// word for elsar_wait (the tag marks the sticky word valid: a fresh
// workspace holds anything).
__global__ void note_status_kernel(uint32_t* ctrl) {
  uint64_t* tag = reinterpret_cast<uint64_t*>(ctrl + kStickyTag);
  if (*tag != kStickyMagic) {
    *tag = kStickyMagic;
    ctrl[kStickyStatus] = ctrl[kStatusWord];
  } else {
    ctrl[kStickyStatus] |= ctrl[kStatusWord];
  }
}

elsar_status device_status(void* d_ws, const Layout& L, cudaStream_t st) {
  uint32_t w = 0;
  cudaError_t e = cudaMemcpyAsync(&w, at<uint32_t>(d_ws, L.ctrl) + kStatusWord, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "status");
  if (w) return fail(ELSAR_ETIMEOUT, "a device-side wait timed out (status word %u)", w);
  return ELSAR_OK;
}

}  // namespace

void elsar::set_last_error(const char* msg) { g_err = msg; }

extern "C" {

void elsar_default_params(elsar_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->num_partitions = 1024;
  p->fine_bins_log2 = 0;
  p->leaf_target = 16;
  p->max_depth = 32;
  p->model_kind = ELSAR_MODEL_RMI;
  p->balance = ELSAR_BALANCE_REFINED;
  p->schedule = ELSAR_SCHED_PERSISTENT;
  p->tile_pairs = 0;
  p->sample_size = 0;
  p->seed = 0x5EEDull;
}

size_t elsar_workspace_size(uint64_t n, const elsar_params* p) {
  Resolved r;
  if (resolve(n, p, &r) != ELSAR_OK) return 0;
  return layout(n, r).total;
}

size_t elsar_model_size(uint64_t n, const elsar_params* p) {
  Resolved r;
  if (resolve(n, p, &r) != ELSAR_OK) return 0;
  return model_bytes_for(r.S, r.log2B, r.T);
}

elsar_status elsar_fit_model(const void* d_records, uint64_t n, const elsar_params* p, void* d_model,
                             size_t model_bytes, void* d_ws, size_t ws_bytes, elsar_stream_t stream) {
  g_err.clear();
  Resolved r;
  elsar_status s = resolve(n, p, &r);
  if (s != ELSAR_OK) return s;
  if (n == 0) return fail(ELSAR_EINVAL, "cannot fit a model on 0 records");
  const Layout L = layout(n, r);
  if ((s = common_checks(n, d_ws, ws_bytes, L)) != ELSAR_OK) return s;
  if (!d_records || !aligned(d_records, 4)) return fail(ELSAR_EINVAL, "records must be non-null and 4-byte aligned");
  if (!d_model || !aligned(d_model, 256)) return fail(ELSAR_EINVAL, "model buffer must be 256-byte aligned");
  if (model_bytes < model_bytes_for(r.S, r.log2B, r.T)) return fail(ELSAR_ENOMEM, "model buffer too small");
  uint32_t launches = 0;
  FitResult fr;
  return do_fit(d_records, n, r, d_model, d_ws, L, (cudaStream_t)stream, &launches, &fr);
}

elsar_status elsar_partition(const void* d_model, const void* d_records, uint64_t n, const elsar_params* p,
                             void* d_pairs, uint32_t* d_bin_offsets, uint64_t* d_part_offsets, void* d_ws,
                             size_t ws_bytes, elsar_stream_t stream) {
  g_err.clear();
  Resolved r;
  elsar_status s = resolve(n, p, &r);
  if (s != ELSAR_OK) return s;
  const Layout L = layout(n, r);
  if ((s = common_checks(n, d_ws, ws_bytes, L)) != ELSAR_OK) return s;
  if (!d_model || !aligned(d_model, 256)) return fail(ELSAR_EINVAL, "model buffer must be 256-byte aligned");
  if ((n && (!d_records || !aligned(d_records, 4))) || (n && (!d_pairs || !aligned(d_pairs, 16))) || !d_bin_offsets ||
      !d_part_offsets)
    return fail(ELSAR_EINVAL, "null or misaligned buffer");
  cudaStream_t st = (cudaStream_t)stream;
  ModelHeader h;
  cudaError_t e = cudaMemcpyAsync(&h, d_model, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "model header");
  if (h.magic != kModelMagic || h.log2B != r.log2B || h.S != r.S || h.T != r.T)
    return fail(ELSAR_EMODEL, "model buffer does not hold a model fitted with these parameters");
  uint32_t launches = 0;
  PartArgs a = part_args(d_model, d_records, n, r, d_pairs, d_bin_offsets, d_part_offsets, d_ws, L, st, &launches);
  e = partition_records(a);
  if (e != cudaSuccess) return cuda_fail(e, "partition");
  return ELSAR_OK;
}

elsar_status elsar_sort_partitions(const void* d_records, uint64_t n, const elsar_params* p, void* d_pairs,
                                   const uint32_t* d_bin_offsets, void* d_out, void* d_ws, size_t ws_bytes,
                                   elsar_stream_t stream) {
  g_err.clear();
  Resolved r;
  elsar_status s = resolve(n, p, &r);
  if (s != ELSAR_OK) return s;
  const Layout L = layout(n, r);
  if ((s = common_checks(n, d_ws, ws_bytes, L)) != ELSAR_OK) return s;
  if (n == 0) return ELSAR_OK;
  if (!d_records || !aligned(d_records, 4) || !d_out || !aligned(d_out, 4) || !d_pairs || !aligned(d_pairs, 16) ||
      !d_bin_offsets)
    return fail(ELSAR_EINVAL, "null or misaligned buffer");
  uint32_t launches = 0;
  return do_sort_partitions(d_records, n, r, d_pairs, d_bin_offsets, d_out, d_ws, L, (cudaStream_t)stream, &launches,
                            nullptr);
}

elsar_status elsar_sort(const void* d_in, void* d_out, uint64_t n, const elsar_params* p, void* d_ws, size_t ws_bytes,
                        elsar_stream_t stream, elsar_stats* stats) {
  g_err.clear();
  Resolved r;
  elsar_status s = resolve(n, p, &r);
  if (s != ELSAR_OK) return s;
  const Layout L = layout(n, r);
  if ((s = common_checks(n, d_ws, ws_bytes, L)) != ELSAR_OK) return s;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (n == 0) return ELSAR_OK;
  if (!d_in || !aligned(d_in, 4) || !d_out || !aligned(d_out, 4)) return fail(ELSAR_EINVAL, "null or misaligned records");
  const uint8_t* i8 = static_cast<const uint8_t*>(d_in);
  const uint8_t* o8 = static_cast<const uint8_t*>(d_out);
  if (i8 < o8 + n * ELSAR_RECORD_BYTES && o8 < i8 + n * ELSAR_RECORD_BYTES)
    return fail(ELSAR_EINVAL, "input and output records overlap");
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t ev[7] = {};
  if (stats)
    for (auto& e : ev) cudaEventCreate(&e);
  if (ev[0]) cudaEventRecord(ev[0], st);
  uint32_t launches = 0;
  FitResult fr;
  void* model = at<void>(d_ws, L.model);
  s = do_fit(d_in, n, r, model, d_ws, L, st, &launches, &fr);
  if (s == ELSAR_OK) {
    if (ev[1]) cudaEventRecord(ev[1], st);
    PartArgs a = part_args(model, d_in, n, r, at<void>(d_ws, L.pairsB), at<uint32_t>(d_ws, L.bin_off),
                           at<uint64_t>(d_ws, L.part_off), d_ws, L, st, &launches);
    // between the scatter passes the pairs wait in the output record buffer
    // (n x 100 bytes, written only by the final gather), 16-byte aligned
    a.mid = reinterpret_cast<void*>((reinterpret_cast<uintptr_t>(d_out) + 15) & ~(uintptr_t)15);
    a.ev[0] = ev[2];
    a.ev[1] = ev[3];
    a.ev[2] = ev[4];
    cudaError_t e = partition_records(a);
    if (e != cudaSuccess) s = cuda_fail(e, "partition");
    if (s == ELSAR_OK && fr.kind == ELSAR_MODEL_MLP && !(r.skip & ELSAR_SKIP_IMBALANCE)) {
      // full-data check of the network's partitions: above 1.1 x the mean, the RMI takes over
      std::vector<uint64_t> off(r.P + 1);
      e = cudaMemcpyAsync(off.data(), at<uint64_t>(d_ws, L.part_off), off.size() * 8, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        s = cuda_fail(e, "partition readback");
      } else {
        uint64_t mx = 0;
        for (uint32_t q = 0; q < r.P; ++q) mx = off[q + 1] - off[q] > mx ? off[q + 1] - off[q] : mx;
        if ((double)mx * r.P > 1.1 * (double)n) {
          fr.kind = ELSAR_MODEL_RMI;
          fr.fallback = 3;
          s = revert_to_rmi(model, r, d_ws, L, st, 3);
          if (s == ELSAR_OK && (e = partition_records(a)) != cudaSuccess) s = cuda_fail(e, "partition");
        }
      }
    }
  }
  if (s == ELSAR_OK)
    s = do_sort_partitions(d_in, n, r, at<void>(d_ws, L.pairsB), at<uint32_t>(d_ws, L.bin_off), d_out, d_ws, L, st,
                           &launches, ev[5]);
  if (s == ELSAR_OK && stats) cudaEventRecord(ev[6], st);
  if (s == ELSAR_OK) {
    if (stats) {
      s = device_status(d_ws, L, st);
    } else {  // no round trip: the status word waits in the sticky word for elsar_wait
      note_status_kernel<<<1, 1, 0, st>>>(at<uint32_t>(d_ws, L.ctrl));
      ++launches;
    }
  }
  if (s == ELSAR_OK && stats) {
    cudaError_t e = cudaEventSynchronize(ev[6]);
    if (e != cudaSuccess) {
      s = cuda_fail(e, "sort");
    } else {
      auto ms = [&](int a, int b) {
        float t = 0;
        cudaEventElapsedTime(&t, ev[a], ev[b]);
        return t;
      };
      stats->pass_ms[0] = ms(0, 1);
      stats->pass_ms[1] = ms(1, 2);
      stats->pass_ms[2] = ms(2, 3) + ms(4, 5);
      stats->pass_ms[3] = ms(3, 4);
      stats->pass_ms[4] = ms(5, 6);
      stats->launches = launches;
      ModelHeader mh = {};
      cudaMemcpy(&mh, model, sizeof mh, cudaMemcpyDeviceToHost);
      stats->model_nodes = mh.num_nodes;
      // the RMI's device loop was counted as one graph launch: count its kernels (six per level)
      if (r.kind != ELSAR_MODEL_RADIX) stats->launches += 6 * mh.levels - 1;
      stats->model_used = fr.kind;
      stats->fallback_reason = fr.fallback;
      stats->judge_buckets = fr.judge_J;
      stats->judge_rmi_max = fr.judge_rmi_max;
      stats->judge_mlp_max = fr.judge_mlp_max;
      stats->F_first_knot = fr.F_first;
      stats->F_last_knot = fr.F_last;
      uint32_t c[4];
      cudaMemcpy(c, at<uint32_t>(d_ws, L.ctrl), sizeof c, cudaMemcpyDeviceToHost);
      stats->num_items = c[kNumItems];
      stats->oversize_items = c[kNumOversize];
      stats->max_bin = c[kMaxBin];
      std::string po((r.P + 1) * 8, '\0');
      cudaMemcpy(&po[0], at<uint64_t>(d_ws, L.part_off), po.size(), cudaMemcpyDeviceToHost);
      const uint64_t* off = reinterpret_cast<const uint64_t*>(po.data());
      for (uint32_t q = 0; q < r.P; ++q)
        if (off[q + 1] - off[q] > stats->max_partition) stats->max_partition = off[q + 1] - off[q];
    }
  }
  if (stats)
    for (auto& e : ev) cudaEventDestroy(e);
  if (s == ELSAR_OK) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_fail(e, "launch");
  }
  return s;
}

elsar_status elsar_sort_host(const void* h_in, void* h_out, uint64_t n, const elsar_params* p, void* d_in,
                             void* d_out, void* d_ws, size_t ws_bytes, elsar_stream_t stream) {
  g_err.clear();
  if (n && (!h_in || !h_out)) return fail(ELSAR_EINVAL, "null host buffer");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = n * ELSAR_RECORD_BYTES;
  cudaError_t e = n ? cudaMemcpyAsync(d_in, h_in, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
  if (e != cudaSuccess) return cuda_fail(e, "copy in");
  elsar_status s = elsar_sort(d_in, d_out, n, p, d_ws, ws_bytes, stream, nullptr);
  if (s != ELSAR_OK) return s;
  if (n && (e = cudaMemcpyAsync(h_out, d_out, bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "copy out");
  return n ? elsar_wait(d_ws, ws_bytes, stream) : ELSAR_OK;  // synchronises
}

elsar_status elsar_sort_host_async(const void* h_in, void* h_out, uint64_t n, const elsar_params* p, void* d_in,
                                   void* d_out, void* d_ws, size_t ws_bytes, elsar_stream_t stream) {
  g_err.clear();
  if (n && (!h_in || !h_out)) return fail(ELSAR_EINVAL, "null host buffer");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = n * ELSAR_RECORD_BYTES;
  cudaError_t e = n ? cudaMemcpyAsync(d_in, h_in, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
  if (e != cudaSuccess) return cuda_fail(e, "copy in");
  elsar_status s = elsar_sort(d_in, d_out, n, p, d_ws, ws_bytes, stream, nullptr);
  if (s != ELSAR_OK) return s;
  if (n && (e = cudaMemcpyAsync(h_out, d_out, bytes, cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(e, "copy out");
  return ELSAR_OK;
}

elsar_status elsar_wait(void* d_ws, size_t ws_bytes, elsar_stream_t stream) {
  g_err.clear();
  if (!d_ws || !aligned(d_ws, 256) || ws_bytes < (kStickyStatus + 1) * 4)
    return fail(ELSAR_EINVAL, "null, misaligned or too small workspace");
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t w[3] = {};
  uint32_t* ctrl = static_cast<uint32_t*>(d_ws);  // the control words open the workspace
  cudaError_t e = cudaMemcpyAsync(w, ctrl + kStickyTag, sizeof w, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "check");
  const uint64_t tag = ((uint64_t)w[1] << 32) | w[0];
  if (tag != kStickyMagic || !w[2]) return ELSAR_OK;
  e = cudaMemsetAsync(ctrl + kStickyStatus, 0, 4, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "check");
  return fail(ELSAR_ETIMEOUT, "a device-side wait timed out in an earlier call (status word %u)", w[2]);
}

// ---------------------------------------------------------------- out of core
namespace {

constexpr uint64_t kOocChunkMin = 8192;
// per chunk record: two input buffers, the pairs, two staging buffers, the stable rank
constexpr size_t kOocChunkBytesPerRecord = 2 * 100 + 16 + 2 * 100 + 2;
// per group record: two input and two output buffers
constexpr size_t kOocGroupBytesPerRecord = 4 * 100;
constexpr size_t kOocSlack = 64ull << 20;

// device address of pinned host memory, or null when the GPU cannot read it
const void* device_view(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

size_t ooc_fixed_bytes(const Resolved& r) {
  return up((size_t)2 << r.log2B) + up((size_t)4 * r.P) + 2 * up((size_t)4 * (r.P + 1)) + 3 * up((size_t)8 * r.P) +
         16 * 256;
}

}  // namespace

extern "C" size_t elsar_ooc_min_workspace(uint64_t n, const elsar_params* p) {
  Resolved r;
  if (resolve(n, p, &r) != ELSAR_OK) return 0;
  return layout(0, r).total + ooc_fixed_bytes(r) + kOocSlack;
}

extern "C" elsar_status elsar_sort_ooc(const void* h_in, void* h_out, uint64_t n, const elsar_params* p, void* d_ws,
                                       size_t ws_bytes, elsar_stream_t stream, elsar_ooc_stats* stats) {
  g_err.clear();
  Resolved r;
  elsar_status s = resolve(n, p, &r);
  if (s != ELSAR_OK) return s;
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (n >= (1ull << 32)) return fail(ELSAR_EUNSUPPORTED, "n must be < 2^32");
  if (n == 0) return ELSAR_OK;
  if (!d_ws || !aligned(d_ws, 256)) return fail(ELSAR_EINVAL, "workspace must be non-null and 256-byte aligned");
  const void* dv_in = h_in ? device_view(h_in) : nullptr;
  uint8_t* dv_out = h_out ? static_cast<uint8_t*>(const_cast<void*>(device_view(h_out))) : nullptr;
  if (!dv_in || !dv_out)
    return fail(ELSAR_EINVAL, "h_in and h_out must be pinned host memory the GPU can read");
  const uint8_t* hi8 = static_cast<const uint8_t*>(h_in);
  uint8_t* ho8 = static_cast<uint8_t*>(h_out);
  if (hi8 < ho8 + n * 100 && ho8 < hi8 + n * 100) return fail(ELSAR_EINVAL, "h_in and h_out overlap");
  if (ws_bytes < elsar_ooc_min_workspace(n, p)) return fail(ELSAR_ENOMEM, "workspace below elsar_ooc_min_workspace");
  cudaStream_t st = (cudaStream_t)stream;
  // the model and its scratch first; the chunk buffers, later the group buffers, after it
  const Layout Lf = layout(0, r);
  uint8_t* rest = static_cast<uint8_t*>(d_ws) + Lf.total;
  const size_t rest_bytes = ws_bytes - Lf.total;

  // side streams for the copies; events order them against the kernels on st
  cudaStream_t up_st = nullptr, down_st = nullptr;
  cudaEvent_t ev_t[5] = {}, in_ready[2] = {}, in_free[2] = {}, out_ready[2] = {}, out_free[2] = {};
  cudaError_t e = cudaStreamCreateWithFlags(&up_st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&down_st, cudaStreamNonBlocking);
  for (auto& ev : ev_t)
    if (e == cudaSuccess) e = cudaEventCreate(&ev);
  for (int i = 0; i < 2; ++i) {
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&in_ready[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&in_free[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&out_ready[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&out_free[i], cudaEventDisableTiming);
  }
  auto cleanup = [&]() {
    if (up_st) cudaStreamSynchronize(up_st);
    if (down_st) cudaStreamSynchronize(down_st);
    for (auto* ev : {&ev_t[0], &ev_t[1], &ev_t[2], &ev_t[3], &ev_t[4], &in_ready[0], &in_ready[1], &in_free[0],
                     &in_free[1], &out_ready[0], &out_ready[1], &out_free[0], &out_free[1]})
      if (*ev) cudaEventDestroy(*ev);
    if (up_st) cudaStreamDestroy(up_st);
    if (down_st) cudaStreamDestroy(down_st);
  };
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "out-of-core setup");
  }
  cudaEventRecord(ev_t[0], st);
  uint64_t h2d = 0, d2h = 0;

  // ---- fit: the sample is read straight from host memory
  uint32_t launches = 0;
  FitResult fr;
  void* model = at<void>(d_ws, Lf.model);
  s = do_fit(dv_in, n, r, model, d_ws, Lf, st, &launches, &fr);
  if (s != ELSAR_OK) {
    cleanup();
    return s;
  }
  cudaEventRecord(ev_t[1], st);

  // ---- chunk buffers
  const size_t fixed = ooc_fixed_bytes(r);
  const size_t per_rec = kOocChunkBytesPerRecord + ((size_t)4 * r.P + 8191) / 8192;
  uint64_t C = rest_bytes > fixed ? (rest_bytes - fixed) / per_rec : 0;
  C = (C / kOocChunkMin) * kOocChunkMin;
  C = std::min<uint64_t>(C, ((n + kOocChunkMin - 1) / kOocChunkMin) * kOocChunkMin);
  C = std::min<uint64_t>(C, 1ull << 30);
  if (C < kOocChunkMin) {
    cleanup();
    return fail(ELSAR_ENOMEM, "device budget too small for a chunk of records");
  }
  size_t o = 0;
  auto carve = [&](size_t bytes) {
    uint8_t* q = rest + o;
    o += up(bytes);
    return q;
  };
  uint8_t* cbuf[2] = {carve(C * 100), carve(C * 100)};
  Pair* cpairs = reinterpret_cast<Pair*>(carve(C * 16));
  uint8_t* stage[2] = {carve(C * 100), carve(C * 100)};
  uint16_t* rank = reinterpret_cast<uint16_t*>(carve(C * 2));
  uint32_t* tile_hist = reinterpret_cast<uint32_t*>(carve(ooc_tiles(C) * r.P * 4));
  uint32_t* pcount = reinterpret_cast<uint32_t*>(carve((size_t)r.P * 4));
  uint32_t* poff_chunk[2] = {reinterpret_cast<uint32_t*>(carve((size_t)(r.P + 1) * 4)),
                             reinterpret_cast<uint32_t*>(carve((size_t)(r.P + 1) * 4))};
  uint16_t* b2p = reinterpret_cast<uint16_t*>(carve((size_t)2 << r.log2B));
  uint64_t* dst_next = reinterpret_cast<uint64_t*>(carve((size_t)8 * r.P));
  uint64_t* dst_cur[2] = {reinterpret_cast<uint64_t*>(carve((size_t)8 * r.P)),
                          reinterpret_cast<uint64_t*>(carve((size_t)8 * r.P))};
  if (o > rest_bytes) {
    cleanup();
    return fail(ELSAR_ENOMEM, "device budget too small for the chunk buffers");
  }
  PartArgs a = part_args(model, nullptr, 0, r, nullptr, at<uint32_t>(d_ws, Lf.bin_off),
                         at<uint64_t>(d_ws, Lf.part_off), d_ws, Lf, st, &launches);
  a.pairs_in_order = cpairs;
  const uint64_t nchunks = (n + C - 1) / C;
  std::vector<uint64_t> part_off(r.P + 1);
  OocSplitArgs sa = {};
  sa.lut = b2p;
  sa.pairs = cpairs;
  sa.P = r.P;
  sa.tile_hist = tile_hist;
  sa.rank = rank;
  sa.part_count = pcount;
  sa.dst_next = dst_next;
  sa.part_end = a.part_off + 1;
  sa.out = dv_out;
  sa.ctrl = a.ctrl;
  auto issue_in = [&](uint64_t c) {
    const int b = (int)(c & 1);
    const uint64_t cn = std::min<uint64_t>(C, n - c * C);
    cudaStreamWaitEvent(up_st, in_free[b], 0);
    cudaMemcpyAsync(cbuf[b], hi8 + c * C * 100, cn * 100, cudaMemcpyHostToDevice, up_st);
    cudaEventRecord(in_ready[b], up_st);
    h2d += cn * 100;
  };
  // pass 1 counts (and runs again if the network's partitions fail the
  // full-data check and the RMI takes over); pass 2 splits and copies out
  int pass = 0;
  while (pass < 2 && s == ELSAR_OK) {
    if (pass == 0) {
      cudaMemsetAsync(a.cursor, 0, (size_t)4 << r.log2B, st);  // the histogram
      cudaMemsetAsync(a.ctrl, 0, 32 * sizeof(uint32_t), st);
    } else {
      cudaMemcpyAsync(dst_next, a.part_off, (size_t)8 * r.P, cudaMemcpyDeviceToDevice, st);
    }
    for (int b = 0; b < 2; ++b) {
      cudaEventRecord(in_free[b], st);
      cudaEventRecord(out_free[b], st);
    }
    issue_in(0);
    for (uint64_t c = 0; c < nchunks && s == ELSAR_OK; ++c) {
      const int b = (int)(c & 1);
      const uint64_t cn = std::min<uint64_t>(C, n - c * C);
      if (c + 1 < nchunks) issue_in(c + 1);
      cudaStreamWaitEvent(st, in_ready[b], 0);
      a.records = cbuf[b];
      a.n = cn;
      if ((e = classify_accumulate(a)) != cudaSuccess) {
        s = cuda_fail(e, "out-of-core classify");
        break;
      }
      if (pass == 1) {
        // stable split by partition into stage[b] (free once its previous
        // copy-out ended), then on the copy stream every piece appended to
        // its partition's range of h_out while the next chunk is split
        sa.chunk = cbuf[b];
        sa.n = cn;
        sa.stage = stage[b];
        sa.chunk_off = poff_chunk[b];
        sa.dst_cur = dst_cur[b];
        cudaStreamWaitEvent(st, out_free[b], 0);
        if ((e = ooc_split_chunk(sa, st)) != cudaSuccess) {
          s = cuda_fail(e, "out-of-core split");
          break;
        }
        cudaEventRecord(out_ready[b], st);
        cudaStreamWaitEvent(down_st, out_ready[b], 0);
        if ((e = ooc_copy_out(sa, down_st)) != cudaSuccess) {
          s = cuda_fail(e, "out-of-core copy-out");
          break;
        }
        cudaEventRecord(out_free[b], down_st);
        launches += 5;
        d2h += cn * 100;
      }
      cudaEventRecord(in_free[b], st);
    }
    if (s != ELSAR_OK) break;
    if (pass == 0) {
      // the exact histogram gives the cuts and the write offsets (Sec. 3.5)
      e = scan_and_cut(a);
      if (e == cudaSuccess) e = cudaMemcpyAsync(part_off.data(), a.part_off, (r.P + 1) * 8, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) {
        s = cuda_fail(e, "out-of-core cuts");
        break;
      }
      if ((s = device_status(d_ws, Lf, st)) != ELSAR_OK) break;  // a classify wait gave up
      uint64_t mx = 0;
      for (uint32_t q = 0; q < r.P; ++q) mx = std::max<uint64_t>(mx, part_off[q + 1] - part_off[q]);
      if (fr.kind == ELSAR_MODEL_MLP && !(r.skip & ELSAR_SKIP_IMBALANCE) && (double)mx * r.P > 1.1 * (double)n) {
        fr.kind = ELSAR_MODEL_RMI;
        fr.fallback = 3;
        s = revert_to_rmi(model, r, d_ws, Lf, st, 3);
        continue;  // count again with the RMI's splitters
      }
      if ((e = ooc_bin_to_part(a.cuts, r.P, 1u << r.log2B, b2p, st)) != cudaSuccess) {
        s = cuda_fail(e, "out-of-core partition map");
        break;
      }
      cudaEventRecord(ev_t[2], st);
    }
    ++pass;
  }
  if (s == ELSAR_OK) {
    e = cudaStreamSynchronize(down_st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(up_st);
    if (e != cudaSuccess) s = cuda_fail(e, "out-of-core copy out");
  }
  if (s == ELSAR_OK) {
    // every partition's range must have been filled exactly
    std::vector<uint64_t> next(r.P);
    e = cudaMemcpyAsync(next.data(), dst_next, (size_t)8 * r.P, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_fail(e, "out-of-core split check");
    for (uint32_t q = 0; q < r.P && s == ELSAR_OK; ++q)
      if (next[q] != part_off[q + 1])
        s = fail(ELSAR_ECUDA, "out-of-core split: partition %u got %llu of %llu records", q,
                 (unsigned long long)(next[q] - part_off[q]), (unsigned long long)(part_off[q + 1] - part_off[q]));
  }
  if (s == ELSAR_OK) s = device_status(d_ws, Lf, st);
  cudaEventRecord(ev_t[3], st);

  // ---- runs of consecutive partitions that fit the budget: in, sorted, back in place
  elsar_params gp;
  if (p) gp = *p;
  else elsar_default_params(&gp);
  gp.model_kind = ELSAR_MODEL_RMI;
  gp.sample_size = 0;
  gp.fine_bins_log2 = 0;
  gp.num_partitions = 0;
  uint64_t G = (rest_bytes / (kOocGroupBytesPerRecord + 64)) & ~63ull;
  while (G > 0 && kOocGroupBytesPerRecord * G + 256 + elsar_workspace_size(G, &gp) > rest_bytes)
    G = (G * 15 / 16) & ~63ull;
  uint64_t maxpart = 0;
  for (uint32_t q = 0; q < r.P; ++q) maxpart = std::max<uint64_t>(maxpart, part_off[q + 1] - part_off[q]);
  if (s == ELSAR_OK && maxpart > G)
    s = fail(ELSAR_EUNSUPPORTED, "a partition of %llu records exceeds the %llu the device budget sorts at once",
             (unsigned long long)maxpart, (unsigned long long)G);
  uint32_t groups = 0;
  if (s == ELSAR_OK) {
    uint8_t* gin[2] = {rest, rest + G * 100};
    uint8_t* gout[2] = {rest + 2 * G * 100, rest + 3 * G * 100};
    uint8_t* gws = rest + up(4 * G * 100);
    const size_t gws_bytes = rest_bytes - up(4 * G * 100);
    std::vector<uint64_t> gb(1, 0);  // group boundaries in records
    for (uint32_t q = 0; q < r.P;) {
      const uint64_t start = part_off[q];
      while (q < r.P && part_off[q + 1] - start <= G) ++q;
      gb.push_back(part_off[q]);
    }
    for (int b = 0; b < 2; ++b) {
      cudaEventRecord(in_free[b], st);
      cudaEventRecord(out_free[b], st);
    }
    auto group_in = [&](size_t g) {
      const int b = (int)(g & 1);
      const uint64_t m = gb[g + 1] - gb[g];
      cudaStreamWaitEvent(up_st, in_free[b], 0);
      cudaMemcpyAsync(gin[b], ho8 + gb[g] * 100, m * 100, cudaMemcpyHostToDevice, up_st);
      cudaEventRecord(in_ready[b], up_st);
      h2d += m * 100;
    };
    const size_t ng = gb.size() - 1;
    group_in(0);
    for (size_t g = 0; g < ng && s == ELSAR_OK; ++g) {
      const int b = (int)(g & 1);
      const uint64_t m = gb[g + 1] - gb[g];
      if (g + 1 < ng) group_in(g + 1);
      cudaStreamWaitEvent(st, in_ready[b], 0);
      cudaStreamWaitEvent(st, out_free[b], 0);
      s = elsar_sort(gin[b], gout[b], m, &gp, gws, gws_bytes, stream, nullptr);
      if (s != ELSAR_OK) break;
      cudaEventRecord(in_free[b], st);
      cudaEventRecord(out_ready[b], st);
      cudaStreamWaitEvent(down_st, out_ready[b], 0);
      cudaMemcpyAsync(ho8 + gb[g] * 100, gout[b], m * 100, cudaMemcpyDeviceToHost, down_st);
      cudaEventRecord(out_free[b], down_st);
      d2h += m * 100;
      ++groups;
    }
    if (s == ELSAR_OK) {
      e = cudaStreamSynchronize(down_st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(up_st);
      if (e != cudaSuccess) s = cuda_fail(e, "out-of-core group copies");
    }
  }
  cudaEventRecord(ev_t[4], st);
  if (s == ELSAR_OK && (e = cudaEventSynchronize(ev_t[4])) != cudaSuccess) s = cuda_fail(e, "out-of-core");
  if (s == ELSAR_OK && stats) {
    for (int i = 0; i < 4; ++i) cudaEventElapsedTime(&stats->phase_ms[i], ev_t[i], ev_t[i + 1]);
    stats->h2d_bytes = h2d;
    stats->d2h_bytes = d2h;
    stats->chunks = (uint32_t)nchunks;
    stats->groups = groups;
    stats->chunk_records = C;
    stats->group_records = G;
    stats->model_used = fr.kind;
    stats->fallback_reason = fr.fallback;
    stats->max_partition = maxpart;
  }
  cleanup();
  return s;
}

size_t elsar_mlp_grad_workspace(uint64_t n) {
  return ((n * 12 * 4 + 255) & ~(size_t)255) + (size_t)kMlpGrid * kMlpParamCount * 4;
}

elsar_status elsar_mlp_eval(const float* d_w, const uint64_t* d_knots, const uint64_t* d_x, uint64_t n, float* d_F,
                            elsar_stream_t stream) {
  g_err.clear();
  if (n >= (1ull << 32)) return fail(ELSAR_EUNSUPPORTED, "n must be < 2^32");
  if (!d_w || !d_knots || (n && (!d_x || !d_F))) return fail(ELSAR_EINVAL, "null buffer");
  if (!n) return ELSAR_OK;
  cudaError_t e = mlp_eval(d_w, d_knots, d_x, n, d_F, (cudaStream_t)stream);
  return e == cudaSuccess ? ELSAR_OK : cuda_fail(e, "mlp eval");
}

elsar_status elsar_mlp_grad(const float* d_w, const uint64_t* d_knots, const uint64_t* d_x, const float* d_y,
                            uint64_t n, float* d_grad, void* d_ws, size_t ws_bytes, elsar_stream_t stream) {
  g_err.clear();
  if (n == 0 || n >= (1ull << 32)) return fail(ELSAR_EINVAL, "n must be in [1, 2^32)");
  if (!d_w || !d_knots || !d_x || !d_y || !d_grad || !d_ws || !aligned(d_ws, 256))
    return fail(ELSAR_EINVAL, "null or misaligned buffer");
  if (ws_bytes < elsar_mlp_grad_workspace(n)) return fail(ELSAR_ENOMEM, "workspace too small");
  float* phi = static_cast<float*>(d_ws);
  float* partial = at<float>(d_ws, (n * 12 * 4 + 255) & ~(size_t)255);
  cudaError_t e = mlp_grad(d_w, d_knots, d_x, d_y, n, phi, partial, kMlpGrid, d_grad, (cudaStream_t)stream);
  return e == cudaSuccess ? ELSAR_OK : cuda_fail(e, "mlp grad");
}

elsar_status elsar_mlp_adam(float* d_w, const float* d_grad, float* d_m, float* d_v, uint32_t t, float lr,
                            elsar_stream_t stream) {
  g_err.clear();
  if (!d_w || !d_grad || !d_m || !d_v) return fail(ELSAR_EINVAL, "null buffer");
  if (t == 0) return fail(ELSAR_EINVAL, "the step number t starts at 1");
  cudaError_t e = mlp_adam_step(d_w, d_grad, d_m, d_v, t, lr, (cudaStream_t)stream);
  return e == cudaSuccess ? ELSAR_OK : cuda_fail(e, "mlp adam");
}

elsar_status elsar_mlp_splitters(const float* d_w, const uint64_t* d_knots, uint32_t log2B, uint64_t* d_t,
                                 elsar_stream_t stream) {
  g_err.clear();
  if (!d_w || !d_knots || !d_t) return fail(ELSAR_EINVAL, "null buffer");
  if (log2B < 1 || log2B > 22) return fail(ELSAR_EINVAL, "log2B must be in [1, 22]");
  cudaError_t e = mlp_splitters(d_w, d_knots, log2B, d_t, (cudaStream_t)stream);
  return e == cudaSuccess ? ELSAR_OK : cuda_fail(e, "mlp splitters");
}

const char* elsar_status_str(elsar_status s) {
  switch (s) {
    case ELSAR_OK: return "ok";
    case ELSAR_EINVAL: return "invalid argument";
    case ELSAR_ENOMEM: return "buffer too small";
    case ELSAR_ECUDA: return "CUDA error";
    case ELSAR_ETIMEOUT: return "device wait timed out";
    case ELSAR_EUNSUPPORTED: return "unsupported size or feature";
    case ELSAR_EMODEL: return "model not fitted";
  }
  return "unknown status";
}

const char* elsar_last_error(void) { return g_err.c_str(); }

}  // extern "C"
