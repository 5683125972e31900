// ELSAR oracle: a plain, slow, single-threaded CPU restatement of the learned
// partition-and-concatenate sort of "Parallel External Sorting of ASCII Records
// Using Learned Models" (arXiv 2305.05671).
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
// bench's CPU-baseline leg may load this library.  It shares no code, header,
// table or constant generator with the CUDA path, and it never reads a value
// produced by it.  Every floating-point step is written out in the order the
// functions below state, compiled with -ffp-contract=off, so nothing is fused
// that is not an explicit std::fma.
//
// What it computes, step by step:
//   encode    Sec. 4: base-95 numerical encoding of the first 9 key bytes
//   sample    Sec. 3.1 / Sec. 6: uniform key sample, 1 % of the input, <= 10M
//   rmi_fit   Sec. 3.1: RMI of linear regressions on the sorted sample, dense
//             regions getting more nodes (leaf clamping keeps it monotone)
//   classify  Sec. 3.3 / Algorithm 1 (the reader loop): p = F_X(encode(x))
//   offsets   Sec. 3.5: write offset = sum of the sizes of earlier partitions
//   sort      Sec. 3.4 / Sec. 4 touch-up: each partition in key byte order
//             (memcmp), ties kept in input order
//   concat    Sec. 3.5: partitions written back to back, no merge
// Beside the method: the radix classifier the paper compares it with (Sec. 3,
// Sec. 3.3), the method with any given classifier (splitters), the choice
// between the learned network and the RMI, and the paper's multi-threaded
// CPU form (Sec. 5) for timing on all host cores.
// Readings of places the paper leaves open are listed beside each function.
//
// Parity of this oracle is pinned by tests/test_oracle_*.py (closed forms,
// brute force, invariants, library least squares); see those files.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

constexpr int kRecord = 100;
constexpr int kKey = 10;

typedef unsigned __int128 u128;
typedef __int128 i128;

// ---------------------------------------------------------------- Sec. 4
// Character c at 1-based position i of an l-character key contributes
// (ASCII(c) - 32) * 95^(l-i); with a 64-bit integer l = 9 (the paper's
// log2 figure of 59.14 bits).  Printable ASCII is 32..126, which is what
// base 95 needs.  The paper leaves other bytes out; reading taken here so that
// the encoding stays monotone in byte order (Eq. 1) for any byte string: at
// the first byte below 32 (above 126) that digit and every later digit become
// 0 (94) -- the key encodes as the smallest (largest) printable key with its
// printable prefix.  The tenth key byte is left to the sort.
uint64_t encode9(const uint8_t* key) {
  uint64_t e = 0;
  int sat = 0;  // 0: none yet, 1: saturate low, 2: saturate high
  for (int i = 0; i < 9; ++i) {
    int c = key[i];
    if (sat == 0 && c < 32) sat = 1;
    if (sat == 0 && c > 126) sat = 2;
    int d = sat == 1 ? 0 : (sat == 2 ? 94 : c - 32);
    e = e * 95u + (uint64_t)d;
  }
  return e;
}

// Variable-length keys (Sec. 4): keys of up to l characters, l the longest,
// with ASCII = 0 at every position past a key's end.  Here the key is the
// first g_key_bytes (l <= 10) bytes of each record; the bytes after them (and,
// in a NUL-padded key field, the NULs past a shorter key's end) count as 0.
// Reading of the padding rule: a 0 byte is below every printable character,
// so by the saturation rule above it and every later digit encode as 0 -- a
// shorter key sorts before every longer key it is a prefix of, as strncmp
// orders NUL-terminated strings -- and byte order compares the padded keys.
int g_key_bytes = 10;

inline void key_of(const uint8_t* rec, uint8_t* k) {
  for (int i = 0; i < kKey; ++i) k[i] = i < g_key_bytes ? rec[i] : 0;
}

inline uint64_t encode_rec(const uint8_t* rec) {
  uint8_t k[kKey];
  key_of(rec, k);
  return encode9(k);
}

// The k-th output of the SplitMix64 generator seeded with `seed`
// (state advances by the golden gamma; Steele, Lea, Flood 2014).
uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ---------------------------------------------------------------- Sec. 3.1
// RMI CDF model.  The paper names the architecture -- starting from the root,
// a key walks through internal linear models, each picking a more specialised
// model below it, until a leaf outputs y ~ P(X <= x) -- says that training
// gives dense regions of the key domain more nodes (so that the leaves act as
// equi-depth bins), and defers the details to the RMI literature.  Readings
// taken here (an adaptive-depth RMI; all numbers are of the sorted sample):
//  * A node covers sample ranks [s, e), n = e - s points.  It is a leaf if
//    n <= 2T, if its points are all equal, if it is at depth Dmax, or if its
//    own router would send its first and last point to the same child.
//    Otherwise it is internal with f = ceil(n / T) children -- unless the
//    children of its whole level would take the tree past 4*ceil(S/T) + 1024
//    nodes, in which case every node of that level is a leaf.
//  * Every node fits ordinary least squares of local rank r = k - s on local
//    coordinate u = (x - base) >> shift, base = its smallest sample, shift =
//    the fewest bits that bring its span under 2^32.  The sums are formed
//    exactly in integers (so no summation order matters); then
//      gamma = max(0, (n*Sur - Su*Sr) / (n*Suu - Su^2))   [each side rounded once]
//      delta = (Sr - gamma*Su) / n.
//  * An internal node routes x to child c = clamp(floor(fma(gamma,u,delta) * f/n), 0, f-1);
//    child c covers the ranks of the points routed to it (contiguous, since
//    the router is monotone).  Children are numbered breadth first.
//  * A leaf outputs F(x) = clamp(fma(gamma/S, u, (s + delta)/S), s/S, e/S):
//    with non-negative slopes and monotone routing this makes F monotone,
//    which concatenation needs (Eq. 1) and an unclamped RMI does not guarantee.
//    Keys below a node's base get u = 0.
struct Node {
  uint64_t s = 0, e = 0, base = 0;
  uint32_t shift = 0, fanout = 0;  // fanout 0: leaf
  uint64_t child0 = 0;
  uint32_t depth = 0;
  double gamma = 0, delta = 0, scale = 0;  // scale = f / n (internal)
  double g = 0, d = 0, lo = 0, hi = 0;     // leaf output constants
};

struct Rmi {
  uint64_t S = 0;
  std::vector<Node> node;
};

inline double pos_or_zero(double v) { return v > 0.0 ? v : 0.0; }

inline uint64_t local_u(const Node& v, uint64_t x) { return x > v.base ? (x - v.base) >> v.shift : 0; }

inline uint32_t route(const Node& v, uint64_t x) {
  double t = std::fma(v.gamma, (double)local_u(v, x), v.delta) * v.scale;
  if (!(t > 0.0)) return 0;
  if (t >= (double)v.fanout) return v.fanout - 1;
  return (uint32_t)t;
}

// exact least squares of local rank on local coordinate over sorted x[s, e)
void fit_linear(const uint64_t* x, Node& v) {
  uint64_t n = v.e - v.s;
  v.base = x[v.s];
  uint64_t span = x[v.e - 1] - v.base;
  uint32_t bits = 0;
  while (bits < 64 && (span >> bits) != 0) ++bits;
  v.shift = bits > 32 ? bits - 32 : 0;
  u128 Su = 0, Suu = 0, Sur = 0;
  for (uint64_t k = v.s; k < v.e; ++k) {
    u128 u = (x[k] - v.base) >> v.shift;
    Su += u;
    Suu += u * u;
    Sur += u * (u128)(k - v.s);
  }
  i128 nn = (i128)n;
  i128 Sr = nn * (nn - 1) / 2;
  i128 Duu = nn * (i128)Suu - (i128)Su * (i128)Su;
  i128 Dur = nn * (i128)Sur - (i128)Su * Sr;
  v.gamma = (n >= 2 && Duu > 0) ? pos_or_zero((double)Dur / (double)Duu) : 0.0;
  v.delta = ((double)Sr - v.gamma * (double)Su) / (double)n;
}

void make_leaf(Node& v, uint64_t S) {
  v.fanout = 0;
  v.scale = 0.0;
  v.lo = (double)v.s / (double)S;
  v.hi = (double)v.e / (double)S;
  if (v.e == v.s) {
    v.base = 0;
    v.shift = 0;
    v.gamma = 0.0;
    v.delta = 0.0;
    v.g = 0.0;
    v.d = v.lo;
    return;
  }
  v.g = v.gamma / (double)S;
  v.d = ((double)v.s + v.delta) / (double)S;
}

// Node budget: a level's nodes split only if the tree then still has at most
// 4*ceil(S/T) + 1024 nodes; otherwise every node of that level is a leaf.
uint64_t node_budget(uint64_t S, uint32_t T) { return 4 * ((S + T - 1) / T) + 1024; }

Rmi rmi_fit(const uint64_t* x, uint64_t S, uint32_t T, uint32_t Dmax) {
  Rmi m;
  m.S = S;
  Node root;
  root.s = 0;
  root.e = S;
  m.node.push_back(root);
  size_t lv0 = 0, lv1 = 1;  // nodes of the current level, numbered breadth first
  while (lv0 < lv1) {
    std::vector<bool> split(lv1 - lv0, false);
    uint64_t children = 0;
    for (size_t i = lv0; i < lv1; ++i) {
      Node& v = m.node[i];
      uint64_t n = v.e - v.s;
      if (n == 0) continue;
      fit_linear(x, v);
      bool sp = n > 2ull * T && v.depth < Dmax && x[v.s] < x[v.e - 1];
      if (sp) {
        v.fanout = (uint32_t)((n + T - 1) / T);
        v.scale = (double)v.fanout / (double)n;
        if (route(v, x[v.s]) == route(v, x[v.e - 1])) sp = false;
        if (!sp) v.fanout = 0;
      }
      split[i - lv0] = sp;
      if (sp) children += v.fanout;
    }
    const bool room = m.node.size() + children <= node_budget(S, T);
    for (size_t i = lv0; i < lv1; ++i) {
      if (!(room && split[i - lv0])) {
        make_leaf(m.node[i], S);
        continue;
      }
      Node v = m.node[i];
      v.child0 = m.node.size();
      std::vector<uint64_t> cs(v.fanout + 1, v.e);
      uint64_t k = v.s;
      for (uint32_t c = 0; c < v.fanout; ++c) {
        while (k < v.e && route(v, x[k]) < c) ++k;
        cs[c] = k;
      }
      m.node[i] = v;
      for (uint32_t c = 0; c < v.fanout; ++c) {
        Node ch;
        ch.s = cs[c];
        ch.e = cs[c + 1];
        ch.depth = v.depth + 1;
        m.node.push_back(ch);
      }
    }
    lv0 = lv1;
    lv1 = m.node.size();
  }
  return m;
}

uint64_t find_leaf(const Rmi& m, uint64_t x) {
  uint64_t i = 0;
  while (m.node[i].fanout) i = m.node[i].child0 + route(m.node[i], x);
  return i;
}

double rmi_cdf(const Rmi& m, uint64_t x) {
  const Node& v = m.node[find_leaf(m, x)];
  double y = std::fma(v.g, (double)local_u(v, x), v.d);
  if (y < v.lo) return v.lo;
  if (y > v.hi) return v.hi;
  return y;
}

// ---------------------------------------------------------------- Sec. 3.3
// Fine bin q = min(B-1, floor(B * F)).  Paper rule (Algorithm 1, reader loop):
// partition p = min(P-1, floor(P * F)), i.e. q / (B/P) for powers of two.
// Refined rule (an addition of this library, not the paper's): the cut c_p of
// partition p is the fine-bin boundary t whose exact cumulative count C(t) is
// closest to p*N/P (ties to the smaller t); partition p = bins [c_p, c_{p+1}).
inline uint32_t fine_bin(double F, uint32_t log2B) {
  uint32_t B = 1u << log2B;
  uint32_t q = (uint32_t)(F * (double)B);
  return q < B ? q : B - 1;
}

std::vector<uint32_t> cuts_of(const std::vector<uint64_t>& counts, uint32_t P, uint32_t log2B, uint64_t N,
                              int balance) {
  uint32_t B = 1u << log2B;
  std::vector<uint32_t> c(P + 1);
  c[0] = 0;
  c[P] = B;
  if (!balance) {
    for (uint32_t p = 1; p < P; ++p) c[p] = p * (B / P);
    return c;
  }
  std::vector<uint64_t> C(B + 1, 0);
  for (uint32_t t = 0; t < B; ++t) C[t + 1] = C[t] + counts[t];
  for (uint32_t p = 1; p < P; ++p) {
    int64_t target = (int64_t)p * (int64_t)N;
    uint32_t best = 0;
    int64_t bestd = -1;
    for (uint32_t t = 0; t <= B; ++t) {
      int64_t d = (int64_t)P * (int64_t)C[t] - target;
      if (d < 0) d = -d;
      if (bestd < 0 || d < bestd) {
        bestd = d;
        best = t;
      }
    }
    c[p] = best;
  }
  return c;
}

inline uint32_t pid_of(const std::vector<uint32_t>& c, uint32_t P, uint32_t q) {
  uint32_t p = 0;
  for (uint32_t k = 1; k < P; ++k)
    if (c[k] <= q) ++p;
  return p;
}

bool key_less(const uint8_t* recs, uint64_t a, uint64_t b) {
  uint8_t ka[kKey], kb[kKey];
  key_of(recs + a * kRecord, ka);
  key_of(recs + b * kRecord, kb);
  return std::memcmp(ka, kb, kKey) < 0;
}

void stable_sort_indices(const uint8_t* recs, std::vector<uint64_t>& idx) {
  std::stable_sort(idx.begin(), idx.end(), [recs](uint64_t a, uint64_t b) { return key_less(recs, a, b); });
}

// Sec. 3.3 - 3.5 given the fine bin q of every record: cuts, partition lists
// in input order, a stable sort of each by memcmp, concatenation.  Optional
// outputs as eo_sort's.
void partition_sort_concat(const uint8_t* in, uint64_t n, const std::vector<uint32_t>& q,
                           const std::vector<uint64_t>& counts, uint32_t P, uint32_t log2B, int balance, uint8_t* out,
                           uint32_t* q_out, uint32_t* pid_out, uint64_t* part_off, uint64_t* bin_counts,
                           uint32_t* cuts_out) {
  const uint32_t B = 1u << log2B;
  std::vector<uint32_t> c = cuts_of(counts, P, log2B, n, balance);
  std::vector<uint32_t> pid_of_bin(B);
  for (uint32_t t = 0; t < B; ++t) pid_of_bin[t] = pid_of(c, P, t);
  std::vector<std::vector<uint64_t>> part(P);
  for (uint64_t i = 0; i < n; ++i) part[pid_of_bin[q[i]]].push_back(i);
  uint64_t off = 0;
  for (uint32_t p = 0; p < P; ++p) {
    if (part_off) part_off[p] = off;
    stable_sort_indices(in, part[p]);
    for (uint64_t i : part[p]) {
      if (out) std::memcpy(out + off * kRecord, in + i * kRecord, kRecord);
      ++off;
    }
  }
  if (part_off) part_off[P] = off;
  for (uint64_t i = 0; i < n; ++i) {
    if (q_out) q_out[i] = q[i];
    if (pid_out) pid_out[i] = pid_of_bin[q[i]];
  }
  if (bin_counts)
    for (uint32_t t = 0; t < B; ++t) bin_counts[t] = counts[t];
  if (cuts_out)
    for (uint32_t p = 0; p <= P; ++p) cuts_out[p] = c[p];
}

// fine bin by splitters t[0..B): the number of q >= 1 with t[q] <= x
inline uint32_t bin_by_splitters(const uint64_t* t, uint32_t B, uint64_t x) {
  return (uint32_t)(std::upper_bound(t + 1, t + B, x) - (t + 1));
}

uint64_t parse_index(const uint8_t* rec, bool* ok) {
  uint64_t v = 0;
  *ok = true;
  for (int j = 0; j < 32; ++j) {
    int c = rec[kKey + j];
    int d;
    if (c >= '0' && c <= '9') d = c - '0';
    else if (c >= 'A' && c <= 'F') d = c - 'A' + 10;
    else { *ok = false; return 0; }
    if (j < 16) { if (d) *ok = false; continue; }
    v = (v << 4) | (uint64_t)d;
  }
  return v;
}

}  // namespace

extern "C" {

uint64_t eo_encode9(const uint8_t* key) { return encode9(key); }

// Key length l (1..10) of every later call: the key is a record's first l
// bytes, padded with 0 bytes (Sec. 4's variable-length keys).  Returns l, or
// 0 if l is out of range (the setting is then unchanged).
int eo_set_key_bytes(int l) {
  if (l < 1 || l > kKey) return 0;
  g_key_bytes = l;
  return l;
}

void eo_encode9_records(const uint8_t* recs, uint64_t n, uint64_t* out) {
  for (uint64_t i = 0; i < n; ++i) out[i] = encode_rec(recs + i * kRecord);
}

uint64_t eo_splitmix64_at(uint64_t seed, uint64_t k) { return splitmix64_at(seed, k); }

// Sec. 3.1 / Sec. 6: 1 % of the input, at least 1000 keys, at most 10M.
// Reading: drawn uniformly over the whole input (not only the first batch of
// one reader thread), with replacement: position k is mulhi64(SplitMix64_k(seed), n).
uint64_t eo_default_sample_size(uint64_t n) {
  if (n == 0) return 0;
  uint64_t s = (n + 99) / 100;
  if (s < 1000) s = 1000;
  if (s > 10000000) s = 10000000;
  return s;
}

void eo_sample(const uint8_t* recs, uint64_t n, uint64_t S, uint64_t seed, uint64_t* out_enc) {
  for (uint64_t k = 0; k < S; ++k) {
    uint64_t i = (uint64_t)(((u128)splitmix64_at(seed, k) * (u128)n) >> 64);
    out_enc[k] = encode_rec(recs + i * kRecord);
  }
}

// Fit on a sorted sample.  Returns the node count, or 0 on bad input.
// The fitted model stays in a small handle table for export and evaluation.
static std::vector<Rmi> g_models;

uint64_t eo_rmi_fit(const uint64_t* sorted, uint64_t S, uint32_t T, uint32_t Dmax, int* handle) {
  if (T < 1 || S >= (1ull << 24)) return 0;
  for (uint64_t k = 1; k < S; ++k)
    if (sorted[k - 1] > sorted[k]) return 0;
  g_models.push_back(rmi_fit(sorted, S, T, Dmax));
  *handle = (int)g_models.size() - 1;
  return g_models.back().node.size();
}

// Node arrays: u64[4] {s, e, base, child0}; u32[3] {shift, fanout, depth};
// f64[7] {gamma, delta, scale, g, d, lo, hi}.
void eo_rmi_export(int handle, uint64_t* nu64, uint32_t* nu32, double* nf64) {
  const Rmi& m = g_models[handle];
  for (size_t i = 0; i < m.node.size(); ++i) {
    const Node& v = m.node[i];
    nu64[4 * i + 0] = v.s;
    nu64[4 * i + 1] = v.e;
    nu64[4 * i + 2] = v.base;
    nu64[4 * i + 3] = v.child0;
    nu32[3 * i + 0] = v.shift;
    nu32[3 * i + 1] = v.fanout;
    nu32[3 * i + 2] = v.depth;
    double f[7] = {v.gamma, v.delta, v.scale, v.g, v.d, v.lo, v.hi};
    for (int t = 0; t < 7; ++t) nf64[7 * i + t] = f[t];
  }
}

void eo_rmi_eval(int handle, const uint64_t* xs, uint64_t m, double* F, uint64_t* leaf) {
  const Rmi& r = g_models[handle];
  for (uint64_t i = 0; i < m; ++i) {
    if (F) F[i] = rmi_cdf(r, xs[i]);
    if (leaf) leaf[i] = find_leaf(r, xs[i]);
  }
}

void eo_rmi_release(void) { g_models.clear(); }

// The whole method (Algorithm 1 without its files):
//   sample -> sort sample -> fit -> per record q, pid -> partition lists in
//   input order -> stable sort each by memcmp -> concatenate.
// Optional outputs (nullable): q[n], pid[n], part_off[P+1], bin_counts[B], cuts[P+1].
int eo_sort(const uint8_t* in, uint64_t n, uint32_t P, uint32_t log2B, uint32_t T, uint32_t Dmax, uint64_t S,
            uint64_t seed, int balance, uint8_t* out, uint32_t* q_out, uint32_t* pid_out, uint64_t* part_off, uint64_t* bin_counts,
            uint32_t* cuts_out) {
  if (P < 1 || (P & (P - 1)) || log2B > 24 || (1u << log2B) < P || T < 1) return 1;
  if (S >= (1ull << 24) || (n > 0 && S == 0)) return 1;  // exact sums need S < 2^24
  if (n == 0) {
    if (part_off)
      for (uint32_t p = 0; p <= P; ++p) part_off[p] = 0;
    return 0;
  }
  std::vector<uint64_t> sample(S);
  eo_sample(in, n, S, seed, sample.data());
  std::sort(sample.begin(), sample.end());
  Rmi m = rmi_fit(sample.data(), S, T, Dmax);
  uint32_t B = 1u << log2B;
  std::vector<uint32_t> q(n);
  std::vector<uint64_t> counts(B, 0);
  for (uint64_t i = 0; i < n; ++i) {
    q[i] = fine_bin(rmi_cdf(m, encode_rec(in + i * kRecord)), log2B);
    counts[q[i]]++;
  }
  partition_sort_concat(in, n, q, counts, P, log2B, balance, out, q_out, pid_out, part_off, bin_counts, cuts_out);
  return 0;
}

// Partition step alone (for full-size checks): fine-bin counts and partition
// offsets of all n records, without sorting.
int eo_classify(const uint8_t* in, uint64_t n, uint32_t P, uint32_t log2B, uint32_t T, uint32_t Dmax, uint64_t S,
                uint64_t seed, int balance, uint64_t* bin_counts, uint64_t* part_off) {
  if (P < 1 || (P & (P - 1)) || log2B > 24 || (1u << log2B) < P || T < 1) return 1;
  if (S >= (1ull << 24) || n == 0 || S == 0) return 1;
  std::vector<uint64_t> sample(S);
  eo_sample(in, n, S, seed, sample.data());
  std::sort(sample.begin(), sample.end());
  Rmi m = rmi_fit(sample.data(), S, T, Dmax);
  uint32_t B = 1u << log2B;
  std::vector<uint64_t> counts(B, 0);
  for (uint64_t i = 0; i < n; ++i) counts[fine_bin(rmi_cdf(m, encode_rec(in + i * kRecord)), log2B)]++;
  std::vector<uint32_t> c = cuts_of(counts, P, log2B, n, balance);
  std::vector<uint64_t> C(B + 1, 0);
  for (uint32_t t = 0; t < B; ++t) C[t + 1] = C[t] + counts[t];
  for (uint32_t p = 0; p <= P; ++p) part_off[p] = C[c[p]];
  for (uint32_t t = 0; t < B; ++t) bin_counts[t] = counts[t];
  return 0;
}

// The plain definition of the result: all records stably sorted by memcmp on
// the 10-byte key (Sec. 7.1 methodology: byte order as memcmp/strncmp).
void eo_stable_sort(const uint8_t* in, uint64_t n, uint8_t* out) {
  std::vector<uint64_t> idx(n);
  for (uint64_t i = 0; i < n; ++i) idx[i] = i;
  stable_sort_indices(in, idx);
  for (uint64_t k = 0; k < n; ++k) std::memcpy(out + k * kRecord, in + idx[k] * kRecord, kRecord);
}

// valsort analogue (Sec. 7.1): returns 0 if `out` is a sorted, stable
// permutation of `in`, else a bit mask: 1 unsorted, 2 not a permutation
// (unparsable/duplicate/out-of-range index, or bytes differ from in[index]),
// 4 equal keys out of input order.  Records carry their input index in hex.
int eo_validate(const uint8_t* in, const uint8_t* out, uint64_t n) {
  int bad = 0;
  std::vector<uint8_t> seen(n, 0);
  uint64_t prev_idx = 0;
  for (uint64_t k = 0; k < n; ++k) {
    const uint8_t* r = out + k * kRecord;
    bool ok;
    uint64_t idx = parse_index(r, &ok);
    if (!ok || idx >= n || seen[idx] || std::memcmp(r, in + idx * kRecord, kRecord) != 0) {
      bad |= 2;
    } else {
      seen[idx] = 1;
    }
    if (k > 0) {
      uint8_t ka[kKey], kb[kKey];
      key_of(out + (k - 1) * kRecord, ka);
      key_of(r, kb);
      int c = std::memcmp(ka, kb, kKey);
      if (c > 0) bad |= 1;
      if (c == 0 && ok && idx < prev_idx) bad |= 4;
    }
    prev_idx = idx;
  }
  return bad;
}

// ---------------------------------------------------------------- radix partitioning (Sec. 3, Sec. 3.3)
// The paper compares its model-based partitions with radix-based ones, which
// give every partition an equal range of the key domain whatever the data
// (sensitive to skew).  Reading taken here: equal-width ranges of the
// printable key domain, i.e. fine bin q = floor(x * B / 95^9) of the key
// encoding x -- the most significant base-95 digits when B is a power of 95,
// equal slices of the same domain for B a power of two.  Exact in 128 bits.
// Its splitters (the smallest encoding of bin >= q) are ceil(q * 95^9 / B).
void eo_radix_bins(const uint64_t* xs, uint64_t n, uint32_t log2B, uint32_t* q) {
  const u128 top = (u128)630249409724609375ull;  // 95^9
  for (uint64_t i = 0; i < n; ++i) q[i] = (uint32_t)(((u128)xs[i] << log2B) / top);
}

void eo_radix_splitters(uint32_t log2B, uint64_t* t) {
  const u128 top = (u128)630249409724609375ull;
  const uint64_t B = 1ull << log2B;
  for (uint64_t q = 0; q < B; ++q) t[q] = (uint64_t)(((u128)q * top + (B - 1)) >> log2B);
}

// Sec. 3.3 - 3.5 with a given classifier: the fine bin of record i is the
// number of splitters t[1..B) at or below its key encoding (t non-decreasing,
// t[0] = 0); then counts, cuts (paper or refined rule), partitions stably
// sorted and concatenated.  `out` may be null (classification only).
int eo_sort_by_splitters(const uint8_t* in, uint64_t n, const uint64_t* t, uint32_t log2B, uint32_t P, int balance,
                         uint8_t* out, uint32_t* q_out, uint32_t* pid_out, uint64_t* part_off, uint64_t* bin_counts,
                         uint32_t* cuts_out) {
  if (P < 1 || (P & (P - 1)) || log2B > 24 || (1u << log2B) < P) return 1;
  const uint32_t B = 1u << log2B;
  for (uint32_t k = 1; k < B; ++k)
    if (t[k] < t[k - 1]) return 1;
  std::vector<uint32_t> q(n);
  std::vector<uint64_t> counts(B, 0);
  for (uint64_t i = 0; i < n; ++i) {
    q[i] = bin_by_splitters(t, B, encode_rec(in + i * kRecord));
    counts[q[i]]++;
  }
  partition_sort_concat(in, n, q, counts, P, log2B, balance, out, q_out, pid_out, part_off, bin_counts, cuts_out);
  return 0;
}

// ---------------------------------------------------------------- the model choice
// The learned network is an addition of this project (the paper's model is
// the RMI); the RMI stays its fallback and judges it.  Given the network's
// weights w (1505 FP32, layout of mlp_oracle.cpp), the rule is:
//   knots   from the sorted sample (seed), as the network was trained on it;
//   check 1 (boundary)  F(T_0) < 1/16 and F(T_12) > 15/16 in FP32, else reason 1;
//   check 2 (judge)     a held-out sample (seed + 1, S keys) put into J judge
//                       buckets (log2J the largest value <= log2B, at least 1,
//                       with 64 * 2^log2J <= S): by the RMI, bucket
//                       floor(fine bin / 2^(log2B - log2J)); by the network, the
//                       number of its J-resolution splitters (those of
//                       min(J-1, floor(J F)), made non-decreasing) at or below
//                       the key.  The network's largest bucket may not hold
//                       more keys than the RMI's, else reason 2;
//   check 3 (full data) the network's partitions of all n records (its
//                       splitters, the configured cut rule): the largest may
//                       not exceed 1.1 times the mean, else reason 3.
// skip bit k-1 skips check k.  Returns the reason (0 = the network is used),
// or -1 on bad input.  diag (nullable, 6 doubles): largest RMI bucket,
// largest network bucket, J, F(T_0), F(T_12), largest network partition
// (0 when check 3 did not run).
extern "C" void eo_mlp_knots(const uint64_t* sorted, uint64_t S, uint64_t* T);
extern "C" void eo_mlp_features(const uint64_t* T, const uint64_t* xs, uint64_t n, float* phi);
extern "C" void eo_mlp_forward32(const float* w, const float* phi, uint64_t n, float* F);
extern "C" void eo_mlp_splitters(const float* w, const uint64_t* T, uint32_t log2B, uint64_t* t);

int eo_model_choice(const uint8_t* in, uint64_t n, uint32_t P, uint32_t log2B, uint32_t T, uint32_t Dmax, uint64_t S,
                    uint64_t seed, int balance, const float* w, uint32_t skip, double* diag) {
  if (n == 0 || S == 0 || S >= (1ull << 24) || log2B < 1 || log2B > 22 || (1u << log2B) < P || P < 1 ||
      (P & (P - 1)) || T < 1)
    return -1;
  const uint32_t B = 1u << log2B;
  std::vector<uint64_t> sample(S), held(S);
  eo_sample(in, n, S, seed, sample.data());
  std::sort(sample.begin(), sample.end());
  Rmi m = rmi_fit(sample.data(), S, T, Dmax);
  uint64_t knots[13];
  eo_mlp_knots(sample.data(), S, knots);
  std::vector<uint64_t> t(B);
  // check 1: F at the first and last knot
  float phi[2 * 12], Fk[2];
  const uint64_t ends[2] = {knots[0], knots[12]};
  eo_mlp_features(knots, ends, 2, phi);
  eo_mlp_forward32(w, phi, 2, Fk);
  // check 2: the held-out judge
  uint32_t log2J = 1;
  while (log2J < log2B && (64ull << (log2J + 1)) <= S) ++log2J;
  const uint32_t J = 1u << log2J;
  eo_sample(in, n, S, seed + 1, held.data());
  std::vector<uint64_t> tJ(J);
  eo_mlp_splitters(w, knots, log2J, tJ.data());
  std::vector<uint64_t> hr(J, 0), hm(J, 0);
  for (uint64_t k = 0; k < S; ++k) {
    hr[fine_bin(rmi_cdf(m, held[k]), log2B) >> (log2B - log2J)]++;
    hm[bin_by_splitters(tJ.data(), J, held[k])]++;
  }
  const uint64_t mr = *std::max_element(hr.begin(), hr.end()), mm = *std::max_element(hm.begin(), hm.end());
  int reason = 0;
  if (!(skip & 1) && !(Fk[0] < 1.0f / 16 && Fk[1] > 1.0f - 1.0f / 16)) reason = 1;
  else if (!(skip & 2) && mm > mr) reason = 2;
  uint64_t maxpart = 0;
  if (reason == 0 && !(skip & 4)) {
    eo_mlp_splitters(w, knots, log2B, t.data());
    std::vector<uint64_t> off(P + 1);
    eo_sort_by_splitters(in, n, t.data(), log2B, P, balance, nullptr, nullptr, nullptr, off.data(), nullptr, nullptr);
    for (uint32_t p = 0; p < P; ++p) maxpart = std::max<uint64_t>(maxpart, off[p + 1] - off[p]);
    if ((double)maxpart * P > 1.1 * (double)n) reason = 3;
  }
  if (diag) {
    diag[0] = (double)mr;
    diag[1] = (double)mm;
    diag[2] = (double)J;
    diag[3] = Fk[0];
    diag[4] = Fk[1];
    diag[5] = (double)maxpart;
  }
  return reason;
}

// ---------------------------------------------------------------- the paper's CPU design, threaded
// eo_sort with the work spread over `threads` host threads the way the paper's
// CPU implementation spreads it (Sec. 5): the records are classified in
// contiguous ranges by all threads, and the partitions are sorted in parallel,
// each thread taking the next unsorted partition (dynamic scheduling).  The
// result is eo_sort's exactly: the classification and cuts are the same
// function, the partition lists keep input order, and each partition is
// sorted stably on its own.  Used to time the oracle on all host cores.
int eo_sort_threads(const uint8_t* in, uint64_t n, uint32_t P, uint32_t log2B, uint32_t T, uint32_t Dmax, uint64_t S,
                    uint64_t seed, int balance, uint8_t* out, uint32_t threads) {
  if (P < 1 || (P & (P - 1)) || log2B > 24 || (1u << log2B) < P || T < 1 || threads < 1) return 1;
  if (S >= (1ull << 24) || (n > 0 && S == 0)) return 1;
  if (n == 0) return 0;
  std::vector<uint64_t> sample(S);
  eo_sample(in, n, S, seed, sample.data());
  std::sort(sample.begin(), sample.end());
  Rmi m = rmi_fit(sample.data(), S, T, Dmax);
  const uint32_t B = 1u << log2B;
  std::vector<uint32_t> q(n);
  std::vector<std::vector<uint64_t>> cnt(threads, std::vector<uint64_t>(B, 0));
  auto ranges = [&](uint32_t k, uint64_t* a, uint64_t* b) {
    *a = n * k / threads;
    *b = n * (k + 1) / threads;
  };
  {
    std::vector<std::thread> pool;
    for (uint32_t k = 0; k < threads; ++k)
      pool.emplace_back([&, k]() {
        uint64_t a, b;
        ranges(k, &a, &b);
        for (uint64_t i = a; i < b; ++i) {
          q[i] = fine_bin(rmi_cdf(m, encode_rec(in + i * kRecord)), log2B);
          cnt[k][q[i]]++;
        }
      });
    for (auto& th : pool) th.join();
  }
  std::vector<uint64_t> counts(B, 0);
  for (uint32_t k = 0; k < threads; ++k)
    for (uint32_t b = 0; b < B; ++b) counts[b] += cnt[k][b];
  std::vector<uint32_t> c = cuts_of(counts, P, log2B, n, balance);
  std::vector<uint32_t> pid_of_bin(B);
  for (uint32_t t = 0; t < B; ++t) pid_of_bin[t] = pid_of(c, P, t);
  std::vector<std::vector<uint64_t>> part(P);
  for (uint64_t i = 0; i < n; ++i) part[pid_of_bin[q[i]]].push_back(i);
  std::vector<uint64_t> off(P + 1, 0);
  for (uint32_t p = 0; p < P; ++p) off[p + 1] = off[p] + part[p].size();
  std::atomic<uint32_t> next(0);
  {
    std::vector<std::thread> pool;
    for (uint32_t k = 0; k < threads; ++k)
      pool.emplace_back([&]() {
        for (uint32_t p = next++; p < P; p = next++) {
          stable_sort_indices(in, part[p]);
          uint64_t o = off[p];
          for (uint64_t i : part[p]) std::memcpy(out + (o++) * kRecord, in + i * kRecord, kRecord);
        }
      });
    for (auto& th : pool) th.join();
  }
  return 0;
}

}  // extern "C"
