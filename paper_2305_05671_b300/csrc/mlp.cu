// The learned CDF alternative: a small monotone MLP (12 features -> 32 -> 32
// -> 1, FP32, non-negative weights) trained on the GPU by this file's own
// forward, backward and Adam kernels.  The paper's model (Sec. 3.1) is the RMI
// in fit.cu; the RMI stays as the network's fallback and as the judge of its
// skew error.  Definitions (shared with the oracle's restatement):
//   knots   T_m = sorted_sample[floor(m (S-1) / 12)], m = 0..12
//   feature phi_m = W_m == 0 ? (x > T_m) : fp32(fp64(clamp(x - T_m, 0, W_m)) * R_m),
//           W_m = T_{m+1} - T_m, R_m = 1 / fp64(W_m)
//   layers  fused multiply-add chains in index order from the bias,
//           sigma(z) = 0.5 + 0.5 z / (1 + |z|); the output adds a non-negative
//           linear skip of the features: z = b3 + sum w3_j h2_j + sum v_m phi_m,
//           F = clamp(z, 0, 1)
//   start   F = sum(phi) / 12 (v = 1/12, w3 = b3 = 0): the interpolation of the
//           sample CDF between the knots, which training then refines
//   splitters by bisection on floor(B F), made non-decreasing by a running max
#include <cmath>

#include "common.cuh"
#include "mlp.cuh"

namespace elsar {

constexpr int kMF = 12, kMH = 32;
constexpr int oW1 = 0, oB1 = oW1 + kMH * kMF, oW2 = oB1 + kMH, oB2 = oW2 + kMH * kMH, oW3 = oB2 + kMH, oB3 = oW3 + kMH,
              oV = oB3 + 1, kMlpParams = oV + kMF;  // 1517
static_assert(kMlpParams == kMlpParamCount, "parameter layout");

struct MlpKnots {
  uint64_t T[kMF + 1];
  uint64_t W[kMF];
  double R[kMF];
};

namespace {

inline uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }

__device__ __forceinline__ void mlp_features(const MlpKnots& k, uint64_t x, float* phi) {
#pragma unroll
  for (int m = 0; m < kMF; ++m) {
    if (k.W[m] == 0) {
      phi[m] = x > k.T[m] ? 1.0f : 0.0f;
    } else {
      uint64_t d = x > k.T[m] ? x - k.T[m] : 0;
      if (d > k.W[m]) d = k.W[m];
      phi[m] = __double2float_rn(__dmul_rn(__ull2double_rn(d), k.R[m]));
    }
  }
}

__device__ __forceinline__ float sigma32(float z) {
  const float r = __fdiv_rn(z, __fadd_rn(1.0f, fabsf(z)));
  return __fmaf_rn(0.5f, r, 0.5f);
}

// d sigma / dz = 0.5 / (1 + |z|)^2
__device__ __forceinline__ float dsigma32(float z) {
  const float d = __fadd_rn(1.0f, fabsf(z));
  return __fdiv_rn(0.5f, __fmul_rn(d, d));
}

__device__ __forceinline__ float mlp_forward(const float* __restrict__ w, const float* phi) {
  float h1[kMH];
#pragma unroll
  for (int j = 0; j < kMH; ++j) {
    float acc = w[oB1 + j];
#pragma unroll
    for (int m = 0; m < kMF; ++m) acc = __fmaf_rn(w[oW1 + j * kMF + m], phi[m], acc);
    h1[j] = sigma32(acc);
  }
  float z = w[oB3];
#pragma unroll 2
  for (int j = 0; j < kMH; ++j) {
    float acc = w[oB2 + j];
#pragma unroll
    for (int i = 0; i < kMH; ++i) acc = __fmaf_rn(w[oW2 + j * kMH + i], h1[i], acc);
    z = __fmaf_rn(w[oW3 + j], sigma32(acc), z);
  }
#pragma unroll
  for (int m = 0; m < kMF; ++m) z = __fmaf_rn(w[oV + m], phi[m], z);
  return z < 0.0f ? 0.0f : (z > 1.0f ? 1.0f : z);
}

__device__ __forceinline__ uint32_t mlp_bin(const float* w, const MlpKnots& k, uint64_t x, uint32_t log2B) {
  float phi[kMF];
  mlp_features(k, x, phi);
  const uint32_t B = 1u << log2B;
  const uint32_t q = (uint32_t)__fmul_rn(mlp_forward(w, phi), (float)B);
  return q < B ? q : B - 1;
}

// knots from the 13 key values T (every kernel builds them in shared memory)
__device__ __forceinline__ void load_knots(const uint64_t* __restrict__ T, MlpKnots& k) {
  if (threadIdx.x == 0) {
    for (int m = 0; m <= kMF; ++m) k.T[m] = T[m];
    for (int m = 0; m < kMF; ++m) {
      k.W[m] = k.T[m + 1] - k.T[m];
      k.R[m] = k.W[m] ? __ddiv_rn(1.0, __ull2double_rn(k.W[m])) : 0.0;
    }
  }
}

__global__ void knots_kernel(const uint64_t* __restrict__ x, uint64_t S, uint64_t* T) {
  if (threadIdx.x <= kMF) T[threadIdx.x] = x[(uint64_t)threadIdx.x * (S - 1) / kMF];
}

__global__ void eval_kernel(const float* __restrict__ w, const uint64_t* __restrict__ T, const uint64_t* __restrict__ x,
                            uint64_t n, float* __restrict__ F) {
  __shared__ float ws[kMlpParams];
  __shared__ MlpKnots k;
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) ws[i] = w[i];
  load_knots(T, k);
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    float phi[kMF];
    mlp_features(k, x[i], phi);
    F[i] = mlp_forward(ws, phi);
  }
}

// bisection per fine bin q (t[0] = 0; 95^9 when no key reaches q)
__global__ void splitter_kernel(const float* __restrict__ w, const uint64_t* __restrict__ T, uint32_t log2B,
                                uint64_t* __restrict__ t) {
  __shared__ float ws[kMlpParams];
  __shared__ MlpKnots k;
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) ws[i] = w[i];
  load_knots(T, k);
  __syncthreads();
  const uint32_t B = 1u << log2B;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < B; q += gridDim.x * blockDim.x) {
    if (q == 0) {
      t[0] = 0;
      continue;
    }
    uint64_t lo = 0, hi = kEncTop;
    while (lo < hi) {
      const uint64_t mid = lo + ((hi - lo) >> 1);
      if (mlp_bin(ws, k, mid, log2B) >= q) hi = mid;
      else lo = mid + 1;
    }
    t[q] = lo;
  }
}

// t[q] = max(t[0..q]) (single CTA, tiles with a running max)
__global__ void __launch_bounds__(1024) running_max_kernel(uint64_t* t, uint32_t log2B) {
  __shared__ uint64_t wmax[32];
  __shared__ uint64_t carry;
  const uint32_t B = 1u << log2B;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < B; base += 1024) {
    const uint32_t q = base + threadIdx.x;
    uint64_t v = q < B ? t[q] : 0;
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= (uint32_t)d) v = max(v, y);
    }
    if (lane == 31) wmax[warp] = v;
    __syncthreads();
    if (warp == 0) {
      uint64_t u = wmax[lane];
      for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, u, d);
        if (lane >= (uint32_t)d) u = max(u, y);
      }
      wmax[lane] = u;
    }
    __syncthreads();
    uint64_t r = max(v, carry);
    if (warp) r = max(r, wmax[warp - 1]);
    if (q < B) t[q] = r;
    __syncthreads();
    if (threadIdx.x == 1023) carry = r;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- training
// training set: every stride-th key of the sorted sample, label rank / S,
// stored minibatch-major: minibatch b holds training samples b, b + nb, ...
__global__ void train_set_kernel(const uint64_t* __restrict__ x, uint64_t S, uint64_t stride, uint64_t ntrain,
                                 uint64_t nb, const uint64_t* __restrict__ T, float* __restrict__ phi,
                                 float* __restrict__ y) {
  __shared__ MlpKnots k;
  load_knots(T, k);
  __syncthreads();
  for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < ntrain; s += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = s % nb, j = s / nb;
    const uint64_t per = ntrain / nb, extra = ntrain % nb;  // minibatch b has per + (b < extra) samples
    const uint64_t pos = b * per + (b < extra ? b : extra) + j;
    const uint64_t r = s * stride;
    float f[kMF];
    mlp_features(k, x[r], f);
    for (int m = 0; m < kMF; ++m) phi[pos * kMF + m] = f[m];
    y[pos] = (float)__ddiv_rn(__ull2double_rn(r), __ull2double_rn(S));
  }
}

__global__ void features_kernel(const uint64_t* __restrict__ x, uint64_t n, const uint64_t* __restrict__ T,
                                float* __restrict__ phi) {
  __shared__ MlpKnots k;
  load_knots(T, k);
  __syncthreads();
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    float f[kMF];
    mlp_features(k, x[i], f);
    for (int m = 0; m < kMF; ++m) phi[i * kMF + m] = f[m];
  }
}

// Start: the output is the linear skip alone, F = sum(phi) / 12; the hidden
// layers start structured -- hidden unit j of layer 1 a soft step of sum(phi)
// at 12 (j + 1/2) / 32, layer 2 passing it on -- with a 1 % jitter from a
// counter-based generator (seed 7), ready for w3 to take them in.
__device__ __forceinline__ float jitter(uint32_t i) {
  uint64_t z = 7ull + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)(z >> 40) * (1.0f / 16777216.0f);
}

__global__ void init_kernel(float* w, float* m, float* v) {
  const float k = 8.0f, a = 4.0f;
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) {
    float val;
    if (i < oB1) val = k * (1.0f + 0.01f * jitter(i));
    else if (i < oW2) val = -k * 12.0f * ((float)(i - oB1) + 0.5f) / 32.0f;
    else if (i < oB2) {
      const int j = (i - oW2) / kMH, c = (i - oW2) % kMH;
      val = (j == c ? a * (1.0f + 0.01f * jitter(i)) : 0.01f * jitter(i));
    } else if (i < oW3) val = -a / 2;
    else if (i < oV) val = 0.0f;  // w3 and b3
    else val = 1.0f / 12.0f;
    w[i] = val;
    m[i] = 0.0f;
    v[i] = 0.0f;
  }
}

constexpr int kChunk = 64;         // samples per CTA pass
constexpr int kQ = 8;              // threads per sample
constexpr int kGradThreads = kChunk * kQ;
constexpr int kUnits = kMH / kQ;   // hidden units per thread and layer
static_assert(kUnits == 4, "a thread's units are one float4 of a weight row");
constexpr int kPad = kMH + 1;
// contraction tasks, one per thread, a whole warp of one kind: 2x2 tiles of
// W2 (j pairs x i pairs), 2x2 tiles of W1 (j pairs x m pairs), then one
// parameter each of b1, b2, W3, b3 and V
constexpr int kW2Tiles = (kMH / 2) * (kMH / 2), kW1Tiles = (kMH / 2) * (kMF / 2);
constexpr int kSingles = kMH + kMH + kMH + 1 + kMF;
constexpr int kW1Task0 = kW2Tiles, kSingleTask0 = (kW2Tiles + kW1Tiles + 31) / 32 * 32;
static_assert(kW2Tiles % 32 == 0 && kSingleTask0 + kSingles <= kGradThreads, "task layout");

constexpr int kGroup = 8;  // blocks whose partial gradients the last of them to finish adds up

__device__ __forceinline__ bool is_weight(int i) {
  return i < oB1 || (i >= oW2 && i < oB2) || (i >= oW3 && i < oB3) || i >= oV;
}

// One Adam step of parameter i on its summed gradient g (Kingma & Ba, with
// the bias corrections c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t)), the
// weights (not the biases) projected to >= 0.
__device__ __forceinline__ void adam_update(int i, float g, float& w, float& m, float& v, float lr, float c1,
                                            float c2) {
  m = 0.9f * m + 0.1f * g;
  v = 0.999f * v + 0.001f * g * g;
  float wi = w - lr * (m * c1) / (sqrtf(v * c2) + 1e-8f);
  if (is_weight(i) && wi < 0.0f) wi = 0.0f;
  w = wi;
}

// The Adam state a training step reads (prev) and the one it writes (next);
// next is written by block 0 only, from the same arithmetic every block runs.
struct AdamIo {
  const float* part;  // previous step's partial gradients (nparts x kMlpParams), or null: no update
  int nparts;
  const float *w, *m, *v;
  float *w_next, *m_next, *v_next;
  float lr, c1, c2;
};

// Where a training step leaves its gradient: one row per block, and one row
// per group of kGroup blocks (the sum of the group's rows in block order),
// written by the group's last block to finish, as its ticket counter tells.
struct GradOut {
  float* block;       // gridDim.x x kMlpParams
  float* group;       // gridDim.x / kGroup x kMlpParams
  unsigned* tickets;  // gridDim.x / kGroup counters, zero between launches
};

// One training step.  Prologue: every block applies the previous step's
// Adam update (summing its group partials in order) to get the weights it
// uses; block 0 also stores the new state.  Then the partial gradient of
// mean (F - y)^2 over a range of one minibatch: eight threads (a quarter of
// a warp) run one sample forward and backward, each through 4 of the 32
// hidden units of a layer; the layer values go through shared memory, the
// output is summed by three shuffles, and each thread keeps the activation
// slopes of its own units in registers.  The weight rows a thread needs are
// one float4 each (W1 and W2 are also kept transposed).  Each thread then
// contracts its task (a 2x2 tile of a weight matrix or one bias/skip
// parameter) over the chunk, in sample order.  Last, the block writes its
// partial gradient, and the last block of its group to finish adds the
// group's rows (a fence and a ticket count, no waiting).
__global__ void __launch_bounds__(kGradThreads)
    grad_kernel(AdamIo io, const float* __restrict__ phi_g, const float* __restrict__ y_g, uint64_t b0, uint32_t cnt,
                float inv_cnt, GradOut out) {
  __shared__ __align__(16) float w[kMlpParams];
  __shared__ __align__(16) float w1t[kMF][kMH];  // w1t[m][j] = W1[j][m]
  __shared__ __align__(16) float w2t[kMH][kMH];  // w2t[i][j] = W2[j][i]
  __shared__ float phi[kChunk][kMF];
  __shared__ float h1[kChunk][kPad], h2[kChunk][kPad], d1[kChunk][kPad], d2[kChunk][kPad];
  __shared__ float dz[kChunk];
  {
    // the thread's parameters i = tid + 512 r; their partial sums are loaded
    // kBatch partials at a time for all of them, so that the loads overlap
    constexpr int kPer = (kMlpParams + kGradThreads - 1) / kGradThreads, kBatch = 9;
    float g[kPer];
#pragma unroll
    for (int r = 0; r < kPer; ++r) g[r] = 0.0f;
    if (io.part) {
      for (int c = 0; c < io.nparts; c += kBatch) {
        float x[kPer][kBatch];
#pragma unroll
        for (int r = 0; r < kPer; ++r)
#pragma unroll
          for (int k = 0; k < kBatch; ++k) {
            const int i = threadIdx.x + kGradThreads * r;
            x[r][k] = (i < kMlpParams && c + k < io.nparts) ? io.part[(uint64_t)(c + k) * kMlpParams + i] : 0.0f;
          }
#pragma unroll
        for (int r = 0; r < kPer; ++r)
#pragma unroll
          for (int k = 0; k < kBatch; ++k)
            if (c + k < io.nparts) g[r] += x[r][k];
      }
    }
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int i = threadIdx.x + kGradThreads * r;
      if (i >= kMlpParams) break;
      float v = io.w[i];
      if (io.part) {
        float mi = io.m[i], vi = io.v[i];
        adam_update(i, g[r], v, mi, vi, io.lr, io.c1, io.c2);
        if (blockIdx.x == 0) {
          io.w_next[i] = v;
          io.m_next[i] = mi;
          io.v_next[i] = vi;
        }
      }
      w[i] = v;
      if (i < oB1) w1t[i % kMF][i / kMF] = v;
      else if (i >= oW2 && i < oB2) w2t[(i - oW2) % kMH][(i - oW2) / kMH] = v;
    }
  }
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const uint32_t chunks = (cnt + kChunk - 1) / kChunk;
  const uint32_t per = (chunks + gridDim.x - 1) / gridDim.x;
  const uint32_t c0 = blockIdx.x * per, c1 = min(chunks, c0 + per);
  const int me = threadIdx.x / kQ, q = threadIdx.x % kQ, j0 = q * kUnits;
  const int task = threadIdx.x;
  __syncthreads();
  for (uint32_t c = c0; c < c1; ++c) {
    const uint32_t s = c * kChunk + me;
    const bool live = s < cnt;
    for (int m = q; m < kMF; m += kQ) phi[me][m] = live ? phi_g[(b0 + s) * kMF + m] : 0.0f;
    const float y = live ? y_g[b0 + s] : 0.0f;
    __syncwarp();
    // layer 1 of my units
    float t[kUnits], ds1[kUnits], ds2[kUnits];
#pragma unroll
    for (int u = 0; u < kUnits; ++u) t[u] = w[oB1 + j0 + u];
#pragma unroll
    for (int m = 0; m < kMF; ++m) {
      const float p = phi[me][m];
      const float4 wv = *reinterpret_cast<const float4*>(&w1t[m][j0]);
      t[0] = __fmaf_rn(wv.x, p, t[0]);
      t[1] = __fmaf_rn(wv.y, p, t[1]);
      t[2] = __fmaf_rn(wv.z, p, t[2]);
      t[3] = __fmaf_rn(wv.w, p, t[3]);
    }
#pragma unroll
    for (int u = 0; u < kUnits; ++u) {
      h1[me][j0 + u] = sigma32(t[u]);
      ds1[u] = dsigma32(t[u]);
      t[u] = w[oB2 + j0 + u];
    }
    __syncwarp();
    // layer 2 of my units and my part of the output
#pragma unroll 8
    for (int i = 0; i < kMH; ++i) {
      const float h = h1[me][i];
      const float4 wv = *reinterpret_cast<const float4*>(&w2t[i][j0]);
      t[0] = __fmaf_rn(wv.x, h, t[0]);
      t[1] = __fmaf_rn(wv.y, h, t[1]);
      t[2] = __fmaf_rn(wv.z, h, t[2]);
      t[3] = __fmaf_rn(wv.w, h, t[3]);
    }
    float z = 0.0f;
#pragma unroll
    for (int u = 0; u < kUnits; ++u) {
      const float hj = sigma32(t[u]);
      h2[me][j0 + u] = hj;
      ds2[u] = dsigma32(t[u]);
      z = __fmaf_rn(w[oW3 + j0 + u], hj, z);
    }
    for (int m = q; m < kMF; m += kQ) z = __fmaf_rn(w[oV + m], phi[me][m], z);
    z += __shfl_xor_sync(0xffffffffu, z, 1);
    z += __shfl_xor_sync(0xffffffffu, z, 2);
    z += __shfl_xor_sync(0xffffffffu, z, 4);
    z += w[oB3];
    const float F = z < 0.0f ? 0.0f : (z > 1.0f ? 1.0f : z);
    const float g = (live && z > 0.0f && z < 1.0f) ? 2.0f * (F - y) * inv_cnt : 0.0f;
    if (q == 0) dz[me] = g;
#pragma unroll
    for (int u = 0; u < kUnits; ++u) d2[me][j0 + u] = g * w[oW3 + j0 + u] * ds2[u];
    __syncwarp();
    // backward into my units of layer 1
    float dh[kUnits] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll 8
    for (int j = 0; j < kMH; ++j) {
      const float d = d2[me][j];
      const float4 wv = *reinterpret_cast<const float4*>(&w[oW2 + j * kMH + j0]);
      dh[0] = __fmaf_rn(d, wv.x, dh[0]);
      dh[1] = __fmaf_rn(d, wv.y, dh[1]);
      dh[2] = __fmaf_rn(d, wv.z, dh[2]);
      dh[3] = __fmaf_rn(d, wv.w, dh[3]);
    }
#pragma unroll
    for (int u = 0; u < kUnits; ++u) d1[me][j0 + u] = dh[u] * ds1[u];
    __syncthreads();
    if (task < kW1Task0) {  // W2[j][i], W2[j][i+1], W2[j+1][i], W2[j+1][i+1]
      const int j = 2 * (task / (kMH / 2)), i = 2 * (task % (kMH / 2));
#pragma unroll 4
      for (int s2 = 0; s2 < kChunk; ++s2) {
        const float a0 = d2[s2][j], a1 = d2[s2][j + 1], e0 = h1[s2][i], e1 = h1[s2][i + 1];
        acc[0] = __fmaf_rn(a0, e0, acc[0]);
        acc[1] = __fmaf_rn(a0, e1, acc[1]);
        acc[2] = __fmaf_rn(a1, e0, acc[2]);
        acc[3] = __fmaf_rn(a1, e1, acc[3]);
      }
    } else if (task < kW1Task0 + kW1Tiles) {  // W1[j][m], W1[j][m+1], W1[j+1][m], W1[j+1][m+1]
      const int k = task - kW1Task0, j = 2 * (k / (kMF / 2)), m = 2 * (k % (kMF / 2));
#pragma unroll 4
      for (int s2 = 0; s2 < kChunk; ++s2) {
        const float a0 = d1[s2][j], a1 = d1[s2][j + 1], e0 = phi[s2][m], e1 = phi[s2][m + 1];
        acc[0] = __fmaf_rn(a0, e0, acc[0]);
        acc[1] = __fmaf_rn(a0, e1, acc[1]);
        acc[2] = __fmaf_rn(a1, e0, acc[2]);
        acc[3] = __fmaf_rn(a1, e1, acc[3]);
      }
    } else if (task >= kSingleTask0 && task < kSingleTask0 + kSingles) {
      const int k = task - kSingleTask0;
      if (k < kMH) {  // b1
        for (int s2 = 0; s2 < kChunk; ++s2) acc[0] += d1[s2][k];
      } else if (k < 2 * kMH) {  // b2
        for (int s2 = 0; s2 < kChunk; ++s2) acc[0] += d2[s2][k - kMH];
      } else if (k < 3 * kMH) {  // W3
        for (int s2 = 0; s2 < kChunk; ++s2) acc[0] = __fmaf_rn(dz[s2], h2[s2][k - 2 * kMH], acc[0]);
      } else if (k == 3 * kMH) {  // b3
        for (int s2 = 0; s2 < kChunk; ++s2) acc[0] += dz[s2];
      } else {  // V
        for (int s2 = 0; s2 < kChunk; ++s2) acc[0] = __fmaf_rn(dz[s2], phi[s2][k - 3 * kMH - 1], acc[0]);
      }
    }
    __syncthreads();
  }
  // my partial gradient into shared memory (h1 is free after the last chunk)
  static_assert(kChunk * kPad >= kMlpParams, "h1 holds a partial gradient");
  float* red = &h1[0][0];
  if (task < kW1Task0) {
    const int j = 2 * (task / (kMH / 2)), i = 2 * (task % (kMH / 2));
    red[oW2 + j * kMH + i] = acc[0];
    red[oW2 + j * kMH + i + 1] = acc[1];
    red[oW2 + (j + 1) * kMH + i] = acc[2];
    red[oW2 + (j + 1) * kMH + i + 1] = acc[3];
  } else if (task < kW1Task0 + kW1Tiles) {
    const int k = task - kW1Task0, j = 2 * (k / (kMF / 2)), m = 2 * (k % (kMF / 2));
    red[oW1 + j * kMF + m] = acc[0];
    red[oW1 + j * kMF + m + 1] = acc[1];
    red[oW1 + (j + 1) * kMF + m] = acc[2];
    red[oW1 + (j + 1) * kMF + m + 1] = acc[3];
  } else if (task >= kSingleTask0 && task < kSingleTask0 + kSingles) {
    const int k = task - kSingleTask0;
    const int p = k < kMH ? oB1 + k : k < 2 * kMH ? oB2 + k - kMH : k < 3 * kMH ? oW3 + k - 2 * kMH
                : k == 3 * kMH ? oB3 : oV + k - 3 * kMH - 1;
    red[p] = acc[0];
  }
  __syncthreads();
  for (int p = threadIdx.x; p < kMlpParams; p += kGradThreads)
    __stcg(&out.block[(uint64_t)blockIdx.x * kMlpParams + p], red[p]);
  __threadfence();
  __syncthreads();
  __shared__ bool last;
  const unsigned grp = blockIdx.x / kGroup;
  if (threadIdx.x == 0) last = atomicAdd(&out.tickets[grp], 1u) == kGroup - 1;
  __syncthreads();
  if (last) {
    __threadfence();
    for (int p = threadIdx.x; p < kMlpParams; p += kGradThreads) {
      float x[kGroup];
#pragma unroll
      for (int k = 0; k < kGroup; ++k) x[k] = __ldcg(&out.block[(uint64_t)(grp * kGroup + k) * kMlpParams + p]);
      float sum = 0.0f;
#pragma unroll
      for (int k = 0; k < kGroup; ++k) sum += x[k];
      out.group[(uint64_t)grp * kMlpParams + p] = sum;
    }
    if (threadIdx.x == 0) out.tickets[grp] = 0;  // ready for the next launch
  }
}

// Sum of the partial gradients in order, then (adam_kernel) the Adam step.
__global__ void reduce_partials_kernel(const float* __restrict__ partial, int nparts, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  float g = 0.0f;
  for (int c = 0; c < nparts; ++c) g += partial[(uint64_t)c * kMlpParams + i];
  out[i] = g;
}

__global__ void adam_kernel(AdamIo io) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  float g = 0.0f;
  for (int c = 0; c < io.nparts; ++c) g += io.part[(uint64_t)c * kMlpParams + i];
  float wi = io.w[i], mi = io.m[i], vi = io.v[i];
  adam_update(i, g, wi, mi, vi, io.lr, io.c1, io.c2);
  io.w_next[i] = wi;
  io.m_next[i] = mi;
  io.v_next[i] = vi;
}

// judge: fine bin of each held-out key under a splitter set (binary search)
__global__ void judge_hist_kernel(const uint64_t* __restrict__ x, uint64_t S, const uint64_t* __restrict__ t,
                                  uint32_t log2B, uint32_t shift, uint32_t* __restrict__ hist) {
  const uint32_t B = 1u << log2B;
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < S; k += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t lo = 0, hi = B - 1;
    const uint64_t v = x[k];
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (t[mid] <= v) lo = mid;
      else hi = mid - 1;
    }
    atomicAdd(hist + (lo >> shift), 1u);
  }
}

}  // namespace

cudaError_t mlp_train(const MlpTrainArgs& a) {
  cudaStream_t st = a.stream;
  const int sms = sm_count();
  const uint64_t stride = a.S / a.ntrain;
  const uint64_t nb = (a.ntrain + a.batch - 1) / a.batch;
  const uint64_t per = a.ntrain / nb, extra = a.ntrain % nb;
  // one CTA per chunk of 64 samples of the largest minibatch, in whole groups
  const int groups = (int)((per + 1 + kChunk * kGroup - 1) / (kChunk * kGroup));
  const int grid = groups * kGroup;
  // a.partial rows: the blocks' partials, two group-partial buffers (steps
  // alternate between them, so a step's prologue reads the previous step's
  // while it writes its own), the second Adam state (w, m, v), the tickets
  if (a.steps == 0 || grid + 2 * groups + 4 > a.grid) return cudaErrorInvalidValue;
  float* gpart[2] = {a.partial + (size_t)grid * kMlpParams, a.partial + (size_t)(grid + groups) * kMlpParams};
  float* alt = a.partial + (size_t)(grid + 2 * groups) * kMlpParams;
  unsigned* tickets = reinterpret_cast<unsigned*>(alt + 3 * kMlpParams);
  cudaError_t e = cudaMemsetAsync(tickets, 0, groups * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  knots_kernel<<<1, 32, 0, st>>>(a.sorted, a.S, a.T);
  train_set_kernel<<<(unsigned)umin64((a.ntrain + 255) / 256, (uint64_t)sms * 8), 256, 0, st>>>(
      a.sorted, a.S, stride, a.ntrain, nb, a.T, a.phi, a.y);
  float* W[2] = {a.w, alt};
  float* M[2] = {a.m, alt + kMlpParams};
  float* V[2] = {a.v, alt + 2 * kMlpParams};
  // the state after k updates is in set (steps - k) mod 2: the last one in a.w
  auto set_of = [&](uint32_t k) { return (int)((a.steps - k) & 1); };
  init_kernel<<<1, 256, 0, st>>>(W[set_of(0)], M[set_of(0)], V[set_of(0)]);
  *a.launches += 3;
  const double pi = 3.14159265358979323846;
  double p1 = 1.0, p2 = 1.0;
  // the update of step k (>= 1; p1, p2 already multiplied k times): state k - 1 -> k
  auto update = [&](uint32_t k) {
    // half-cosine decay of the learning rate from lr to lr_min over the steps
    const double f = a.steps > 1 ? (double)(k - 1) / (double)(a.steps - 1) : 0.0;
    const double lr = a.lr_min + (a.lr - a.lr_min) * 0.5 * (1.0 + cos(pi * f));
    const int from = set_of(k - 1), to = set_of(k);
    AdamIo io = {gpart[k & 1], groups, W[from], M[from], V[from], W[to], M[to], V[to],
                 (float)lr, (float)(1.0 / (1.0 - p1)), (float)(1.0 / (1.0 - p2))};
    return io;
  };
  for (uint32_t t = 1; t <= a.steps; ++t) {
    const uint64_t b = (t - 1) % nb;  // minibatch b holds training samples b, b + nb, ...
    const uint64_t b0 = b * per + (b < extra ? b : extra);
    const uint32_t cnt = (uint32_t)(per + (b < extra ? 1 : 0));
    AdamIo io = {};
    io.w = W[set_of(0)];
    if (t >= 2) {  // this launch first applies step t - 1's update
      p1 *= 0.9;
      p2 *= 0.999;
      io = update(t - 1);
    }
    grad_kernel<<<grid, kGradThreads, 0, st>>>(io, a.phi, a.y, b0, cnt, 1.0f / (float)cnt,
                                               GradOut{a.partial, gpart[t & 1], tickets});
  }
  p1 *= 0.9;
  p2 *= 0.999;
  adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(update(a.steps));
  *a.launches += a.steps + 1;
  return cudaGetLastError();
}

cudaError_t mlp_adam_step(float* w, const float* grad, float* m, float* v, uint32_t t, float lr, cudaStream_t st) {
  // the trainer's bias corrections: running products of the decay rates in FP64, then one rounding
  double p1 = 1.0, p2 = 1.0;
  for (uint32_t k = 0; k < t; ++k) {
    p1 *= 0.9;
    p2 *= 0.999;
  }
  const AdamIo io = {grad, 1, w, m, v, w, m, v, lr, (float)(1.0 / (1.0 - p1)), (float)(1.0 / (1.0 - p2))};
  adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(io);
  return cudaGetLastError();
}

cudaError_t mlp_splitters(const float* w, const uint64_t* T, uint32_t log2B, uint64_t* t, cudaStream_t st) {
  const uint32_t B = 1u << log2B;
  splitter_kernel<<<(B + 127) / 128, 128, 0, st>>>(w, T, log2B, t);
  running_max_kernel<<<1, 1024, 0, st>>>(t, log2B);
  return cudaGetLastError();
}

cudaError_t mlp_eval(const float* w, const uint64_t* T, const uint64_t* x, uint64_t n, float* F, cudaStream_t st) {
  const int sms = sm_count();
  eval_kernel<<<(unsigned)umin64((n + 255) / 256 + 1, (uint64_t)sms * 8), 256, 0, st>>>(w, T, x, n, F);
  return cudaGetLastError();
}

cudaError_t mlp_grad(const float* w, const uint64_t* T, const uint64_t* x, const float* y, uint64_t n, float* phi,
                     float* partial, int grid, float* out, cudaStream_t st) {
  const int sms = sm_count();
  features_kernel<<<(unsigned)umin64((n + 255) / 256 + 1, (uint64_t)sms * 8), 256, 0, st>>>(x, n, T, phi);
  AdamIo io = {};
  io.w = w;
  // partial rows: the blocks', the groups', the tickets
  const int groups = (grid - 1) / (kGroup + 1), blocks = groups * kGroup;
  if (groups < 1) return cudaErrorInvalidValue;
  float* gpart = partial + (size_t)blocks * kMlpParams;
  unsigned* tickets = reinterpret_cast<unsigned*>(gpart + (size_t)groups * kMlpParams);
  cudaError_t e = cudaMemsetAsync(tickets, 0, groups * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  grad_kernel<<<blocks, kGradThreads, 0, st>>>(io, phi, y, 0, (uint32_t)n, 1.0f / (float)n,
                                               GradOut{partial, gpart, tickets});
  reduce_partials_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(gpart, groups, out);
  return cudaGetLastError();
}

cudaError_t judge_histogram(const uint64_t* x, uint64_t S, const uint64_t* t, uint32_t log2B, uint32_t log2J,
                            uint32_t* hist, cudaStream_t st) {
  const int sms = sm_count();
  cudaMemsetAsync(hist, 0, sizeof(uint32_t) << log2J, st);
  judge_hist_kernel<<<(unsigned)umin64((S + 255) / 256 + 1, (uint64_t)sms * 8), 256, 0, st>>>(x, S, t, log2B,
                                                                                               log2B - log2J, hist);
  return cudaGetLastError();
}

}  // namespace elsar
