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

constexpr int kChunk = 64;  // samples per CTA pass (one per thread)
constexpr int kPad = kMH + 1;
constexpr int kOwn = (kMlpParams + kChunk - 1) / kChunk;  // parameters each thread contracts (24)

// Partial gradient of mean (F - y)^2 over a range of one minibatch: each
// thread runs one sample forward and backward into shared memory, then every
// thread contracts its own parameters over the chunk (fixed order).
__global__ void __launch_bounds__(kChunk) grad_kernel(const float* __restrict__ w_g, const float* __restrict__ phi_g,
                                                      const float* __restrict__ y_g, uint64_t b0, uint32_t cnt,
                                                      float inv_cnt, float* __restrict__ partial) {
  __shared__ float w[kMlpParams];
  __shared__ float phi[kChunk][kMF];
  __shared__ float h1[kChunk][kPad], h2[kChunk][kPad], d1[kChunk][kPad], d2[kChunk][kPad];
  __shared__ float dz[kChunk];
  for (int i = threadIdx.x; i < kMlpParams; i += kChunk) w[i] = w_g[i];
  float acc[kOwn];
#pragma unroll
  for (int r = 0; r < kOwn; ++r) acc[r] = 0.0f;
  const uint32_t chunks = (cnt + kChunk - 1) / kChunk;
  const uint32_t per = (chunks + gridDim.x - 1) / gridDim.x;
  const uint32_t c0 = blockIdx.x * per, c1 = min(chunks, c0 + per);
  const int me = threadIdx.x;
  __syncthreads();
  for (uint32_t c = c0; c < c1; ++c) {
    const uint32_t s = c * kChunk + me;
    const bool live = s < cnt;
#pragma unroll
    for (int m = 0; m < kMF; ++m) phi[me][m] = live ? phi_g[(b0 + s) * kMF + m] : 0.0f;
    const float y = live ? y_g[b0 + s] : 0.0f;
    // layer 1: h1 and sigma'(pre1) (kept in d1 until the backward pass)
    for (int j = 0; j < kMH; ++j) {
      float t = w[oB1 + j];
#pragma unroll
      for (int m = 0; m < kMF; ++m) t = __fmaf_rn(w[oW1 + j * kMF + m], phi[me][m], t);
      h1[me][j] = sigma32(t);
      d1[me][j] = dsigma32(t);
    }
    // layer 2 and output: h2 and sigma'(pre2) (kept in d2)
    float z = w[oB3];
    for (int j = 0; j < kMH; ++j) {
      float t = w[oB2 + j];
#pragma unroll 8
      for (int i = 0; i < kMH; ++i) t = __fmaf_rn(w[oW2 + j * kMH + i], h1[me][i], t);
      const float hj = sigma32(t);
      h2[me][j] = hj;
      d2[me][j] = dsigma32(t);
      z = __fmaf_rn(w[oW3 + j], hj, z);
    }
#pragma unroll
    for (int m = 0; m < kMF; ++m) z = __fmaf_rn(w[oV + m], phi[me][m], z);
    const float F = z < 0.0f ? 0.0f : (z > 1.0f ? 1.0f : z);
    const float g = (live && z > 0.0f && z < 1.0f) ? 2.0f * (F - y) * inv_cnt : 0.0f;
    dz[me] = g;
    float dh1[kMH];
#pragma unroll
    for (int i = 0; i < kMH; ++i) dh1[i] = 0.0f;
    for (int j = 0; j < kMH; ++j) {
      const float dp2 = g * w[oW3 + j] * d2[me][j];
      d2[me][j] = dp2;
#pragma unroll
      for (int i = 0; i < kMH; ++i) dh1[i] = __fmaf_rn(dp2, w[oW2 + j * kMH + i], dh1[i]);
    }
#pragma unroll
    for (int i = 0; i < kMH; ++i) d1[me][i] = dh1[i] * d1[me][i];
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kOwn; ++r) {
      const int p = me + kChunk * r;
      if (p >= kMlpParams) break;
      float sum = 0.0f;
      if (p < oB1) {
        const int j = p / kMF, m = p % kMF;
        for (int s2 = 0; s2 < kChunk; ++s2) sum = __fmaf_rn(d1[s2][j], phi[s2][m], sum);
      } else if (p < oW2) {
        const int j = p - oB1;
        for (int s2 = 0; s2 < kChunk; ++s2) sum += d1[s2][j];
      } else if (p < oB2) {
        const int j = (p - oW2) / kMH, i = (p - oW2) % kMH;
        for (int s2 = 0; s2 < kChunk; ++s2) sum = __fmaf_rn(d2[s2][j], h1[s2][i], sum);
      } else if (p < oW3) {
        const int j = p - oB2;
        for (int s2 = 0; s2 < kChunk; ++s2) sum += d2[s2][j];
      } else if (p < oB3) {
        const int j = p - oW3;
        for (int s2 = 0; s2 < kChunk; ++s2) sum = __fmaf_rn(dz[s2], h2[s2][j], sum);
      } else if (p == oB3) {
        for (int s2 = 0; s2 < kChunk; ++s2) sum += dz[s2];
      } else {
        const int m = p - oV;
        for (int s2 = 0; s2 < kChunk; ++s2) sum = __fmaf_rn(dz[s2], phi[s2][m], sum);
      }
      acc[r] += sum;
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < kOwn; ++r) {
    const int p = me + kChunk * r;
    if (p < kMlpParams) partial[(uint64_t)blockIdx.x * kMlpParams + p] = acc[r];
  }
}

__global__ void reduce_partials_kernel(const float* __restrict__ partial, int nparts, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  float g = 0.0f;
  for (int c = 0; c < nparts; ++c) g += partial[(uint64_t)c * kMlpParams + i];
  out[i] = g;
}

__device__ __forceinline__ bool is_weight(int i) {
  return i < oB1 || (i >= oW2 && i < oB2) || (i >= oW3 && i < oB3) || i >= oV;
}

// Adam on the summed partial gradients (fixed order), weights projected to >= 0.
__global__ void adam_kernel(const float* __restrict__ partial, int nparts, float* w, float* m, float* v, float lr,
                            float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  float g = 0.0f;
  for (int c = 0; c < nparts; ++c) g += partial[(uint64_t)c * kMlpParams + i];
  const float mi = 0.9f * m[i] + 0.1f * g;
  const float vi = 0.999f * v[i] + 0.001f * g * g;
  m[i] = mi;
  v[i] = vi;
  float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
  if (is_weight(i) && wi < 0.0f) wi = 0.0f;
  w[i] = wi;
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
  knots_kernel<<<1, 32, 0, st>>>(a.sorted, a.S, a.T);
  const uint64_t stride = a.S / a.ntrain;
  const uint64_t nb = (a.ntrain + a.batch - 1) / a.batch;
  train_set_kernel<<<(unsigned)umin64((a.ntrain + 255) / 256, (uint64_t)sms * 8), 256, 0, st>>>(
      a.sorted, a.S, stride, a.ntrain, nb, a.T, a.phi, a.y);
  init_kernel<<<1, 256, 0, st>>>(a.w, a.m, a.v);
  *a.launches += 3;
  const uint64_t per = a.ntrain / nb, extra = a.ntrain % nb;
  // one CTA per chunk of 64 samples of the largest minibatch, at most a.grid
  const int grid = (int)umin64((uint64_t)a.grid, (per + 1 + kChunk - 1) / kChunk);
  const double pi = 3.14159265358979323846;
  double p1 = 1.0, p2 = 1.0;
  for (uint32_t t = 1; t <= a.steps; ++t) {
    const uint64_t b = (t - 1) % nb;  // minibatch b holds training samples b, b + nb, ...
    const uint64_t b0 = b * per + (b < extra ? b : extra);
    const uint32_t cnt = (uint32_t)(per + (b < extra ? 1 : 0));
    grad_kernel<<<grid, kChunk, 0, st>>>(a.w, a.phi, a.y, b0, cnt, 1.0f / (float)cnt, a.partial);
    p1 *= 0.9;
    p2 *= 0.999;
    // half-cosine decay of the learning rate from lr to lr_min over the steps
    const double f = a.steps > 1 ? (double)(t - 1) / (double)(a.steps - 1) : 0.0;
    const double lr = a.lr_min + (a.lr - a.lr_min) * 0.5 * (1.0 + cos(pi * f));
    adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(a.partial, grid, a.w, a.m, a.v, (float)lr,
                                                           (float)(1.0 / (1.0 - p1)), (float)(1.0 / (1.0 - p2)));
    *a.launches += 2;
  }
  return cudaGetLastError();
}

cudaError_t mlp_adam_step(float* w, const float* grad, float* m, float* v, uint32_t t, float lr, cudaStream_t st) {
  // the trainer's bias corrections: running products of the decay rates in FP64, then one rounding
  double p1 = 1.0, p2 = 1.0;
  for (uint32_t k = 0; k < t; ++k) {
    p1 *= 0.9;
    p2 *= 0.999;
  }
  adam_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(grad, 1, w, m, v, lr, (float)(1.0 / (1.0 - p1)),
                                                         (float)(1.0 / (1.0 - p2)));
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
  grad_kernel<<<grid, kChunk, 0, st>>>(w, phi, y, 0, (uint32_t)n, 1.0f / (float)n, partial);
  reduce_partials_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(partial, grid, out);
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
