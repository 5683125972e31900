// ELSAR oracle, learned part: the monotone MLP CDF model the GPU path trains
// as an alternative to the paper's RMI (the paper's Sec. 3.1 model is an RMI;
// this network is an addition, so its definition below is this project's).
//
// TEST INFRASTRUCTURE ONLY (see elsar_oracle.cpp).  Shares no code with the
// CUDA path.  Compiled with -ffp-contract=off: every fused multiply-add is an
// explicit std::fma / std::fmaf.
//
// Definition:
//   knots   T_m = sorted_sample[floor(m (S-1) / 12)], m = 0..12
//   feature phi_m(x) = W_m == 0 ? (x > T_m) : fp32(fp64(min(max(x - T_m, 0), W_m)) * R_m),
//           W_m = T_{m+1} - T_m, R_m = 1.0 / fp64(W_m)     (m = 0..11; exact integer ramps)
//   layer   h1_j = sigma(b1_j + sum_m W1_jm phi_m), h2_j = sigma(b2_j + sum_i W2_ji h1_i),
//           z = b3 + sum_j w3_j h2_j + sum_m v_m phi_m, F = clamp(z, 0, 1); all weights
//           (W1, W2, w3 and the linear skip v from the features to the output) >= 0
//   sigma(z) = 0.5 + 0.5 z / (1 + |z|)
//   sums    in index order as a chain of fused multiply-adds starting from the bias
//           (the output: b3, then the w3 terms, then the v terms)
//   start   v_m = 1/12, w3 = 0, b3 = 0: F starts as sum(phi) / 12, the linear
//           interpolation of the sample CDF between the knots; the hidden layers
//           start as structured soft steps (eo_mlp_init)
//   bins    fine-bin splitters t_q = smallest x in [0, 95^9] with min(B-1, floor(B F(x))) >= q,
//           found by bisection, then t_q = max(t_q, t_{q-1}); the fine bin of x is
//           #{q >= 1 : t_q <= x}, monotone in x whatever FP32 rounding does to F
//   training (FP64 here): MSE of F against rank/S on the sample, Adam
//           (beta 0.9 / 0.999, eps 1e-8) with the learning rate decayed from lr
//           to lr_min over the steps by a half cosine, weights projected to >= 0
//           after every step.
// Parity: FP64 forward/backward pinned by closed forms and central finite
// differences, the Adam step by its closed forms (first step, constant and
// alternating gradients, projection of weights only), the splitters by the
// exact bracket bin(t_q) >= q > bin(t_q - 1) (tests/test_oracle_mlp.py).  The
// GPU trains in FP32, so trained weights are not compared bit for bit; the
// FP32 forward and the splitters are compared exactly for given weights, and
// one Adam step within FP32 rounding.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

constexpr int kF = 12, kH = 32;
constexpr uint64_t kEncTop = 630249409724609375ull;  // 95^9
// parameter vector layout
constexpr int oW1 = 0, oB1 = oW1 + kH * kF, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH, oB3 = oW3 + kH,
              oV = oB3 + 1, kParams = oV + kF;  // 1517

struct Knots {
  uint64_t T[kF + 1];
  uint64_t W[kF];
  double R[kF];
};

Knots make_knots(const uint64_t* sorted, uint64_t S) {
  Knots k;
  for (int m = 0; m <= kF; ++m) k.T[m] = sorted[(uint64_t)m * (S - 1) / kF];
  for (int m = 0; m < kF; ++m) {
    k.W[m] = k.T[m + 1] - k.T[m];
    k.R[m] = k.W[m] ? 1.0 / (double)k.W[m] : 0.0;
  }
  return k;
}

void features32(const Knots& k, uint64_t x, float* phi) {
  for (int m = 0; m < kF; ++m) {
    if (k.W[m] == 0) {
      phi[m] = x > k.T[m] ? 1.0f : 0.0f;
      continue;
    }
    uint64_t d = x > k.T[m] ? x - k.T[m] : 0;
    if (d > k.W[m]) d = k.W[m];
    phi[m] = (float)((double)d * k.R[m]);
  }
}

// ---- FP32 forward, the operation order of the definition
float sigma32(float z) {
  float a = std::fabs(z);
  float r = z / (1.0f + a);
  return std::fmaf(0.5f, r, 0.5f);
}

float forward32(const float* w, const float* phi) {
  float h1[kH], h2[kH];
  for (int j = 0; j < kH; ++j) {
    float acc = w[oB1 + j];
    for (int m = 0; m < kF; ++m) acc = std::fmaf(w[oW1 + j * kF + m], phi[m], acc);
    h1[j] = sigma32(acc);
  }
  for (int j = 0; j < kH; ++j) {
    float acc = w[oB2 + j];
    for (int i = 0; i < kH; ++i) acc = std::fmaf(w[oW2 + j * kH + i], h1[i], acc);
    h2[j] = sigma32(acc);
  }
  float z = w[oB3];
  for (int j = 0; j < kH; ++j) z = std::fmaf(w[oW3 + j], h2[j], z);
  for (int m = 0; m < kF; ++m) z = std::fmaf(w[oV + m], phi[m], z);
  return z < 0.0f ? 0.0f : (z > 1.0f ? 1.0f : z);
}

// ---- FP64 forward and backward (plain chain rule)
double sigma64(double z) { return 0.5 + 0.5 * z / (1.0 + std::fabs(z)); }
double dsigma64(double z) {
  double d = 1.0 + std::fabs(z);
  return 0.5 / (d * d);
}

struct Acts {
  double p1[kH], h1[kH], p2[kH], h2[kH], z, F;
};

void forward64(const double* w, const double* phi, Acts& a) {
  for (int j = 0; j < kH; ++j) {
    double acc = w[oB1 + j];
    for (int m = 0; m < kF; ++m) acc += w[oW1 + j * kF + m] * phi[m];
    a.p1[j] = acc;
    a.h1[j] = sigma64(acc);
  }
  for (int j = 0; j < kH; ++j) {
    double acc = w[oB2 + j];
    for (int i = 0; i < kH; ++i) acc += w[oW2 + j * kH + i] * a.h1[i];
    a.p2[j] = acc;
    a.h2[j] = sigma64(acc);
  }
  double z = w[oB3];
  for (int j = 0; j < kH; ++j) z += w[oW3 + j] * a.h2[j];
  for (int m = 0; m < kF; ++m) z += w[oV + m] * phi[m];
  a.z = z;
  a.F = z < 0.0 ? 0.0 : (z > 1.0 ? 1.0 : z);
}

// gradient of (F - y)^2 with respect to every parameter, added into g
void backward64(const double* w, const double* phi, double y, const Acts& a, double* g) {
  double dF = 2.0 * (a.F - y);
  double dz = (a.z > 0.0 && a.z < 1.0) ? dF : 0.0;
  g[oB3] += dz;
  for (int m = 0; m < kF; ++m) g[oV + m] += dz * phi[m];
  double dp2[kH];
  for (int j = 0; j < kH; ++j) {
    g[oW3 + j] += dz * a.h2[j];
    dp2[j] = dz * w[oW3 + j] * dsigma64(a.p2[j]);
  }
  double dh1[kH] = {0};
  for (int j = 0; j < kH; ++j) {
    g[oB2 + j] += dp2[j];
    for (int i = 0; i < kH; ++i) {
      g[oW2 + j * kH + i] += dp2[j] * a.h1[i];
      dh1[i] += dp2[j] * w[oW2 + j * kH + i];
    }
  }
  for (int j = 0; j < kH; ++j) {
    double dp1 = dh1[j] * dsigma64(a.p1[j]);
    g[oB1 + j] += dp1;
    for (int m = 0; m < kF; ++m) g[oW1 + j * kF + m] += dp1 * phi[m];
  }
}

bool is_weight(int i) { return i < oB1 || (i >= oW2 && i < oB2) || (i >= oW3 && i < oB3) || i >= oV; }

}  // namespace

extern "C" {

int eo_mlp_params(void) { return kParams; }

// Starting point: the output is the linear skip alone, F = sum(phi) / 12 (the
// interpolation of the sample CDF between the knots); the hidden layers start
// structured -- hidden unit j of layer 1 a soft step of sum(phi) at
// 12 (j + 1/2) / 32, layer 2 passing it on -- with a 1 % jitter from the
// SplitMix64 counter stream with seed 7, ready for w3 to take them in.
void eo_mlp_init(float* w) {
  auto jitter = [](uint32_t i) {
    uint64_t z = 7ull + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (float)(z >> 40) * (1.0f / 16777216.0f);
  };
  const float k = 8.0f, a = 4.0f;
  for (int i = 0; i < kParams; ++i) {
    float v;
    if (i < oB1) v = k * (1.0f + 0.01f * jitter(i));
    else if (i < oW2) v = -k * 12.0f * ((float)(i - oB1) + 0.5f) / 32.0f;
    else if (i < oB2) {
      int j = (i - oW2) / kH, c = (i - oW2) % kH;
      v = j == c ? a * (1.0f + 0.01f * jitter(i)) : 0.01f * jitter(i);
    } else if (i < oW3) v = -a / 2;
    else if (i < oV) v = 0.0f;  // w3 and b3
    else v = 1.0f / 12.0f;
    w[i] = v;
  }
}

// knots (13 u64) of a sorted sample
void eo_mlp_knots(const uint64_t* sorted, uint64_t S, uint64_t* T) {
  Knots k = make_knots(sorted, S);
  for (int m = 0; m <= kF; ++m) T[m] = k.T[m];
}

// FP32 features of each x (12 per key)
void eo_mlp_features(const uint64_t* T, const uint64_t* xs, uint64_t n, float* phi) {
  Knots k;
  for (int m = 0; m <= kF; ++m) k.T[m] = T[m];
  for (int m = 0; m < kF; ++m) {
    k.W[m] = k.T[m + 1] - k.T[m];
    k.R[m] = k.W[m] ? 1.0 / (double)k.W[m] : 0.0;
  }
  for (uint64_t i = 0; i < n; ++i) features32(k, xs[i], phi + i * kF);
}

// FP32 forward on given features
void eo_mlp_forward32(const float* w, const float* phi, uint64_t n, float* F) {
  for (uint64_t i = 0; i < n; ++i) F[i] = forward32(w, phi + i * kF);
}

// FP64 forward on given features (double weights)
void eo_mlp_forward64(const double* w, const double* phi, uint64_t n, double* F) {
  Acts a;
  for (uint64_t i = 0; i < n; ++i) {
    forward64(w, phi + i * kF, a);
    F[i] = a.F;
  }
}

// FP64 gradient of the mean squared error over n samples
void eo_mlp_grad64(const double* w, const double* phi, const double* y, uint64_t n, double* g) {
  for (int i = 0; i < kParams; ++i) g[i] = 0.0;
  Acts a;
  for (uint64_t s = 0; s < n; ++s) {
    forward64(w, phi + s * kF, a);
    backward64(w, phi + s * kF, y[s], a, g);
  }
  for (int i = 0; i < kParams; ++i) g[i] /= (double)n;
}

// One step of Adam (Kingma & Ba 2015, Algorithm 1) at step number t >= 1 on
// the gradient g: the moment estimates m, v are updated in place, corrected
// for their zero start (divided by 1 - beta^t), and every parameter moves by
// lr * mhat / (sqrt(vhat) + eps); then the weights (not the biases) are
// projected back onto >= 0, which keeps the network monotone.
void eo_mlp_adam64(double* w, const double* g, double* m, double* v, uint64_t t, double lr) {
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  for (int i = 0; i < kParams; ++i) {
    m[i] = b1 * m[i] + (1 - b1) * g[i];
    v[i] = b2 * v[i] + (1 - b2) * g[i] * g[i];
    double mh = m[i] / (1 - std::pow(b1, (double)t));
    double vh = v[i] / (1 - std::pow(b2, (double)t));
    w[i] -= lr * mh / (std::sqrt(vh) + eps);
    if (is_weight(i) && w[i] < 0.0) w[i] = 0.0;
  }
}

// The learning rate of step t (1-based) of `steps`: a half cosine from lr to lr_min.
double eo_mlp_lr_at(uint64_t t, uint64_t steps, double lr, double lr_min) {
  const double pi = 3.14159265358979323846;
  const double f = steps > 1 ? (double)(t - 1) / (double)(steps - 1) : 0.0;
  return lr_min + (lr - lr_min) * 0.5 * (1.0 + std::cos(pi * f));
}

// FP64 training (Adam + projection) on features/labels: `steps` minibatch
// steps, step t taking minibatch (t - 1) mod nb, where minibatch b holds
// samples b, b + nb, b + 2 nb, ... (nb = ceil(n / batch)); w in/out.
void eo_mlp_train64(double* w, const double* phi, const double* y, uint64_t n, uint32_t batch, uint32_t steps,
                    double lr, double lr_min, double* loss_out) {
  std::vector<double> mom(kParams, 0.0), vel(kParams, 0.0), g(kParams);
  uint64_t nb = (n + batch - 1) / batch;
  Acts a;
  for (uint64_t t = 1; t <= steps; ++t) {
    const uint64_t b = (t - 1) % nb;
    for (int i = 0; i < kParams; ++i) g[i] = 0.0;
    uint64_t cnt = 0;
    for (uint64_t s = b; s < n; s += nb, ++cnt) {
      forward64(w, phi + s * kF, a);
      backward64(w, phi + s * kF, y[s], a, g.data());
    }
    for (int i = 0; i < kParams; ++i) g[i] /= (double)cnt;
    eo_mlp_adam64(w, g.data(), mom.data(), vel.data(), t, eo_mlp_lr_at(t, steps, lr, lr_min));
  }
  if (loss_out) {
    double l = 0.0;
    for (uint64_t s = 0; s < n; ++s) {
      forward64(w, phi + s * kF, a);
      l += (a.F - y[s]) * (a.F - y[s]);
    }
    *loss_out = l / (double)n;
  }
}

// Fine-bin splitters of the FP32 model by bisection (t[0] = 0), and the bins
// of given keys by the splitters.
void eo_mlp_splitters(const float* w, const uint64_t* T, uint32_t log2B, uint64_t* t) {
  Knots k;
  for (int m = 0; m <= kF; ++m) k.T[m] = T[m];
  for (int m = 0; m < kF; ++m) {
    k.W[m] = k.T[m + 1] - k.T[m];
    k.R[m] = k.W[m] ? 1.0 / (double)k.W[m] : 0.0;
  }
  const uint32_t B = 1u << log2B;
  float phi[kF];
  t[0] = 0;
  for (uint32_t q = 1; q < B; ++q) {
    uint64_t lo = 0, hi = kEncTop;
    while (lo < hi) {
      uint64_t mid = lo + (hi - lo) / 2;
      features32(k, mid, phi);
      float F = forward32(w, phi);
      uint32_t b = (uint32_t)(F * (float)B);
      if (b > B - 1) b = B - 1;
      if (b >= q) hi = mid;
      else lo = mid + 1;
    }
    t[q] = lo < t[q - 1] ? t[q - 1] : lo;  // kept non-decreasing (rounding could make F dip)
  }
}

// fine bin = #{q >= 1 : t_q <= x} (t non-decreasing)
void eo_bins_by_splitters(const uint64_t* t, uint32_t log2B, const uint64_t* xs, uint64_t n, uint32_t* q) {
  const uint32_t B = 1u << log2B;
  for (uint64_t i = 0; i < n; ++i) q[i] = (uint32_t)(std::upper_bound(t + 1, t + B, xs[i]) - (t + 1));
}

}  // extern "C"
