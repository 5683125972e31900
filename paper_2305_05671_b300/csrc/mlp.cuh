// Host interface of the monotone MLP CDF kernels (mlp.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace elsar {

constexpr int kMlpParamCount = 1517;  // 12*32 + 32 + 32*32 + 32 + 32 + 1 + 12 (the linear skip)

struct MlpTrainArgs {
  const uint64_t* sorted;  // sorted sample (S keys)
  uint64_t S, ntrain, batch;
  uint32_t steps;   // minibatch steps; step t takes minibatch (t - 1) mod nb
  float lr, lr_min; // learning rate decayed from lr to lr_min by a half cosine
  uint64_t* T;     // 13 knots (written)
  float* w;        // kMlpParamCount weights (written)
  float* m;        // Adam state (kMlpParamCount each)
  float* v;
  float* phi;      // ntrain * 12 features
  float* y;        // ntrain labels
  float* partial;  // grid * kMlpParamCount: partial gradients (per block, per group), a second Adam state
  int grid;
  cudaStream_t stream;
  uint32_t* launches;
};

cudaError_t mlp_train(const MlpTrainArgs& a);
cudaError_t mlp_splitters(const float* w, const uint64_t* T, uint32_t log2B, uint64_t* t, cudaStream_t st);
cudaError_t mlp_eval(const float* w, const uint64_t* T, const uint64_t* x, uint64_t n, float* F, cudaStream_t st);
cudaError_t mlp_grad(const float* w, const uint64_t* T, const uint64_t* x, const float* y, uint64_t n, float* phi,
                     float* partial, int grid, float* out, cudaStream_t st);
// one Adam step (step number t >= 1) on a given gradient, with the update training applies
cudaError_t mlp_adam_step(float* w, const float* grad, float* m, float* v, uint32_t t, float lr, cudaStream_t st);
cudaError_t judge_histogram(const uint64_t* x, uint64_t S, const uint64_t* t, uint32_t log2B, uint32_t log2J,
                            uint32_t* hist, cudaStream_t st);

}  // namespace elsar
