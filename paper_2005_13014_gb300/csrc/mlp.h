// mlp.h - host interface of the cost-model MLP kernels (k_mlp.cu).
#pragma once

#include <cuda_runtime.h>

namespace oec {

struct MlpDims {
  int F, H;   // features, hidden width
  int param_count() const { return H * F + H + H * H + H + H + 1; }
};

// device work buffers for batches of up to `cap` rows
struct MlpWork {
  int cap = 0;
  float *Z1 = nullptr, *A1 = nullptr, *Z2 = nullptr, *A2 = nullptr, *y = nullptr;
  float *dy = nullptr, *dZ2 = nullptr, *dZ1 = nullptr, *partial = nullptr;
  float* Xs = nullptr;   // standardised features
};

cudaError_t mlp_standardise(const float* X, int n, int F, const float* mu, const float* inv_sigma, float* out,
                            cudaStream_t st);

cudaError_t mlp_forward(const MlpDims& d, const float* P, const float* X, int n, MlpWork& w, float* y, cudaStream_t st);
cudaError_t mlp_gradient(const MlpDims& d, const float* P, const float* X, const float* t, int n, MlpWork& w,
                         float* G, float* loss, cudaStream_t st);
cudaError_t mlp_adam(float* P, const float* G, float* m, float* v, int count, float lr, float b1, float b2, float eps,
                     int step, cudaStream_t st);

}  // namespace oec
