// costmodel.cpp - the learned cost model's handle (include/oec.h,
// oec_costmodel_*): parameters, Adam state and work buffers on the device,
// driven by the MLP kernels of k_mlp.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <new>
#include <vector>

#include "../../include/oec.h"
#include "api_internal.h"
#include "mlp.h"

struct oec_costmodel {
  oec::MlpDims dims{0, 0};
  float* P = nullptr;   // parameters
  float* G = nullptr;   // gradient
  float* m = nullptr;   // Adam first moment
  float* v = nullptr;   // Adam second moment
  int step = 0;
  float* mu = nullptr;          // feature standardisation (x - mu) * inv_sigma
  float* inv_sigma = nullptr;
  oec::MlpWork work;
  int dev = 0;
};

namespace {

void free_work(oec::MlpWork& w) {
  float* bufs[] = {w.Z1, w.A1, w.Z2, w.A2, w.y, w.dy, w.dZ2, w.dZ1, w.partial, w.Xs};
  for (float* b : bufs)
    if (b) cudaFree(b);
  w = oec::MlpWork();
}

int ensure_work(oec_costmodel* c, int n) {
  if (n <= c->work.cap) return OEC_OK;
  free_work(c->work);
  const size_t nh = sizeof(float) * (size_t)n * c->dims.H, n1 = sizeof(float) * (size_t)n;
  float** bufs[] = {&c->work.Z1, &c->work.A1, &c->work.Z2, &c->work.A2, &c->work.dZ2, &c->work.dZ1};
  for (float** b : bufs)
    if (cudaMalloc(b, nh) != cudaSuccess) return oec::cuda_fail(cudaGetLastError(), "cost-model work buffers");
  if (cudaMalloc(&c->work.Xs, sizeof(float) * (size_t)n * c->dims.F) != cudaSuccess)
    return oec::cuda_fail(cudaGetLastError(), "cost-model work buffers");
  if (cudaMalloc(&c->work.y, n1) != cudaSuccess || cudaMalloc(&c->work.dy, n1) != cudaSuccess ||
      cudaMalloc(&c->work.partial, sizeof(float) * ((n + 255) / 256 + 1)) != cudaSuccess)
    return oec::cuda_fail(cudaGetLastError(), "cost-model work buffers");
  c->work.cap = n;
  return OEC_OK;
}

}  // namespace

using namespace oec;

extern "C" {

int oec_costmodel_create(int n_features, int hidden, const float* params, oec_costmodel_t* out) {
  clear_error();
  if (!out || n_features < 1 || n_features > 256 || hidden < 1 || hidden > 128)
    return fail(OEC_ERR_INVALID_ARG, "need 1..256 features, 1..128 hidden units and an output handle");
  *out = nullptr;
  oec_costmodel* c = new (std::nothrow) oec_costmodel();
  if (!c) return fail(OEC_ERR_INVALID_ARG, "out of host memory");
  c->dims = MlpDims{n_features, hidden};
  cudaGetDevice(&c->dev);
  const size_t bytes = sizeof(float) * c->dims.param_count();
  cudaError_t e = cudaMalloc(&c->P, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->G, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->m, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->v, bytes);
  if (e == cudaSuccess) e = cudaMemset(c->m, 0, bytes);
  if (e == cudaSuccess) e = cudaMemset(c->v, 0, bytes);
  if (e == cudaSuccess) e = params ? cudaMemcpy(c->P, params, bytes, cudaMemcpyHostToDevice) : cudaMemset(c->P, 0, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&c->mu, sizeof(float) * n_features);
  if (e == cudaSuccess) e = cudaMalloc(&c->inv_sigma, sizeof(float) * n_features);
  if (e == cudaSuccess) {
    std::vector<float> z(n_features, 0.0f), o(n_features, 1.0f);
    e = cudaMemcpy(c->mu, z.data(), sizeof(float) * n_features, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->inv_sigma, o.data(), sizeof(float) * n_features, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    oec_costmodel_destroy(c);
    return cuda_fail(e, "cost-model allocation");
  }
  *out = c;
  return OEC_OK;
}

int oec_costmodel_param_count(oec_costmodel_t c) {
  clear_error();
  if (!c) return fail(OEC_ERR_INVALID_ARG, "null model");
  return c->dims.param_count();
}

int oec_costmodel_get_params(oec_costmodel_t c, float* host, int count) {
  clear_error();
  if (!c || !host || count != c->dims.param_count()) return fail(OEC_ERR_INVALID_ARG, "bad argument");
  cudaError_t e = cudaMemcpy(host, c->P, sizeof(float) * count, cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? OEC_OK : cuda_fail(e, "cost-model parameters");
}

int oec_costmodel_set_params(oec_costmodel_t c, const float* host, int count) {
  clear_error();
  if (!c || !host || count != c->dims.param_count()) return fail(OEC_ERR_INVALID_ARG, "bad argument");
  cudaError_t e = cudaMemcpy(c->P, host, sizeof(float) * count, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(c->m, 0, sizeof(float) * count);
  if (e == cudaSuccess) e = cudaMemset(c->v, 0, sizeof(float) * count);
  c->step = 0;
  return e == cudaSuccess ? OEC_OK : cuda_fail(e, "cost-model parameters");
}

int oec_costmodel_predict(oec_costmodel_t c, const float* X, int n, float* y, void* stream) {
  clear_error();
  if (!c || !X || !y || n < 1) return fail(OEC_ERR_INVALID_ARG, "bad argument");
  int rc = ensure_work(c, n);
  if (rc) return rc;
  cudaError_t e = mlp_standardise(X, n, c->dims.F, c->mu, c->inv_sigma, c->work.Xs, (cudaStream_t)stream);
  if (e == cudaSuccess) e = mlp_forward(c->dims, c->P, c->work.Xs, n, c->work, y, (cudaStream_t)stream);
  return e == cudaSuccess ? OEC_OK : cuda_fail(e, "cost-model forward");
}

int oec_costmodel_gradient(oec_costmodel_t c, const float* X, const float* t, int n, float* grad, float* loss,
                           void* stream) {
  clear_error();
  if (!c || !X || !t || !grad || !loss || n < 1) return fail(OEC_ERR_INVALID_ARG, "bad argument");
  int rc = ensure_work(c, n);
  if (rc) return rc;
  cudaError_t e = mlp_standardise(X, n, c->dims.F, c->mu, c->inv_sigma, c->work.Xs, (cudaStream_t)stream);
  if (e == cudaSuccess) e = mlp_gradient(c->dims, c->P, c->work.Xs, t, n, c->work, grad, loss, (cudaStream_t)stream);
  return e == cudaSuccess ? OEC_OK : cuda_fail(e, "cost-model gradient");
}

int oec_costmodel_train_step(oec_costmodel_t c, const float* X, const float* t, int n, float lr, float beta1,
                             float beta2, float eps, float* loss, void* stream) {
  clear_error();
  if (!c || !X || !t || !loss || n < 1) return fail(OEC_ERR_INVALID_ARG, "bad argument");
  int rc = ensure_work(c, n);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = mlp_standardise(X, n, c->dims.F, c->mu, c->inv_sigma, c->work.Xs, st);
  if (e == cudaSuccess) e = mlp_gradient(c->dims, c->P, c->work.Xs, t, n, c->work, c->G, loss, st);
  if (e == cudaSuccess) e = mlp_adam(c->P, c->G, c->m, c->v, c->dims.param_count(), lr, beta1, beta2, eps, ++c->step, st);
  return e == cudaSuccess ? OEC_OK : cuda_fail(e, "cost-model training step");
}

int oec_costmodel_set_normalization(oec_costmodel_t c, const float* mu, const float* sigma) {
  clear_error();
  if (!c || !mu || !sigma) return fail(OEC_ERR_INVALID_ARG, "null argument");
  std::vector<float> inv(c->dims.F);
  for (int f = 0; f < c->dims.F; ++f) inv[f] = sigma[f] > 0.0f ? 1.0f / sigma[f] : 1.0f;
  cudaError_t e = cudaMemcpy(c->mu, mu, sizeof(float) * c->dims.F, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->inv_sigma, inv.data(), sizeof(float) * c->dims.F, cudaMemcpyHostToDevice);
  return e == cudaSuccess ? OEC_OK : cuda_fail(e, "cost-model normalisation");
}

void oec_costmodel_destroy(oec_costmodel_t c) {
  if (!c) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(c->dev);
  cudaDeviceSynchronize();
  free_work(c->work);
  float* bufs[] = {c->P, c->G, c->m, c->v, c->mu, c->inv_sigma};
  for (float* b : bufs)
    if (b) cudaFree(b);
  cudaSetDevice(cur);
  delete c;
}

}  // extern "C"
