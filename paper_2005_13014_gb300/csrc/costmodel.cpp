// costmodel.cpp - the learned cost model's handle (include/oec.h,
// oec_costmodel_*): parameters, Adam state and work buffers on the device,
// driven by the MLP kernels of k_mlp.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
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
  std::vector<float> mu_host, sigma_host;   // as last set (checkpoints)
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
  c->mu_host.assign(mu, mu + c->dims.F);
  c->sigma_host.assign(sigma, sigma + c->dims.F);
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

// ---- checkpoints: magic, F, H, parameter count, parameters, mu, sigma ------
int oec_costmodel_save(oec_costmodel_t c, const char* path) {
  clear_error();
  if (!c || !path) return fail(OEC_ERR_INVALID_ARG, "null argument");
  const int n = oec_costmodel_param_count(c);
  std::vector<float> P(n);
  int rc = oec_costmodel_get_params(c, P.data(), n);
  if (rc) return rc;
  std::vector<float> mu(c->mu_host), sg(c->sigma_host);
  mu.resize(c->dims.F, 0.0f);
  sg.resize(c->dims.F, 1.0f);
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(OEC_ERR_INVALID_ARG, "cannot write %s", path);
  const char magic[8] = {'O', 'E', 'C', 'M', 'L', 'P', '1', 0};
  const int32_t hdr[3] = {c->dims.F, c->dims.H, n};
  bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int32_t), 3, f) == 3 &&
            std::fwrite(P.data(), sizeof(float), n, f) == (size_t)n &&
            std::fwrite(mu.data(), sizeof(float), mu.size(), f) == mu.size() &&
            std::fwrite(sg.data(), sizeof(float), sg.size(), f) == sg.size();
  ok = (std::fclose(f) == 0) && ok;
  return ok ? OEC_OK : fail(OEC_ERR_INVALID_ARG, "short write to %s", path);
}

int oec_costmodel_load(const char* path, oec_costmodel_t* out) {
  clear_error();
  if (!path || !out) return fail(OEC_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(OEC_ERR_INVALID_ARG, "cannot read %s", path);
  char magic[8];
  int32_t hdr[3];
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "OECMLP1", 8) == 0 &&
            std::fread(hdr, sizeof(int32_t), 3, f) == 3 && hdr[0] > 0 && hdr[1] > 0 && hdr[2] > 0 &&
            hdr[0] <= 4096 && hdr[1] <= 4096;
  std::vector<float> P, mu, sg;
  if (ok) {
    P.resize(hdr[2]);
    mu.resize(hdr[0]);
    sg.resize(hdr[0]);
    ok = std::fread(P.data(), sizeof(float), P.size(), f) == P.size() &&
         std::fread(mu.data(), sizeof(float), mu.size(), f) == mu.size() &&
         std::fread(sg.data(), sizeof(float), sg.size(), f) == sg.size();
  }
  std::fclose(f);
  if (!ok) return fail(OEC_ERR_INVALID_ARG, "%s is not a cost-model checkpoint", path);
  oec_costmodel_t c = nullptr;
  int rc = oec_costmodel_create(hdr[0], hdr[1], P.data(), &c);
  if (rc) return rc;
  if (oec_costmodel_param_count(c) != hdr[2]) {
    oec_costmodel_destroy(c);
    return fail(OEC_ERR_INVALID_ARG, "%s: parameter count does not match its dimensions", path);
  }
  rc = oec_costmodel_set_normalization(c, mu.data(), sg.data());
  if (rc) {
    oec_costmodel_destroy(c);
    return rc;
  }
  *out = c;
  return OEC_OK;
}

// ---- model-guided schedule selection ------------------------------------------
int oec_program_autotune_model(oec_program_t p, oec_costmodel_t m, const oec_field_desc* in, int n_in,
                               const oec_field_desc* out, int n_out, const int64_t lb[3], const int64_t ub[3],
                               const int64_t halo[3], const double* params, int n_params, int top_k, int reps,
                               void* cuda_stream, float* pred, int* best) {
  clear_error();
  if (!p || !m || !out || n_out < 1 || !lb || !ub || !halo || !best) return fail(OEC_ERR_INVALID_ARG, "null argument");
  const int nc = oec_program_candidates(p, nullptr, 0);
  if (nc < 1) return nc < 0 ? nc : fail(OEC_ERR_UNSUPPORTED, "no candidate schedules");
  std::vector<oec_schedule> cand(nc);
  oec_program_candidates(p, cand.data(), nc);
  const int64_t ext[3] = {ub[0] - lb[0], ub[1] - lb[1], ub[2] - lb[2]};
  const int64_t sj = out[0].stride[1], sk = out[0].stride[2];
  const int F = m->dims.F;
  std::vector<float> X((size_t)nc * F);
  for (int c = 0; c < nc; ++c) {
    const int nf = oec_program_features(p, ext, sj, sk, &cand[c], &X[(size_t)c * F], F);
    if (nf < 0) return nf;
    if (nf != F) return fail(OEC_ERR_INVALID_ARG, "the model takes %d features, the program gives %d", F, nf);
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  float *dX = nullptr, *dy = nullptr;
  std::vector<float> y(nc);
  cudaError_t e = cudaMalloc(&dX, sizeof(float) * X.size());
  if (e == cudaSuccess) e = cudaMalloc(&dy, sizeof(float) * nc);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dX, X.data(), sizeof(float) * X.size(), cudaMemcpyHostToDevice, st);
  int rc = e == cudaSuccess ? oec_costmodel_predict(m, dX, nc, dy, cuda_stream) : OEC_OK;
  if (e == cudaSuccess && rc == OEC_OK) e = cudaMemcpyAsync(y.data(), dy, sizeof(float) * nc, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && rc == OEC_OK) e = cudaStreamSynchronize(st);
  if (dX) cudaFree(dX);
  if (dy) cudaFree(dy);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "cost-model prediction");
  if (pred) std::copy(y.begin(), y.end(), pred);
  std::vector<int> order(nc);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return y[a] < y[b]; });
  if (top_k <= 0) {
    std::string why;
    for (int c : order)
      if (schedule_ok(p->kind, cand[c], why)) {
        p->sched = cand[c];
        *best = c;
        return OEC_OK;
      }
    return fail(OEC_ERR_UNSUPPORTED, "no valid candidate schedule");
  }
  const int k = std::min(top_k, nc);
  std::vector<oec_schedule> sub(k);
  for (int x = 0; x < k; ++x) sub[x] = cand[order[x]];
  std::vector<double> t(k);
  int bi = -1;
  rc = oec_program_autotune(p, in, n_in, out, n_out, lb, ub, halo, params, n_params, sub.data(), k, reps < 1 ? 1 : reps,
                            cuda_stream, t.data(), &bi);
  if (rc) return rc;
  *best = order[bi];
  return OEC_OK;
}

}  // extern "C"
