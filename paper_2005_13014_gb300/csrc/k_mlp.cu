// k_mlp.cu - the cost model's MLP (features -> H -> H -> 1, ReLU) in FP32:
// forward, mean-squared-error gradient, backward and Adam (Kingma & Ba, 2015).
// Every reduction runs in a fixed order (no atomics), so training is
// bit-reproducible. The paper has no learned component; this predicts the
// best schedule for a stencil program from the autotuner's timings.
//
// Parameters are one flat FP32 array: W1 [H][F], b1 [H], W2 [H][H], b2 [H],
// W3 [1][H], b3 [1].
#include <cuda_runtime.h>

#include "kcommon.cuh"
#include "mlp.h"

namespace oec {
namespace {

constexpr int ROWS = 16;   // rows of X per CTA in the dense layers

// Z[n][o] = sum_f X[n][f] W[o][f] + b[o];  A = relu(Z) (or A = Z when !relu)
__global__ void dense_fwd(const float* __restrict__ X, int n, int fin, const float* __restrict__ W,
                          const float* __restrict__ b, int fout, float* __restrict__ Z, float* __restrict__ A,
                          int relu) {
  extern __shared__ float sm[];
  float* sW = sm;                  // fout * fin
  float* sX = sm + fout * fin;     // ROWS * fin
  const int r0 = blockIdx.x * ROWS;
  for (int x = threadIdx.x; x < fout * fin; x += blockDim.x) sW[x] = W[x];
  for (int x = threadIdx.x; x < ROWS * fin; x += blockDim.x) {
    const int r = r0 + x / fin;
    sX[x] = r < n ? X[(size_t)r * fin + x % fin] : 0.0f;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < ROWS * fout; x += blockDim.x) {
    const int r = x / fout, o = x % fout;
    if (r0 + r >= n) continue;
    float acc = b[o];
    for (int f = 0; f < fin; ++f) acc = fmaf(sX[r * fin + f], sW[o * fin + f], acc);
    const size_t idx = (size_t)(r0 + r) * fout + o;
    if (Z) Z[idx] = acc;
    A[idx] = relu ? fmaxf(acc, 0.0f) : acc;
  }
}

// dy = 2 (y - t) / n; per-CTA partial sums of (y - t)^2 in a fixed tree order
__global__ void mse_grad(const float* __restrict__ y, const float* __restrict__ t, int n, float* __restrict__ dy,
                         float* __restrict__ partial) {
  __shared__ float s[256];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float e = 0.0f;
  if (i < n) {
    const float r = y[i] - t[i];
    dy[i] = 2.0f * r / (float)n;
    e = r * r;
  }
  s[threadIdx.x] = e;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = s[0];
}

__global__ void sum_partials(const float* __restrict__ partial, int m, int n, float* __restrict__ loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    float acc = 0.0f;
    for (int x = 0; x < m; ++x) acc += partial[x];
    *loss = acc / (float)n;
  }
}

// dW[o][i] = sum_n dZ[n][o] A[n][i]  (A = nullptr: column of ones, i.e. db)
// one thread per (o, i), sum over n in order
__global__ void weight_grad(const float* __restrict__ dZ, int n, int fout, const float* __restrict__ A, int fin,
                            float* __restrict__ dW) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int cols = A ? fin : 1;
  if (x >= fout * cols) return;
  const int o = x / cols, i = x % cols;
  float acc = 0.0f;
  for (int r = 0; r < n; ++r) acc = fmaf(dZ[(size_t)r * fout + o], A ? A[(size_t)r * fin + i] : 1.0f, acc);
  dW[x] = acc;
}

// dZp[n][i] = (sum_o dZ[n][o] W[o][i]) * (Zp[n][i] > 0)
__global__ void input_grad(const float* __restrict__ dZ, int n, int fout, const float* __restrict__ W, int fin,
                           const float* __restrict__ Zp, float* __restrict__ dZp) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n * fin) return;
  const int r = x / fin, i = x % fin;
  float acc = 0.0f;
  for (int o = 0; o < fout; ++o) acc = fmaf(dZ[(size_t)r * fout + o], W[o * fin + i], acc);
  dZp[x] = Zp[x] > 0.0f ? acc : 0.0f;
}

__global__ void adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                     int count, float lr, float b1, float b2, float eps, float bc1, float bc2) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= count) return;
  const float gx = g[x];
  const float mx = b1 * m[x] + (1.0f - b1) * gx;
  const float vx = b2 * v[x] + (1.0f - b2) * gx * gx;
  m[x] = mx;
  v[x] = vx;
  p[x] -= lr * (mx / bc1) / (sqrtf(vx / bc2) + eps);
}

__global__ void standardise(const float* __restrict__ X, int n, int F, const float* __restrict__ mu,
                            const float* __restrict__ inv_sigma, float* __restrict__ out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n * F) return;
  const int f = x % F;
  out[x] = (X[x] - mu[f]) * inv_sigma[f];
}

size_t dense_smem(int fin, int fout) { return sizeof(float) * (size_t)(fout * fin + ROWS * fin); }

}  // namespace

cudaError_t mlp_standardise(const float* X, int n, int F, const float* mu, const float* inv_sigma, float* out,
                            cudaStream_t st) {
  standardise<<<ceil_div(n * F, 256), 256, 0, st>>>(X, n, F, mu, inv_sigma, out);
  return cudaGetLastError();
}

cudaError_t mlp_forward(const MlpDims& d, const float* P, const float* X, int n, MlpWork& w, float* y, cudaStream_t st) {
  const int F = d.F, H = d.H;
  const float *W1 = P, *b1 = W1 + H * F, *W2 = b1 + H, *b2 = W2 + H * H, *W3 = b2 + H, *b3 = W3 + H;
  const unsigned g = (unsigned)ceil_div(n, ROWS);
  dense_fwd<<<g, 128, dense_smem(F, H), st>>>(X, n, F, W1, b1, H, w.Z1, w.A1, 1);
  dense_fwd<<<g, 128, dense_smem(H, H), st>>>(w.A1, n, H, W2, b2, H, w.Z2, w.A2, 1);
  dense_fwd<<<g, 128, dense_smem(H, 1), st>>>(w.A2, n, H, W3, b3, 1, nullptr, y, 0);
  return cudaGetLastError();
}

cudaError_t mlp_gradient(const MlpDims& d, const float* P, const float* X, const float* t, int n, MlpWork& w,
                         float* G, float* loss, cudaStream_t st) {
  const int F = d.F, H = d.H;
  const float *W1 = P, *W2 = W1 + H * F + H, *W3 = W2 + H * H + H;
  float *gW1 = G, *gb1 = gW1 + H * F, *gW2 = gb1 + H, *gb2 = gW2 + H * H, *gW3 = gb2 + H, *gb3 = gW3 + H;
  cudaError_t e = mlp_forward(d, P, X, n, w, w.y, st);
  if (e != cudaSuccess) return e;
  const int nb = ceil_div(n, 256);
  mse_grad<<<nb, 256, 0, st>>>(w.y, t, n, w.dy, w.partial);
  sum_partials<<<1, 32, 0, st>>>(w.partial, nb, n, loss);
  // layer 3
  weight_grad<<<ceil_div(H, 128), 128, 0, st>>>(w.dy, n, 1, w.A2, H, gW3);
  weight_grad<<<1, 128, 0, st>>>(w.dy, n, 1, nullptr, H, gb3);
  input_grad<<<ceil_div(n * H, 256), 256, 0, st>>>(w.dy, n, 1, W3, H, w.Z2, w.dZ2);
  // layer 2
  weight_grad<<<ceil_div(H * H, 128), 128, 0, st>>>(w.dZ2, n, H, w.A1, H, gW2);
  weight_grad<<<ceil_div(H, 128), 128, 0, st>>>(w.dZ2, n, H, nullptr, H, gb2);
  input_grad<<<ceil_div(n * H, 256), 256, 0, st>>>(w.dZ2, n, H, W2, H, w.Z1, w.dZ1);
  // layer 1
  weight_grad<<<ceil_div(H * F, 128), 128, 0, st>>>(w.dZ1, n, H, X, F, gW1);
  weight_grad<<<ceil_div(H, 128), 128, 0, st>>>(w.dZ1, n, H, nullptr, F, gb1);
  return cudaGetLastError();
}

cudaError_t mlp_adam(float* P, const float* G, float* m, float* v, int count, float lr, float b1, float b2, float eps,
                     int step, cudaStream_t st) {
  const float bc1 = 1.0f - powf(b1, (float)step), bc2 = 1.0f - powf(b2, (float)step);
  adam<<<ceil_div(count, 256), 256, 0, st>>>(P, G, m, v, count, lr, b1, b2, eps, bc1, bc2);
  return cudaGetLastError();
}

}  // namespace oec
