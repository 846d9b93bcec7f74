// k_hdiff_vec.cu - horizontal diffusion on vectorised warp rows, for fields
// whose rows are 16-byte aligned: OEC_STAGE_WARP (each warp loads its rows
// with 16-byte vector loads, the next levels held in registers) and
// OEC_STAGE_TMA (a CTA's window of every level copied by the tensor memory
// accelerator into a shared-memory ring, one cp.async.bulk.tensor per level,
// completion tracked on an mbarrier). Both evaluate the same per-warp row
// arithmetic (vec_rows): lap -> limited fluxes -> out, paper Table II hdiffsa,
// each Laplacian and flux once per column (stencil inlining, §V-A).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "arith.cuh"
#include "kcommon.cuh"
#include "kernels.h"
#include "tma.cuh"
#include "k_hdiff_vec.cuh"

namespace oec {
namespace {

// bounded-wait give-ups (see device_wait_timeouts)
__device__ unsigned g_wait_timeouts;

// One CTA of the warp-row kernel: 4 warps, U rows each, k_chunk levels
template <class P, int U, class Off, int NB, bool SEP>
__global__ void __launch_bounds__(128)
hdiff_vec_kernel(const typename P::S* __restrict__ in, const typename P::S* __restrict__ coeff,
                 typename P::S* __restrict__ out, int ni, int nj, int nk, int64_t sj, int64_t sk, int kchunk,
                 int64_t osj, int64_t osk, int nkz, const typename P::S* __restrict__ in1,
                 typename P::S* __restrict__ out1) {
  hdiff_vec_block<P, U, Off, NB, SEP>(in, coeff, out, ni, nj, nk, sj, sk, kchunk, osj, osk, nkz, in1, out1,
                                      blockIdx.x, blockIdx.y, blockIdx.z);
}

template <class P, int U>
cudaError_t run_vec(const oec_schedule& s, const Dom& d, const typename P::S* in, const typename P::S* coeff,
                    typename P::S* out, cudaStream_t st) {
  constexpr int W = 32 * Vec16<typename P::S>::V;
  const int kc = (s.k_chunk <= 0 || s.k_chunk > d.nk) ? d.nk : s.k_chunk;
  dim3 g(ceil_div(d.ni, W), ceil_div(d.nj, 4 * U), ceil_div(d.nk, kc));
  if (use_int32(s, d))
    hdiff_vec_kernel<P, U, int, 2, false><<<g, 128, 0, st>>>(in, coeff, out, d.ni, d.nj, d.nk, d.sj, d.sk, kc, 0, 0, 0,
                                                             nullptr, nullptr);
  else
    hdiff_vec_kernel<P, U, int64_t, 2, false><<<g, 128, 0, st>>>(in, coeff, out, d.ni, d.nj, d.nk, d.sj, d.sk, kc, 0,
                                                                 0, 0, nullptr, nullptr);
  launched(st);
  return cudaGetLastError();
}

// the vector-row kernel as the staged producer: in0 -> out0 and in1 -> out1
// (domain layout osj, osk) in one launch
template <class P, int U>
cudaError_t run_vec_to(const oec_schedule& s, const Dom& d, int64_t osj, int64_t osk, const typename P::S* in0,
                       const typename P::S* in1, const typename P::S* coeff, typename P::S* out0,
                       typename P::S* out1, cudaStream_t st) {
  constexpr int W = 32 * Vec16<typename P::S>::V;
  const int kc = (s.k_chunk <= 0 || s.k_chunk > d.nk) ? d.nk : s.k_chunk, nkz = ceil_div(d.nk, kc);
  dim3 g(ceil_div(d.ni, W), ceil_div(d.nj, 4 * U), 2 * nkz);
  if (use_int32(s, d))
    hdiff_vec_kernel<P, U, int, 2, true><<<g, 128, 0, st>>>(in0, coeff, out0, d.ni, d.nj, d.nk, d.sj, d.sk, kc, osj,
                                                            osk, nkz, in1, out1);
  else
    hdiff_vec_kernel<P, U, int64_t, 2, true><<<g, 128, 0, st>>>(in0, coeff, out0, d.ni, d.nj, d.nk, d.sj, d.sk, kc,
                                                                osj, osk, nkz, in1, out1);
  launched(st);
  return cudaGetLastError();
}

// ---- OEC_STAGE_TMA: tensor-memory-accelerator ring ---------------------------
template <class S, int U>
struct TmaGeom {
  static constexpr int V = Vec16<S>::V, W = 32 * V, TJ = 4 * U;
  static constexpr int BX = W + 2 * V, BY = TJ + 4;                  // window box: columns i0-V .., rows j0-2 ..
  static constexpr int WIN = BX * BY, COE = W * TJ;                  // elements per stage
  static constexpr int STAGE = WIN + COE;
  static constexpr int D = 4;                                        // ring stages
  static constexpr size_t SMEM = size_t(D) * STAGE * sizeof(S) + D * sizeof(unsigned long long);
};

// Persistent: grid = SMs x resident CTAs. The work units are (tile, level)
// pairs, level fastest (a tile is W columns x 4U rows); CTA b streams the
// contiguous range [b N / G, (b+1) N / G). Thread 0 keeps D units of window +
// coeff in flight across tile boundaries: after every warp is done with unit
// u (barrier) it refills that stage with unit u+D. Each warp copies its row
// strip out of the stage into registers and runs vec_rows. A wait that gives
// up counts a timeout, and the CTA stops after waiting (bounded) for the
// copies it still has in flight.
template <class P, int U>
__global__ void __launch_bounds__(128)
hdiff_tma_kernel(const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tco, int cxi, int cyi,
                 int czi, int cxc, int cyc, int czc, typename P::S* __restrict__ out, int ni, int nj, int nk,
                 int64_t sj, int64_t sk, int ntx, long long nunits) {
  typedef typename P::S S;
  typedef TmaGeom<S, U> G;
  constexpr int V = G::V, W = G::W, D = G::D;
  extern __shared__ __align__(128) unsigned char smem[];
  S* ring = reinterpret_cast<S*>(smem);
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + size_t(D) * G::STAGE * sizeof(S));
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const long long u0 = (long long)blockIdx.x * nunits / gridDim.x;
  const long long u1 = (long long)(blockIdx.x + 1) * nunits / gridDim.x;
  auto unit = [&](long long u, int& i0, int& j0, int& k) {
    k = (int)(u % nk);
    const long long t = u / nk;
    i0 = (int)(t % ntx) * W;
    j0 = (int)(t / ntx) * G::TJ;
  };
  if (tid == 0) {
    for (int x = 0; x < D; ++x) mbar_init(smem_u32(&bars[x]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](long long u) {   // thread 0 only
    int i0, j0, k;
    unit(u, i0, j0, k);
    const int sl = (int)((u - u0) % D);
    S* st_ = ring + (size_t)sl * G::STAGE;
    const unsigned bar = smem_u32(&bars[sl]);
    mbar_expect_tx(bar, G::STAGE * sizeof(S));
    tma_load_3d(st_, &tin, cxi + i0 - V, cyi + j0 - 2, czi + k, bar);
    tma_load_3d(st_ + G::WIN, &tco, cxc + i0, cyc + j0, czc + k, bar);
  };
  if (tid == 0)
    for (long long u = u0; u < min(u1, u0 + D); ++u) issue(u);
  long long issued_to = min(u1, u0 + D);   // units [u0, issued_to) have been issued (thread 0's view)
  long long failed_at = -1;
  for (long long u = u0; u < u1; ++u) {
    const int sl = (int)((u - u0) % D);
    const bool ok = mbar_wait(smem_u32(&bars[sl]), (unsigned)(((u - u0) / D) & 1));
    if (__syncthreads_or(!ok)) {
      failed_at = u;
      if (tid == 0) atomicAdd(&g_wait_timeouts, 1u);
      break;
    }
    int i0, j0, k;
    unit(u, i0, j0, k);
    const int c0 = i0 + V * lane, jb = j0 + wid * U;
    const S* stg = ring + (size_t)sl * G::STAGE;
    if (jb < nj) {
      // this warp's strip: window rows wid*U .. wid*U+U+3, columns V + V lane ..
      VecWin<S, U, V> w;
      const S* wrow = stg + (size_t)(wid * U) * G::BX;
#pragma unroll
      for (int r = 0; r < U + 4; ++r)
        vsplit<S, V>(*reinterpret_cast<const typename Vec16<S>::T*>(wrow + r * G::BX + V + V * lane), w.v[r]);
      const int ea_col = lane == 0 ? V - 1 : V + W, eb_col = lane == 0 ? V - 2 : V + W + 1;
#pragma unroll
      for (int r = 0; r < U + 2; ++r) w.ea[r] = wrow[(r + 1) * G::BX + ea_col];
#pragma unroll
      for (int r = 0; r < U; ++r) {
        w.eb[r] = wrow[(r + 2) * G::BX + eb_col];
        vsplit<S, V>(*reinterpret_cast<const typename Vec16<S>::T*>(stg + G::WIN + (size_t)(wid * U + r) * W + V * lane),
                     w.cf[r]);
      }
      vec_rows<P, U>(w, lane, c0, jb, ni, nj, out + ((int64_t)k * sk + (int64_t)jb * sj + c0), sj);
    }
    __syncthreads();   // every warp is done with this stage
    if (tid == 0 && u + D < u1) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      issue(u + D);
      issued_to = u + D + 1;
    }
  }
  if (failed_at >= 0 && tid == 0) {
    // wait (bounded) for the copies still in flight before the CTA exits
    for (long long u = failed_at; u < issued_to; ++u)
      mbar_wait(smem_u32(&bars[(u - u0) % D]), (unsigned)(((u - u0) / D) & 1));
  }
}

template <class P, int U>
cudaError_t run_tma(const oec_schedule& s, const Dom& d, const TmaField& fin, const TmaField& fco,
                    typename P::S* out, cudaStream_t st) {
  typedef typename P::S S;
  typedef TmaGeom<S, U> G;
  if (fin.corner[0] % G::V != 0 || fco.corner[0] % G::V != 0) return cudaErrorMisalignedAddress;
  CUtensorMap tin, tco;
  if (!encode_map<S>(&tin, fin, d.sj, d.sk, G::BX, G::BY) || !encode_map<S>(&tco, fco, d.sj, d.sk, G::W, G::TJ))
    return cudaErrorNotSupported;
  static std::once_flag attr;
  static int per_sm = 1;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(hdiff_tma_kernel<P, U>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, hdiff_tma_kernel<P, U>, 128, G::SMEM) == cudaSuccess && n > 0)
      per_sm = n;
  });
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int ntx = ceil_div(d.ni, G::W), nty = ceil_div(d.nj, G::TJ);
  const long long nunits = (long long)ntx * nty * d.nk;
  const long long grid = std::min<long long>(nunits, (long long)sms * per_sm);
  hdiff_tma_kernel<P, U><<<(unsigned)grid, 128, G::SMEM, st>>>(tin, tco, (int)fin.corner[0], (int)fin.corner[1],
                                                               (int)fin.corner[2], (int)fco.corner[0],
                                                               (int)fco.corner[1], (int)fco.corner[2], out, d.ni,
                                                               d.nj, d.nk, d.sj, d.sk, ntx, nunits);
  launched(st);
  return cudaGetLastError();
}

}  // namespace

// cuTensorMapEncodeTiled from the CUDA driver API, looked up once
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

namespace {
// an mbarrier that nothing arrives on: the wait gives up after `polls` polls,
// counts a timeout and the kernel returns (no copies were issued)
__global__ void wait_selftest_kernel(unsigned polls) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(smem_u32(&bar), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait_n(smem_u32(&bar), 0u, polls)) atomicAdd(&g_wait_timeouts, 1u);
}
}  // namespace

cudaError_t wait_selftest_launch(unsigned polls, cudaStream_t st) {
  wait_selftest_kernel<<<1, 32, 0, st>>>(polls);
  return cudaGetLastError();
}

unsigned* wait_timeout_counter() {
  static unsigned* addr = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_wait_timeouts) == cudaSuccess) addr = (unsigned*)p;
  });
  return addr;
}

cudaError_t hdiff_warp_launch(const oec_schedule& s, int dtype, const Dom& d, const void* in, const void* coeff,
                              void* out, cudaStream_t st) {
#define OEC_VEC_U(P, T)                                                                       \
  switch (s.unroll) {                                                                         \
    case 1: return run_vec<P, 1>(s, d, (const T*)in, (const T*)coeff, (T*)out, st);          \
    case 2: return run_vec<P, 2>(s, d, (const T*)in, (const T*)coeff, (T*)out, st);          \
    case 4: return run_vec<P, 4>(s, d, (const T*)in, (const T*)coeff, (T*)out, st);          \
  }                                                                                           \
  return cudaErrorInvalidValue;
  if (dtype == OEC_F64) {
    if (s.arith == 1) { OEC_VEC_U(P64D, double) }
    OEC_VEC_U(P64, double)
  }
  OEC_VEC_U(P32, float)
#undef OEC_VEC_U
}

cudaError_t hdiff_warp_to_compute(const oec_schedule& s, const Dom& d, int64_t osj, int64_t osk, const float* in0,
                                  const float* in1, const float* coeff, float* out0, float* out1, cudaStream_t st) {
  switch (s.unroll) {
    case 2: return run_vec_to<P32, 2>(s, d, osj, osk, in0, in1, coeff, out0, out1, st);
    case 4: return run_vec_to<P32, 4>(s, d, osj, osk, in0, in1, coeff, out0, out1, st);
    default: return run_vec_to<P32, 1>(s, d, osj, osk, in0, in1, coeff, out0, out1, st);
  }
}

cudaError_t hdiff_tma_launch(const oec_schedule& s, int dtype, const Dom& d, const TmaField& in, const TmaField& coeff,
                             void* out, cudaStream_t st) {
#define OEC_TMA_U(P, T)                                                     \
  switch (s.unroll) {                                                       \
    case 1: return run_tma<P, 1>(s, d, in, coeff, (T*)out, st);             \
    case 2: return run_tma<P, 2>(s, d, in, coeff, (T*)out, st);             \
    case 4: return run_tma<P, 4>(s, d, in, coeff, (T*)out, st);             \
  }                                                                         \
  return cudaErrorInvalidValue;
  if (dtype == OEC_F64) {
    if (s.arith == 1) { OEC_TMA_U(P64D, double) }
    OEC_TMA_U(P64, double)
  }
  OEC_TMA_U(P32, float)
#undef OEC_TMA_U
}

int device_wait_timeouts(cudaStream_t st, unsigned* count) {
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return (int)e;
  unsigned v = 0, zero = 0;
  e = cudaMemcpyFromSymbol(&v, g_wait_timeouts, sizeof(v));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_wait_timeouts, &zero, sizeof(zero));
  *count = v;
  return (int)e;
}

}  // namespace oec
