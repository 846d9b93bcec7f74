// k_hdiff.cu - horizontal diffusion (5-point Laplacian -> i/j fluxes with a sign
// limiter -> flux divergence; the program whose shape Table II lists as hdiffsa)
// in three forms:
//   fused, SMEM staging: each CTA stages an (TI+4) x (TJ+4) input window of one
//     level in shared memory and evaluates every stage once per point of its
//     overlapped tile (overlapped tiling, paper §VII-D), marching over a chunk
//     of levels;
//   fused, REGS staging: every thread recomputes the Laplacians and fluxes it
//     needs (stencil inlining, paper §V-A), U outputs per thread along j
//     sharing their Laplacians (stencil unrolling + CSE, paper §V-A);
//   unfused: one kernel per stencil.apply (lap, flx, fly, out) with the
//     temporaries in device memory over their inferred ranges (paper §V-B),
//     the paper's "original" level (§VII-C).
#include "kcommon.cuh"
#include "kernels.h"

namespace oec {
namespace {

template <typename T, int TI, int TJ>
__global__ void __launch_bounds__(TI * TJ)
hdiff_smem_kernel(const T* __restrict__ in, const T* __restrict__ coeff, T* __restrict__ out, int ni, int nj,
                  int nk, int64_t sj, int64_t sk, int64_t osj, int64_t osk, int kchunk) {
  constexpr int NT = TI * TJ, WI = TI + 4, WJ = TJ + 4;
  __shared__ T s_in[WJ][WI];
  __shared__ T s_lap[TJ + 2][TI + 2];
  __shared__ T s_flx[TJ][TI + 1];
  __shared__ T s_fly[TJ + 1][TI];
  const int tid = threadIdx.x, tx = tid % TI, ty = tid / TI;
  const int i0 = blockIdx.x * TI, j0 = blockIdx.y * TJ;
  const int k0 = blockIdx.z * kchunk, k1 = min(nk, k0 + kchunk);
  const int vi = min(TI, ni - i0), vj = min(TJ, nj - j0);   // valid part of a ragged tile
  for (int k = k0; k < k1; ++k) {
    const T* pin = in + (int64_t)k * sk + (int64_t)(j0 - 2) * sj + (i0 - 2);
    for (int idx = tid; idx < WI * WJ; idx += NT) {
      const int r = idx / WI, c = idx - r * WI;
      if (c < vi + 4 && r < vj + 4) s_in[r][c] = ldg(pin + (int64_t)r * sj + c);
    }
    __syncthreads();
    // lap(i0-1+c, j0-1+r)
    for (int idx = tid; idx < (TI + 2) * (TJ + 2); idx += NT) {
      const int r = idx / (TI + 2), c = idx - r * (TI + 2);
      if (c < vi + 2 && r < vj + 2)
        s_lap[r][c] = hd_lap(s_in[r + 1][c + 1], s_in[r + 1][c], s_in[r + 1][c + 2], s_in[r][c + 1], s_in[r + 2][c + 1]);
    }
    __syncthreads();
    // flx(i0-1+c, j0+r) and fly(i0+c, j0-1+r)
    for (int idx = tid; idx < (TI + 1) * TJ; idx += NT) {
      const int r = idx / (TI + 1), c = idx - r * (TI + 1);
      if (c < vi + 1 && r < vj)
        s_flx[r][c] = hd_flux(s_lap[r + 1][c + 1], s_lap[r + 1][c], s_in[r + 2][c + 2], s_in[r + 2][c + 1]);
    }
    for (int idx = tid; idx < TI * (TJ + 1); idx += NT) {
      const int r = idx / TI, c = idx - r * TI;
      if (c < vi && r < vj + 1)
        s_fly[r][c] = hd_flux(s_lap[r + 1][c + 1], s_lap[r][c + 1], s_in[r + 2][c + 2], s_in[r + 1][c + 2]);
    }
    __syncthreads();
    if (tx < vi && ty < vj) {
      const int64_t o = (int64_t)k * sk + (int64_t)(j0 + ty) * sj + (i0 + tx);
      out[(int64_t)k * osk + (int64_t)(j0 + ty) * osj + (i0 + tx)] =
          hd_out(s_in[ty + 2][tx + 2], ldg(coeff + o), s_flx[ty][tx + 1], s_flx[ty][tx], s_fly[ty + 1][tx], s_fly[ty][tx]);
    }
    __syncthreads();
  }
}

template <typename T, int U>
__global__ void hdiff_regs_kernel(const T* __restrict__ in, const T* __restrict__ coeff, T* __restrict__ out, int ni,
                                  int nj, int nk, int64_t sj, int64_t sk, int64_t osj, int64_t osk, int kchunk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int jb = (blockIdx.y * blockDim.y + threadIdx.y) * U;
  if (i >= ni || jb >= nj) return;
  const int jmax = nj + 1 - jb;          // last row offset inside the halo-2 window
  const int k0 = blockIdx.z * kchunk, k1 = min(nk, k0 + kchunk);
  for (int k = k0; k < k1; ++k) {
    const T* p = in + (int64_t)k * sk + (int64_t)jb * sj + i;
    auto at = [&](int di, int dj) { return ldg(p + (int64_t)min(dj, jmax) * sj + di); };
    T lc[U + 2], lw[U], le[U];   // lap(i, jb-1+r); lap(i-1, jb+r); lap(i+1, jb+r)
#pragma unroll
    for (int r = 0; r < U + 2; ++r) {
      const int dj = r - 1;
      lc[r] = hd_lap(at(0, dj), at(-1, dj), at(1, dj), at(0, dj - 1), at(0, dj + 1));
    }
#pragma unroll
    for (int r = 0; r < U; ++r) {
      lw[r] = hd_lap(at(-1, r), at(-2, r), at(0, r), at(-1, r - 1), at(-1, r + 1));
      le[r] = hd_lap(at(1, r), at(0, r), at(2, r), at(1, r - 1), at(1, r + 1));
    }
#pragma unroll
    for (int r = 0; r < U; ++r) {
      if (jb + r < nj) {
        const T c = at(0, r);
        const T flx = hd_flux(le[r], lc[r + 1], at(1, r), c);
        const T flx_m = hd_flux(lc[r + 1], lw[r], c, at(-1, r));
        const T fly = hd_flux(lc[r + 2], lc[r + 1], at(0, r + 1), c);
        const T fly_m = hd_flux(lc[r + 1], lc[r], c, at(0, r - 1));
        const int64_t o = (int64_t)k * sk + (int64_t)(jb + r) * sj + i;
        out[(int64_t)k * osk + (int64_t)(jb + r) * osj + i] = hd_out(c, ldg(coeff + o), flx, flx_m, fly, fly_m);
      }
    }
  }
}

// ---- unfused: one kernel per stage, temporaries over their inferred ranges ---
// lap over [-1, ni+1) x [-1, nj+1): element (i, j, k) at ((k*(nj+2) + j+1)*(ni+2) + i+1)
template <typename T>
__global__ void hdiff_lap_kernel(const T* __restrict__ in, T* __restrict__ lap, int ni, int nj, int nk, int64_t sj,
                                 int64_t sk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x - 1;
  const int j = blockIdx.y * blockDim.y + threadIdx.y - 1;
  const int k = blockIdx.z;
  if (i >= ni + 1 || j >= nj + 1) return;
  const T* p = in + (int64_t)k * sk + (int64_t)j * sj + i;
  lap[((int64_t)k * (nj + 2) + (j + 1)) * (ni + 2) + (i + 1)] = hd_lap(ldg(p), ldg(p - 1), ldg(p + 1), ldg(p - sj), ldg(p + sj));
}
// flx over [-1, ni) x [0, nj): ((k*nj + j)*(ni+1) + i+1)
template <typename T>
__global__ void hdiff_flx_kernel(const T* __restrict__ in, const T* __restrict__ lap, T* __restrict__ flx, int ni,
                                 int nj, int nk, int64_t sj, int64_t sk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x - 1;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= ni || j >= nj) return;
  const T* p = in + (int64_t)k * sk + (int64_t)j * sj + i;
  const T* l = lap + ((int64_t)k * (nj + 2) + (j + 1)) * (ni + 2) + (i + 1);
  flx[((int64_t)k * nj + j) * (ni + 1) + (i + 1)] = hd_flux(ldg(l + 1), ldg(l), ldg(p + 1), ldg(p));
}
// fly over [0, ni) x [-1, nj): ((k*(nj+1) + j+1)*ni + i)
template <typename T>
__global__ void hdiff_fly_kernel(const T* __restrict__ in, const T* __restrict__ lap, T* __restrict__ fly, int ni,
                                 int nj, int nk, int64_t sj, int64_t sk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y - 1;
  const int k = blockIdx.z;
  if (i >= ni || j >= nj) return;
  const T* p = in + (int64_t)k * sk + (int64_t)j * sj + i;
  const T* l = lap + ((int64_t)k * (nj + 2) + (j + 1)) * (ni + 2) + (i + 1);
  fly[((int64_t)k * (nj + 1) + (j + 1)) * ni + i] = hd_flux(ldg(l + (ni + 2)), ldg(l), ldg(p + sj), ldg(p));
}
template <typename T>
__global__ void hdiff_out_kernel(const T* __restrict__ in, const T* __restrict__ coeff, const T* __restrict__ flx,
                                 const T* __restrict__ fly, T* __restrict__ out, int ni, int nj, int nk, int64_t sj,
                                 int64_t sk, int64_t osj, int64_t osk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= ni || j >= nj) return;
  const int64_t o = (int64_t)k * sk + (int64_t)j * sj + i;
  const T* fx = flx + ((int64_t)k * nj + j) * (ni + 1) + (i + 1);
  const T* fy = fly + ((int64_t)k * (nj + 1) + (j + 1)) * ni + i;
  out[(int64_t)k * osk + (int64_t)j * osj + i] = hd_out(ldg(in + o), ldg(coeff + o), ldg(fx), ldg(fx - 1), ldg(fy), ldg(fy - ni));
}

struct Tmp {
  size_t lap, flx, fly, total;
};
Tmp unfused_layout(int dtype, const Dom& d) {
  const size_t e = dtype == OEC_F64 ? 8 : 4;
  Tmp t;
  t.lap = 0;
  t.flx = align_up(t.lap + e * size_t(d.ni + 2) * (d.nj + 2) * d.nk, 256);
  t.fly = align_up(t.flx + e * size_t(d.ni + 1) * d.nj * d.nk, 256);
  t.total = align_up(t.fly + e * size_t(d.ni) * (d.nj + 1) * d.nk, 256);
  return t;
}

template <typename T>
cudaError_t run_unfused(const Dom& d, int64_t osj, int64_t osk, const T* in, const T* coeff, T* out, char* scratch,
                        cudaStream_t st) {
  Tmp t = unfused_layout(sizeof(T) == 8 ? OEC_F64 : OEC_F32, d);
  T* lap = (T*)(scratch + t.lap);
  T* flx = (T*)(scratch + t.flx);
  T* fly = (T*)(scratch + t.fly);
  dim3 b(32, 8);
  hdiff_lap_kernel<T><<<dim3(ceil_div(d.ni + 2, 32), ceil_div(d.nj + 2, 8), d.nk), b, 0, st>>>(in, lap, d.ni, d.nj, d.nk, d.sj, d.sk);
  hdiff_flx_kernel<T><<<dim3(ceil_div(d.ni + 1, 32), ceil_div(d.nj, 8), d.nk), b, 0, st>>>(in, lap, flx, d.ni, d.nj, d.nk, d.sj, d.sk);
  hdiff_fly_kernel<T><<<dim3(ceil_div(d.ni, 32), ceil_div(d.nj + 1, 8), d.nk), b, 0, st>>>(in, lap, fly, d.ni, d.nj, d.nk, d.sj, d.sk);
  hdiff_out_kernel<T><<<dim3(ceil_div(d.ni, 32), ceil_div(d.nj, 8), d.nk), b, 0, st>>>(in, coeff, flx, fly, out, d.ni, d.nj, d.nk, d.sj, d.sk, osj, osk);
  return cudaGetLastError();
}

int kchunk_of(const oec_schedule& s, int nk) { return (s.k_chunk <= 0 || s.k_chunk > nk) ? nk : s.k_chunk; }

template <typename T, int TI, int TJ>
cudaError_t run_smem(const oec_schedule& s, const Dom& d, int64_t osj, int64_t osk, const T* in, const T* coeff, T* out,
                     cudaStream_t st) {
  const int kc = kchunk_of(s, d.nk);
  dim3 g(ceil_div(d.ni, TI), ceil_div(d.nj, TJ), ceil_div(d.nk, kc));
  hdiff_smem_kernel<T, TI, TJ><<<g, TI * TJ, 0, st>>>(in, coeff, out, d.ni, d.nj, d.nk, d.sj, d.sk, osj, osk, kc);
  return cudaGetLastError();
}

template <typename T, int U>
cudaError_t run_regs(const oec_schedule& s, const Dom& d, int64_t osj, int64_t osk, const T* in, const T* coeff, T* out,
                     cudaStream_t st) {
  const int kc = kchunk_of(s, d.nk);
  dim3 b(s.tile_i, s.tile_j / U);
  dim3 g(ceil_div(d.ni, s.tile_i), ceil_div(d.nj, s.tile_j), ceil_div(d.nk, kc));
  hdiff_regs_kernel<T, U><<<g, b, 0, st>>>(in, coeff, out, d.ni, d.nj, d.nk, d.sj, d.sk, osj, osk, kc);
  return cudaGetLastError();
}

#define OEC_SMEM_TILES(X) X(32, 4) X(32, 8) X(64, 2) X(64, 4) X(64, 8) X(128, 2) X(128, 4)

template <typename T>
cudaError_t dispatch(const oec_schedule& s, const Dom& d, int64_t osj, int64_t osk, const T* in, const T* coeff, T* out,
                     void* scratch, cudaStream_t st) {
  if (s.fusion == OEC_FUSE_NONE) return run_unfused<T>(d, osj, osk, in, coeff, out, (char*)scratch, st);
  if (s.staging == OEC_STAGE_SMEM) {
#define X(a, b) if (s.tile_i == a && s.tile_j == b) return run_smem<T, a, b>(s, d, osj, osk, in, coeff, out, st);
    OEC_SMEM_TILES(X)
#undef X
    return cudaErrorInvalidValue;
  }
  switch (s.unroll) {
    case 1: return run_regs<T, 1>(s, d, osj, osk, in, coeff, out, st);
    case 2: return run_regs<T, 2>(s, d, osj, osk, in, coeff, out, st);
    case 4: return run_regs<T, 4>(s, d, osj, osk, in, coeff, out, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool hdiff_schedule_ok(const oec_schedule& s, std::string& why) {
  if (s.fusion == OEC_FUSE_NONE) return true;
  if (s.fusion != OEC_FUSE_INLINE) { why = "fusion must be OEC_FUSE_INLINE or OEC_FUSE_NONE"; return false; }
  if (s.k_chunk < 0) { why = "k_chunk must be >= 0"; return false; }
  if (s.staging == OEC_STAGE_SMEM) {
#define X(a, b) if (s.tile_i == a && s.tile_j == b && s.unroll == 1) return true;
    OEC_SMEM_TILES(X)
#undef X
    why = "SMEM staging supports tiles 32x4, 32x8, 64x2, 64x4, 64x8, 128x2, 128x4 with unroll 1";
    return false;
  }
  if (s.staging != OEC_STAGE_REGS) { why = "unknown staging"; return false; }
  if (s.unroll != 1 && s.unroll != 2 && s.unroll != 4) { why = "unroll must be 1, 2 or 4"; return false; }
  if (s.tile_i < 16 || s.tile_i > 256 || s.tile_i % 16) { why = "tile_i must be a multiple of 16 in [16, 256]"; return false; }
  if (s.tile_j < s.unroll || s.tile_j % s.unroll || s.tile_j > 64) { why = "tile_j must be a multiple of unroll, <= 64"; return false; }
  if (s.tile_i * (s.tile_j / s.unroll) > 1024) { why = "more than 1024 threads per CTA"; return false; }
  return true;
}

size_t hdiff_scratch_bytes(const oec_schedule& s, int dtype, const Dom& d) {
  return s.fusion == OEC_FUSE_NONE ? unfused_layout(dtype, d).total : 0;
}

cudaError_t hdiff_launch(const oec_schedule& s, int dtype, const Dom& d, const void* in, const void* coeff, void* out,
                         void* scratch, cudaStream_t st) {
  if (dtype == OEC_F64)
    return dispatch<double>(s, d, d.sj, d.sk, (const double*)in, (const double*)coeff, (double*)out, scratch, st);
  return dispatch<float>(s, d, d.sj, d.sk, (const float*)in, (const float*)coeff, (float*)out, scratch, st);
}

cudaError_t hdiff_launch_strided(const oec_schedule& s, int dtype, const Dom& d, const void* in, const void* coeff,
                                 void* out, int64_t osj, int64_t osk, cudaStream_t st) {
  if (s.fusion == OEC_FUSE_NONE) return cudaErrorInvalidValue;   // needs scratch; not used here
  if (dtype == OEC_F64)
    return dispatch<double>(s, d, osj, osk, (const double*)in, (const double*)coeff, (double*)out, nullptr, st);
  return dispatch<float>(s, d, osj, osk, (const float*)in, (const float*)coeff, (float*)out, nullptr, st);
}

}  // namespace oec
