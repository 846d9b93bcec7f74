// k_vadvc.cu - horizontal diffusion of u and v followed by implicit vertical
// advection: per (i, j) column a tridiagonal system
//   a_k x_{k-1} + b_k x_k + c_k x_{k+1} = d_k
// with wf(k) = (w + w(i+1))/2, a_k = -wf(k)/4 (k >= 1), c_k = wf(k+1)/4
// (k <= K-2), b_k = dtr + |a_k| + |c_k| (strictly diagonally dominant),
// d_k = dtr*phi_k - (a_k (phi_{k-1} - phi_k) + c_k (phi_{k+1} - phi_k))/2 with
// the column-end terms left out, solved by the Thomas algorithm (forward
// elimination, back substitution; the paper names Thomas for vertical implicit
// integration in §VII-B) for phi = hdiff(u) and hdiff(v) with one matrix.
//
// T is the storage/stencil type, R the type of the Thomas recurrence (double
// in both precisions: FP32 fields keep the recurrence in FP64).
//
// Fused form: one CTA owns TI x TJ columns, a thread per column. Marching up
// the column, the CTA evaluates hdiff of u and v one level ahead in shared
// memory (the producer inlined into the sweep, paper §V-A), builds row k and
// eliminates it; c'_k, d'_k go to a scratch array (R, layout [3][k][column])
// that the back substitution reads on the way down.
// Staged form: the hdiff kernel writes hdiff(u), hdiff(v) to scratch over the
// domain, then a column kernel runs the sweep.
#include "kcommon.cuh"
#include "kernels.h"

namespace oec {
namespace {

template <typename T>
struct HV {
  const T* u; const T* v; const T* w; const T* coeff;
  T* uo; T* vo;
  int ni, nj, nk;
  int64_t sj, sk;
};

// One row of the system and its right-hand sides for both fields.
template <typename T>
__device__ __forceinline__ void hv_row(bool lo, bool hi, T wf_c, T wf_p, T dtr, T um, T uc, T up, T vm, T vc, T vp,
                                       T& a, T& b, T& c, T& du, T& dv) {
  a = lo ? T(-0.25) * wf_c : T(0);
  c = hi ? T(0.25) * wf_p : T(0);
  b = dtr + fabs(a) + fabs(c);
  if (lo && hi) {
    du = dtr * uc - T(0.5) * (a * (um - uc) + c * (up - uc));
    dv = dtr * vc - T(0.5) * (a * (vm - vc) + c * (vp - vc));
  } else if (hi) {
    du = dtr * uc - T(0.5) * (c * (up - uc));
    dv = dtr * vc - T(0.5) * (c * (vp - vc));
  } else if (lo) {
    du = dtr * uc - T(0.5) * (a * (um - uc));
    dv = dtr * vc - T(0.5) * (a * (vm - vc));
  } else {
    du = dtr * uc;
    dv = dtr * vc;
  }
}

template <typename T, typename R, int TI, int TJ>
__global__ void __launch_bounds__(TI * TJ)
hv_fused_kernel(HV<T> p, T dtr, R* __restrict__ scr) {
  constexpr int NT = TI * TJ, WI = TI + 4, WJ = TJ + 4;
  __shared__ T s_in[2][WJ][WI];
  __shared__ T s_lap[2][TJ + 2][TI + 2];
  __shared__ T s_flx[2][TJ][TI + 1];
  __shared__ T s_fly[2][TJ + 1][TI];
  const int tid = threadIdx.x, tx = tid % TI, ty = tid / TI;
  const int i0 = blockIdx.x * TI, j0 = blockIdx.y * TJ;
  const int vi = min(TI, p.ni - i0), vj = min(TJ, p.nj - j0);
  const bool active = tx < vi && ty < vj;
  const int i = i0 + tx, j = j0 + ty;
  const int nk = p.nk;
  const int64_t ncol = (int64_t)p.ni * p.nj, col = (int64_t)j * p.ni + i;
  const int64_t plane = ncol * nk;

  // hdiff of u and v at level k for every column of the tile (all threads call)
  auto level = [&](int k, T& ud, T& vd) {
    const int64_t base = (int64_t)k * p.sk + (int64_t)(j0 - 2) * p.sj + (i0 - 2);
    for (int idx = tid; idx < 2 * WI * WJ; idx += NT) {
      const int f = idx / (WI * WJ), rem = idx - f * WI * WJ, r = rem / WI, c = rem - r * WI;
      if (c < vi + 4 && r < vj + 4) s_in[f][r][c] = ldg((f ? p.v : p.u) + base + (int64_t)r * p.sj + c);
    }
    __syncthreads();
    for (int idx = tid; idx < 2 * (TI + 2) * (TJ + 2); idx += NT) {
      const int f = idx / ((TI + 2) * (TJ + 2)), rem = idx - f * (TI + 2) * (TJ + 2);
      const int r = rem / (TI + 2), c = rem - r * (TI + 2);
      if (c < vi + 2 && r < vj + 2)
        s_lap[f][r][c] = hd_lap(s_in[f][r + 1][c + 1], s_in[f][r + 1][c], s_in[f][r + 1][c + 2], s_in[f][r][c + 1],
                                s_in[f][r + 2][c + 1]);
    }
    __syncthreads();
    for (int idx = tid; idx < 2 * (TI + 1) * TJ; idx += NT) {
      const int f = idx / ((TI + 1) * TJ), rem = idx - f * (TI + 1) * TJ, r = rem / (TI + 1), c = rem - r * (TI + 1);
      if (c < vi + 1 && r < vj)
        s_flx[f][r][c] = hd_flux(s_lap[f][r + 1][c + 1], s_lap[f][r + 1][c], s_in[f][r + 2][c + 2], s_in[f][r + 2][c + 1]);
    }
    for (int idx = tid; idx < 2 * TI * (TJ + 1); idx += NT) {
      const int f = idx / (TI * (TJ + 1)), rem = idx - f * TI * (TJ + 1), r = rem / TI, c = rem - r * TI;
      if (c < vi && r < vj + 1)
        s_fly[f][r][c] = hd_flux(s_lap[f][r + 1][c + 1], s_lap[f][r][c + 1], s_in[f][r + 2][c + 2], s_in[f][r + 1][c + 2]);
    }
    __syncthreads();
    if (active) {
      const T cf = ldg(p.coeff + (int64_t)k * p.sk + (int64_t)j * p.sj + i);
      ud = hd_out(s_in[0][ty + 2][tx + 2], cf, s_flx[0][ty][tx + 1], s_flx[0][ty][tx], s_fly[0][ty + 1][tx], s_fly[0][ty][tx]);
      vd = hd_out(s_in[1][ty + 2][tx + 2], cf, s_flx[1][ty][tx + 1], s_flx[1][ty][tx], s_fly[1][ty + 1][tx], s_fly[1][ty][tx]);
    }
    __syncthreads();
  };
  auto wf = [&](int k) -> T {
    if (!active) return T(0);
    const T* q = p.w + (int64_t)k * p.sk + (int64_t)j * p.sj + i;
    return T(0.5) * (ldg(q) + ldg(q + 1));
  };

  T um = 0, uc = 0, up = 0, vm = 0, vc = 0, vp = 0;
  level(0, uc, vc);
  if (nk > 1) level(1, up, vp);
  T wf_c = wf(0), wf_p = nk > 1 ? wf(1) : T(0);
  R cp = 0, dpu = 0, dpv = 0;
  for (int k = 0; k < nk; ++k) {
    T a, b, c, du, dv;
    hv_row(k > 0, k < nk - 1, wf_c, wf_p, dtr, um, uc, up, vm, vc, vp, a, b, c, du, dv);
    const R m = k == 0 ? R(b) : R(b) - R(a) * cp;
    const R inv = R(1) / m;
    cp = R(c) * inv;
    dpu = (R(du) - R(a) * dpu) * inv;
    dpv = (R(dv) - R(a) * dpv) * inv;
    if (active) {
      R* s = scr + (int64_t)k * ncol + col;
      s[0] = cp;
      s[plane] = dpu;
      s[2 * plane] = dpv;
    }
    um = uc; uc = up; vm = vc; vc = vp;
    wf_c = wf_p;
    if (k + 2 < nk) {
      level(k + 2, up, vp);
      wf_p = wf(k + 2);
    }
  }
  if (!active) return;
  R xu = dpu, xv = dpv;
  int64_t o = (int64_t)(nk - 1) * p.sk + (int64_t)j * p.sj + i;
  p.uo[o] = T(xu);
  p.vo[o] = T(xv);
  for (int k = nk - 2; k >= 0; --k) {
    const R* s = scr + (int64_t)k * ncol + col;
    const R ck = s[0];
    xu = s[plane] - ck * xu;
    xv = s[2 * plane] - ck * xv;
    o -= p.sk;
    p.uo[o] = T(xu);
    p.vo[o] = T(xv);
  }
}

// Staged form, second kernel: the column sweep over precomputed hdiff(u),
// hdiff(v) (ud, vd: domain layout, pitch ni, plane ni*nj).
template <typename T, typename R>
__global__ void vadvc_kernel(HV<T> p, const T* __restrict__ ud, const T* __restrict__ vd, T dtr, R* __restrict__ scr) {
  const int64_t ncol = (int64_t)p.ni * p.nj;
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= ncol) return;
  const int i = int(col % p.ni), j = int(col / p.ni);
  const int nk = p.nk;
  const int64_t plane = ncol * nk;
  auto wf = [&](int k) -> T {
    const T* q = p.w + (int64_t)k * p.sk + (int64_t)j * p.sj + i;
    return T(0.5) * (ldg(q) + ldg(q + 1));
  };
  T um = 0, uc = ldg(ud + col), up = nk > 1 ? ldg(ud + ncol + col) : T(0);
  T vm = 0, vc = ldg(vd + col), vp = nk > 1 ? ldg(vd + ncol + col) : T(0);
  T wf_c = wf(0), wf_p = nk > 1 ? wf(1) : T(0);
  R cp = 0, dpu = 0, dpv = 0;
  for (int k = 0; k < nk; ++k) {
    T a, b, c, du, dv;
    hv_row(k > 0, k < nk - 1, wf_c, wf_p, dtr, um, uc, up, vm, vc, vp, a, b, c, du, dv);
    const R m = k == 0 ? R(b) : R(b) - R(a) * cp;
    const R inv = R(1) / m;
    cp = R(c) * inv;
    dpu = (R(du) - R(a) * dpu) * inv;
    dpv = (R(dv) - R(a) * dpv) * inv;
    R* s = scr + (int64_t)k * ncol + col;
    s[0] = cp;
    s[plane] = dpu;
    s[2 * plane] = dpv;
    um = uc; uc = up; vm = vc; vc = vp;
    wf_c = wf_p;
    if (k + 2 < nk) {
      up = ldg(ud + (int64_t)(k + 2) * ncol + col);
      vp = ldg(vd + (int64_t)(k + 2) * ncol + col);
      wf_p = wf(k + 2);
    }
  }
  R xu = dpu, xv = dpv;
  int64_t o = (int64_t)(nk - 1) * p.sk + (int64_t)j * p.sj + i;
  p.uo[o] = T(xu);
  p.vo[o] = T(xv);
  for (int k = nk - 2; k >= 0; --k) {
    const R* s = scr + (int64_t)k * ncol + col;
    const R ck = s[0];
    xu = s[plane] - ck * xu;
    xv = s[2 * plane] - ck * xv;
    o -= p.sk;
    p.uo[o] = T(xu);
    p.vo[o] = T(xv);
  }
}

size_t elem(int dtype) { return dtype == OEC_F64 ? 8 : 4; }

struct Layout {
  size_t thomas, ud, vd, total;
};
Layout layout(const oec_schedule& s, int dtype, const Dom& d) {
  const size_t pts = size_t(d.ni) * d.nj * d.nk;
  Layout l;
  l.thomas = 0;
  l.ud = align_up(3 * sizeof(double) * pts, 256);
  if (s.fusion == OEC_FUSE_NONE) {
    l.vd = align_up(l.ud + elem(dtype) * pts, 256);
    l.total = align_up(l.vd + elem(dtype) * pts, 256);
  } else {
    l.vd = l.ud;
    l.total = l.ud;
  }
  return l;
}

#define OEC_HV_TILES(X) X(32, 1) X(32, 2) X(32, 4) X(64, 1) X(64, 2) X(128, 1)

template <typename T>
cudaError_t dispatch(const oec_schedule& s, int dtype, const Dom& d, const HV<T>& p, double dtr, char* scratch,
                     cudaStream_t st) {
  Layout l = layout(s, dtype, d);
  double* scr = (double*)(scratch + l.thomas);
  if (s.fusion == OEC_FUSE_NONE) {
    T* ud = (T*)(scratch + l.ud);
    T* vd = (T*)(scratch + l.vd);
    // hdiff(u) and hdiff(v) into domain-layout temporaries: the fused hdiff
    // kernel with the temporaries' strides (pitch ni, plane ni*nj)
    oec_schedule hs{};
    hs.fusion = OEC_FUSE_INLINE;
    hs.staging = OEC_STAGE_SMEM;
    hs.tile_i = 64;
    hs.tile_j = 4;
    hs.unroll = 1;
    cudaError_t e = hdiff_launch_strided(hs, dtype, d, p.u, p.coeff, ud, d.ni, (int64_t)d.ni * d.nj, st);
    if (e != cudaSuccess) return e;
    e = hdiff_launch_strided(hs, dtype, d, p.v, p.coeff, vd, d.ni, (int64_t)d.ni * d.nj, st);
    if (e != cudaSuccess) return e;
    const int64_t ncol = (int64_t)d.ni * d.nj;
    vadvc_kernel<T, double><<<(unsigned)((ncol + 127) / 128), 128, 0, st>>>(p, ud, vd, T(dtr), scr);
    return cudaGetLastError();
  }
#define X(a, b)                                                                                  \
  if (s.tile_i == a && s.tile_j == b) {                                                          \
    dim3 g(ceil_div(d.ni, a), ceil_div(d.nj, b));                                                \
    hv_fused_kernel<T, double, a, b><<<g, a * b, 0, st>>>(p, T(dtr), scr);                       \
    return cudaGetLastError();                                                                   \
  }
  OEC_HV_TILES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace

bool hdiff_vadvc_schedule_ok(const oec_schedule& s, std::string& why) {
  if (s.fusion == OEC_FUSE_NONE) return true;
  if (s.fusion != OEC_FUSE_INLINE) { why = "fusion must be OEC_FUSE_INLINE or OEC_FUSE_NONE"; return false; }
#define X(a, b) if (s.tile_i == a && s.tile_j == b) return true;
  OEC_HV_TILES(X)
#undef X
  why = "hdiff+vadvc column tiles: 32x1, 32x2, 32x4, 64x1, 64x2, 128x1";
  return false;
}

size_t hdiff_vadvc_scratch_bytes(const oec_schedule& s, int dtype, const Dom& d) { return layout(s, dtype, d).total; }

cudaError_t hdiff_vadvc_launch(const oec_schedule& s, int dtype, const Dom& d, const void* u, const void* v,
                               const void* w, const void* coeff, void* u_out, void* v_out, double dtr, void* scratch,
                               cudaStream_t st) {
  if (dtype == OEC_F64) {
    HV<double> p{(const double*)u, (const double*)v, (const double*)w, (const double*)coeff,
                 (double*)u_out, (double*)v_out, d.ni, d.nj, d.nk, d.sj, d.sk};
    return dispatch<double>(s, dtype, d, p, dtr, (char*)scratch, st);
  }
  HV<float> p{(const float*)u, (const float*)v, (const float*)w, (const float*)coeff,
              (float*)u_out, (float*)v_out, d.ni, d.nj, d.nk, d.sj, d.sk};
  return dispatch<float>(s, dtype, d, p, dtr, (char*)scratch, st);
}

}  // namespace oec
