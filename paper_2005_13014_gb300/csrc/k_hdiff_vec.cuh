// k_hdiff_vec.cuh - the vectorised warp-row arithmetic of horizontal
// diffusion (OEC_STAGE_WARP / OEC_STAGE_TMA, k_hdiff_vec.cu) and the warp-row
// kernel's block body, shared with the persistent staged batch kernel
// (k_vadvc.cu). Rows must be 16-byte aligned (checked by the callers).
#pragma once

#include "arith.cuh"
#include "kcommon.cuh"

namespace oec {
namespace {

template <class S> struct Vec16;
template <> struct Vec16<float> { typedef float4 T; static constexpr int V = 4; };
template <> struct Vec16<double> { typedef double2 T; static constexpr int V = 2; };
template <class S, int V> __device__ __forceinline__ void vsplit(const typename Vec16<S>::T& t, S (&d)[V]);
template <> __device__ __forceinline__ void vsplit<float, 4>(const float4& t, float (&d)[4]) {
  d[0] = t.x; d[1] = t.y; d[2] = t.z; d[3] = t.w;
}
template <> __device__ __forceinline__ void vsplit<double, 2>(const double2& t, double (&d)[2]) {
  d[0] = t.x; d[1] = t.y;
}
template <class S, int V> __device__ __forceinline__ typename Vec16<S>::T vjoin(const S (&d)[V]);
template <> __device__ __forceinline__ float4 vjoin<float, 4>(const float (&d)[4]) {
  return make_float4(d[0], d[1], d[2], d[3]);
}
template <> __device__ __forceinline__ double2 vjoin<double, 2>(const double (&d)[2]) { return make_double2(d[0], d[1]); }

// The values one warp row-strip of one level needs: U output rows of W = 32 V
// columns (lane l: columns c0 = i0 + V l .. c0 + V - 1).
template <class S, int U, int V>
struct VecWin {
  S v[U + 4][V];   // rows jb-2 .. jb+U+1, this lane's columns
  S ea[U + 2];     // lane 0: column i0-1, lane 31: column i0+W; rows jb-1 .. jb+U
  S eb[U];         // lane 0: column i0-2, lane 31: column i0+W+1; rows jb .. jb+U-1
  S cf[U][V];      // coeff, rows jb .. jb+U-1
};

// The arithmetic of one warp row-strip: Laplacians of rows jb-1 .. jb+U at
// the lane's columns (neighbours across the vector boundary from the adjacent
// lanes; lanes 0 and 31 use their outer columns and evaluate the Laplacian
// outside the warp), fluxes once per column, outputs written to q0 + o sj
// (row jb+o) where the point lies in the domain.
template <class P, int U>
__device__ __forceinline__ void vec_rows(const VecWin<typename P::S, U, Vec16<typename P::S>::V>& w, int lane, int c0,
                                         int jb, int ni, int nj, typename P::S* q0, int64_t sj) {
  typedef typename P::S S;
  typedef typename P::C C;
  typedef typename Vec16<S>::T VT;
  constexpr int V = Vec16<S>::V;
  auto at = [&](int r, int x) { return cvt<C>(w.v[r][x]); };
  C lap[U + 2][V], inr[U + 2];
#pragma unroll
  for (int q = 0; q < U + 2; ++q) {
    const int r = q + 1;
    C left = shfl_up_(at(r, V - 1), 1), right = shfl_down_(at(r, 0), 1);
    if (lane == 0) left = cvt<C>(w.ea[q]);
    if (lane == 31) right = cvt<C>(w.ea[q]);
    inr[q] = right;
#pragma unroll
    for (int x = 0; x < V; ++x)
      lap[q][x] = hlap(at(r, x), x > 0 ? at(r, x - 1) : left, x < V - 1 ? at(r, x + 1) : right, at(r - 1, x),
                       at(r + 1, x));
  }
  C fly[U + 1][V];   // between rows jb-1+q and jb+q
#pragma unroll
  for (int q = 0; q < U + 1; ++q)
#pragma unroll
    for (int x = 0; x < V; ++x) fly[q][x] = hflux(lap[q + 1][x], lap[q][x], at(q + 2, x), at(q + 1, x));
  const bool vout_full = c0 + V - 1 < ni;
#pragma unroll
  for (int o = 0; o < U; ++o) {
    const int q = o + 1, r = o + 2;
    const C le = lane == 0 ? hlap(cvt<C>(w.ea[q]), cvt<C>(w.eb[o]), at(r, 0), cvt<C>(w.ea[q - 1]), cvt<C>(w.ea[q + 1]))
                           : hlap(cvt<C>(w.ea[q]), at(r, V - 1), cvt<C>(w.eb[o]), cvt<C>(w.ea[q - 1]), cvt<C>(w.ea[q + 1]));
    C lapr = shfl_down_(lap[q][0], 1);
    if (lane == 31) lapr = le;
    C flx[V];
#pragma unroll
    for (int x = 0; x < V; ++x)
      flx[x] = x < V - 1 ? hflux(lap[q][x + 1], lap[q][x], at(r, x + 1), at(r, x))
                         : hflux(lapr, lap[q][x], inr[q], at(r, x));
    C flxl = shfl_up_(flx[V - 1], 1);
    if (lane == 0) flxl = hflux(lap[q][0], le, at(r, 0), cvt<C>(w.ea[q]));
    if (jb + o < nj) {
      S res[V];
#pragma unroll
      for (int x = 0; x < V; ++x)
        res[x] = cvt<S>(hout(at(r, x), cvt<C>(w.cf[o][x]), flx[x], x > 0 ? flx[x - 1] : flxl, fly[o + 1][x], fly[o][x]));
      S* q2 = q0 + (int64_t)o * sj;
      if (vout_full) {
        *reinterpret_cast<VT*>(q2) = vjoin<S, V>(res);
      } else {
#pragma unroll
        for (int x = 0; x < V; ++x)
          if (c0 + x < ni) q2[x] = res[x];
      }
    }
  }
}

// ---- OEC_STAGE_WARP: vector loads from global memory ------------------------
// The level loop keeps NB register windows in rotation (unrolled by NB, no
// copies): a window is refilled with level k+NB right after level k is
// computed, so the loads of NB-1 levels are in flight during each level.
//
// SEP: the output has its own layout (pitch osj, plane osk; rows 16-byte
// aligned) and grid z covers two fields (z < nkz: in -> out, else in1 ->
// out1), as the FP32 producer of the staged hdiff+vadvc form uses it.
template <class P, int U, class Off, int NB, bool SEP>
__device__ __forceinline__ void hdiff_vec_block(const typename P::S* __restrict__ in,
                                                const typename P::S* __restrict__ coeff,
                                                typename P::S* __restrict__ out, int ni, int nj, int nk, int64_t sj,
                                                int64_t sk, int kchunk, int64_t osj, int64_t osk, int nkz,
                                                const typename P::S* __restrict__ in1,
                                                typename P::S* __restrict__ out1, int bx, int by, int bz) {
  typedef typename P::S S;
  typedef typename Vec16<S>::T VT;
  constexpr int V = Vec16<S>::V, W = 32 * V;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int i0 = bx * W, c0 = i0 + V * lane;
  const int jb = (by * 4 + wid) * U;
  if (jb >= nj) return;                                  // whole warp
  const int jmax = nj + 1 - jb;                          // last row offset inside the halo-2 window
  int z = bz;
  if (SEP && z >= nkz) {
    in = in1;
    out = out1;
    z -= nkz;
  }
  const int k0 = z * kchunk, k1 = min(nk, k0 + kchunk);
  const bool vin_full = c0 + V - 1 <= ni + 1;            // whole vector inside the input range [-2, ni+2)
  const bool vout_full = c0 + V - 1 < ni;                // whole vector inside the domain
  const bool edge = lane == 0 || lane == 31;
  const int ca = lane == 0 ? i0 - 1 : i0 + W, cb = lane == 0 ? i0 - 2 : i0 + W + 1;
  const bool ea_ok = edge && ca <= ni + 1, eb_ok = edge && cb <= ni + 1;
  Off roff[U + 4];
#pragma unroll
  for (int x = 0; x < U + 4; ++x) roff[x] = (Off)min(x - 2, jmax) * (Off)sj;
  const Off ksk = (Off)sk;
  Off lev = (Off)k0 * ksk + (Off)jb * (Off)sj;
  auto load = [&](VecWin<S, U, V>& w, Off l) {
#pragma unroll
    for (int r = 0; r < U + 4; ++r) {
      const S* q = in + (l + roff[r] + c0);
      if (vin_full) {
        vsplit<S, V>(__ldg(reinterpret_cast<const VT*>(q)), w.v[r]);
      } else {
#pragma unroll
        for (int x = 0; x < V; ++x) w.v[r][x] = c0 + x <= ni + 1 ? ldg(q + x) : S(0);
      }
    }
#pragma unroll
    for (int r = 0; r < U + 2; ++r) w.ea[r] = ea_ok ? ldg(in + (l + roff[r + 1] + ca)) : S(0);
#pragma unroll
    for (int r = 0; r < U; ++r) {
      w.eb[r] = eb_ok ? ldg(in + (l + roff[r + 2] + cb)) : S(0);
      if (jb + r < nj) {
        const S* q = coeff + (l + roff[r + 2] + c0);
        if (vout_full) {
          vsplit<S, V>(__ldg(reinterpret_cast<const VT*>(q)), w.cf[r]);
        } else {
#pragma unroll
          for (int x = 0; x < V; ++x) w.cf[r][x] = c0 + x < ni ? ldg(q + x) : S(0);
        }
      }
    }
  };
  VecWin<S, U, V> win[NB];
#pragma unroll
  for (int x = 0; x < NB; ++x)
    if (k0 + x < k1) load(win[x], lev + (Off)x * ksk);
  for (int k = k0; k < k1; k += NB, lev += (Off)NB * ksk) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      if (k + b >= k1) break;
      const Off lx = lev + (Off)b * ksk;
      if (SEP)
        vec_rows<P, U>(win[b], lane, c0, jb, ni, nj, out + ((int64_t)(k + b) * osk + (int64_t)jb * osj + c0), osj);
      else
        vec_rows<P, U>(win[b], lane, c0, jb, ni, nj, out + (lx + c0), sj);
      if (k + b + NB < k1) load(win[b], lx + (Off)NB * ksk);
    }
  }
}

}  // namespace
}  // namespace oec
