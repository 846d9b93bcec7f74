// k_hdiff_fixed.cuh - the exact fixed-point FP64 hdiff tile (arith 2): one
// CTA's block body, used by the fixed-point hdiff kernel (k_hdiff.cu).
// Arithmetic in fixedpt.cuh.
#pragma once

#include "arith.cuh"
#include "fixedpt.cuh"
#include "kcommon.cuh"

namespace oec {
namespace {

// shared memory of one tile (bytes): raw window (two levels), fixed-point
// window, limiter keys, Laplacian, and the two exponent slots
template <int TI, int TJ>
struct FixedSmem {
  static constexpr int WI = TI + 4, WJ = TJ + 4, NW = WI * WJ, LI = TI + 2, LJ = TJ + 2, NL = LI * LJ;
  static constexpr size_t FIX = size_t(2) * NW * 8, KEY = FIX + size_t(NW) * 8, LAP = KEY + size_t(NW) * 8,
                          EMAX = LAP + size_t(NL) * 8, BYTES = EMAX + 16;
};

// One CTA: a TI x TJ tile of one field over a chunk of levels, TI x TJ / U
// threads. Per level: (1) the (TI+4) x (TJ+4) window of raw values is loaded
// and its largest exponent E reduced; (2) the window is converted to fixed
// point at scale E, with the limiter keys; (3) the Laplacian over (TI+2) x
// (TJ+2); (4) every thread walks its U output points up j, forming the
// limited fluxes from the Laplacian and keys planes (the flux across the edge
// between two of its points is formed once), the divergence, and one FP64
// FMA. The raw window and the exponent slot are double-buffered, so the next
// level's load overlaps this level's step (4) and a level costs three
// barriers.
template <class OutT, int TI, int TJ, int U, class Off>
__device__ __forceinline__ void hdiff_fixed_block(const double* __restrict__ in0, const double* __restrict__ in1,
                                                  const double* __restrict__ coeff, OutT* __restrict__ out0,
                                                  OutT* __restrict__ out1, int ni, int nj, int nk, int64_t sj,
                                                  int64_t sk, int64_t osj, int64_t osk, int kchunk, int nkz, int bx,
                                                  int by, int bz, unsigned char* smem) {
  typedef FixedSmem<TI, TJ> SM;
  static_assert(TJ % U == 0, "whole rows per thread");
  constexpr int NT = TI * TJ / U, WI = SM::WI, NW = SM::NW, LI = SM::LI, NL = SM::NL;
  constexpr int QW = (NW + NT - 1) / NT, QL = (NL + NT - 1) / NT;
  double(*s_raw)[NW] = reinterpret_cast<double(*)[NW]>(smem);
  long long* s_fix = reinterpret_cast<long long*>(smem + SM::FIX);
  long long* s_key = reinterpret_cast<long long*>(smem + SM::KEY);
  long long* s_lap = reinterpret_cast<long long*>(smem + SM::LAP);
  unsigned* s_emax = reinterpret_cast<unsigned*>(smem + SM::EMAX);
  const int tid = threadIdx.x, tx = tid % TI, ty = (tid / TI) * U;   // first of the thread's U rows
  const int i0 = bx * TI, j0 = by * TJ;
  const bool second = bz >= nkz;
  const double* __restrict__ in = second ? in1 : in0;
  OutT* __restrict__ out = second ? out1 : out0;
  const int kz = second ? bz - nkz : bz;
  const int k0 = kz * kchunk, k1 = min(nk, k0 + kchunk);
  const int vi = min(TI, ni - i0), vj = min(TJ, nj - j0);
  // this thread's positions, fixed for every level: window copies (offset
  // from the window corner), Laplacian positions (window centre), its output
  Off wg[QW];
  bool wok[QW];
#pragma unroll
  for (int q = 0; q < QW; ++q) {
    const int idx = tid + q * NT, r = idx / WI, c = idx - r * WI;
    wok[q] = idx < NW && c < vi + 4 && r < vj + 4;
    wg[q] = (Off)r * (Off)sj + c;
  }
  int lw[QL];
  bool lok[QL];
#pragma unroll
  for (int q = 0; q < QL; ++q) {
    const int idx = tid + q * NT, r = idx / LI, c = idx - r * LI;
    lok[q] = idx < NL && c < vi + 2 && r < vj + 2;
    lw[q] = (r + 1) * WI + c + 1;
  }
  const bool own = tx < vi && ty < vj;
  const int ow = (ty + 2) * WI + tx + 2, ol = (ty + 1) * LI + tx + 1;
  const double* __restrict__ wcorner = in + ((Off)(j0 - 2) * (Off)sj + (i0 - 2));
  const Off oin = (Off)(j0 + ty) * (Off)sj + (i0 + tx), oout = (Off)(j0 + ty) * (Off)osj + (i0 + tx);
  if (tid < 2) s_emax[tid] = 0u;
  __syncthreads();
  // the window values of the next level are loaded into registers while the
  // current level is computed
  double nx[QW];
  auto fetch = [&](int k) {
    const double* pin = wcorner + (Off)k * (Off)sk;
#pragma unroll
    for (int q = 0; q < QW; ++q)
      if (wok[q]) nx[q] = ldg(pin + wg[q]);
  };
  if (k0 < k1) fetch(k0);
  int bf = 0;
  for (int k = k0; k < k1; ++k, bf ^= 1) {
    // (1) raw window and its largest exponent
    unsigned emax = 0u;
#pragma unroll
    for (int q = 0; q < QW; ++q)
      if (wok[q]) {
        const double x = nx[q];
        s_raw[bf][tid + q * NT] = x;
        emax = max(emax, (unsigned)(__double_as_longlong(x) >> 52) & 0x7FFu);
      }
    if (k + 1 < k1) fetch(k + 1);
    emax = __reduce_max_sync(0xFFFFFFFFu, emax);
    if ((tid & 31) == 0) atomicMax(&s_emax[bf], emax);
    __syncthreads();
    // (2) fixed point at scale E, and the limiter keys
    const unsigned E = max(s_emax[bf], 100u);
#pragma unroll
    for (int q = 0; q < QW; ++q)
      if (wok[q]) {
        const int idx = tid + q * NT;
        const double x = s_raw[bf][idx];
        s_fix[idx] = fx_of(x, E);
        s_key[idx] = fx_key(x);
      }
    __syncthreads();
    if (tid == 0) s_emax[bf] = 0u;   // read by everyone before the barrier; next written two levels on
    // (3) Laplacian
#pragma unroll
    for (int q = 0; q < QL; ++q)
      if (lok[q]) {
        const long long* f = s_fix + lw[q];
        s_lap[tid + q * NT] = (f[0] << 2) - f[-1] - f[1] - f[-WI] - f[WI];
      }
    __syncthreads();
    // (4) limited fluxes, divergence, output; fyb is the flux across the
    // edge below the current point
    if (own) {
      const long long* L = s_lap + ol;
      const long long* K = s_key + ow;
      long long fyb = fx_flux(L[0], L[-LI], K[0], K[-WI]);
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (ty + u < vj) {
          const long long lc = L[u * LI], kc = K[u * WI];
          const long long fxp = fx_flux(L[u * LI + 1], lc, K[u * WI + 1], kc);
          const long long fxm = fx_flux(lc, L[u * LI - 1], kc, K[u * WI - 1]);
          const long long fya = fx_flux(L[(u + 1) * LI], lc, K[(u + 1) * WI], kc);
          const long long div = (fxp - fxm) + (fya - fyb);
          fyb = fya;
          const double dv = fx_scaled(div, E);
          const double r =
              __fma_rn(-ldg(coeff + ((Off)k * (Off)sk + oin + (Off)u * (Off)sj)), dv, s_raw[bf][ow + u * WI]);
          out[(Off)k * (Off)osk + oout + (Off)u * (Off)osj] = cvt<OutT>(r);
        }
      }
    }
  }
}

}  // namespace
}  // namespace oec
