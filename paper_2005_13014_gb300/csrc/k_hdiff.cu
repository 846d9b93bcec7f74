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
// Each form is templated on an arithmetic policy (arith.cuh): FP32, native
// FP64, or FP64 storage with double-float arithmetic on the FP32 pipes.
#include "arith.cuh"
#include "fixedpt.cuh"
#include "kcommon.cuh"
#include "kernels.h"
#include "k_hdiff_fixed.cuh"

namespace oec {
namespace {

// Two independent fields may share a launch: blocks with blockIdx.z >= nkz
// work on (in1, out1) (nkz = number of k-chunks; in1 == nullptr: one field).
template <class P, class OutT, int TI, int TJ>
__global__ void __launch_bounds__(TI * TJ)
hdiff_smem_kernel(const typename P::S* __restrict__ in0, const typename P::S* __restrict__ in1,
                  const typename P::S* __restrict__ coeff, OutT* __restrict__ out0, OutT* __restrict__ out1, int ni,
                  int nj, int nk, int64_t sj, int64_t sk, int64_t osj, int64_t osk, int kchunk, int nkz) {
  typedef typename P::S S;
  typedef typename P::C C;
  constexpr int NT = TI * TJ, WI = TI + 4, WJ = TJ + 4;
  __shared__ C s_in[WJ][WI];
  __shared__ C s_lap[TJ + 2][TI + 2];
  __shared__ C s_flx[TJ][TI + 1];
  __shared__ C s_fly[TJ + 1][TI];
  const int tid = threadIdx.x, tx = tid % TI, ty = tid / TI;
  const int i0 = blockIdx.x * TI, j0 = blockIdx.y * TJ;
  const bool second = (int)blockIdx.z >= nkz;
  const S* __restrict__ in = second ? in1 : in0;
  OutT* __restrict__ out = second ? out1 : out0;
  const int kz = second ? blockIdx.z - nkz : blockIdx.z;
  const int k0 = kz * kchunk, k1 = min(nk, k0 + kchunk);
  const int vi = min(TI, ni - i0), vj = min(TJ, nj - j0);   // valid part of a ragged tile
  for (int k = k0; k < k1; ++k) {
    const S* pin = in + (int64_t)k * sk + (int64_t)(j0 - 2) * sj + (i0 - 2);
    for (int idx = tid; idx < WI * WJ; idx += NT) {
      const int r = idx / WI, c = idx - r * WI;
      if (c < vi + 4 && r < vj + 4) s_in[r][c] = cvt<C>(ldg(pin + (int64_t)r * sj + c));
    }
    __syncthreads();
    // lap(i0-1+c, j0-1+r)
    for (int idx = tid; idx < (TI + 2) * (TJ + 2); idx += NT) {
      const int r = idx / (TI + 2), c = idx - r * (TI + 2);
      if (c < vi + 2 && r < vj + 2)
        s_lap[r][c] = hlap(s_in[r + 1][c + 1], s_in[r + 1][c], s_in[r + 1][c + 2], s_in[r][c + 1], s_in[r + 2][c + 1]);
    }
    __syncthreads();
    // flx(i0-1+c, j0+r) and fly(i0+c, j0-1+r)
    for (int idx = tid; idx < (TI + 1) * TJ; idx += NT) {
      const int r = idx / (TI + 1), c = idx - r * (TI + 1);
      if (c < vi + 1 && r < vj)
        s_flx[r][c] = hflux(s_lap[r + 1][c + 1], s_lap[r + 1][c], s_in[r + 2][c + 2], s_in[r + 2][c + 1]);
    }
    for (int idx = tid; idx < TI * (TJ + 1); idx += NT) {
      const int r = idx / TI, c = idx - r * TI;
      if (c < vi && r < vj + 1)
        s_fly[r][c] = hflux(s_lap[r + 1][c + 1], s_lap[r][c + 1], s_in[r + 2][c + 2], s_in[r + 1][c + 2]);
    }
    __syncthreads();
    if (tx < vi && ty < vj) {
      const int64_t o = (int64_t)k * sk + (int64_t)(j0 + ty) * sj + (i0 + tx);
      out[(int64_t)k * osk + (int64_t)(j0 + ty) * osj + (i0 + tx)] = cvt<OutT>(
          hout(s_in[ty + 2][tx + 2], cvt<C>(ldg(coeff + o)), s_flx[ty][tx + 1], s_flx[ty][tx], s_fly[ty + 1][tx], s_fly[ty][tx]));
    }
    __syncthreads();
  }
}

// REGS form (the paper's model: every thread recomputes what it reads): a
// thread owns U consecutive rows of one column and walks its k-chunk. The
// values one level needs (the cross of offsets -2..2 around the U rows, and
// coeff) are loaded into registers one level ahead, so the next level's loads
// are in flight while the current level is computed.
template <class S, int U>
struct RegsWin {
  S c0[U + 4];           // (i,   jb-2 .. jb+U+1)
  S m1[U + 2], p1[U + 2];  // (i-1 / i+1, jb-1 .. jb+U)
  S m2[U], p2[U];          // (i-2 / i+2, jb .. jb+U-1)
  S cf[U];               // coeff (i, jb .. jb+U-1)
};

//
// SEP: the output has its own layout (pitch osj, plane osk) and type OutT, and
// grid z covers two fields (z < nkz: in -> out, else in1 -> out1), as the
// producer of the staged hdiff+vadvc form uses it; otherwise out shares the
// input's layout.
template <class P, int U, class Off, int NB, class OutT, bool SEP>
__global__ void hdiff_regs_kernel(const typename P::S* __restrict__ in, const typename P::S* __restrict__ coeff,
                                  OutT* __restrict__ out, int ni, int nj, int nk, int64_t sj, int64_t sk,
                                  int kchunk, int64_t osj, int64_t osk, int nkz, const typename P::S* __restrict__ in1,
                                  OutT* __restrict__ out1) {
  typedef typename P::S S;
  typedef typename P::C C;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int jb = (blockIdx.y * blockDim.y + threadIdx.y) * U;
  if (i >= ni || jb >= nj) return;
  const int jmax = nj + 1 - jb;          // last row offset inside the halo-2 window
  int z = blockIdx.z;
  if (SEP && z >= nkz) {
    in = in1;
    out = out1;
    z -= nkz;
  }
  const int k0 = z * kchunk, k1 = min(nk, k0 + kchunk);
  // element offsets from the level's (i, jb): rows jb-2 .. jb+U+1 (clamped to
  // the window), computed once; the level offset advances by sk
  Off roff[U + 4];
#pragma unroll
  for (int x = 0; x < U + 4; ++x) roff[x] = (Off)min(x - 2, jmax) * (Off)sj;
  const Off ksk = (Off)sk;
  Off lev = (Off)k0 * ksk + (Off)jb * (Off)sj + i;
  const Off oksk = (Off)osk;
  Off olev = (Off)k0 * oksk + (Off)jb * (Off)osj + i;   // SEP output offset of the level
  auto load = [&](RegsWin<S, U>& w, Off l) {
#pragma unroll
    for (int x = 0; x < U + 4; ++x) w.c0[x] = ldg(in + (l + roff[x]));
#pragma unroll
    for (int x = 0; x < U + 2; ++x) {
      w.m1[x] = ldg(in + (l + roff[x + 1] - 1));
      w.p1[x] = ldg(in + (l + roff[x + 1] + 1));
    }
#pragma unroll
    for (int x = 0; x < U; ++x) {
      w.m2[x] = ldg(in + (l + roff[x + 2] - 2));
      w.p2[x] = ldg(in + (l + roff[x + 2] + 2));
      if (jb + x < nj) w.cf[x] = ldg(coeff + (l + roff[x + 2]));
    }
  };
  // NB register windows, used in rotation with the level loop unrolled by
  // NB: window x holds level k+x; after computing it, it is refilled with
  // level k+x+NB, so NB-1 levels of compute cover every load's latency
  RegsWin<S, U> win[NB];
#pragma unroll
  for (int x = 0; x < NB; ++x)
    if (k0 + x < k1) load(win[x], lev + (Off)x * ksk);
  for (int k = k0; k < k1; k += NB, lev += (Off)NB * ksk, olev += (Off)NB * oksk) {
#pragma unroll
    for (int x = 0; x < NB; ++x) {
      if (k + x >= k1) break;
      const RegsWin<S, U>& cur = win[x];
      const Off lx = lev + (Off)x * ksk;
      // at(di, dj): the value at (i + di, jb + dj)
      auto at = [&](int di, int dj) {
        return cvt<C>(di == 0 ? cur.c0[dj + 2] : di == -1 ? cur.m1[dj + 1] : di == 1 ? cur.p1[dj + 1]
                      : di == -2 ? cur.m2[dj] : cur.p2[dj]);
      };
      C lc[U + 2], lw[U], le[U];   // lap(i, jb-1+r); lap(i-1, jb+r); lap(i+1, jb+r)
#pragma unroll
      for (int r = 0; r < U + 2; ++r) {
        const int dj = r - 1;
        lc[r] = hlap(at(0, dj), at(-1, dj), at(1, dj), at(0, dj - 1), at(0, dj + 1));
      }
#pragma unroll
      for (int r = 0; r < U; ++r) {
        lw[r] = hlap(at(-1, r), at(-2, r), at(0, r), at(-1, r - 1), at(-1, r + 1));
        le[r] = hlap(at(1, r), at(0, r), at(2, r), at(1, r - 1), at(1, r + 1));
      }
#pragma unroll
      for (int r = 0; r < U; ++r) {
        if (jb + r < nj) {
          const C c = at(0, r);
          const C flx = hflux(le[r], lc[r + 1], at(1, r), c);
          const C flx_m = hflux(lc[r + 1], lw[r], c, at(-1, r));
          const C fly = hflux(lc[r + 2], lc[r + 1], at(0, r + 1), c);
          const C fly_m = hflux(lc[r + 1], lc[r], c, at(0, r - 1));
          const Off o = SEP ? olev + (Off)x * oksk + (Off)r * (Off)osj : lx + roff[r + 2];
          out[o] = cvt<OutT>(hout(c, cvt<C>(cur.cf[r]), flx, flx_m, fly, fly_m));
        }
      }
      if (k + x + NB < k1) load(win[x], lx + (Off)NB * ksk);
    }
  }
}

// ---- k-streaming hdiff (OEC_STAGE_STREAM) ----------------------------------
// A CTA owns a TI x TJ tile and walks a chunk of levels. The raw window of
// level k+D-1 ((TI+4) x (TJ+4) values) and its coeff tile are copied
// asynchronously into a D-slot shared-memory ring while level k is computed,
// so each SM keeps D-1 levels of loads in flight: a bandwidth-bound kernel
// needs bytes in flight, not more threads. Per level: a barrier that makes
// level k's copies visible and frees level k-1's slot for the next copy; the
// Laplacian plane of the tile plus one ring, once per point; a barrier; then
// every point forms its four limited fluxes from that plane and its window
// values, and the divergence (overlapped tiling, paper §VII-D).
template <class P, int TI, int TJ>
struct StreamDepth {
  static constexpr int v = sizeof(typename P::S) == 4 ? 4 : 3;   // ring slots (<= 48 KB static)
};

template <class P, int TI, int TJ>
__global__ void __launch_bounds__(TI * TJ)
hdiff_stream_kernel(const typename P::S* __restrict__ in, const typename P::S* __restrict__ coeff,
                    typename P::S* __restrict__ out, int ni, int nj, int nk, int64_t sj, int64_t sk, int kchunk) {
  typedef typename P::S S;
  typedef typename P::C C;
  constexpr int D = StreamDepth<P, TI, TJ>::v;
  constexpr int NT = TI * TJ, WI = TI + 4, WJ = TJ + 4, NW = WI * WJ, QW = (NW + NT - 1) / NT;
  constexpr int LI = TI + 2, LJ = TJ + 2, NL = LI * LJ, QL = (NL + NT - 1) / NT;
  constexpr int SLOT = NW + NT;   // one level: window, then the coeff tile
  __shared__ __align__(16) S s_ring[D * SLOT];
  __shared__ C s_lap[NL];
  const int tid = threadIdx.x, tx = tid % TI, ty = tid / TI;
  const int i0 = blockIdx.x * TI, j0 = blockIdx.y * TJ;
  const int k0 = blockIdx.z * kchunk, k1 = min(nk, k0 + kchunk);
  const int vi = min(TI, ni - i0), vj = min(TJ, nj - j0);   // valid part of a ragged tile
  const bool own = tx < vi && ty < vj;
  // every offset this thread uses, computed once: window copies (global
  // offset from the level's window corner, ring offset), Laplacian positions
  // (window centre, plane slot), and its own output point
  int64_t wg[QW];
  int ws[QW];
  bool wok[QW];
#pragma unroll
  for (int q = 0; q < QW; ++q) {
    const int idx = tid + q * NT, r = idx / WI, c = idx - r * WI;
    wok[q] = idx < NW && c < vi + 4 && r < vj + 4;
    wg[q] = (int64_t)r * sj + c;
    ws[q] = idx;
  }
  int lw[QL], ll[QL];
  bool lok[QL];
#pragma unroll
  for (int q = 0; q < QL; ++q) {
    const int idx = tid + q * NT, r = idx / LI, c = idx - r * LI;
    lok[q] = idx < NL && c < vi + 2 && r < vj + 2;
    lw[q] = (r + 1) * WI + c + 1;
    ll[q] = idx;
  }
  const int ow = (ty + 2) * WI + tx + 2, ol = (ty + 1) * LI + tx + 1;
  const S* __restrict__ wcorner = in + (int64_t)(j0 - 2) * sj + (i0 - 2);
  const int64_t oc = (int64_t)(j0 + ty) * sj + (i0 + tx);
  auto issue = [&](int k, S* slot) {
    if (k < k1) {
      const S* pin = wcorner + (int64_t)k * sk;
#pragma unroll
      for (int q = 0; q < QW; ++q)
        if (wok[q]) cp_async(slot + ws[q], pin + wg[q]);
      if (own) cp_async(slot + NW + tid, coeff + (int64_t)k * sk + oc);
    }
    cp_async_commit();
  };
#pragma unroll
  for (int x = 0; x < D - 1; ++x) issue(k0 + x, s_ring + x * SLOT);
  int sl = 0;   // ring slot of level k
  for (int k = k0; k < k1; ++k) {
    cp_async_wait<D - 2>();   // this thread's copies of level k have landed
    __syncthreads();          // everyone's have; everyone is done with level k-1
    issue(k + D - 1, s_ring + (sl == 0 ? D - 1 : sl - 1) * SLOT);   // into level k-1's slot
    const S* W = s_ring + sl * SLOT;
#pragma unroll
    for (int q = 0; q < QL; ++q)
      if (lok[q]) {
        const S* p = W + lw[q];
        s_lap[ll[q]] = hlap(cvt<C>(p[0]), cvt<C>(p[-1]), cvt<C>(p[1]), cvt<C>(p[-WI]), cvt<C>(p[WI]));
      }
    __syncthreads();
    if (own) {
      const S* p = W + ow;
      const C* L = s_lap + ol;
      const C c0 = cvt<C>(p[0]), lc = L[0];
      const C fxp = hflux(L[1], lc, cvt<C>(p[1]), c0), fxm = hflux(lc, L[-1], c0, cvt<C>(p[-1]));
      const C fyp = hflux(L[LI], lc, cvt<C>(p[WI]), c0), fym = hflux(lc, L[-LI], c0, cvt<C>(p[-WI]));
      out[(int64_t)k * sk + oc] = cvt<S>(hout(c0, cvt<C>(W[NW + tid]), fxp, fxm, fyp, fym));
    }
    sl = sl == D - 1 ? 0 : sl + 1;
  }
  cp_async_wait<0>();
}

template <class P, int TI, int TJ>
cudaError_t run_stream(const oec_schedule& s, const Dom& d, const typename P::S* in, const typename P::S* coeff,
                       typename P::S* out, cudaStream_t st) {
  const int kc = (s.k_chunk <= 0 || s.k_chunk > d.nk) ? d.nk : s.k_chunk;
  dim3 g(ceil_div(d.ni, TI), ceil_div(d.nj, TJ), ceil_div(d.nk, kc));
  hdiff_stream_kernel<P, TI, TJ><<<g, TI * TJ, 0, st>>>(in, coeff, out, d.ni, d.nj, d.nk, d.sj, d.sk, kc);
  launched(st);
  return cudaGetLastError();
}

// ---- exact fixed-point FP64 hdiff (arith 2): block body in k_hdiff_fixed.cuh --
template <class OutT, int TI, int TJ, int U, class Off>
__global__ void __launch_bounds__(TI * TJ / U)
hdiff_fixed_kernel(const double* __restrict__ in0, const double* __restrict__ in1, const double* __restrict__ coeff,
                   OutT* __restrict__ out0, OutT* __restrict__ out1, int ni, int nj, int nk, int64_t sj, int64_t sk,
                   int64_t osj, int64_t osk, int kchunk, int nkz) {
  __shared__ __align__(16) unsigned char smem[FixedSmem<TI, TJ>::BYTES];
  hdiff_fixed_block<OutT, TI, TJ, U, Off>(in0, in1, coeff, out0, out1, ni, nj, nk, sj, sk, osj, osk, kchunk, nkz,
                                          blockIdx.x, blockIdx.y, blockIdx.z, smem);
}

template <class OutT, int TI, int TJ, int U>
cudaError_t run_fixed(const oec_schedule& s, const Dom& d, int64_t osj, int64_t osk, const double* in,
                      const double* coeff, OutT* out, cudaStream_t st, const double* in1 = nullptr,
                      OutT* out1 = nullptr) {
  const int kc = (s.k_chunk <= 0 || s.k_chunk > d.nk) ? d.nk : s.k_chunk;
  const int nkz = ceil_div(d.nk, kc);
  dim3 g(ceil_div(d.ni, TI), ceil_div(d.nj, TJ), nkz * (in1 ? 2 : 1));
  constexpr int NT = TI * TJ / U;
  if (use_int32(s, d))
    hdiff_fixed_kernel<OutT, TI, TJ, U, int><<<g, NT, 0, st>>>(in, in1, coeff, out, out1, d.ni, d.nj, d.nk, d.sj,
                                                               d.sk, osj, osk, kc, nkz);
  else
    hdiff_fixed_kernel<OutT, TI, TJ, U, int64_t><<<g, NT, 0, st>>>(in, in1, coeff, out, out1, d.ni, d.nj, d.nk, d.sj,
                                                                   d.sk, osj, osk, kc, nkz);
  launched(st);
  return cudaGetLastError();
}

// ---- unfused: one kernel per stage, temporaries (compute type) over their
// inferred ranges ----------------------------------------------------------
// lap over [-1, ni+1) x [-1, nj+1): element (i, j, k) at ((k*(nj+2) + j+1)*(ni+2) + i+1)
template <class P>
__global__ void hdiff_lap_kernel(const typename P::S* __restrict__ in, typename P::C* __restrict__ lap, int ni, int nj,
                                 int nk, int64_t sj, int64_t sk) {
  typedef typename P::C C;
  const int i = blockIdx.x * blockDim.x + threadIdx.x - 1;
  const int j = blockIdx.y * blockDim.y + threadIdx.y - 1;
  const int k = blockIdx.z;
  if (i >= ni + 1 || j >= nj + 1) return;
  const typename P::S* p = in + (int64_t)k * sk + (int64_t)j * sj + i;
  lap[((int64_t)k * (nj + 2) + (j + 1)) * (ni + 2) + (i + 1)] =
      hlap(cvt<C>(ldg(p)), cvt<C>(ldg(p - 1)), cvt<C>(ldg(p + 1)), cvt<C>(ldg(p - sj)), cvt<C>(ldg(p + sj)));
}
// flx over [-1, ni) x [0, nj): ((k*nj + j)*(ni+1) + i+1)
template <class P>
__global__ void hdiff_flx_kernel(const typename P::S* __restrict__ in, const typename P::C* __restrict__ lap,
                                 typename P::C* __restrict__ flx, int ni, int nj, int nk, int64_t sj, int64_t sk) {
  typedef typename P::C C;
  const int i = blockIdx.x * blockDim.x + threadIdx.x - 1;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= ni || j >= nj) return;
  const typename P::S* p = in + (int64_t)k * sk + (int64_t)j * sj + i;
  const C* l = lap + ((int64_t)k * (nj + 2) + (j + 1)) * (ni + 2) + (i + 1);
  flx[((int64_t)k * nj + j) * (ni + 1) + (i + 1)] = hflux(l[1], l[0], cvt<C>(ldg(p + 1)), cvt<C>(ldg(p)));
}
// fly over [0, ni) x [-1, nj): ((k*(nj+1) + j+1)*ni + i)
template <class P>
__global__ void hdiff_fly_kernel(const typename P::S* __restrict__ in, const typename P::C* __restrict__ lap,
                                 typename P::C* __restrict__ fly, int ni, int nj, int nk, int64_t sj, int64_t sk) {
  typedef typename P::C C;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y - 1;
  const int k = blockIdx.z;
  if (i >= ni || j >= nj) return;
  const typename P::S* p = in + (int64_t)k * sk + (int64_t)j * sj + i;
  const C* l = lap + ((int64_t)k * (nj + 2) + (j + 1)) * (ni + 2) + (i + 1);
  fly[((int64_t)k * (nj + 1) + (j + 1)) * ni + i] = hflux(l[ni + 2], l[0], cvt<C>(ldg(p + sj)), cvt<C>(ldg(p)));
}
template <class P>
__global__ void hdiff_out_kernel(const typename P::S* __restrict__ in, const typename P::S* __restrict__ coeff,
                                 const typename P::C* __restrict__ flx, const typename P::C* __restrict__ fly,
                                 typename P::S* __restrict__ out, int ni, int nj, int nk, int64_t sj, int64_t sk) {
  typedef typename P::C C;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int k = blockIdx.z;
  if (i >= ni || j >= nj) return;
  const int64_t o = (int64_t)k * sk + (int64_t)j * sj + i;
  const C* fx = flx + ((int64_t)k * nj + j) * (ni + 1) + (i + 1);
  const C* fy = fly + ((int64_t)k * (nj + 1) + (j + 1)) * ni + i;
  out[o] = cvt<typename P::S>(hout(cvt<C>(ldg(in + o)), cvt<C>(ldg(coeff + o)), fx[0], fx[-1], fy[0], fy[-ni]));
}

struct Tmp {
  size_t lap, flx, fly, total;
};
Tmp unfused_layout(size_t e, const Dom& d) {
  Tmp t;
  t.lap = 0;
  t.flx = align_up(t.lap + e * size_t(d.ni + 2) * (d.nj + 2) * d.nk, 256);
  t.fly = align_up(t.flx + e * size_t(d.ni + 1) * d.nj * d.nk, 256);
  t.total = align_up(t.fly + e * size_t(d.ni) * (d.nj + 1) * d.nk, 256);
  return t;
}

template <class P>
cudaError_t run_unfused(const Dom& d, const typename P::S* in, const typename P::S* coeff, typename P::S* out,
                        char* scratch, cudaStream_t st) {
  typedef typename P::C C;
  Tmp t = unfused_layout(sizeof(C), d);
  C* lap = (C*)(scratch + t.lap);
  C* flx = (C*)(scratch + t.flx);
  C* fly = (C*)(scratch + t.fly);
  dim3 b(32, 8);
  hdiff_lap_kernel<P><<<dim3(ceil_div(d.ni + 2, 32), ceil_div(d.nj + 2, 8), d.nk), b, 0, st>>>(in, lap, d.ni, d.nj, d.nk, d.sj, d.sk);
  launched(st);
  hdiff_flx_kernel<P><<<dim3(ceil_div(d.ni + 1, 32), ceil_div(d.nj, 8), d.nk), b, 0, st>>>(in, lap, flx, d.ni, d.nj, d.nk, d.sj, d.sk);
  launched(st);
  hdiff_fly_kernel<P><<<dim3(ceil_div(d.ni, 32), ceil_div(d.nj + 1, 8), d.nk), b, 0, st>>>(in, lap, fly, d.ni, d.nj, d.nk, d.sj, d.sk);
  launched(st);
  hdiff_out_kernel<P><<<dim3(ceil_div(d.ni, 32), ceil_div(d.nj, 8), d.nk), b, 0, st>>>(in, coeff, flx, fly, out, d.ni, d.nj, d.nk, d.sj, d.sk);
  launched(st);
  return cudaGetLastError();
}

int kchunk_of(const oec_schedule& s, int nk) { return (s.k_chunk <= 0 || s.k_chunk > nk) ? nk : s.k_chunk; }

template <class P, class OutT, int TI, int TJ>
cudaError_t run_smem(const oec_schedule& s, const Dom& d, int64_t osj, int64_t osk, const typename P::S* in,
                     const typename P::S* coeff, OutT* out, cudaStream_t st, const typename P::S* in1 = nullptr,
                     OutT* out1 = nullptr) {
  const int kc = kchunk_of(s, d.nk);
  const int nkz = ceil_div(d.nk, kc);
  dim3 g(ceil_div(d.ni, TI), ceil_div(d.nj, TJ), nkz * (in1 ? 2 : 1));
  hdiff_smem_kernel<P, OutT, TI, TJ><<<g, TI * TJ, 0, st>>>(in, in1, coeff, out, out1, d.ni, d.nj, d.nk, d.sj, d.sk,
                                                              osj, osk, kc, nkz); launched(st);
  return cudaGetLastError();
}

#ifndef REGS_NB
#define REGS_NB 2   // register windows in rotation (prefetch distance REGS_NB - 1 levels)
#endif
template <class P, int U>
cudaError_t run_regs(const oec_schedule& s, const Dom& d, const typename P::S* in, const typename P::S* coeff,
                     typename P::S* out, cudaStream_t st) {
  const int kc = kchunk_of(s, d.nk);
  dim3 b(s.tile_i, s.tile_j / U);
  dim3 g(ceil_div(d.ni, s.tile_i), ceil_div(d.nj, s.tile_j), ceil_div(d.nk, kc));
  typedef typename P::S S;
  if (use_int32(s, d))
    hdiff_regs_kernel<P, U, int, REGS_NB, S, false><<<g, b, 0, st>>>(in, coeff, out, d.ni, d.nj, d.nk, d.sj, d.sk, kc,
                                                                     0, 0, 0, nullptr, nullptr);
  else
    hdiff_regs_kernel<P, U, int64_t, REGS_NB, S, false><<<g, b, 0, st>>>(in, coeff, out, d.ni, d.nj, d.nk, d.sj, d.sk,
                                                                         kc, 0, 0, 0, nullptr, nullptr);
  launched(st);
  return cudaGetLastError();
}

// the REGS kernel as the staged producer: fields in0 -> out0 and in1 -> out1
// (domain layout osj, osk, type OutT) in one launch
template <class P, int U, class OutT>
cudaError_t run_regs_to(const oec_schedule& s, const Dom& d, int64_t osj, int64_t osk, const typename P::S* in0,
                        const typename P::S* in1, const typename P::S* coeff, OutT* out0, OutT* out1,
                        cudaStream_t st) {
  const int kc = kchunk_of(s, d.nk), nkz = ceil_div(d.nk, kc);
  dim3 b(s.tile_i, s.tile_j / U);
  dim3 g(ceil_div(d.ni, s.tile_i), ceil_div(d.nj, s.tile_j), 2 * nkz);
  if (use_int32(s, d))
    hdiff_regs_kernel<P, U, int, REGS_NB, OutT, true><<<g, b, 0, st>>>(in0, coeff, out0, d.ni, d.nj, d.nk, d.sj,
                                                                       d.sk, kc, osj, osk, nkz, in1, out1);
  else
    hdiff_regs_kernel<P, U, int64_t, REGS_NB, OutT, true><<<g, b, 0, st>>>(in0, coeff, out0, d.ni, d.nj, d.nk, d.sj,
                                                                           d.sk, kc, osj, osk, nkz, in1, out1);
  launched(st);
  return cudaGetLastError();
}

#define OEC_SMEM_TILES(X) X(32, 4) X(32, 8) X(64, 2) X(64, 4) X(64, 8) X(128, 2) X(128, 4)
// fixed-point hdiff: tile_i, tile_j, rows per thread
#define OEC_FIXED_TILES(X)                                                                                   \
  X(32, 4, 1) X(32, 8, 1) X(64, 2, 1) X(64, 4, 1) X(64, 8, 1) X(128, 2, 1) X(128, 4, 1) X(32, 8, 2) X(32, 16, 1) \
  X(32, 16, 2) X(32, 16, 4) X(64, 8, 2)
#define OEC_STREAM_TILES(X) X(32, 4) X(32, 8) X(64, 4) X(64, 8) X(128, 2) X(128, 4)

template <class P>
cudaError_t dispatch(const oec_schedule& s, const Dom& d, const typename P::S* in, const typename P::S* coeff,
                     typename P::S* out, void* scratch, cudaStream_t st) {
  typedef typename P::S S;
  if (s.fusion == OEC_FUSE_NONE) return run_unfused<P>(d, in, coeff, out, (char*)scratch, st);
  if (s.staging == OEC_STAGE_STREAM) {
#define X(a, b) if (s.tile_i == a && s.tile_j == b) return run_stream<P, a, b>(s, d, in, coeff, out, st);
    OEC_STREAM_TILES(X)
#undef X
    return cudaErrorInvalidValue;
  }
  if (s.staging == OEC_STAGE_SMEM) {
#define X(a, b) if (s.tile_i == a && s.tile_j == b) return run_smem<P, S, a, b>(s, d, d.sj, d.sk, in, coeff, out, st);
    OEC_SMEM_TILES(X)
#undef X
    return cudaErrorInvalidValue;
  }
  switch (s.unroll) {
    case 1: return run_regs<P, 1>(s, d, in, coeff, out, st);
    case 2: return run_regs<P, 2>(s, d, in, coeff, out, st);
    case 4: return run_regs<P, 4>(s, d, in, coeff, out, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool hdiff_schedule_ok(const oec_schedule& s, std::string& why) {
  if (s.arith < 0 || s.arith > 2) { why = "arith must be 0 (native), 1 (double-float) or 2 (fixed point)"; return false; }
  if (s.arith == 2) {
    if (s.fusion != OEC_FUSE_INLINE || s.staging != OEC_STAGE_SMEM) {
      why = "fixed-point arithmetic runs the fused SMEM-staged kernel";
      return false;
    }
    if (s.k_chunk < 0) { why = "k_chunk must be >= 0"; return false; }
#define X(a, b, u) if (s.tile_i == a && s.tile_j == b && s.unroll == u) return true;
    OEC_FIXED_TILES(X)
#undef X
    why = "fixed-point tiles (tile_i x tile_j, unroll): 32x4 1, 32x8 1/2, 64x2 1, 64x4 1, 64x8 1/2, 128x2 1, "
          "128x4 1, 32x16 1/2/4";
    return false;
  }
  if (s.fusion == OEC_FUSE_NONE) return true;
  if (s.fusion != OEC_FUSE_INLINE) { why = "fusion must be OEC_FUSE_INLINE or OEC_FUSE_NONE"; return false; }
  if (s.k_chunk < 0) { why = "k_chunk must be >= 0"; return false; }
  if (s.staging == OEC_STAGE_WARP || s.staging == OEC_STAGE_TMA) {
    if (s.unroll != 1 && s.unroll != 2 && s.unroll != 4) { why = "WARP/TMA staging: unroll (rows per warp) 1, 2 or 4"; return false; }
    return true;
  }
  if (s.staging == OEC_STAGE_STREAM) {
#define X(a, b) if (s.tile_i == a && s.tile_j == b && s.unroll == 1) return true;
    OEC_STREAM_TILES(X)
#undef X
    why = "STREAM staging supports tiles 32x4, 32x8, 64x4, 64x8, 128x2, 128x4 with unroll 1";
    return false;
  }
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

static size_t compute_bytes(const oec_schedule& s, int dtype) { return dtype == OEC_F32 ? 4 : 8; }

size_t hdiff_scratch_bytes(const oec_schedule& s, int dtype, const Dom& d) {
  return s.fusion == OEC_FUSE_NONE ? unfused_layout(compute_bytes(s, dtype), d).total : 0;
}

cudaError_t hdiff_launch(const oec_schedule& s, int dtype, const Dom& d, const void* in, const void* coeff, void* out,
                         void* scratch, cudaStream_t st) {
  if (s.fusion == OEC_FUSE_INLINE && s.staging == OEC_STAGE_WARP) return hdiff_warp_launch(s, dtype, d, in, coeff, out, st);
  if (dtype == OEC_F64 && s.arith == 2) {
#define X(a, b, u)                                                                                            \
  if (s.tile_i == a && s.tile_j == b && s.unroll == u)                                                        \
    return run_fixed<double, a, b, u>(s, d, d.sj, d.sk, (const double*)in, (const double*)coeff, (double*)out, st);
    OEC_FIXED_TILES(X)
#undef X
    return cudaErrorInvalidValue;
  }
  if (dtype == OEC_F64) {
    if (s.arith == 1)
      return dispatch<P64D>(s, d, (const double*)in, (const double*)coeff, (double*)out, scratch, st);
    return dispatch<P64>(s, d, (const double*)in, (const double*)coeff, (double*)out, scratch, st);
  }
  return dispatch<P32>(s, d, (const float*)in, (const float*)coeff, (float*)out, scratch, st);
}

cudaError_t hdiff_to_compute(const oec_schedule& sched, int dtype, const Dom& d, const void* in0, const void* in1,
                             const void* coeff, void* out0, void* out1, cudaStream_t st) {
  const int64_t osj = d.ni, osk = (int64_t)d.ni * d.nj;
  // FP32 fields with WARP staging whose rows are 16-byte aligned (inputs at
  // the domain corner, strides, and ni for the outputs): the vector-row
  // kernel (unroll rows per warp, k_chunk levels per CTA); unaligned fields
  // take the REGS kernel below
  if (dtype == OEC_F32 && sched.staging == OEC_STAGE_WARP) {
    const bool aligned = ((uintptr_t)in0 | (uintptr_t)in1 | (uintptr_t)coeff | (uintptr_t)out0 | (uintptr_t)out1) % 16 == 0 &&
                         d.sj % 4 == 0 && d.sk % 4 == 0 && d.ni % 4 == 0;
    if (aligned)
      return hdiff_warp_to_compute(sched, d, osj, osk, (const float*)in0, (const float*)in1, (const float*)coeff,
                                   (float*)out0, (float*)out1, st);
  }
  // FP32 fields with REGS staging: the REGS kernel (CTA tile_i x tile_j/unroll
  // threads, unroll rows per thread, k_chunk levels per CTA); a tile it cannot
  // run falls back to 64 x 4, unroll 1
  if (dtype == OEC_F32 && (sched.staging == OEC_STAGE_REGS || sched.staging == OEC_STAGE_WARP)) {
    oec_schedule s = sched;
    const int u = s.unroll;
    const bool ok = (u == 1 || u == 2 || u == 4) && s.tile_i >= 16 && s.tile_i <= 256 && s.tile_i % 16 == 0 &&
                    s.tile_j >= u && s.tile_j % u == 0 && s.tile_j <= 64 && s.tile_i * (s.tile_j / u) <= 1024;
    if (!ok) {
      s.tile_i = 64;
      s.tile_j = 4;
      s.unroll = 1;
    }
    const float* i0 = (const float*)in0;
    const float* i1 = (const float*)in1;
    const float* cf = (const float*)coeff;
    switch (s.unroll) {
      case 2: return run_regs_to<P32, 2, float>(s, d, osj, osk, i0, i1, cf, (float*)out0, (float*)out1, st);
      case 4: return run_regs_to<P32, 4, float>(s, d, osj, osk, i0, i1, cf, (float*)out0, (float*)out1, st);
      default: return run_regs_to<P32, 1, float>(s, d, osj, osk, i0, i1, cf, (float*)out0, (float*)out1, st);
    }
  }
  // FP64 arith 2: the fixed-point kernel on the schedule's tile and rows per
  // thread when they name one of its tiles, else 64 x 4, one row
  if (dtype == OEC_F64 && sched.arith == 2) {
    oec_schedule s = sched;
    if (s.k_chunk <= 0) s.k_chunk = 4;
    const double* i0 = (const double*)in0;
    const double* i1 = (const double*)in1;
    const double* cf = (const double*)coeff;
#define X(a, b, u) \
  if (s.tile_i == a && s.tile_j == b && s.unroll == u) return run_fixed<df64, a, b, u>(s, d, osj, osk, i0, cf, (df64*)out0, st, i1, (df64*)out1);
    OEC_FIXED_TILES(X)
#undef X
    return run_fixed<df64, 64, 4, 1>(s, d, osj, osk, i0, cf, (df64*)out0, st, i1, (df64*)out1);
  }
  // otherwise the SMEM tile kernel: the schedule's tile and k_chunk pick its
  // tile when they name one of its tiles; otherwise 64 x 4, 4 levels per CTA
  oec_schedule s = sched;
  bool known = false;
#define X(a, b) known = known || (s.tile_i == a && s.tile_j == b);
  OEC_SMEM_TILES(X)
#undef X
  if (!known) {
    s.tile_i = 64;
    s.tile_j = 4;
  }
  if (s.k_chunk <= 0) s.k_chunk = 4;
#define X(a, b)                                                                                                  \
  if (s.tile_i == a && s.tile_j == b) {                                                                          \
    if (dtype == OEC_F64) {                                                                                      \
      if (s.arith == 1)                                                                                          \
        return run_smem<P64D, df64, a, b>(s, d, osj, osk, (const double*)in0, (const double*)coeff, (df64*)out0, \
                                          st, (const double*)in1, (df64*)out1);                                  \
      return run_smem<P64, double, a, b>(s, d, osj, osk, (const double*)in0, (const double*)coeff,               \
                                         (double*)out0, st, (const double*)in1, (double*)out1);                  \
    }                                                                                                            \
    return run_smem<P32, float, a, b>(s, d, osj, osk, (const float*)in0, (const float*)coeff, (float*)out0, st,  \
                                      (const float*)in1, (float*)out1);                                          \
  }
  OEC_SMEM_TILES(X)
#undef X
  return cudaErrorInvalidValue;
}

}  // namespace oec
