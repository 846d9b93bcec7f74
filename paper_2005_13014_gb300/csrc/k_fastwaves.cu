// k_fastwaves.cu - the fastwaves-like program (the shape Table II lists as
// fastwavesuv: six applies, nine inputs, two outputs, no control flow):
//   S1 ppgk = wgtfac*pp + (1 - wgtfac)*pp(k-1)
//   S2 ppgc = ppgk(k+1) - ppgk
//   S3 ppgu = (pp(i+1) - pp) + 0.25*(ppgc(i+1) + ppgc)*((hhl(k+1) + hhl)
//             - (hhl(i+1,k+1) + hhl(i+1))) / ((hhl(k+1) - hhl) + (hhl(i+1,k+1) - hhl(i+1)))
//   S4 ppgv = S3 along j
//   S5 div  = (-u(i+2) + 8u(i+1) - 8u(i-1) + u(i-2))/12 + (same for v along j)
//   S6 u_out = u_in + dt*((utens - ppgu*2*fx/(rho(i+1) + rho)) + alpha*(div(i+1) - div)),
//      v_out likewise along j.
// Forms:
//   fused REGS: a thread computes U consecutive levels of one column,
//     recomputing S1/S2/S5 at the three (i,j) positions it needs (stencil
//     inlining, paper §V-A) and reusing ppgk(k+1) as the next level's ppgk(k)
//     (k-unrolling with CSE; paper §VII-C notes the 3-D reuse unrolling brings
//     to fastwaves);
//   fused SMEM: a CTA streams its (i, j) tile up a chunk of levels, keeping the
//     S1 plane of the previous level in shared memory and S2/S5 of the current
//     level on the tile plus one row/column (the execution model of overlapped
//     tiling + k-streaming, paper §VII-D);
//   unfused: one kernel per stage, temporaries over their inferred ranges.
// Templated on an arithmetic policy (arith.cuh): S storage, C compute type.
#include <mutex>

#include "arith.cuh"
#include "kcommon.cuh"
#include "kernels.h"
#include "tma.cuh"

namespace oec {
namespace {

template <typename T>
struct FW {
  const T *u_in, *v_in, *utens, *vtens, *pp, *rho, *wgtfac, *hhl, *fx;
  T *u_out, *v_out;
  int ni, nj, nk;
  int64_t sj, sk;
};

template <class C>
__device__ __forceinline__ C fw_ppgk(C wg, C pp, C pp_km1) { return wg * pp + (kc<C>(1.0f) - wg) * pp_km1; }
template <class C>
__device__ __forceinline__ C fw_pgrad(C pp_n, C pp, C pc_n, C pc, C h_k1, C h, C hn_k1, C hn) {
  return (pp_n - pp) + fdiv_(mul_p2(pc_n + pc, 0.25f) * ((h_k1 + h) - (hn_k1 + hn)), (h_k1 - h) + (hn_k1 - hn));
}
template <class C>
__device__ __forceinline__ C fw_d4(C m2, C m1, C p1, C p2) {
  return div12(-p2 + mul_p2(p1, 8.0f) - mul_p2(m1, 8.0f) + m2);
}
template <class C>
__device__ __forceinline__ C fw_out(C uin, C dt, C tens, C pg, C fx, C rho_n, C rho, C alpha, C div_n, C div) {
  return uin + dt * ((tens - fdiv_(mul_p2(pg, 2.0f) * fx, rho_n + rho)) + alpha * (div_n - div));
}

template <class P>
__device__ __forceinline__ typename P::C ld(const typename P::S* q) { return cvt<typename P::C>(ldg(q)); }

// element offsets o of type Off (int where every offset of the domain fits)
template <class P, class Off>
__device__ __forceinline__ typename P::C ppgk_at(const FW<typename P::S>& p, Off o) {
  return fw_ppgk(ld<P>(p.wgtfac + o), ld<P>(p.pp + o), ld<P>(p.pp + (o - (Off)p.sk)));
}
template <class P, class Off>
__device__ __forceinline__ typename P::C div_at(const FW<typename P::S>& p, Off o) {
  const typename P::S* u = p.u_in + o;
  const typename P::S* v = p.v_in + o;
  const Off sj = (Off)p.sj;
  return fw_d4(ld<P>(u - 2), ld<P>(u - 1), ld<P>(u + 1), ld<P>(u + 2)) +
         fw_d4(ld<P>(v - 2 * sj), ld<P>(v - sj), ld<P>(v + sj), ld<P>(v + 2 * sj));
}

template <class P, class Off>
__device__ __forceinline__ void fw_point(const FW<typename P::S>& p, Off o, typename P::C pc, typename P::C pc_e,
                                         typename P::C pc_n, typename P::C dv, typename P::C dv_e, typename P::C dv_n,
                                         typename P::C dt, typename P::C alpha) {
  typedef typename P::C C;
  typedef typename P::S S;
  const Off sj = (Off)p.sj, sk = (Off)p.sk;
  const C pp = ld<P>(p.pp + o), h = ld<P>(p.hhl + o), h1 = ld<P>(p.hhl + o + sk);
  const C ppgu = fw_pgrad(ld<P>(p.pp + o + 1), pp, pc_e, pc, h1, h, ld<P>(p.hhl + o + 1 + sk), ld<P>(p.hhl + o + 1));
  const C ppgv = fw_pgrad(ld<P>(p.pp + o + sj), pp, pc_n, pc, h1, h, ld<P>(p.hhl + o + sj + sk), ld<P>(p.hhl + o + sj));
  const C fx = ld<P>(p.fx + o), rho = ld<P>(p.rho + o);
  p.u_out[o] = cvt<S>(fw_out(ld<P>(p.u_in + o), dt, ld<P>(p.utens + o), ppgu, fx, ld<P>(p.rho + o + 1), rho, alpha, dv_e, dv));
  p.v_out[o] = cvt<S>(fw_out(ld<P>(p.v_in + o), dt, ld<P>(p.vtens + o), ppgv, fx, ld<P>(p.rho + o + sj), rho, alpha, dv_n, dv));
}

template <class P, int U>
__global__ void fw_regs_kernel(FW<typename P::S> p, double dt_d, double alpha_d) {
  typedef typename P::C T;
  const T dt = kd<T>(dt_d), alpha = kd<T>(alpha_d);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int kb = blockIdx.z * U;
  if (i >= p.ni || j >= p.nj) return;
  const int64_t col = (int64_t)j * p.sj + i;
  T pk[U + 1], pk_e[U + 1], pk_n[U + 1];   // ppgk at (i,j), (i+1,j), (i,j+1), levels kb..kb+U
#pragma unroll
  for (int r = 0; r <= U; ++r) {
    const int64_t o = (int64_t)min(kb + r, p.nk) * p.sk + col;   // clamp: levels past nk unused
    pk[r] = ppgk_at<P>(p, o);
    pk_e[r] = ppgk_at<P>(p, o + 1);
    pk_n[r] = ppgk_at<P>(p, o + p.sj);
  }
#pragma unroll
  for (int r = 0; r < U; ++r) {
    if (kb + r < p.nk) {
      const int64_t o = (int64_t)(kb + r) * p.sk + col;
      fw_point<P>(p, o, pk[r + 1] - pk[r], pk_e[r + 1] - pk_e[r], pk_n[r + 1] - pk_n[r], div_at<P>(p, o),
                  div_at<P>(p, o + 1), div_at<P>(p, o + p.sj), dt, alpha);
    }
  }
}

// k-streaming form (OEC_STAGE_STREAM): a thread walks its column up a chunk
// of levels and carries, from level k to k+1, ppgk, pp and hhl of the three
// columns it needs ((i,j), (i+1,j), (i,j+1)): per level it loads only level
// k+1 of pp, wgtfac, hhl there, the stencil of u and v for the divergence at
// the three points, and the point's own inputs (35 loads; the REGS form makes
// 59). Element offsets are 32-bit where the fields allow it, and the next
// level's loads are issued before the current level is computed (two
// register windows in rotation).
template <class S>
struct FwWin {
  S pp1[3], wg1[3], hh1[3];   // level k+1 at (i,j), (i+1,j), (i,j+1)
  S ur0[6];                   // u_in(i-2 .. i+3, j)
  S ur1[4];                   // u_in(i-2, i-1, i+1, i+2; j+1)
  S vc0[6];                   // v_in(i, j-2 .. j+3)
  S vc1[4];                   // v_in(i+1; j-2, j-1, j+1, j+2)
  S fx, rho, rho_e, rho_n, ut, vt;
};

template <class P, class Off>
__global__ void fw_stream_kernel(FW<typename P::S> p, double dt_d, double alpha_d, int kchunk) {
  typedef typename P::C T;
  typedef typename P::S S;
  const T dt = kd<T>(dt_d), alpha = kd<T>(alpha_d);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= p.ni || j >= p.nj) return;
  const int k0 = blockIdx.z * kchunk, k1 = min(p.nk, k0 + kchunk);
  const Off sj = (Off)p.sj, sk = (Off)p.sk;
  const Off col = (Off)j * sj + i;
  const Off cn[3] = {0, 1, sj};   // the three columns, relative to (i,j)
  auto ld = [&](const S* f, Off o) { return ldg(f + o); };
  auto load = [&](FwWin<S>& w, int k) {   // level k's window (pp, wgtfac, hhl of level k+1)
    const Off o = (Off)k * sk + col, o1 = o + sk;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      w.pp1[c] = ld(p.pp, o1 + cn[c]);
      w.wg1[c] = ld(p.wgtfac, o1 + cn[c]);
      w.hh1[c] = ld(p.hhl, o1 + cn[c]);
    }
#pragma unroll
    for (int x = 0; x < 6; ++x) w.ur0[x] = ld(p.u_in, o + (x - 2));
    w.ur1[0] = ld(p.u_in, o + sj - 2);
    w.ur1[1] = ld(p.u_in, o + sj - 1);
    w.ur1[2] = ld(p.u_in, o + sj + 1);
    w.ur1[3] = ld(p.u_in, o + sj + 2);
#pragma unroll
    for (int x = 0; x < 6; ++x) w.vc0[x] = ld(p.v_in, o + (Off)(x - 2) * sj);
    w.vc1[0] = ld(p.v_in, o + 1 - 2 * sj);
    w.vc1[1] = ld(p.v_in, o + 1 - sj);
    w.vc1[2] = ld(p.v_in, o + 1 + sj);
    w.vc1[3] = ld(p.v_in, o + 1 + 2 * sj);
    w.fx = ld(p.fx, o);
    w.rho = ld(p.rho, o);
    w.rho_e = ld(p.rho, o + 1);
    w.rho_n = ld(p.rho, o + sj);
    w.ut = ld(p.utens, o);
    w.vt = ld(p.vtens, o);
  };
  // carried state at level k: ppgk(k), pp(k), hhl(k) of the three columns
  T pk[3], ppv[3], hh[3];
  {
    const Off o = (Off)k0 * sk + col;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ppv[c] = cvt<T>(ld(p.pp, o + cn[c]));
      pk[c] = fw_ppgk(cvt<T>(ld(p.wgtfac, o + cn[c])), ppv[c], cvt<T>(ld(p.pp, o + cn[c] - sk)));
      hh[c] = cvt<T>(ld(p.hhl, o + cn[c]));
    }
  }
  FwWin<S> win[2];
  load(win[0], k0);
  if (k0 + 1 < k1) load(win[1], k0 + 1);
  for (int k = k0; k < k1; k += 2) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      if (k + b >= k1) break;
      const FwWin<S>& w = win[b];
      const Off o = (Off)(k + b) * sk + col;
      T pk1[3], pc[3], h1[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pk1[c] = fw_ppgk(cvt<T>(w.wg1[c]), cvt<T>(w.pp1[c]), ppv[c]);
        pc[c] = pk1[c] - pk[c];
        h1[c] = cvt<T>(w.hh1[c]);
      }
      const T ppgu = fw_pgrad(ppv[1], ppv[0], pc[1], pc[0], h1[0], hh[0], h1[1], hh[1]);
      const T ppgv = fw_pgrad(ppv[2], ppv[0], pc[2], pc[0], h1[0], hh[0], h1[2], hh[2]);
      auto U0 = [&](int x) { return cvt<T>(w.ur0[x + 2]); };   // u_in(i+x, j)
      auto V0 = [&](int y) { return cvt<T>(w.vc0[y + 2]); };   // v_in(i, j+y)
      // divergence at (i,j), (i+1,j), (i,j+1)
      const T dv = fw_d4(U0(-2), U0(-1), U0(1), U0(2)) + fw_d4(V0(-2), V0(-1), V0(1), V0(2));
      const T dv_e = fw_d4(U0(-1), U0(0), U0(2), U0(3)) +
                     fw_d4(cvt<T>(w.vc1[0]), cvt<T>(w.vc1[1]), cvt<T>(w.vc1[2]), cvt<T>(w.vc1[3]));
      const T dv_n = fw_d4(cvt<T>(w.ur1[0]), cvt<T>(w.ur1[1]), cvt<T>(w.ur1[2]), cvt<T>(w.ur1[3])) +
                     fw_d4(V0(-1), V0(0), V0(2), V0(3));
      const T fx = cvt<T>(w.fx), rho = cvt<T>(w.rho);
      p.u_out[o] = cvt<S>(fw_out(U0(0), dt, cvt<T>(w.ut), ppgu, fx, cvt<T>(w.rho_e), rho, alpha, dv_e, dv));
      p.v_out[o] = cvt<S>(fw_out(V0(0), dt, cvt<T>(w.vt), ppgv, fx, cvt<T>(w.rho_n), rho, alpha, dv_n, dv));
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pk[c] = pk1[c];
        ppv[c] = cvt<T>(w.pp1[c]);
        hh[c] = h1[c];
      }
      if (k + b + 2 < k1) load(win[b], k + b + 2);
    }
  }
}

// k-streaming with the divergence's inputs staged: as fw_stream_kernel, but a
// CTA's u_in and v_in windows of each level ((TJ+1) x (TI+5) of u: rows j, j+1,
// columns i-2 .. i+3; (TJ+5) x (TI+1) of v: rows j-2 .. j+3, columns i, i+1)
// are copied asynchronously into a D-level shared-memory ring, D-1 levels
// ahead, so the 20 stencil reads of a point come from shared memory and the
// loads in flight do not occupy registers. The point's 15 other values (pp,
// wgtfac, hhl of the next level at three columns; fx, rho at three columns,
// utens, vtens) keep the two-window register prefetch. Same arithmetic, in
// the same order, as fw_stream_kernel.
template <class P, int TI, int TJ, class Off>
__global__ void __launch_bounds__(TI * TJ) fw_tile_kernel(FW<typename P::S> p, double dt_d, double alpha_d, int kchunk) {
  typedef typename P::C T;
  typedef typename P::S S;
  constexpr int NT = TI * TJ, UI = TI + 5, UJ = TJ + 1, VI = TI + 1, VJ = TJ + 5;
  constexpr int NU = UI * UJ, NV = VI * VJ, SLOT = NU + NV, Q = (SLOT + NT - 1) / NT, D = 4;
  __shared__ __align__(16) S ring[D * SLOT];
  const T dt = kd<T>(dt_d), alpha = kd<T>(alpha_d);
  const int tid = threadIdx.x, tx = tid % TI, ty = tid / TI;
  const int i0 = blockIdx.x * TI, j0 = blockIdx.y * TJ;
  const int i = i0 + tx, j = j0 + ty;
  const bool own = i < p.ni && j < p.nj;
  const int k0 = blockIdx.z * kchunk, k1 = min(p.nk, k0 + kchunk);
  const Off sj = (Off)p.sj, sk = (Off)p.sk;
  // this thread's copies: element e of the slot (u window, then v window),
  // its offset from the field's level base and whether the point exists
  // (u: columns up to ni+2, rows up to nj; v: columns up to ni, rows up to
  // nj+2: what the domain's points read)
  Off goff[Q];
  int cfield[Q];   // 0 none, 1 u, 2 v
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int e = tid + q * NT;
    cfield[q] = 0;
    goff[q] = 0;
    if (e < NU) {
      const int r = e / UI, c = e - r * UI, ii = i0 - 2 + c, jj = j0 + r;
      if (ii <= p.ni + 2 && jj <= p.nj) {
        cfield[q] = 1;
        goff[q] = (Off)jj * sj + ii;
      }
    } else if (e < SLOT) {
      const int f = e - NU, r = f / VI, c = f - r * VI, ii = i0 + c, jj = j0 - 2 + r;
      if (ii <= p.ni && jj <= p.nj + 2) {
        cfield[q] = 2;
        goff[q] = (Off)jj * sj + ii;
      }
    }
  }
  auto issue = [&](int k, S* slot) {
    if (k < k1) {
      const Off ko = (Off)k * sk;
#pragma unroll
      for (int q = 0; q < Q; ++q)
        if (cfield[q]) cp_async(slot + tid + q * NT, (cfield[q] == 1 ? p.u_in : p.v_in) + (ko + goff[q]));
    }
    cp_async_commit();
  };
  const Off col = (Off)j * sj + i;
  const Off cn[3] = {0, 1, sj};
  auto ld = [&](const S* f, Off o) { return ldg(f + o); };
  struct Win {
    S pp1[3], wg1[3], hh1[3];
    S fx, rho, rho_e, rho_n, ut, vt;
  };
  auto load = [&](Win& w, int k) {
    const Off o = (Off)k * sk + col, o1 = o + sk;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      w.pp1[c] = ld(p.pp, o1 + cn[c]);
      w.wg1[c] = ld(p.wgtfac, o1 + cn[c]);
      w.hh1[c] = ld(p.hhl, o1 + cn[c]);
    }
    w.fx = ld(p.fx, o);
    w.rho = ld(p.rho, o);
    w.rho_e = ld(p.rho, o + 1);
    w.rho_n = ld(p.rho, o + sj);
    w.ut = ld(p.utens, o);
    w.vt = ld(p.vtens, o);
  };
#pragma unroll
  for (int x = 0; x < D - 1; ++x) issue(k0 + x, ring + x * SLOT);
  T pk[3], ppv[3], hh[3];
  Win win[2];
  if (own) {
    const Off o = (Off)k0 * sk + col;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ppv[c] = cvt<T>(ld(p.pp, o + cn[c]));
      pk[c] = fw_ppgk(cvt<T>(ld(p.wgtfac, o + cn[c])), ppv[c], cvt<T>(ld(p.pp, o + cn[c] - sk)));
      hh[c] = cvt<T>(ld(p.hhl, o + cn[c]));
    }
    load(win[0], k0);
    if (k0 + 1 < k1) load(win[1], k0 + 1);
  }
  int sl = 0;   // ring slot of level k
  for (int k = k0; k < k1; k += 2) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      if (k + b >= k1) break;
      cp_async_wait<D - 2>();   // this thread's copies of level k+b have landed
      __syncthreads();          // everyone's have; everyone is done with level k+b-1
      issue(k + b + D - 1, ring + (sl == 0 ? D - 1 : sl - 1) * SLOT);   // into level k+b-1's slot
      const S* W = ring + sl * SLOT;
      sl = sl == D - 1 ? 0 : sl + 1;
      if (!own) continue;
      const Win& w = win[b];
      const Off o = (Off)(k + b) * sk + col;
      T pk1[3], pc[3], h1[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pk1[c] = fw_ppgk(cvt<T>(w.wg1[c]), cvt<T>(w.pp1[c]), ppv[c]);
        pc[c] = pk1[c] - pk[c];
        h1[c] = cvt<T>(w.hh1[c]);
      }
      const T ppgu = fw_pgrad(ppv[1], ppv[0], pc[1], pc[0], h1[0], hh[0], h1[1], hh[1]);
      const T ppgv = fw_pgrad(ppv[2], ppv[0], pc[2], pc[0], h1[0], hh[0], h1[2], hh[2]);
      const S* su = W + ty * UI + tx + 2;    // u_in(i, j); the next row is j+1
      const S* sv = W + NU + (ty + 2) * VI + tx;   // v_in(i, j); the next column is i+1
      auto U0 = [&](int x) { return cvt<T>(su[x]); };             // u_in(i+x, j)
      auto U1 = [&](int x) { return cvt<T>(su[UI + x]); };        // u_in(i+x, j+1)
      auto V0 = [&](int y) { return cvt<T>(sv[y * VI]); };        // v_in(i, j+y)
      auto V1 = [&](int y) { return cvt<T>(sv[y * VI + 1]); };    // v_in(i+1, j+y)
      const T dv = fw_d4(U0(-2), U0(-1), U0(1), U0(2)) + fw_d4(V0(-2), V0(-1), V0(1), V0(2));
      const T dv_e = fw_d4(U0(-1), U0(0), U0(2), U0(3)) + fw_d4(V1(-2), V1(-1), V1(1), V1(2));
      const T dv_n = fw_d4(U1(-2), U1(-1), U1(1), U1(2)) + fw_d4(V0(-1), V0(0), V0(2), V0(3));
      const T fx = cvt<T>(w.fx), rho = cvt<T>(w.rho);
      p.u_out[o] = cvt<S>(fw_out(U0(0), dt, cvt<T>(w.ut), ppgu, fx, cvt<T>(w.rho_e), rho, alpha, dv_e, dv));
      p.v_out[o] = cvt<S>(fw_out(V0(0), dt, cvt<T>(w.vt), ppgv, fx, cvt<T>(w.rho_n), rho, alpha, dv_n, dv));
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pk[c] = pk1[c];
        ppv[c] = cvt<T>(w.pp1[c]);
        hh[c] = h1[c];
      }
      if (k + b + 2 < k1) load(win[b], k + b + 2);
    }
  }
  cp_async_wait<0>();
}

// k-streaming with every input staged by the tensor memory accelerator
// (OEC_STAGE_TMA): per level a CTA's nine boxes (u_in rows j, j+1, columns
// i-2 .. i+3; v_in rows j-2 .. j+3, columns i, i+1; pp, wgtfac, hhl of level
// k+1 and rho at columns i, i+1, rows j, j+1; fx, utens, vtens at the points)
// are copied by one thread with cp.async.bulk.tensor into a D-stage ring,
// completion counted on the stage's mbarrier, D levels ahead. A box starts at
// the 16-byte boundary at or below its first column; its element offset o
// into the box is the same for every tile, since tiles start at multiples of
// TI. Same arithmetic, in the same order, as fw_stream_kernel. A wait that
// gives up counts a timeout and the CTA stops after waiting (bounded) for the
// copies it still has in flight.
template <class S, int TI, int TJ>
struct FwTmaGeom {
  static constexpr int E = 16 / (int)sizeof(S);   // elements per 16 bytes
  static constexpr int rup(int x) { return (x + E - 1) / E * E; }
  static constexpr int BXU = rup(TI + 5 + E - 1), BYU = TJ + 1;   // u_in
  static constexpr int BXV = rup(TI + 1 + E - 1), BYV = TJ + 5;   // v_in
  static constexpr int BXC = rup(TI + 1 + E - 1), BYC = TJ + 1;   // pp, wgtfac, hhl (level k+1), rho
  static constexpr int BXP = rup(TI + E - 1), BYP = TJ;           // fx, utens, vtens
  static constexpr size_t al(size_t b) { return (b + 127) / 128 * 128; }
  static constexpr size_t SU = al(size_t(BXU) * BYU * sizeof(S)), SV = al(size_t(BXV) * BYV * sizeof(S));
  static constexpr size_t SC = al(size_t(BXC) * BYC * sizeof(S)), SP = al(size_t(BXP) * BYP * sizeof(S));
  // byte offsets in a stage (128-byte aligned), fields in FASTWAVES input
  // order: u_in, v_in, utens, vtens, pp, rho, wgtfac, hhl, fx
  __host__ __device__ static constexpr size_t off(int f) {
    return f == 0 ? 0 : f == 1 ? SU : f <= 3 ? SU + SV + (f - 2) * SP : f <= 7 ? SU + SV + 2 * SP + (f - 4) * SC
                                                                              : SU + SV + 2 * SP + 4 * SC;
  }
  static constexpr size_t STAGE = SU + SV + 3 * SP + 4 * SC;
  static constexpr unsigned TX =
      unsigned((size_t(BXU) * BYU + size_t(BXV) * BYV + 4 * size_t(BXC) * BYC + 3 * size_t(BXP) * BYP) * sizeof(S));
  static constexpr int D = 4;
  static constexpr size_t SMEM = D * STAGE + D * sizeof(unsigned long long);
};

struct FwMaps {
  CUtensorMap m[9];
  int x0[9], y0[9], z0[9], o[9];   // box corner of the tile at (0, 0, k = 0), element offset of the first column
};

template <class P, int TI, int TJ, class Off>
__global__ void __launch_bounds__(TI * TJ) fw_tma_kernel(const __grid_constant__ FwMaps mp, FW<typename P::S> p,
                                                          double dt_d, double alpha_d, int kchunk,
                                                          unsigned* __restrict__ timeouts) {
  typedef typename P::C T;
  typedef typename P::S S;
  typedef FwTmaGeom<S, TI, TJ> G;
  constexpr int D = G::D;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* bars = reinterpret_cast<unsigned long long*>(smem + size_t(D) * G::STAGE);
  const T dt = kd<T>(dt_d), alpha = kd<T>(alpha_d);
  const int tid = threadIdx.x, tx = tid % TI, ty = tid / TI;
  const int i0 = blockIdx.x * TI, j0 = blockIdx.y * TJ;
  const int i = i0 + tx, j = j0 + ty;
  const bool own = i < p.ni && j < p.nj;
  const int k0 = blockIdx.z * kchunk, k1 = min(p.nk, k0 + kchunk);
  if (tid == 0) {
    for (int x = 0; x < D; ++x) mbar_init(smem_u32(&bars[x]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int k) {   // thread 0 only: level k into stage (k - k0) % D
    const int sl = (k - k0) % D;
    unsigned char* st_ = smem + size_t(sl) * G::STAGE;
    const unsigned bar = smem_u32(&bars[sl]);
    mbar_expect_tx(bar, G::TX);
#pragma unroll
    for (int f = 0; f < 9; ++f) tma_load_3d(st_ + G::off(f), &mp.m[f], mp.x0[f] + i0, mp.y0[f] + j0, mp.z0[f] + k, bar);
  };
  if (tid == 0)
    for (int k = k0; k < min(k1, k0 + D); ++k) issue(k);
  int issued_to = min(k1, k0 + D);   // levels [k0, issued_to) issued (thread 0's view)
  int failed_at = -1;
  const Off sj = (Off)p.sj, sk = (Off)p.sk;
  const Off col = (Off)j * sj + i;
  const Off cn[3] = {0, 1, sj};
  T pk[3], ppv[3], hh[3];
  if (own) {
    const Off o = (Off)k0 * sk + col;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ppv[c] = cvt<T>(ldg(p.pp + (o + cn[c])));
      pk[c] = fw_ppgk(cvt<T>(ldg(p.wgtfac + (o + cn[c]))), ppv[c], cvt<T>(ldg(p.pp + (o + cn[c] - sk))));
      hh[c] = cvt<T>(ldg(p.hhl + (o + cn[c])));
    }
  }
  for (int k = k0; k < k1; ++k) {
    const int sl = (k - k0) % D;
    const bool ok = mbar_wait(smem_u32(&bars[sl]), (unsigned)(((k - k0) / D) & 1));
    if (__syncthreads_or(!ok)) {
      failed_at = k;
      if (tid == 0) atomicAdd(timeouts, 1u);
      break;
    }
    if (own) {
      const unsigned char* st_ = smem + size_t(sl) * G::STAGE;
      auto box = [&](int f) { return reinterpret_cast<const S*>(st_ + G::off(f)); };
      const S* su = box(0) + ty * G::BXU + mp.o[0] + 2 + tx;   // u_in(i, j); next row j+1
      const S* sv = box(1) + (ty + 2) * G::BXV + mp.o[1] + tx;   // v_in(i, j); next column i+1
      const int cp = ty * G::BXC + tx, pq = ty * G::BXP + tx;
      const S* spp = box(4) + cp + mp.o[4];
      const S* srh = box(5) + cp + mp.o[5];
      const S* swg = box(6) + cp + mp.o[6];
      const S* shh = box(7) + cp + mp.o[7];
      const int cc[3] = {0, 1, G::BXC};
      T pk1[3], pc[3], h1[3], pp1[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pp1[c] = cvt<T>(spp[cc[c]]);
        pk1[c] = fw_ppgk(cvt<T>(swg[cc[c]]), pp1[c], ppv[c]);
        pc[c] = pk1[c] - pk[c];
        h1[c] = cvt<T>(shh[cc[c]]);
      }
      const T ppgu = fw_pgrad(ppv[1], ppv[0], pc[1], pc[0], h1[0], hh[0], h1[1], hh[1]);
      const T ppgv = fw_pgrad(ppv[2], ppv[0], pc[2], pc[0], h1[0], hh[0], h1[2], hh[2]);
      auto U0 = [&](int x) { return cvt<T>(su[x]); };
      auto U1 = [&](int x) { return cvt<T>(su[G::BXU + x]); };
      auto V0 = [&](int y) { return cvt<T>(sv[y * G::BXV]); };
      auto V1 = [&](int y) { return cvt<T>(sv[y * G::BXV + 1]); };
      const T dv = fw_d4(U0(-2), U0(-1), U0(1), U0(2)) + fw_d4(V0(-2), V0(-1), V0(1), V0(2));
      const T dv_e = fw_d4(U0(-1), U0(0), U0(2), U0(3)) + fw_d4(V1(-2), V1(-1), V1(1), V1(2));
      const T dv_n = fw_d4(U1(-2), U1(-1), U1(1), U1(2)) + fw_d4(V0(-1), V0(0), V0(2), V0(3));
      const T fx = cvt<T>(box(8)[pq + mp.o[8]]), rho = cvt<T>(srh[0]);
      const T ut = cvt<T>(box(2)[pq + mp.o[2]]), vt = cvt<T>(box(3)[pq + mp.o[3]]);
      const Off o = (Off)k * sk + col;
      p.u_out[o] = cvt<S>(fw_out(U0(0), dt, ut, ppgu, fx, cvt<T>(srh[1]), rho, alpha, dv_e, dv));
      p.v_out[o] = cvt<S>(fw_out(V0(0), dt, vt, ppgv, fx, cvt<T>(srh[G::BXC]), rho, alpha, dv_n, dv));
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        pk[c] = pk1[c];
        ppv[c] = pp1[c];
        hh[c] = h1[c];
      }
    }
    __syncthreads();   // every thread is done with this stage
    if (tid == 0 && k + D < k1) {
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      issue(k + D);
      issued_to = k + D + 1;
    }
  }
  if (failed_at >= 0 && tid == 0)
    for (int k = failed_at; k < issued_to; ++k) mbar_wait(smem_u32(&bars[(k - k0) % D]), (unsigned)(((k - k0) / D) & 1));
}

template <class P, int TI, int TJ, class Off>
__global__ void __launch_bounds__(TI * TJ) fw_smem_kernel(FW<typename P::S> p, double dt_d, double alpha_d, int kchunk) {
  typedef typename P::C T;
  const T dt = kd<T>(dt_d), alpha = kd<T>(alpha_d);
  constexpr int NT = TI * TJ, PI = TI + 1, PJ = TJ + 1;
  __shared__ T s_pk[2][PJ][PI];
  __shared__ T s_pc[PJ][PI];
  __shared__ T s_dv[PJ][PI];
  const int tid = threadIdx.x, tx = tid % TI, ty = tid / TI;
  const int i0 = blockIdx.x * TI, j0 = blockIdx.y * TJ;
  const int k0 = blockIdx.z * kchunk, k1 = min(p.nk, k0 + kchunk);
  const int vi = min(TI, p.ni - i0), vj = min(TJ, p.nj - j0);
  const Off sj = (Off)p.sj, sk = (Off)p.sk, tile = (Off)j0 * sj + i0;
  int cur = 0;
  for (int idx = tid; idx < PI * PJ; idx += NT) {
    const int b = idx / PI, a = idx - b * PI;
    if (a < vi + 1 && b < vj + 1) s_pk[cur][b][a] = ppgk_at<P>(p, (Off)k0 * sk + tile + (Off)b * sj + a);
  }
  for (int k = k0; k < k1; ++k) {
    __syncthreads();
    for (int idx = tid; idx < PI * PJ; idx += NT) {
      const int b = idx / PI, a = idx - b * PI;
      if (a < vi + 1 && b < vj + 1) {
        const Off o = (Off)k * sk + tile + (Off)b * sj + a;
        const T pk1 = ppgk_at<P>(p, o + sk);
        s_pc[b][a] = pk1 - s_pk[cur][b][a];
        s_pk[cur ^ 1][b][a] = pk1;
        s_dv[b][a] = div_at<P>(p, o);
      }
    }
    __syncthreads();
    if (tx < vi && ty < vj) {
      const Off o = (Off)k * sk + tile + (Off)ty * sj + tx;
      fw_point<P>(p, o, s_pc[ty][tx], s_pc[ty][tx + 1], s_pc[ty + 1][tx], s_dv[ty][tx], s_dv[ty][tx + 1],
                  s_dv[ty + 1][tx], dt, alpha);
    }
    cur ^= 1;
  }
}

// ---- unfused: one kernel per stage ----------------------------------------
// temporaries: pk  [0,ni+1) x [0,nj+1) x [0,nk+1)   pitch ni+1, plane (ni+1)(nj+1)
//              pc, dv [0,ni+1) x [0,nj+1) x [0,nk)
//              pu, pv domain                        pitch ni, plane ni*nj
template <class P, class T = typename P::C>
__global__ void fw_s1(FW<typename P::S> p, T* pk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i > p.ni || j > p.nj) return;
  pk[((int64_t)k * (p.nj + 1) + j) * (p.ni + 1) + i] = ppgk_at<P>(p, (int64_t)k * p.sk + (int64_t)j * p.sj + i);
}
template <class P, class T = typename P::C>
__global__ void fw_s2(FW<typename P::S> p, const T* __restrict__ pk, T* __restrict__ pc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i > p.ni || j > p.nj) return;
  const int64_t plane = (int64_t)(p.nj + 1) * (p.ni + 1), o = ((int64_t)k * (p.nj + 1) + j) * (p.ni + 1) + i;
  pc[o] = pk[o + plane] - pk[o];
}
template <class P, int DIR, class T = typename P::C>
__global__ void fw_s34(FW<typename P::S> p, const T* __restrict__ pc, T* __restrict__ pg) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i >= p.ni || j >= p.nj) return;
  const int64_t o = (int64_t)k * p.sk + (int64_t)j * p.sj + i;
  const int64_t n = DIR == 0 ? 1 : p.sj;                 // neighbour in the field's storage
  const int64_t t = ((int64_t)k * (p.nj + 1) + j) * (p.ni + 1) + i;
  const int64_t tn = DIR == 0 ? 1 : (p.ni + 1);          // neighbour in the temporary
  pg[((int64_t)k * p.nj + j) * p.ni + i] =
      fw_pgrad(ld<P>(p.pp + o + n), ld<P>(p.pp + o), pc[t + tn], pc[t], ld<P>(p.hhl + o + p.sk), ld<P>(p.hhl + o),
               ld<P>(p.hhl + o + n + p.sk), ld<P>(p.hhl + o + n));
}
template <class P, class T = typename P::C>
__global__ void fw_s5(FW<typename P::S> p, T* dv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i > p.ni || j > p.nj) return;
  dv[((int64_t)k * (p.nj + 1) + j) * (p.ni + 1) + i] = div_at<P>(p, (int64_t)k * p.sk + (int64_t)j * p.sj + i);
}
template <class P, class T = typename P::C>
__global__ void fw_s6(FW<typename P::S> p, const T* __restrict__ pu, const T* __restrict__ pv, const T* __restrict__ dv,
                      double dt_d, double alpha_d) {
  typedef typename P::S S;
  const T dt = kd<T>(dt_d), alpha = kd<T>(alpha_d);
  const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y, k = blockIdx.z;
  if (i >= p.ni || j >= p.nj) return;
  const int64_t o = (int64_t)k * p.sk + (int64_t)j * p.sj + i;
  const int64_t t = ((int64_t)k * (p.nj + 1) + j) * (p.ni + 1) + i;
  const int64_t d = ((int64_t)k * p.nj + j) * p.ni + i;
  const T fx = ld<P>(p.fx + o), rho = ld<P>(p.rho + o), dvc = dv[t];
  p.u_out[o] = cvt<S>(fw_out(ld<P>(p.u_in + o), dt, ld<P>(p.utens + o), pu[d], fx, ld<P>(p.rho + o + 1), rho, alpha, dv[t + 1], dvc));
  p.v_out[o] = cvt<S>(fw_out(ld<P>(p.v_in + o), dt, ld<P>(p.vtens + o), pv[d], fx, ld<P>(p.rho + o + p.sj), rho, alpha,
                             dv[t + (p.ni + 1)], dvc));
}

struct Tmp {
  size_t pk, pc, dv, pu, pv, total;
};
Tmp tmp_layout(size_t e, const Dom& d) {
  const size_t plane1 = size_t(d.ni + 1) * (d.nj + 1), dom = size_t(d.ni) * d.nj * d.nk;
  Tmp t;
  t.pk = 0;
  t.pc = align_up(t.pk + e * plane1 * (d.nk + 1), 256);
  t.dv = align_up(t.pc + e * plane1 * d.nk, 256);
  t.pu = align_up(t.dv + e * plane1 * d.nk, 256);
  t.pv = align_up(t.pu + e * dom, 256);
  t.total = align_up(t.pv + e * dom, 256);
  return t;
}

int kchunk_of(const oec_schedule& s, int nk) { return (s.k_chunk <= 0 || s.k_chunk > nk) ? nk : s.k_chunk; }

// every element offset the k-streaming kernel forms (halo 3 in i/j, 1 in k)
// fits in a 32-bit int
bool offsets_fit_fw(const Dom& d) {
  const int64_t hi = (int64_t)(d.nk + 1) * d.sk + (int64_t)(d.nj + 3) * d.sj + d.ni + 3;
  const int64_t lo = -(d.sk + 3 * d.sj + 3);
  return hi < INT32_MAX && lo > INT32_MIN;
}
// 32-bit offsets unless the schedule asks for 64-bit ones or they do not fit
bool fw_int32(const oec_schedule& s, const Dom& d) { return s.index_bits != OEC_INDEX_64 && offsets_fit_fw(d); }

// tiles of the TMA-staged kernel (TI a multiple of 16 elements keeps every
// box corner on a 16-byte boundary)
#define OEC_FWTMA_TILES(X) X(32, 4) X(32, 8) X(64, 4)

template <class P, int TI, int TJ>
cudaError_t run_fw_tma(const oec_schedule& s, const Dom& d, const TmaField* tf, const FW<typename P::S>& p, double dt,
                       double alpha, cudaStream_t st) {
  typedef typename P::S S;
  typedef FwTmaGeom<S, TI, TJ> G;
  static_assert(TI % G::E == 0, "tile columns on 16-byte boundaries");
  // per field (FASTWAVES input order): columns and rows before the point
  // that its box starts at, level offset, box extents
  const int hx[9] = {2, 0, 0, 0, 0, 0, 0, 0, 0}, hy[9] = {0, 2, 0, 0, 0, 0, 0, 0, 0};
  const int kz[9] = {0, 0, 0, 0, 1, 0, 1, 1, 0};
  const int bx[9] = {G::BXU, G::BXV, G::BXP, G::BXP, G::BXC, G::BXC, G::BXC, G::BXC, G::BXP};
  const int by[9] = {G::BYU, G::BYV, G::BYP, G::BYP, G::BYC, G::BYC, G::BYC, G::BYC, G::BYP};
  FwMaps mp;
  for (int f = 0; f < 9; ++f) {
    const int64_t cx = tf[f].corner[0] - hx[f];
    const int o = (int)(((cx % G::E) + G::E) % G::E);
    mp.x0[f] = (int)(cx - o);
    mp.o[f] = o;
    mp.y0[f] = (int)(tf[f].corner[1] - hy[f]);
    mp.z0[f] = (int)(tf[f].corner[2] + kz[f]);
    if (mp.x0[f] % G::E != 0) return cudaErrorMisalignedAddress;
    if (!encode_map<S>(&mp.m[f], tf[f], d.sj, d.sk, bx[f], by[f])) return cudaErrorNotSupported;
  }
  unsigned* timeouts = wait_timeout_counter();
  if (!timeouts) return cudaErrorNotSupported;
  const int kc = (s.k_chunk <= 0 || s.k_chunk > d.nk) ? d.nk : s.k_chunk;
  dim3 g(ceil_div(d.ni, TI), ceil_div(d.nj, TJ), ceil_div(d.nk, kc));
  static std::once_flag attr;
  std::call_once(attr, [] {
    cudaFuncSetAttribute(fw_tma_kernel<P, TI, TJ, int>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::SMEM);
    cudaFuncSetAttribute(fw_tma_kernel<P, TI, TJ, int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)G::SMEM);
  });
  if (fw_int32(s, d))
    fw_tma_kernel<P, TI, TJ, int><<<g, TI * TJ, G::SMEM, st>>>(mp, p, dt, alpha, kc, timeouts);
  else
    fw_tma_kernel<P, TI, TJ, int64_t><<<g, TI * TJ, G::SMEM, st>>>(mp, p, dt, alpha, kc, timeouts);
  launched(st);
  return cudaGetLastError();
}

#define OEC_FW_TILES(X) X(32, 4) X(32, 8) X(64, 2) X(64, 4) X(128, 2)
// shared-memory u/v windows in the k-streaming form (OEC_STAGE_STREAM, unroll 2)
#define OEC_FWTILE_TILES(X) X(32, 4) X(32, 8) X(64, 4) X(128, 2)

template <class P>
cudaError_t dispatch(const oec_schedule& s, const Dom& d, const FW<typename P::S>& p, double dt, double alpha,
                     char* scratch, cudaStream_t st, const TmaField* tf) {
  if (s.fusion == OEC_FUSE_INLINE && s.staging == OEC_STAGE_TMA) {
    if (!tf) return cudaErrorInvalidValue;
#define X(a, b) if (s.tile_i == a && s.tile_j == b) return run_fw_tma<P, a, b>(s, d, tf, p, dt, alpha, st);
    OEC_FWTMA_TILES(X)
#undef X
    return cudaErrorInvalidValue;
  }
  typedef typename P::C T;
  if (s.fusion == OEC_FUSE_NONE) {
    Tmp t = tmp_layout(sizeof(T), d);
    T *pk = (T*)(scratch + t.pk), *pc = (T*)(scratch + t.pc), *dv = (T*)(scratch + t.dv);
    T *pu = (T*)(scratch + t.pu), *pv = (T*)(scratch + t.pv);
    dim3 b(32, 8);
    dim3 g1(ceil_div(d.ni + 1, 32), ceil_div(d.nj + 1, 8), d.nk + 1), g(ceil_div(d.ni + 1, 32), ceil_div(d.nj + 1, 8), d.nk);
    dim3 gd(ceil_div(d.ni, 32), ceil_div(d.nj, 8), d.nk);
    fw_s1<P><<<g1, b, 0, st>>>(p, pk); launched(st);
    fw_s2<P><<<g, b, 0, st>>>(p, pk, pc); launched(st);
    fw_s34<P, 0><<<gd, b, 0, st>>>(p, pc, pu); launched(st);
    fw_s34<P, 1><<<gd, b, 0, st>>>(p, pc, pv); launched(st);
    fw_s5<P><<<g, b, 0, st>>>(p, dv); launched(st);
    fw_s6<P><<<gd, b, 0, st>>>(p, pu, pv, dv, dt, alpha); launched(st);
    return cudaGetLastError();
  }
  if (s.staging == OEC_STAGE_STREAM && s.unroll == 2) {
    const int kc = kchunk_of(s, d.nk);
#define X(a, b)                                                                                       \
  if (s.tile_i == a && s.tile_j == b) {                                                               \
    dim3 g(ceil_div(d.ni, a), ceil_div(d.nj, b), ceil_div(d.nk, kc));                                 \
    if (fw_int32(s, d))                                                                            \
      fw_tile_kernel<P, a, b, int><<<g, a * b, 0, st>>>(p, dt, alpha, kc);                            \
    else                                                                                              \
      fw_tile_kernel<P, a, b, int64_t><<<g, a * b, 0, st>>>(p, dt, alpha, kc);                        \
    launched(st);                                                                                     \
    return cudaGetLastError();                                                                        \
  }
    OEC_FWTILE_TILES(X)
#undef X
    return cudaErrorInvalidValue;
  }
  if (s.staging == OEC_STAGE_STREAM) {
    const int kc = kchunk_of(s, d.nk);
    dim3 b(s.tile_i, s.tile_j);
    dim3 g(ceil_div(d.ni, s.tile_i), ceil_div(d.nj, s.tile_j), ceil_div(d.nk, kc));
    if (fw_int32(s, d))
      fw_stream_kernel<P, int><<<g, b, 0, st>>>(p, dt, alpha, kc);
    else
      fw_stream_kernel<P, int64_t><<<g, b, 0, st>>>(p, dt, alpha, kc);
    launched(st);
    return cudaGetLastError();
  }
  if (s.staging == OEC_STAGE_SMEM) {
    const int kc = kchunk_of(s, d.nk);
#define X(a, b)                                                                                 \
  if (s.tile_i == a && s.tile_j == b) {                                                         \
    dim3 g(ceil_div(d.ni, a), ceil_div(d.nj, b), ceil_div(d.nk, kc));                           \
    if (fw_int32(s, d))                                                                      \
      fw_smem_kernel<P, a, b, int><<<g, a * b, 0, st>>>(p, dt, alpha, kc);                      \
    else                                                                                        \
      fw_smem_kernel<P, a, b, int64_t><<<g, a * b, 0, st>>>(p, dt, alpha, kc);                  \
    launched(st);                                                                               \
    return cudaGetLastError();                                                                  \
  }
    OEC_FW_TILES(X)
#undef X
    return cudaErrorInvalidValue;
  }
  dim3 b(s.tile_i, s.tile_j);
  dim3 g(ceil_div(d.ni, s.tile_i), ceil_div(d.nj, s.tile_j), ceil_div(d.nk, s.unroll));
  switch (s.unroll) {
    case 1: fw_regs_kernel<P, 1><<<g, b, 0, st>>>(p, dt, alpha); launched(st); break;
    case 2: fw_regs_kernel<P, 2><<<g, b, 0, st>>>(p, dt, alpha); launched(st); break;
    case 4: fw_regs_kernel<P, 4><<<g, b, 0, st>>>(p, dt, alpha); launched(st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

bool fastwaves_schedule_ok(const oec_schedule& s, std::string& why) {
  if (s.arith != 0 && s.arith != 1) { why = "arith must be 0 (native) or 1 (double-float)"; return false; }
  if (s.fusion == OEC_FUSE_NONE) return true;
  if (s.fusion != OEC_FUSE_INLINE) { why = "fusion must be OEC_FUSE_INLINE or OEC_FUSE_NONE"; return false; }
  if (s.k_chunk < 0) { why = "k_chunk must be >= 0"; return false; }
  if (s.staging == OEC_STAGE_SMEM) {
#define X(a, b) if (s.tile_i == a && s.tile_j == b) return true;
    OEC_FW_TILES(X)
#undef X
    why = "fastwaves SMEM tiles: 32x4, 32x8, 64x2, 64x4, 128x2";
    return false;
  }
  if (s.staging == OEC_STAGE_TMA) {
#define X(a, b) if (s.tile_i == a && s.tile_j == b && s.unroll == 1) return true;
    OEC_FWTMA_TILES(X)
#undef X
    why = "fastwaves TMA tiles: 32x4, 32x8, 64x4 with unroll 1";
    return false;
  }
  if (s.staging != OEC_STAGE_REGS && s.staging != OEC_STAGE_STREAM) { why = "unknown staging"; return false; }
  if (s.staging == OEC_STAGE_STREAM && s.unroll == 2) {
#define X(a, b) if (s.tile_i == a && s.tile_j == b) return true;
    OEC_FWTILE_TILES(X)
#undef X
    why = "fastwaves STREAM with shared-memory u/v windows (unroll 2): tiles 32x4, 32x8, 64x4, 128x2";
    return false;
  }
  if (s.staging == OEC_STAGE_STREAM && s.unroll != 1) { why = "fastwaves STREAM: unroll 1 or 2"; return false; }
  if (s.staging == OEC_STAGE_REGS && s.unroll != 1 && s.unroll != 2 && s.unroll != 4) {
    why = "unroll (along k) must be 1, 2 or 4";
    return false;
  }
  if (s.tile_i < 16 || s.tile_i > 256 || s.tile_i % 16 || s.tile_j < 1 || s.tile_j > 16 || s.tile_i * s.tile_j > 1024) {
    why = "tile_i a multiple of 16 in [16,256], tile_j in [1,16], at most 1024 threads";
    return false;
  }
  return true;
}

size_t fastwaves_scratch_bytes(const oec_schedule& s, int dtype, const Dom& d) {
  return s.fusion == OEC_FUSE_NONE ? tmp_layout(dtype == OEC_F64 ? 8 : 4, d).total : 0;
}

cudaError_t fastwaves_launch(const oec_schedule& s, int dtype, const Dom& d, const FastwavesPtrs& f, double dt,
                             double alpha, void* scratch, cudaStream_t st, const TmaField* tf) {
  if (dtype == OEC_F64) {
    typedef double T;
    FW<T> p{(const T*)f.u_in, (const T*)f.v_in, (const T*)f.utens, (const T*)f.vtens, (const T*)f.pp,
            (const T*)f.rho, (const T*)f.wgtfac, (const T*)f.hhl, (const T*)f.fx, (T*)f.u_out, (T*)f.v_out,
            d.ni, d.nj, d.nk, d.sj, d.sk};
    if (s.arith == 1) return dispatch<P64D>(s, d, p, dt, alpha, (char*)scratch, st, tf);
    return dispatch<P64>(s, d, p, dt, alpha, (char*)scratch, st, tf);
  }
  typedef float T;
  FW<T> p{(const T*)f.u_in, (const T*)f.v_in, (const T*)f.utens, (const T*)f.vtens, (const T*)f.pp,
          (const T*)f.rho, (const T*)f.wgtfac, (const T*)f.hhl, (const T*)f.fx, (T*)f.u_out, (T*)f.v_out,
          d.ni, d.nj, d.nk, d.sj, d.sk};
  return dispatch<P32>(s, d, p, dt, alpha, (char*)scratch, st, tf);
}

}  // namespace oec
