// k_vadvc_seg.cu - the column sweep of the staged hdiff+vadvc form as a
// partitioned Thomas solve (schedule field sweep = OEC_SWEEP_SEGMENTS4 or
// OEC_SWEEP_SEGMENTS8): every column is cut into NSEG segments of consecutive
// levels, one thread each, so each thread's dependent chain covers nk/NSEG
// levels instead of the twisted form's nk/2.
//
// A segment holds the rows [s, e) of the column's system
//   a_k x_{k-1} + b_k x_k + c_k x_{k+1} = d_k
// (built from hdiff(u), hdiff(v) and w exactly as the twisted sweep builds
// them). Its thread
//  1. eliminates downwards with the coupling to the unknown x_{s-1} of the
//     segment below carried as a spike:
//       m = b_k - a_k G_{k-1},  G_k = c_k / m,  E_k = (d_k - a_k E_{k-1}) / m,
//       H_k = -a_k H_{k-1} / m  (H_{s-1} = -1, G_{s-1} = E_{s-1} = 0),
//     so that x_k = E_k - G_k x_{k+1} - H_k x_{s-1};
//  2. substitutes upwards to x_k = P_k + Q_k x_e + T_k x_{s-1}:
//       P_{e-1} = E_{e-1}, Q_{e-1} = -G_{e-1}, T_{e-1} = -H_{e-1};
//       P_k = E_k - G_k P_{k+1}, Q_k = -G_k Q_{k+1}, T_k = -H_k - G_k T_{k+1};
//  3. with the first (f_p = x_s) and last (l_p = x_{e-1}) rows of every
//     segment p of its column, solves the reduced system
//       f_p = P_s + Q_s f_{p+1} + T_s l_{p-1},  l_p = P_e + Q_e f_{p+1} + T_e l_{p-1}
//     by one pass up the segments (l_{p-1} = alpha + beta f_p) and one down;
//  4. forms x_k = P_k + Q_k f_{p+1} + T_k l_{p-1} for its rows.
// The bottom segment has a_0 = 0 (so H = T = 0), the top one c_{nk-1} = 0 (Q =
// 0). The system is strictly diagonally dominant, so every pivot, and the
// reduced system's 1 - T_s beta, stays away from zero without pivoting.
// Warp w of a CTA is segment w of the CTA's 32 columns (lane = column), so
// every level's values move as coalesced rows of 32 columns. Per level a thread
// keeps G, H, E_u, E_v, then P_u, P_v, Q, T, in its own scratch slots
// ([k][4][column]); the values of a level pass through a shared-memory ring
// filled by cp.async DEPTH-1 levels ahead.
#include <cmath>
#include <type_traits>

#include "arith.cuh"
#include "kcommon.cuh"
#include "kernels.h"
#include "k_vadvc.cuh"

namespace oec {
namespace {

template <class C, class S> __device__ __forceinline__ C wsum2(S a, S b) { return cvt<C>(a) + cvt<C>(b); }
template <> __device__ __forceinline__ df64 wsum2<df64, double>(double a, double b) { return df_from_double(a + b); }

template <class P, int NSEG, int DEPTH>
struct SegSmem {
  typedef typename P::S S;
  typedef typename P::C C;
  typedef typename P::R R;
  static constexpr int NT = 32 * NSEG;
  struct Fwd {
    C u[DEPTH][NT], v[DEPTH][NT];
    S w0[DEPTH][NT], w1[DEPTH][NT];
  };
  struct Back {
    R q[4][DEPTH][NT];
  };
  union {
    Fwd f;
    Back b;
  } ring;
  R red[8][NSEG][32];   // per segment and column: P_s u/v, Q_s, T_s, P_e u/v, Q_e, T_e
};

__host__ __device__ __forceinline__ int seg_lo(int p, int nk, int nseg) { return int((int64_t)nk * p / nseg); }

template <class P, int NSEG, int DEPTH, bool DTR_P2, class Off>
__global__ void __launch_bounds__(32 * NSEG)
hv_segments_kernel(HV<typename P::S> p, const typename P::C* __restrict__ ud, const typename P::C* __restrict__ vd,
                   double dtr_d, typename P::R* __restrict__ scr) {
  typedef typename P::S S;
  typedef typename P::C C;
  typedef typename P::R R;
  typedef SegSmem<P, NSEG, DEPTH> SM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM& sm = *reinterpret_cast<SM*>(smem_raw);
  const int t = threadIdx.x, lane = t & 31, seg = t >> 5;
  const int64_t ncol = (int64_t)p.ni * p.nj;
  const int64_t col = (int64_t)blockIdx.x * 32 + lane;
  const bool active = col < ncol;
  const int i = active ? int(col % p.ni) : 0, j = active ? int(col / p.ni) : 0;
  const int nk = p.nk;
  const int s = seg_lo(seg, nk, NSEG), e = seg_lo(seg + 1, nk, NSEG);
  const int L = active ? e - s : 0;   // this thread's rows
  const C dtr = cvt<C>(dtr_d);
  const float dtr_f = (float)dtr_d;
  auto times_dtr = [&](C x) { return DTR_P2 ? mul_p2(x, dtr_f) : dtr * x; };
  const int64_t cbase = (int64_t)j * p.sj + i;
  const S* __restrict__ wcol = p.w + cbase;
  const Off ncol_o = (Off)ncol, col_o = (Off)col, sk_o = (Off)p.sk;
  const R zero = cvt<R>(0.0f);

  // ---- 1. rows and downward elimination; ring slot q holds level s - 1 + q
  auto issue = [&](int q) {
    if (L > 0 && q <= L + 1) {
      const int lv = s - 1 + q;
      if (lv >= 0 && lv < nk) {
        const int sl = q % DEPTH;
        const Off o = (Off)lv * ncol_o + col_o;
        cp_async(&sm.ring.f.u[sl][t], ud + o);
        cp_async(&sm.ring.f.v[sl][t], vd + o);
        cp_async(&sm.ring.f.w0[sl][t], wcol + (Off)lv * sk_o);
        cp_async(&sm.ring.f.w1[sl][t], wcol + (Off)lv * sk_o + 1);
      }
    }
    cp_async_commit();
  };
  // wf of the edge between the levels of slots q-1 and q (w at slot q's level)
  auto wf_at = [&](int q) {
    const int sl = q % DEPTH;
    return mul_p2(wsum2<C>(sm.ring.f.w0[sl][t], sm.ring.f.w1[sl][t]), 0.5f);
  };
#pragma unroll 1
  for (int q = 0; q < DEPTH - 1; ++q) issue(q);
  C uc = zero_<C>(), vc = zero_<C>(), pbu = zero_<C>(), pbv = zero_<C>(), ak = zero_<C>();
  if (L > 0) {
    cp_async_wait<DEPTH - 3>();   // slots 0 and 1 (levels s-1 and s) have landed
    uc = sm.ring.f.u[1][t];
    vc = sm.ring.f.v[1][t];
    if (s >= 1) {   // the edge below row s
      const C wfs = wf_at(1);
      pbu = wfs * subf(uc, sm.ring.f.u[0][t]);
      pbv = wfs * subf(vc, sm.ring.f.v[0][t]);
      ak = mul_p2(wfs, -0.25f);
    }
  }
  R G = zero, H = cvt<R>(-1.0f), Eu = zero, Ev = zero;
#pragma unroll 2
  for (int r = 0; r < L; ++r) {
    issue(r + DEPTH - 1);
    cp_async_wait<DEPTH - 3>();   // slot r+2 (level k+1) has landed
    const int k = s + r;
    const bool lo = k >= 1, hi = k <= nk - 2;
    C un = zero_<C>(), vn = zero_<C>(), pau = zero_<C>(), pav = zero_<C>(), ck = zero_<C>(), an = zero_<C>();
    if (hi) {   // the edge above row k
      const int sl = (r + 2) % DEPTH;
      un = sm.ring.f.u[sl][t];
      vn = sm.ring.f.v[sl][t];
      const C wfn = wf_at(r + 2);
      pau = wfn * subf(un, uc);
      pav = wfn * subf(vn, vc);
      ck = mul_p2(wfn, 0.25f);
      an = mul_p2(wfn, -0.25f);
    }
    const C b = addf(addf(dtr, abs_(ak)), abs_(ck));
    C du = times_dtr(uc), dv = times_dtr(vc);
    if (lo && hi) {
      du = subf(du, mul_p2(addf(pbu, pau), 0.125f));
      dv = subf(dv, mul_p2(addf(pbv, pav), 0.125f));
    } else if (lo) {
      du = subf(du, mul_p2(pbu, 0.125f));
      dv = subf(dv, mul_p2(pbv, 0.125f));
    } else if (hi) {
      du = subf(du, mul_p2(pau, 0.125f));
      dv = subf(dv, mul_p2(pav, 0.125f));
    }
    const R ra = cvt<R>(ak);
    const R m = subf(cvt<R>(b), ra * G);
    const R inv = rcp_pivot(m);
    G = cvt<R>(ck) * inv;
    H = -((ra * H) * inv);
    Eu = subf(cvt<R>(du), ra * Eu) * inv;
    Ev = subf(cvt<R>(dv), ra * Ev) * inv;
    R* sp = scr + ((Off)k * 4 * ncol_o + col_o);
    sp[0] = G;
    sp[ncol_o] = H;
    sp[2 * ncol_o] = Eu;
    sp[3 * ncol_o] = Ev;
    uc = un;
    vc = vn;
    pbu = pau;
    pbv = pav;
    ak = an;
  }
  cp_async_wait<0>();
  __syncthreads();          // every thread is done with the forward ring
  __threadfence_block();    // this thread's scratch stores precede its copies below

  // ---- 2. upward substitution; back-ring slot q holds the q-th row from the top
  auto issue_b = [&](int q) {
    if (q < L) {
      const int sl = q % DEPTH;
      const R* sp = scr + ((Off)(e - 1 - q) * 4 * ncol_o + col_o);
#pragma unroll
      for (int x = 0; x < 4; ++x) cp_async(&sm.ring.b.q[x][sl][t], sp + (Off)x * ncol_o);
    }
    cp_async_commit();
  };
#pragma unroll 1
  for (int q = 0; q < DEPTH - 1; ++q) issue_b(q);
  R Pu = zero, Pv = zero, Q = zero, T = zero;
  R Pue = zero, Pve = zero, Qe = zero, Te = zero;   // the segment's last row
#pragma unroll 2
  for (int q = 0; q < L; ++q) {
    issue_b(q + DEPTH - 1);
    cp_async_wait<DEPTH - 1>();   // row q has landed
    const int sl = q % DEPTH;
    const R Gk = sm.ring.b.q[0][sl][t], Hk = sm.ring.b.q[1][sl][t];
    const R Euk = sm.ring.b.q[2][sl][t], Evk = sm.ring.b.q[3][sl][t];
    if (q == 0) {
      Pu = Euk;
      Pv = Evk;
      Q = -Gk;
      T = -Hk;
      Pue = Pu;
      Pve = Pv;
      Qe = Q;
      Te = T;
    } else {
      Pu = subf(Euk, Gk * Pu);
      Pv = subf(Evk, Gk * Pv);
      Q = -(Gk * Q);
      T = subf(-Hk, Gk * T);
    }
    R* sp = scr + ((Off)(e - 1 - q) * 4 * ncol_o + col_o);
    sp[0] = Pu;
    sp[ncol_o] = Pv;
    sp[2 * ncol_o] = Q;
    sp[3 * ncol_o] = T;
  }
  cp_async_wait<0>();

  // ---- 3. the reduced system of the column's segments (every thread of the
  // column runs it; empty segments are skipped)
  sm.red[0][seg][lane] = Pu;    // first row (the last one substituted)
  sm.red[1][seg][lane] = Pv;
  sm.red[2][seg][lane] = Q;
  sm.red[3][seg][lane] = T;
  sm.red[4][seg][lane] = Pue;   // last row
  sm.red[5][seg][lane] = Pve;
  sm.red[6][seg][lane] = Qe;
  sm.red[7][seg][lane] = Te;
  __syncthreads();
  __threadfence_block();   // this thread's stores of step 2 precede its copies below
  R gu[NSEG], gv[NSEG], dl[NSEG], au[NSEG], av[NSEG], bt[NSEG];
  {
    R alu = zero, alv = zero, be = zero;   // l of the segment below = alpha + beta f
    const R one = cvt<R>(1.0f);
#pragma unroll
    for (int x = 0; x < NSEG; ++x) {
      gu[x] = gv[x] = dl[x] = au[x] = av[x] = bt[x] = zero;
      if (seg_lo(x + 1, nk, NSEG) > seg_lo(x, nk, NSEG)) {
        const R Ts = sm.red[3][x][lane], Qs = sm.red[2][x][lane];
        const R Tl = sm.red[7][x][lane], Ql = sm.red[6][x][lane];
        const R inv = rcp_pivot(subf(one, Ts * be));
        gu[x] = addf(sm.red[0][x][lane], Ts * alu) * inv;
        gv[x] = addf(sm.red[1][x][lane], Ts * alv) * inv;
        dl[x] = Qs * inv;
        alu = addf(sm.red[4][x][lane], Tl * addf(alu, be * gu[x]));
        alv = addf(sm.red[5][x][lane], Tl * addf(alv, be * gv[x]));
        be = addf(Ql, Tl * (be * dl[x]));
        au[x] = alu;
        av[x] = alv;
        bt[x] = be;
      }
    }
  }
  R fu_up = zero, fv_up = zero, lu_dn = zero, lv_dn = zero;   // f of the segment above, l of the one below
  {
    R fnu = zero, fnv = zero;
    bool below = false;
#pragma unroll
    for (int x = NSEG - 1; x >= 0; --x) {
      if (seg_lo(x + 1, nk, NSEG) > seg_lo(x, nk, NSEG)) {
        if (x == seg) {
          fu_up = fnu;
          fv_up = fnv;
        }
        if (x < seg && !below) {
          lu_dn = addf(au[x], bt[x] * fnu);
          lv_dn = addf(av[x], bt[x] * fnv);
          below = true;
        }
        const R fu = addf(gu[x], dl[x] * fnu), fv = addf(gv[x], dl[x] * fnv);
        fnu = fu;
        fnv = fv;
      }
    }
  }

  // ---- 4. the solution of the segment's rows, bottom up
  auto issue_f = [&](int q) {
    if (q < L) {
      const int sl = q % DEPTH;
      const R* sp = scr + ((Off)(s + q) * 4 * ncol_o + col_o);
#pragma unroll
      for (int x = 0; x < 4; ++x) cp_async(&sm.ring.b.q[x][sl][t], sp + (Off)x * ncol_o);
    }
    cp_async_commit();
  };
  if (L == 0) return;
#pragma unroll 1
  for (int q = 0; q < DEPTH - 1; ++q) issue_f(q);
  Off o = (Off)s * sk_o + (Off)cbase;
#pragma unroll 2
  for (int q = 0; q < L; ++q) {
    issue_f(q + DEPTH - 1);
    cp_async_wait<DEPTH - 1>();
    const int sl = q % DEPTH;
    const R Pk = sm.ring.b.q[0][sl][t], Pvk = sm.ring.b.q[1][sl][t];
    const R Qk = sm.ring.b.q[2][sl][t], Tk = sm.ring.b.q[3][sl][t];
    const R xu = addf(addf(Pk, Qk * fu_up), Tk * lu_dn);
    const R xv = addf(addf(Pvk, Qk * fv_up), Tk * lv_dn);
    p.uo[o] = cvt<S>(xu);
    p.vo[o] = cvt<S>(xv);
    o += sk_o;
  }
  cp_async_wait<0>();
}

template <class P, int NSEG>
cudaError_t launch_seg(const Dom& d, const HV<typename P::S>& p, const typename P::C* ud, const typename P::C* vd,
                       double dtr, typename P::R* scr, bool p2, bool o32, cudaStream_t st) {
  constexpr int DEPTH = NSEG == 8 ? 4 : 6;   // 48 KB (8 segments) / 32 KB of shared memory per CTA
  typedef SegSmem<P, NSEG, DEPTH> SM;
  const unsigned grid = (unsigned)(((int64_t)d.ni * d.nj + 31) / 32);
  const void* fn = p2 ? (o32 ? (const void*)hv_segments_kernel<P, NSEG, DEPTH, true, int>
                             : (const void*)hv_segments_kernel<P, NSEG, DEPTH, true, int64_t>)
                      : (o32 ? (const void*)hv_segments_kernel<P, NSEG, DEPTH, false, int>
                             : (const void*)hv_segments_kernel<P, NSEG, DEPTH, false, int64_t>);
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SM));
  if (e != cudaSuccess) return e;
  if (p2) {
    if (o32)
      hv_segments_kernel<P, NSEG, DEPTH, true, int><<<grid, 32 * NSEG, sizeof(SM), st>>>(p, ud, vd, dtr, scr);
    else
      hv_segments_kernel<P, NSEG, DEPTH, true, int64_t><<<grid, 32 * NSEG, sizeof(SM), st>>>(p, ud, vd, dtr, scr);
  } else {
    if (o32)
      hv_segments_kernel<P, NSEG, DEPTH, false, int><<<grid, 32 * NSEG, sizeof(SM), st>>>(p, ud, vd, dtr, scr);
    else
      hv_segments_kernel<P, NSEG, DEPTH, false, int64_t><<<grid, 32 * NSEG, sizeof(SM), st>>>(p, ud, vd, dtr, scr);
  }
  return cudaGetLastError();
}

template <class P>
cudaError_t dispatch_seg(int nseg, const Dom& d, const HV<typename P::S>& p, const void* ud, const void* vd,
                         double dtr, void* scr, bool p2, bool o32, cudaStream_t st) {
  typedef typename P::C C;
  typedef typename P::R R;
  if (nseg == 4) return launch_seg<P, 4>(d, p, (const C*)ud, (const C*)vd, dtr, (R*)scr, p2, o32, st);
  if (nseg == 8) return launch_seg<P, 8>(d, p, (const C*)ud, (const C*)vd, dtr, (R*)scr, p2, o32, st);
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t hdiff_vadvc_segments_launch(int nseg, int dtype, int arith, const Dom& d, const void* u, const void* v,
                                        const void* w, const void* coeff, void* u_out, void* v_out,
                                        const void* ud, const void* vd, double dtr, void* scr, bool o32,
                                        cudaStream_t st) {
  int e2 = 0;
  const bool p2 = std::frexp(dtr, &e2) == 0.5 && e2 > -120 && e2 < 120;
  if (dtype == OEC_F64) {
    HV<double> p{(const double*)u, (const double*)v, (const double*)w, (const double*)coeff,
                 (double*)u_out, (double*)v_out, d.ni, d.nj, d.nk, d.sj, d.sk};
    if (arith >= 1) return dispatch_seg<P64D>(nseg, d, p, ud, vd, dtr, scr, p2, o32, st);
    return dispatch_seg<P64>(nseg, d, p, ud, vd, dtr, scr, false, o32, st);
  }
  HV<float> p{(const float*)u, (const float*)v, (const float*)w, (const float*)coeff,
              (float*)u_out, (float*)v_out, d.ni, d.nj, d.nk, d.sj, d.sk};
  if (arith >= 1) return dispatch_seg<P32D>(nseg, d, p, ud, vd, dtr, scr, false, o32, st);
  return dispatch_seg<P32>(nseg, d, p, ud, vd, dtr, scr, false, o32, st);
}

}  // namespace oec
