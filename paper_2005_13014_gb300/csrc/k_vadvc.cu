// k_vadvc.cu - horizontal diffusion of u and v followed by implicit vertical
// advection: per (i, j) column a tridiagonal system
//   a_k x_{k-1} + b_k x_k + c_k x_{k+1} = d_k
// with wf(k) = (w + w(i+1))/2, a_k = -wf(k)/4 (k >= 1), c_k = wf(k+1)/4
// (k <= K-2), b_k = dtr + |a_k| + |c_k| (strictly diagonally dominant),
// d_k = dtr*phi_k - (a_k (phi_{k-1} - phi_k) + c_k (phi_{k+1} - phi_k))/2 with
// the column-end terms left out, solved by the Thomas algorithm (forward
// elimination, back substitution; the paper names Thomas for vertical implicit
// integration, §VII-B) for phi = hdiff(u) and hdiff(v) with one matrix.
//
// Fused form (the producer inlined into the column sweep, paper §V-A): one CTA
// owns TI x TJ columns and walks up them in chunks of KC levels. Per chunk all
// 2*TI*TJ threads evaluate hdiff of u and v for the chunk's levels on an
// overlapped tile in shared memory; then one thread per column runs the
// chunk's elimination steps (lagging one level, since row k needs phi_{k+1}).
// c'_k, d'_k go to a per-tile scratch slot ([k][3][column]) that the back
// substitution reads on the way down.
// Staged form: hdiff writes hdiff(u), hdiff(v) to scratch, then a column
// kernel runs the sweep from a shared-memory ring filled by asynchronous
// copies.
// Batched form: a persistent kernel pulls (member, tile) items of an ensemble
// of domains from an atomic counter and runs the fused tile sweep on each.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <mutex>
#include <type_traits>

#include "arith.cuh"
#include "kcommon.cuh"
#include "kernels.h"
#include "k_vadvc.cuh"
#include "k_hdiff_vec.cuh"

namespace oec {
namespace {

// One row of the system and its right-hand sides for both fields (compute type C).
template <class C>
__device__ __forceinline__ void hv_row(bool lo, bool hi, C wf_c, C wf_p, C dtr, C um, C uc, C up, C vm, C vc, C vp,
                                       C& a, C& b, C& c, C& du, C& dv) {
  a = lo ? -mul_p2(wf_c, 0.25f) : zero_<C>();
  c = hi ? mul_p2(wf_p, 0.25f) : zero_<C>();
  b = dtr + abs_(a) + abs_(c);
  const C tu = dtr * uc, tv = dtr * vc;
  if (lo && hi) {
    du = tu - mul_p2(a * (um - uc) + c * (up - uc), 0.5f);
    dv = tv - mul_p2(a * (vm - vc) + c * (vp - vc), 0.5f);
  } else if (hi) {
    du = tu - mul_p2(c * (up - uc), 0.5f);
    dv = tv - mul_p2(c * (vp - vc), 0.5f);
  } else if (lo) {
    du = tu - mul_p2(a * (um - uc), 0.5f);
    dv = tv - mul_p2(a * (vm - vc), 0.5f);
  } else {
    du = tu;
    dv = tv;
  }
}

template <class P, int TI, int TJ, int KC>
struct HVSmem {
  typedef typename P::S S;
  typedef typename P::C C;
  static constexpr int WI = TI + 4, WJ = TJ + 4, NC = TI * TJ, NT = 2 * NC, RING = KC + 2;
  static constexpr int QW = (WJ * WI + NT - 1) / NT;        // window positions per thread
  static constexpr int QR = (TJ * (TI + 1) + NT - 1) / NT;  // w-row positions per thread
  C win[2][KC][WJ][WI];
  C lap[2][KC][TJ + 2][TI + 2];
  C flx[2][KC][TJ][TI + 1];
  C fly[2][KC][TJ + 1][TI];
  C ring[2][RING][NC];
  S wrow[KC][TJ][TI + 1];
  S cf[KC][NC];
  C wf[KC][NC];
  int item;
};

// The fused sweep of one tile (all 2*TI*TJ threads of the CTA call it). Every
// thread owns fixed positions of each plane (window, Laplacian, fluxes,
// outputs) and loops over both fields and the chunk's levels there, so index
// arithmetic is paid once per chunk. In the elimination phase thread t works
// on column t % NC for field t / NC (u or v); both threads of a column carry
// the shared c' recurrence.
template <class P, int TI, int TJ, int KC>
__device__ void hv_tile(const HV<typename P::S>& p, int i0, int j0, typename P::R* __restrict__ slot,
                        typename P::C dtr, HVSmem<P, TI, TJ, KC>& sm) {
  typedef typename P::S S;
  typedef typename P::C C;
  typedef typename P::R R;
  typedef HVSmem<P, TI, TJ, KC> SM;
  constexpr int NC = SM::NC, NT = SM::NT, RING = SM::RING, WI = SM::WI, WJ = SM::WJ;
  constexpr int QW = SM::QW, QR = SM::QR;
  const int tid = threadIdx.x;
  const int vi = min(TI, p.ni - i0), vj = min(TJ, p.nj - j0);
  const int nk = p.nk;
  // elimination-phase role: column q, field f
  const int q = tid % NC, fld = tid / NC;
  const int tx = q % TI, ty = q / TI;
  const bool col = tx < vi && ty < vj;
  const int64_t cbase = (int64_t)(j0 + ty) * p.sj + (i0 + tx);
  const S* __restrict__ src = fld ? p.v : p.u;
  S* __restrict__ dst = fld ? p.vo : p.uo;

  // ---- per-thread load positions (computed once per tile) -----------------
  int64_t woff[QW];
  bool wok[QW];
#pragma unroll
  for (int x = 0; x < QW; ++x) {
    const int e = tid + x * NT, r = e / WI, c = e % WI;
    wok[x] = e < WJ * WI && c < vi + 4 && r < vj + 4;
    woff[x] = (int64_t)(j0 - 2 + r) * p.sj + (i0 - 2 + c);
  }
  int64_t roff[QR];
  bool rok[QR];
#pragma unroll
  for (int x = 0; x < QR; ++x) {
    const int e = tid + x * NT, r = e / (TI + 1), c = e % (TI + 1);
    rok[x] = e < TJ * (TI + 1) && c < vi + 1 && r < vj;
    roff[x] = (int64_t)(j0 + r) * p.sj + (i0 + c);
  }
  const bool cfok = tid < NC && col;
  S pw[QW][2][KC], pr[QR][KC], pc[KC];
  auto issue = [&](int k0, int nl) {
#pragma unroll
    for (int l = 0; l < KC; ++l) {
      if (l < nl) {
        const int64_t ko = (int64_t)(k0 + l) * p.sk;
#pragma unroll
        for (int x = 0; x < QW; ++x)
          if (wok[x]) {
            pw[x][0][l] = ldg(p.u + ko + woff[x]);
            pw[x][1][l] = ldg(p.v + ko + woff[x]);
          }
#pragma unroll
        for (int x = 0; x < QR; ++x)
          if (rok[x]) pr[x][l] = ldg(p.w + ko + roff[x]);
        if (cfok) pc[l] = ldg(p.coeff + ko + cbase);
      }
    }
  };
  auto land = [&](int nl) {
#pragma unroll
    for (int l = 0; l < KC; ++l) {
      if (l < nl) {
#pragma unroll
        for (int x = 0; x < QW; ++x)
          if (wok[x]) {
            const int e = tid + x * NT;
            (&sm.win[0][l][0][0])[e] = cvt<C>(pw[x][0][l]);
            (&sm.win[1][l][0][0])[e] = cvt<C>(pw[x][1][l]);
          }
#pragma unroll
        for (int x = 0; x < QR; ++x)
          if (rok[x]) (&sm.wrow[l][0][0])[tid + x * NT] = pr[x][l];
        if (cfok) sm.cf[l][q] = pc[l];
      }
    }
  };

  C um = zero_<C>(), uc = zero_<C>(), wf_c = zero_<C>();
  R cp = cvt<R>(0.0f), dp = cvt<R>(0.0f);
  int knext = 0;   // next elimination step
  issue(0, min(KC, nk));
  land(min(KC, nk));
  __syncthreads();

  for (int k0 = 0; k0 < nk; k0 += KC) {
    const int nl = min(KC, nk - k0);
    // ---- phase A: hdiff of u and v (and wf) for levels [k0, k0+nl) ----------
    for (int e = tid; e < (TJ + 2) * (TI + 2); e += NT) {
      const int r = e / (TI + 2), c = e % (TI + 2);
      if (c < vi + 2 && r < vj + 2) {
#pragma unroll
        for (int f = 0; f < 2; ++f)
#pragma unroll
          for (int l = 0; l < KC; ++l)
            if (l < nl) {
              const auto& W = sm.win[f][l];
              sm.lap[f][l][r][c] = hlap(W[r + 1][c + 1], W[r + 1][c], W[r + 1][c + 2], W[r][c + 1], W[r + 2][c + 1]);
            }
      }
    }
    if (tid < NC && col) {
#pragma unroll
      for (int l = 0; l < KC; ++l)
        if (l < nl) sm.wf[l][q] = mul_p2(cvt<C>(sm.wrow[l][ty][tx]) + cvt<C>(sm.wrow[l][ty][tx + 1]), 0.5f);
    }
    __syncthreads();
    for (int e = tid; e < TJ * (TI + 1) + (TJ + 1) * TI; e += NT) {
      if (e < TJ * (TI + 1)) {
        const int r = e / (TI + 1), c = e % (TI + 1);
        if (c < vi + 1 && r < vj) {
#pragma unroll
          for (int f = 0; f < 2; ++f)
#pragma unroll
            for (int l = 0; l < KC; ++l)
              if (l < nl) {
                const auto& W = sm.win[f][l];
                const auto& L = sm.lap[f][l];
                sm.flx[f][l][r][c] = hflux(L[r + 1][c + 1], L[r + 1][c], W[r + 2][c + 2], W[r + 2][c + 1]);
              }
        }
      } else {
        const int g = e - TJ * (TI + 1), r = g / TI, c = g % TI;
        if (c < vi && r < vj + 1) {
#pragma unroll
          for (int f = 0; f < 2; ++f)
#pragma unroll
            for (int l = 0; l < KC; ++l)
              if (l < nl) {
                const auto& W = sm.win[f][l];
                const auto& L = sm.lap[f][l];
                sm.fly[f][l][r][c] = hflux(L[r + 1][c + 1], L[r][c + 1], W[r + 2][c + 2], W[r + 1][c + 2]);
              }
        }
      }
    }
    __syncthreads();
    if (col) {   // thread (q, fld): hdiff output of field fld at column q
#pragma unroll
      for (int l = 0; l < KC; ++l)
        if (l < nl)
          sm.ring[fld][(k0 + l) % RING][q] =
              hout(sm.win[fld][l][ty + 2][tx + 2], cvt<C>(sm.cf[l][q]), sm.flx[fld][l][ty][tx + 1], sm.flx[fld][l][ty][tx],
                   sm.fly[fld][l][ty + 1][tx], sm.fly[fld][l][ty][tx]);
    }
    __syncthreads();
    // the next chunk's loads fly while this chunk's elimination steps run
    const int k0n = k0 + KC, nln = min(KC, nk - k0n);
    if (k0n < nk) issue(k0n, nln);
    // ---- phase B: elimination steps whose rows are now complete -------------
    const int last_avail = k0 + nl - 1;
    const int kend = last_avail == nk - 1 ? nk - 1 : last_avail - 1;
    if (col) {
      if (knext == 0) {
        wf_c = sm.wf[0][q];
        uc = sm.ring[fld][0][q];
      }
      for (int k = knext; k <= kend; ++k) {
        const bool lo = k > 0, hi = k + 1 < nk;
        const C up = hi ? sm.ring[fld][(k + 1) % RING][q] : zero_<C>();
        const C wf_p = hi ? sm.wf[k + 1 - k0][q] : zero_<C>();
        const C a = lo ? -mul_p2(wf_c, 0.25f) : zero_<C>();
        const C c = hi ? mul_p2(wf_p, 0.25f) : zero_<C>();
        const C b = dtr + abs_(a) + abs_(c);
        const C t = dtr * uc;
        C d;
        if (lo && hi) d = t - mul_p2(a * (um - uc) + c * (up - uc), 0.5f);
        else if (hi) d = t - mul_p2(c * (up - uc), 0.5f);
        else if (lo) d = t - mul_p2(a * (um - uc), 0.5f);
        else d = t;
        const R ra = cvt<R>(a);
        const R m = k == 0 ? cvt<R>(b) : subf(cvt<R>(b), ra * cp);
        const R inv = rcp_(m);
        cp = cvt<R>(c) * inv;
        dp = subf(cvt<R>(d), ra * dp) * inv;
        R* s = slot + (int64_t)k * 3 * NC + q;
        if (fld == 0) s[0] = cp;
        s[(1 + fld) * NC] = dp;
        um = uc;
        uc = up;
        wf_c = wf_p;
      }
    }
    knext = kend + 1;
    __syncthreads();
    if (k0n < nk) {
      land(nln);
      __syncthreads();
    }
  }
  // ---- back substitution (thread per column and field), loads batched ------
  if (col) {
    constexpr int BK = 8;
    R x = dp;
    int64_t o = (int64_t)(nk - 1) * p.sk + cbase;
    dst[o] = cvt<S>(x);
    for (int kt = nk - 2; kt >= 0; kt -= BK) {
      R c_[BK], d_[BK];
#pragma unroll
      for (int y = 0; y < BK; ++y) {
        if (kt - y >= 0) {
          const R* s = slot + (int64_t)(kt - y) * 3 * NC + q;
          c_[y] = s[0];
          d_[y] = s[(1 + fld) * NC];
        }
      }
#pragma unroll
      for (int y = 0; y < BK; ++y) {
        if (kt - y >= 0) {
          x = subf(d_[y], c_[y] * x);
          o -= p.sk;
          dst[o] = cvt<S>(x);
        }
      }
    }
  }
  __syncthreads();
  (void)src;
}

template <class P, int TI, int TJ, int KC>
__global__ void __launch_bounds__(2 * TI * TJ)
hv_fused_kernel(HV<typename P::S> p, double dtr, typename P::R* __restrict__ scr) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<HVSmem<P, TI, TJ, KC>*>(smem_raw);
  const int tile = blockIdx.y * gridDim.x + blockIdx.x;
  hv_tile<P, TI, TJ, KC>(p, blockIdx.x * TI, blockIdx.y * TJ, scr + (int64_t)tile * 3 * p.nk * TI * TJ,
                         cvt<typename P::C>(dtr), sm);
}

template <class P, int TI, int TJ, int KC>
__global__ void __launch_bounds__(2 * TI * TJ)
hv_batch_kernel(const HVMember* __restrict__ members, int n_members, int total_items, int* __restrict__ counter,
                double dtr, typename P::R* __restrict__ scr, int64_t slot_elems) {
  typedef typename P::S S;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<HVSmem<P, TI, TJ, KC>*>(smem_raw);
  typename P::R* slot = scr + (int64_t)blockIdx.x * slot_elems;
  for (;;) {
    if (threadIdx.x == 0) sm.item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = sm.item;
    __syncthreads();
    if (item >= total_items) break;
    int m = 0;
    while (m + 1 < n_members && members[m + 1].tile_begin <= item) ++m;
    const HVMember& mb = members[m];
    const int t = item - mb.tile_begin;
    HV<S> p{(const S*)mb.u, (const S*)mb.v, (const S*)mb.w, (const S*)mb.coeff, (S*)mb.uo, (S*)mb.vo,
            mb.ni, mb.nj, mb.nk, mb.sj, mb.sk};
    hv_tile<P, TI, TJ, KC>(p, (t % mb.tiles_i) * TI, (t / mb.tiles_i) * TJ, slot, cvt<typename P::C>(dtr), sm);
  }
}

// w(i) + w(i+1) in the compute type: for FP64 fields with double-float
// compute, the binary64 sum rounded once by one FP64 add and then split into a
// pair (one conversion instead of two and a pair addition); otherwise the
// compute type's own sum.
template <class C, class S> __device__ __forceinline__ C wsum(S a, S b) { return cvt<C>(a) + cvt<C>(b); }
template <> __device__ __forceinline__ df64 wsum<df64, double>(double a, double b) { return df_from_double(a + b); }

// Staged form, column sweep over hdiff(u), hdiff(v) held in the compute type
// (domain layout, pitch ni, plane ni*nj), by twisted factorisation: the
// column's rows [0, m) are eliminated upwards from level 0 and its rows
// [m, nk) downwards from the top level at the same time (m = ceil(nk/2)),
// the two halves meet in a 2 x 2 system for x_{m-1}, x_m, and each half
// substitutes back outwards. The operation count is that of the Thomas
// algorithm; each thread's sequential chain is half a column long. Both
// halves run one instruction stream: a half walks its levels in direction
// dir (+1 up, -1 down), and for a row the coupling to the level behind it is
// beta (a_k going up, c_k going down) and to the level ahead gamma:
//   m_k = b_k - beta_k g_prev,  g_k = gamma_k / m_k,
//   e_k = (d_k - beta_k e_prev) / m_k,   x_k = e_k - g_k x_ahead.
// Warp layout: lanes 0..15 eliminate 16 columns upwards, lanes 16..31 the same
// columns downwards (partner = lane ^ 16); NC columns per CTA, consecutive in
// (j, i) order. A thread solves both fields (one shared g recurrence). The
// values a level needs (hdiff(u), hdiff(v) there, w for the edge behind it)
// are copied asynchronously into a shared-memory ring DEPTH levels ahead, and
// row s+1 is built while row s is eliminated. g, e_u, e_v go to scratch
// ([k][g, e_u, e_v][column]) and come back through the same kind of ring for
// the back substitution. Each thread reads only ring entries its own copies
// wrote; the one barrier separates the two uses of the ring. DTR_P2: dtr is a
// power of two in float range, so dtr * phi is an exact scaling (for
// double-float, two float multiplies instead of a pair product).
// L2 use: the scratch rows have a pitch of ncolp columns (a multiple of 16),
// so each 128-byte line of scratch (16 columns of one value at one level)
// belongs to one half-warp. The DISCARD form (for scratch larger than L2;
// scr 128-byte aligned) stores scratch with evict-last priority and reads
// and writes the streamed fields with evict-first priority, so that the
// recurrence values of the columns in flight stay in L2 until the back
// substitution reads them, and then drops those lines from L2 without
// writing them back, four back steps (12 lines of a half-warp, one per lane)
// at a time. The values of a half's last step are used from registers and
// not stored.
// shared-memory ring of one block of the column sweep (bytes)
template <class P, int NC, int DEPTH>
__host__ __device__ constexpr size_t thomas_ring_bytes() {
  constexpr size_t FB = size_t(DEPTH) * 2 * NC * (2 * sizeof(typename P::C) + 2 * sizeof(typename P::S));
  constexpr size_t BB = size_t(DEPTH) * 2 * NC * 3 * sizeof(typename P::R);
  return FB > BB ? FB : BB;
}

// One block of the column sweep: NC columns (2 NC threads), the block-th
// group of NC columns of the domain; ring: thomas_ring_bytes() of shared
// memory, 16-byte aligned.
template <class P, int NC, int DEPTH, bool DTR_P2, class Off, bool DISCARD>
__device__ __forceinline__ void hv_thomas_block(const HV<typename P::S>& p, const typename P::C* __restrict__ ud,
                                                const typename P::C* __restrict__ vd, double dtr_d,
                                                typename P::R* __restrict__ scr, int64_t ncolp, int64_t block,
                                                unsigned char* ring) {
  typedef typename P::S S;
  typedef typename P::C C;
  typedef typename P::R R;
  constexpr int NT = 2 * NC;
  C(*su)[NT] = reinterpret_cast<C(*)[NT]>(ring);
  C(*sv)[NT] = su + DEPTH;
  S(*sw0)[NT] = reinterpret_cast<S(*)[NT]>(sv + DEPTH);
  S(*sw1)[NT] = sw0 + DEPTH;
  const int t = threadIdx.x, lane = t & 31;
  const bool down = lane >= 16;
  const int64_t ncol = (int64_t)p.ni * p.nj;
  const int64_t col = block * NC + (t >> 5) * 16 + (lane & 15);
  const bool active = col < ncol;   // inactive threads only join the barrier and the exchange
  // the active lanes of this thread's half-warp (they share scratch lines)
  const unsigned hmask = __ballot_sync(0xFFFFFFFFu, active) & (0xFFFFu << (lane & 16));
  uint64_t keep = 0, stream = 0;
  if (DISCARD) {
    keep = l2_evict_last();
    stream = l2_evict_first();
  }
  // loads and stores with the L2 priorities in the DISCARD form, plain otherwise
  auto ld_async = [&](auto* dst, const auto* src, uint64_t pol) {
    if (DISCARD) cp_async_l2(dst, src, pol); else cp_async(dst, src);
  };
  auto st_g = [&](auto* dst, auto v, uint64_t pol) {
    if (DISCARD) st_l2(dst, v, pol); else *dst = v;
  };
  const int i = active ? int(col % p.ni) : 0, j = active ? int(col / p.ni) : 0;
  const int nk = p.nk, mid = (nk + 1) / 2;
  const int nsteps = active ? (down ? nk - mid : mid) : 0;
  const C dtr = cvt<C>(dtr_d);
  const float dtr_f = (float)dtr_d;
  auto times_dtr = [&](C x) { return DTR_P2 ? mul_p2(x, dtr_f) : dtr * x; };
  const int64_t cbase = (int64_t)j * p.sj + i;
  const S* __restrict__ wcol = p.w + cbase;
  // element offsets per level in Off (32-bit when every offset fits)
  const Off ncol_o = (Off)ncol, ncolp_o = (Off)ncolp, col_o = (Off)col, sk_o = (Off)p.sk;
  // level of step s, and the level whose w gives the edge behind step s
  // (the edge between levels k-1 and k belongs to w at level k)
  auto lev = [&](int st) { return down ? nk - 1 - st : st; };
  auto wlev = [&](int st) { return down ? nk - st : st; };
  auto issue = [&](int st) {
    if (active && st <= nsteps) {
      const int sl = st % DEPTH, k = lev(st), kw = wlev(st);
      if (k >= 0 && k < nk) {
        const Off o = (Off)k * ncol_o + col_o;
        ld_async(&su[sl][t], ud + o, stream);
        ld_async(&sv[sl][t], vd + o, stream);
      }
      if (kw < nk) {
        ld_async(&sw0[sl][t], wcol + (Off)kw * sk_o, stream);
        ld_async(&sw1[sl][t], wcol + (Off)kw * sk_o + 1, stream);
      }
    }
    cp_async_commit();
  };
  // wf of the edge held in slot st (zero where there is none)
  auto wf_of = [&](int st) {
    const int sl = st % DEPTH;
    return wlev(st) < nk ? mul_p2(wsum<C>(sw0[sl][t], sw1[sl][t]), 0.5f) : zero_<C>();
  };
  const float sgn = down ? -1.0f : 1.0f;   // beta = -sgn wf_behind / 4, gamma = sgn wf_ahead / 4
  R g = cvt<R>(0.0f), eu = cvt<R>(0.0f), ev = cvt<R>(0.0f);
#pragma unroll 1
  for (int st = 0; st < DEPTH - 1; ++st) issue(st);
  cp_async_wait<DEPTH - 3>();   // slots 0 and 1 have landed
  // row of step 0: no level behind; ahead: slot 1 (absent only when nk == 1)
  const bool ahead0 = nsteps > 0 && lev(1) >= 0 && lev(1) < nk;
  // pu, pv: wf * (phi(next) - phi) of the edge ahead of the current row,
  // unscaled. The explicit part of a row is -(beta (phi(k-1) - phi(k)) +
  // gamma (phi(k+1) - phi(k))) / 2 = -sgn/8 (p_behind + p_ahead), and a row's
  // p_ahead is the next row's p_behind, so each product is formed once. The
  // scalings by +-1/4, 1/2 and +-1/8 are exact, so this is bit for bit the
  // value of the two products written out.
  C u1 = zero_<C>(), v1 = zero_<C>(), wfa = zero_<C>(), pu = zero_<C>(), pv = zero_<C>();
  C beta = zero_<C>(), gamma = zero_<C>(), b = dtr, ru = zero_<C>(), rv = zero_<C>();
  const float sgn8 = 0.125f * sgn;
  if (nsteps > 0) {
    const C u0 = su[0][t], v0 = sv[0][t];
    if (ahead0) {
      u1 = su[1][t];
      v1 = sv[1][t];
      wfa = wf_of(1);
      pu = wfa * subf(u1, u0);
      pv = wfa * subf(v1, v0);
      gamma = mul_p2(wfa, 0.25f * sgn);
    }
    b = addf(dtr, abs_(gamma));
    ru = times_dtr(u0);
    rv = times_dtr(v0);
    if (ahead0) {
      ru = subf(ru, mul_p2(pu, sgn8));
      rv = subf(rv, mul_p2(pv, sgn8));
    }
  }
  // elimination of the row of step st (step 0 needs no special case:
  // beta = 0 and g = 0 make m = b exactly)
  auto eliminate = [&](int st, bool store) {
    const R rb = cvt<R>(beta);
    const R m = fms_(cvt<R>(b), rb, g);
    const R inv = rcp_pivot(m);
    g = cvt<R>(gamma) * inv;
    eu = fms_(cvt<R>(ru), rb, eu) * inv;
    ev = fms_(cvt<R>(rv), rb, ev) * inv;
    if (store) {
      R* sp = scr + ((Off)lev(st) * 3 * ncolp_o + col_o);
      st_g(sp, g, keep);
      st_g(sp + ncolp_o, eu, keep);
      st_g(sp + 2 * ncolp_o, ev, keep);
    }
  };
  // row of step st+1 (it has a level behind; hi: it has one ahead)
  auto build_next = [&](int st, bool hi) {
    C u2 = zero_<C>(), v2 = zero_<C>(), wf2 = zero_<C>(), qu = zero_<C>(), qv = zero_<C>();
    if (hi) {
      const int sl = (st + 2) % DEPTH;
      u2 = su[sl][t];
      v2 = sv[sl][t];
      wf2 = wf_of(st + 2);
      qu = wf2 * subf(u2, u1);
      qv = wf2 * subf(v2, v1);
    }
    beta = mul_p2(wfa, -0.25f * sgn);
    gamma = hi ? mul_p2(wf2, 0.25f * sgn) : zero_<C>();
    b = addf(addf(dtr, abs_(beta)), abs_(gamma));
    const C tu = times_dtr(u1), tv = times_dtr(v1);
    if (hi) {
      ru = subf(tu, mul_p2(addf(pu, qu), sgn8));
      rv = subf(tv, mul_p2(addf(pv, qv), sgn8));
    } else {
      ru = subf(tu, mul_p2(pu, sgn8));
      rv = subf(tv, mul_p2(pv, sgn8));
    }
    u1 = u2;
    v1 = v2;
    pu = qu;
    pv = qv;
    wfa = wf2;
  };
  // every row a half builds has a level ahead (the other half's first row is
  // there), except the single row of a one-level column
  int st = 0;
#pragma unroll 2
  for (; st + 1 < nsteps; ++st) {
    issue(st + DEPTH - 1);
    cp_async_wait<DEPTH - 3>();   // slot st+2 has landed
    eliminate(st, true);
    build_next(st, true);
  }
  if (st < nsteps) {
    issue(st + DEPTH - 1);
    eliminate(st, false);
  }
  cp_async_wait<0>();
  // the halves meet: x_lo = x_{mid-1} (upward half's last row), x_hi = x_mid
  const R g_o = shfl_xor_(g, 16), eu_o = shfl_xor_(eu, 16), ev_o = shfl_xor_(ev, 16);
  const R g_lo = down ? g_o : g, g_hi = down ? g : g_o;
  const R inv = rcp_pivot(fms_(cvt<R>(1.0f), g_lo, g_hi));
  R xu, xv;
  {
    const R eu_lo = down ? eu_o : eu, eu_hi = down ? eu : eu_o;
    const R ev_lo = down ? ev_o : ev, ev_hi = down ? ev : ev_o;
    const R xu_lo = fms_(eu_lo, g_lo, eu_hi) * inv, xv_lo = fms_(ev_lo, g_lo, ev_hi) * inv;
    xu = down ? fms_(eu_hi, g_hi, xu_lo) : xu_lo;
    xv = down ? fms_(ev_hi, g_hi, xv_lo) : xv_lo;
  }
  __syncthreads();   // every thread is done with the forward ring
  __threadfence_block();   // this thread's scratch stores precede its copies below
  R(*sg)[NT] = reinterpret_cast<R(*)[NT]>(ring);
  R(*seu)[NT] = sg + DEPTH;
  R(*sev)[NT] = seu + DEPTH;
  // back substitution outwards: back step mm handles step nsteps-2-mm
  auto issue_b = [&](int mm) {
    const int sb = nsteps - 2 - mm;
    if (sb >= 0) {
      const int sl = mm % DEPTH;
      const R* sp = scr + ((Off)lev(sb) * 3 * ncolp_o + col_o);
      cp_async(&sg[sl][t], sp);
      cp_async(&seu[sl][t], sp + ncolp_o);
      cp_async(&sev[sl][t], sp + 2 * ncolp_o);
    }
    cp_async_commit();
  };
  if (nsteps == 0) return;
#pragma unroll 1
  for (int mm = 0; mm < DEPTH - 1; ++mm) issue_b(mm);
  Off o = (Off)lev(nsteps - 1) * sk_o + (Off)cbase;
  const Off ostep = down ? sk_o : -sk_o;   // outwards
  st_g(p.uo + o, cvt<S>(xu), stream);
  st_g(p.vo + o, cvt<S>(xv), stream);
  // the half-warp's first column: its scratch lines start there. Lane l < 12
  // of the half drops the line of value l % 3 of back step first + l / 3.
  const int lh = lane & 15;
  const R* hline = scr + (col_o - (Off)lh);
  auto drop4 = [&](int first, int n) {
    __syncwarp(hmask);   // every lane of the half has its copies of these steps
    if (lh < 3 * n) l2_discard(hline + ((Off)lev(nsteps - 2 - (first + lh / 3)) * 3 + lh % 3) * ncolp_o);
  };
#pragma unroll 4
  for (int mm = 0; mm < nsteps - 1; ++mm) {
    issue_b(mm + DEPTH - 1);
    cp_async_wait<DEPTH - 1>();   // back step mm's values have landed
    const int sl = mm % DEPTH;
    if (DISCARD && (mm & 3) == 3) drop4(mm - 3, 4);
    const R gk = sg[sl][t];
    xu = fms_(seu[sl][t], gk, xu);
    xv = fms_(sev[sl][t], gk, xv);
    o += ostep;
    st_g(p.uo + o, cvt<S>(xu), stream);
    st_g(p.vo + o, cvt<S>(xv), stream);
  }
  if (DISCARD && ((nsteps - 1) & 3)) drop4((nsteps - 1) & ~3, (nsteps - 1) & 3);
  cp_async_wait<0>();
}

template <class P, int NC, int DEPTH, bool DTR_P2, class Off, bool DISCARD>
__global__ void __launch_bounds__(2 * NC) hv_thomas_kernel(HV<typename P::S> p, const typename P::C* __restrict__ ud,
                                                           const typename P::C* __restrict__ vd, double dtr_d,
                                                           typename P::R* __restrict__ scr, int64_t ncolp) {
  __shared__ __align__(16) unsigned char ring[thomas_ring_bytes<P, NC, DEPTH>()];
  hv_thomas_block<P, NC, DEPTH, DTR_P2, Off, DISCARD>(p, ud, vd, dtr_d, scr, ncolp, blockIdx.x, ring);
}

// The same column sweep with the two fields in separate warps (schedule
// field sweep = OEC_SWEEP_SPLIT): warp 0 of a CTA solves 16 columns for u,
// warp 1 the same columns for v (lanes 0..15 upwards, 16..31 downwards, as
// above). Each thread builds the matrix part of its rows (w, beta, gamma, b,
// the g recurrence) itself, so that part is computed twice per column, but
// every thread's sequential chain carries one right-hand side instead of two
// and twice as many warps share the SMs: the sweep is bound by the latency of
// its dependent chains, not by instruction throughput. Per level a thread
// writes g and its e to its field's half of the scratch ([field][k][g, e][column]).
template <class P, int DEPTH, bool DTR_P2, class Off>
__global__ void __launch_bounds__(64) hv_thomas_split_kernel(HV<typename P::S> p, const typename P::C* __restrict__ ud,
                                                             const typename P::C* __restrict__ vd, double dtr_d,
                                                             typename P::R* __restrict__ scr) {
  typedef typename P::S S;
  typedef typename P::C C;
  typedef typename P::R R;
  constexpr int NT = 64;
  constexpr size_t FB = size_t(DEPTH) * NT * (sizeof(C) + 2 * sizeof(S));
  constexpr size_t BB = size_t(DEPTH) * NT * 2 * sizeof(R);
  __shared__ __align__(16) unsigned char ring[FB > BB ? FB : BB];
  C(*sphi)[NT] = reinterpret_cast<C(*)[NT]>(ring);
  S(*sw0)[NT] = reinterpret_cast<S(*)[NT]>(sphi + DEPTH);
  S(*sw1)[NT] = sw0 + DEPTH;
  const int t = threadIdx.x, lane = t & 31, fld = t >> 5;
  const bool down = lane >= 16;
  const int64_t ncol = (int64_t)p.ni * p.nj;
  const int64_t col = (int64_t)blockIdx.x * 16 + (lane & 15);
  const bool active = col < ncol;
  const int i = active ? int(col % p.ni) : 0, j = active ? int(col / p.ni) : 0;
  const int nk = p.nk, mid = (nk + 1) / 2;
  const int nsteps = active ? (down ? nk - mid : mid) : 0;
  const C dtr = cvt<C>(dtr_d);
  const float dtr_f = (float)dtr_d;
  auto times_dtr = [&](C x) { return DTR_P2 ? mul_p2(x, dtr_f) : dtr * x; };
  const int64_t cbase = (int64_t)j * p.sj + i;
  const S* __restrict__ wcol = p.w + cbase;
  const C* __restrict__ phi = fld ? vd : ud;
  const Off ncol_o = (Off)ncol, col_o = (Off)col, sk_o = (Off)p.sk;
  R* __restrict__ fscr = scr + (Off)fld * (Off)2 * (Off)nk * ncol_o;   // this field's [k][g, e][column]
  auto lev = [&](int st) { return down ? nk - 1 - st : st; };
  auto wlev = [&](int st) { return down ? nk - st : st; };
  auto issue = [&](int st) {
    if (active && st <= nsteps) {
      const int sl = st % DEPTH, k = lev(st), kw = wlev(st);
      if (k >= 0 && k < nk) cp_async(&sphi[sl][t], phi + ((Off)k * ncol_o + col_o));
      if (kw < nk) {
        cp_async(&sw0[sl][t], wcol + (Off)kw * sk_o);
        cp_async(&sw1[sl][t], wcol + (Off)kw * sk_o + 1);
      }
    }
    cp_async_commit();
  };
  auto wf_of = [&](int st) {
    const int sl = st % DEPTH;
    return wlev(st) < nk ? mul_p2(wsum<C>(sw0[sl][t], sw1[sl][t]), 0.5f) : zero_<C>();
  };
  const float sgn = down ? -1.0f : 1.0f;
  R g = cvt<R>(0.0f), e = cvt<R>(0.0f);
#pragma unroll 1
  for (int st = 0; st < DEPTH - 1; ++st) issue(st);
  cp_async_wait<DEPTH - 3>();   // slots 0 and 1 have landed
  const bool ahead0 = nsteps > 0 && lev(1) >= 0 && lev(1) < nk;
  C f1 = zero_<C>(), wfa = zero_<C>(), pf = zero_<C>();
  C beta = zero_<C>(), gamma = zero_<C>(), b = dtr, rf = zero_<C>();
  const float sgn8 = 0.125f * sgn;
  if (nsteps > 0) {
    const C f0 = sphi[0][t];
    if (ahead0) {
      f1 = sphi[1][t];
      wfa = wf_of(1);
      pf = wfa * subf(f1, f0);
      gamma = mul_p2(wfa, 0.25f * sgn);
    }
    b = addf(dtr, abs_(gamma));
    rf = times_dtr(f0);
    if (ahead0) rf = subf(rf, mul_p2(pf, sgn8));
  }
  auto eliminate = [&](int st) {
    const R rb = cvt<R>(beta);
    const R m = fms_(cvt<R>(b), rb, g);
    const R inv = rcp_pivot(m);
    g = cvt<R>(gamma) * inv;
    e = fms_(cvt<R>(rf), rb, e) * inv;
    R* sp = fscr + ((Off)lev(st) * 2 * ncol_o + col_o);
    sp[0] = g;
    sp[ncol_o] = e;
  };
  auto build_next = [&](int st, bool hi) {
    C f2 = zero_<C>(), wf2 = zero_<C>(), qf = zero_<C>();
    if (hi) {
      const int sl = (st + 2) % DEPTH;
      f2 = sphi[sl][t];
      wf2 = wf_of(st + 2);
      qf = wf2 * subf(f2, f1);
    }
    beta = mul_p2(wfa, -0.25f * sgn);
    gamma = hi ? mul_p2(wf2, 0.25f * sgn) : zero_<C>();
    b = addf(addf(dtr, abs_(beta)), abs_(gamma));
    const C tf = times_dtr(f1);
    rf = hi ? subf(tf, mul_p2(addf(pf, qf), sgn8)) : subf(tf, mul_p2(pf, sgn8));
    f1 = f2;
    pf = qf;
    wfa = wf2;
  };
  int st = 0;
#pragma unroll 2
  for (; st + 1 < nsteps; ++st) {
    issue(st + DEPTH - 1);
    cp_async_wait<DEPTH - 3>();   // slot st+2 has landed
    eliminate(st);
    build_next(st, true);
  }
  if (st < nsteps) {
    issue(st + DEPTH - 1);
    eliminate(st);
  }
  cp_async_wait<0>();
  // the halves meet (x_lo = x_{mid-1}, x_hi = x_mid)
  const R g_o = shfl_xor_(g, 16), e_o = shfl_xor_(e, 16);
  const R g_lo = down ? g_o : g, g_hi = down ? g : g_o;
  const R inv = rcp_pivot(fms_(cvt<R>(1.0f), g_lo, g_hi));
  R x;
  {
    const R e_lo = down ? e_o : e, e_hi = down ? e : e_o;
    const R x_lo = fms_(e_lo, g_lo, e_hi) * inv;
    x = down ? fms_(e_hi, g_hi, x_lo) : x_lo;
  }
  __syncthreads();          // every thread is done with the forward ring
  __threadfence_block();    // this thread's scratch stores precede its copies below
  R(*sg)[NT] = reinterpret_cast<R(*)[NT]>(ring);
  R(*se)[NT] = sg + DEPTH;
  auto issue_b = [&](int mm) {
    const int sb = nsteps - 2 - mm;
    if (sb >= 0) {
      const int sl = mm % DEPTH;
      const R* sp = fscr + ((Off)lev(sb) * 2 * ncol_o + col_o);
      cp_async(&sg[sl][t], sp);
      cp_async(&se[sl][t], sp + ncol_o);
    }
    cp_async_commit();
  };
  if (nsteps == 0) return;
#pragma unroll 1
  for (int mm = 0; mm < DEPTH - 1; ++mm) issue_b(mm);
  S* __restrict__ out = fld ? p.vo : p.uo;
  Off o = (Off)lev(nsteps - 1) * sk_o + (Off)cbase;
  const Off ostep = down ? sk_o : -sk_o;
  out[o] = cvt<S>(x);
#pragma unroll 4
  for (int mm = 0; mm < nsteps - 1; ++mm) {
    issue_b(mm + DEPTH - 1);
    cp_async_wait<DEPTH - 1>();
    const int sl = mm % DEPTH;
    x = fms_(se[sl][t], sg[sl][t], x);
    o += ostep;
    out[o] = cvt<S>(x);
  }
  cp_async_wait<0>();
}

size_t csize(int dtype, int arith) { return dtype == OEC_F32 ? 4 : 8; }   // compute type bytes
size_t rsize() { return 8; }                                                // double or df64

template <class P, int TI, int TJ, int KC>
cudaError_t launch_fused(const Dom& d, const HV<typename P::S>& p, double dtr, void* scratch, cudaStream_t st) {
  typedef HVSmem<P, TI, TJ, KC> SM;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(hv_fused_kernel<P, TI, TJ, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(SM));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 g(ceil_div(d.ni, TI), ceil_div(d.nj, TJ));
  hv_fused_kernel<P, TI, TJ, KC><<<g, 2 * TI * TJ, sizeof(SM), st>>>(p, dtr, (typename P::R*)scratch); launched(st);
  return cudaGetLastError();
}

// the dynamic shared-memory attribute is set by batch_occupancy() at batch
// creation, before any stream capture
template <class P, int TI, int TJ, int KC>
cudaError_t launch_batch(const HVBatchLaunch& b, cudaStream_t st) {
  typedef HVSmem<P, TI, TJ, KC> SM;
  hv_batch_kernel<P, TI, TJ, KC><<<b.grid, 2 * TI * TJ, sizeof(SM), st>>>(
      b.members, b.n_members, b.total_items, b.counter, b.dtr, (typename P::R*)b.scratch, b.slot_elems); launched(st);
  return cudaGetLastError();
}

template <class P, int TI, int TJ, int KC>
int batch_occupancy() {
  typedef HVSmem<P, TI, TJ, KC> SM;
  cudaFuncSetAttribute(hv_batch_kernel<P, TI, TJ, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SM));
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, hv_batch_kernel<P, TI, TJ, KC>, 2 * TI * TJ, sizeof(SM)) !=
      cudaSuccess)
    return 1;
  return n > 0 ? n : 1;
}

// tiles (TI, TJ) and levels per chunk: KC keeps the shared memory of the
// 8-byte compute types under ~64 KB
#define OEC_HV_TILES(X) X(16, 4) X(32, 2) X(8, 8) X(32, 4) X(8, 4) X(16, 2)
template <int TI, int TJ, int CB> struct KCOf {
  static constexpr int v = (TI * TJ >= 128) ? (CB == 4 ? 4 : 2) : (TI * TJ >= 64) ? (CB == 4 ? 8 : 4) : (CB == 4 ? 16 : 8);
};

template <class P>
cudaError_t dispatch_fused(const oec_schedule& s, const Dom& d, const HV<typename P::S>& p, double dtr, void* scratch,
                           cudaStream_t st) {
  constexpr int CB = sizeof(typename P::C);
#define X(a, b) \
  if (s.tile_i == a && s.tile_j == b) return launch_fused<P, a, b, KCOf<a, b, CB>::v>(d, p, dtr, scratch, st);
  OEC_HV_TILES(X)
#undef X
  return cudaErrorInvalidValue;
}

template <class P>
cudaError_t dispatch_batch(const oec_schedule& s, const HVBatchLaunch& b, cudaStream_t st) {
  constexpr int CB = sizeof(typename P::C);
#define X(a, c) \
  if (s.tile_i == a && s.tile_j == c) return launch_batch<P, a, c, KCOf<a, c, CB>::v>(b, st);
  OEC_HV_TILES(X)
#undef X
  return cudaErrorInvalidValue;
}

template <class P>
int occupancy_of(const oec_schedule& s) {
  constexpr int CB = sizeof(typename P::C);
#define X(a, c) \
  if (s.tile_i == a && s.tile_j == c) return batch_occupancy<P, a, c, KCOf<a, c, CB>::v>();
  OEC_HV_TILES(X)
#undef X
  return 1;
}

// the pair sweep drops its read scratch lines from L2 when its scratch is
// larger than this
constexpr size_t kDiscardAboveBytes = size_t(48) << 20;

// scratch row pitch of the pair sweep: the columns rounded up to 16, so that
// a 128-byte line of 8-byte values holds one half-warp's columns only
int64_t pair_pitch(int64_t ncol) { return (ncol + 15) / 16 * 16; }

// column-scratch elements (recurrence values) of one slab of `rows` j-rows
size_t sweep_scratch_elems(const oec_schedule& s, const Dom& d, int rows) {
  const int64_t ncol = (int64_t)d.ni * rows;
  return s.sweep == OEC_SWEEP_PAIR ? size_t(3) * pair_pitch(ncol) * d.nk : size_t(4) * ncol * d.nk;
}

// one FP32 domain of at least this many columns runs the staged form as one
// persistent launch (measured: 512x512x137 68.8 against 56.8 G points/s,
// 256x256x80 60.4 against 57.9; on smaller domains the two kernels)
constexpr int64_t kPSSingleMinCols = 65536;
bool pstaged_single_ok(const oec_schedule& s, int dtype, const Dom& d) {
  return hdiff_vadvc_pstaged_ok(s, dtype) && s.slabs <= 1 && (int64_t)d.ni * d.nj >= kPSSingleMinCols;
}

struct Layout {
  size_t thomas, ud, vd, counters, total;
};
Layout layout(const oec_schedule& s, int dtype, const Dom& d) {
  const size_t pts = size_t(d.ni) * d.nj * d.nk;
  Layout l;
  l.thomas = 0;
  if (s.fusion == OEC_FUSE_NONE) {
    // column scratch: g, e_u, e_v per point (pair sweep; each slab's rows
    // padded to 16 columns), the split and partitioned sweeps keep g, e per
    // field
    const int ns = std::min(std::max(s.slabs, 1), std::min(d.nj, kMaxSlabs));
    const size_t pad = ns > 1 ? size_t(3) * 16 * ns * d.nk : 0;   // slab starts on 128 bytes
    l.ud = align_up(rsize() * (sweep_scratch_elems(s, d, d.nj) + pad), 256);
    l.vd = align_up(l.ud + csize(dtype, s.arith) * pts, 256);
    l.counters = align_up(l.vd + csize(dtype, s.arith) * pts, 256);
    // the persistent single-domain form's row-block counters and ticket
    const size_t nc = pstaged_single_ok(s, dtype, d) ? size_t(ceil_div(d.nj, 4 * s.unroll)) + 1 : 0;
    l.total = align_up(l.counters + sizeof(int) * nc, 256);
  } else {
    // one slot of 3 x nk x (TI*TJ) recurrence values per tile
    const size_t tiles = size_t(ceil_div(d.ni, s.tile_i)) * ceil_div(d.nj, s.tile_j);
    l.ud = l.vd = l.counters = l.total = align_up(3 * rsize() * tiles * d.nk * s.tile_i * s.tile_j, 256);
  }
  return l;
}

// the column sweep of the staged form over ud, vd (domain layout of d)
template <class P>
cudaError_t launch_sweep(const oec_schedule& s, const Dom& d, const HV<typename P::S>& p,
                         const typename P::C* ud, const typename P::C* vd, typename P::R* scr, double dtr,
                         cudaStream_t st, bool batch_member = false) {
  typedef typename P::C C;
  // pair sweep: 64 threads, two warps of 16 columns. Ring depth: with FP64
  // fields 8 levels (measured at 128x128x80: 34.8 us against 36.9 us at 16 and
  // 38.9 at 4; larger FP64 domains 1-3% faster too); with FP32 fields 16
  // (512x512x137: 8 levels 4% slower), or 12 when every CTA of the 16-level
  // ring would be resident at once (128x128x80: 26.3 us against 27.6 at 16)
  constexpr bool f64 = std::is_same<typename P::S, double>::value;
  constexpr int NC = 32, DEPTH = f64 ? 8 : 16, DEPTH_SMALL = f64 ? 8 : 12, DEPTH_SPLIT = 16;
  constexpr int64_t kSmallCols = 152 * 7 * NC;
  const int64_t ncol = (int64_t)d.ni * d.nj;
  int e2 = 0;
  const bool p2 = std::is_same<C, df64>::value && std::frexp(dtr, &e2) == 0.5 && e2 > -120 && e2 < 120;
  // 32-bit offsets: the fields' (as for the producer) and the column
  // scratch's (3 or 4 values per point) all fit
  const bool o32 = use_int32(s, d) && 4 * pair_pitch(ncol) * d.nk < INT32_MAX;
  if (s.sweep == OEC_SWEEP_SEGMENTS4 || s.sweep == OEC_SWEEP_SEGMENTS8) {
    cudaError_t e = hdiff_vadvc_segments_launch(s.sweep, std::is_same<typename P::S, double>::value ? OEC_F64 : OEC_F32,
                                                s.arith, d, p.u, p.v, p.w, p.coeff, p.uo, p.vo, ud, vd, dtr, scr, o32,
                                                st);
    if (e != cudaSuccess) return e;
    launched(st);
    return cudaSuccess;
  }
  if (s.sweep == OEC_SWEEP_SPLIT) {
    const unsigned grid = (unsigned)((ncol + 15) / 16);
#define OEC_SPLIT(P2, OFF) hv_thomas_split_kernel<P, DEPTH_SPLIT, P2, OFF><<<grid, 64, 0, st>>>(p, ud, vd, dtr, scr)
    if (p2) {
      if (o32) { OEC_SPLIT(true, int); } else { OEC_SPLIT(true, int64_t); }
    } else {
      if (o32) { OEC_SPLIT(false, int); } else { OEC_SPLIT(false, int64_t); }
    }
#undef OEC_SPLIT
  } else {
    const unsigned grid = (unsigned)((ncol + NC - 1) / NC);
    // the L2 form pays for batch members whose scratch cannot stay in L2
    // anyway (on smaller domains, and for one apply alone, its few extra
    // instructions per step cost more than the traffic it saves)
    const bool discard = batch_member && (uintptr_t)scr % 128 == 0 &&
                         size_t(24) * pair_pitch(ncol) * d.nk > kDiscardAboveBytes;
    const bool small = ncol <= kSmallCols;
#define OEC_PAIR(P2, OFF, D, DP) \
  hv_thomas_kernel<P, NC, DP, P2, OFF, D><<<grid, 2 * NC, 0, st>>>(p, ud, vd, dtr, scr, pair_pitch(ncol))
#define OEC_PAIR_D(P2, OFF)                      \
  if (discard) {                                 \
    OEC_PAIR(P2, OFF, true, DEPTH);              \
  } else if (small) {                            \
    OEC_PAIR(P2, OFF, false, DEPTH_SMALL);       \
  } else {                                       \
    OEC_PAIR(P2, OFF, false, DEPTH);             \
  }
    if (p2) {
      if (o32) { OEC_PAIR_D(true, int); } else { OEC_PAIR_D(true, int64_t); }
    } else {
      if (o32) { OEC_PAIR_D(false, int); } else { OEC_PAIR_D(false, int64_t); }
    }
#undef OEC_PAIR_D
#undef OEC_PAIR
  }
  launched(st);
  return cudaGetLastError();
}

// ---- persistent staged batch ------------------------------------------------
// Every CTA (128 threads) takes work items in ticket order from an atomic
// counter until none is left. A producer item is one CTA of the warp-row hdiff
// kernel for one member (both fields into its hdiff(u), hdiff(v) buffers);
// when it is done its thread 0 releases one count on the member's row-block
// counter. A sweep item is one block of 64 columns of the column sweep; its
// thread 0 first waits until the counters of the row blocks those columns
// need are complete. Tickets put every producer item that a sweep item needs
// before it, and producer items never wait, so every wait ends without any
// assumption on which CTAs are resident: the items it waits for were taken by
// running CTAs. The host orders the items so that a sweep item comes well
// after its producers (the rows in between stay in L2). A wait is bounded: it
// gives up after `polls` polls, counts a timeout and skips the item.
constexpr int kPSDepth = 8;     // column sweep ring depth (16: 1.4-5% slower)
constexpr int kPSCols = 64;     // columns per sweep item (128 threads)

__device__ __forceinline__ bool ps_wait_geq(const int* p, int need, unsigned polls) {
  for (unsigned n = 0; n < polls; ++n) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    if (v >= need) return true;
    __nanosleep(256);
  }
  return false;
}

// One domain's ticket order in closed form (PSLaunch without tables). Column
// group g (columns 64g .. 64g+63) needs the row blocks of its first and last
// column; it is placed after the producer items of row block hi + lag, where
// hi is its last column's row block, or after the last block. Row block b
// then starts at ticket b * per_block + before(b), where before(b) counts the
// groups whose last column lies in a row block below b - lag.
__host__ __device__ inline int64_t ps_groups_before(const PSLaunch& L, int b) {
  if (b >= L.blocks) return L.groups;
  const int h = b - 1 - L.lag;
  if (h < 0) return 0;
  const int64_t lim = (int64_t)(h + 1) * L.rows * L.single.ni;   // first column beyond row block h
  if (lim >= (int64_t)L.single.ni * L.single.nj) return L.groups;
  return lim / kPSCols;   // groups whose last column (64g + 63) lies below lim
}

__host__ __device__ PSItem ps_decode(const PSLaunch& L, int t) {
  auto start = [&](int b) { return (int64_t)b * L.per_block + ps_groups_before(L, b); };
  int lo = 0, hi = L.blocks - 1;   // the row block b with start(b) <= t < start(b + 1)
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (start(mid) <= t) lo = mid; else hi = mid - 1;
  }
  const int b = lo;
  const int64_t r = t - start(b);
  if (r < L.per_block) return PSItem{0, int(r % L.tiles_i), b, int(r / L.tiles_i)};
  const int64_t g = ps_groups_before(L, b) + (r - L.per_block);
  const int64_t ncol = (int64_t)L.single.ni * L.single.nj;
  const int64_t c1 = g * kPSCols + kPSCols - 1 < ncol - 1 ? g * kPSCols + kPSCols - 1 : ncol - 1;
  return PSItem{~0, int(g), int((g * kPSCols) / L.single.ni) / L.rows, int(c1 / L.single.ni) / L.rows};
}

template <class P, int U, class Off, bool DISCARD>
__global__ void __launch_bounds__(2 * kPSCols) hv_pstaged_kernel(PSLaunch L) {
  typedef typename P::S S;
  typedef typename P::C C;
  typedef typename P::R R;
  extern __shared__ __align__(16) unsigned char ps_ring[];
  __shared__ int s_item, s_ok;
  __shared__ PSItem s_pi;
  for (;;) {
    if (threadIdx.x == 0) {
      s_item = atomicAdd(L.ticket, 1);
      if (s_item < L.n_items) s_pi = L.items ? L.items[s_item] : ps_decode(L, s_item);
    }
    __syncthreads();
    const int it = s_item;
    if (it >= L.n_items) break;
    const PSItem item = s_pi;
    if (item.x >= 0) {   // producer
      const PSMember& m = L.items ? L.members[item.x] : L.single;
      // one register window (the next level loads after this one's rows):
      // with two, the 2-row producer's registers hold the kernel at three
      // CTAs per SM (164 registers); with one, four (125), and the column
      // sweep items' chains gain the warps (512x512x80: 71.6 against 68.9 G
      // points/s; 32-member ensemble 1.78 against 1.85 ms)
      hdiff_vec_block<P, U, Off, 1, true>((const S*)m.u, (const S*)m.coeff, (S*)m.ud, m.ni, m.nj, m.nk, m.sj, m.sk,
                                          m.kchunk, m.ni, (int64_t)m.ni * m.nj, m.nkz, (const S*)m.v, (S*)m.vd,
                                          item.y, item.z, item.w);
      __syncthreads();   // every store of this item is issued
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(L.done + m.row_base + item.z, 1);
      }
    } else {             // column sweep
      const PSMember& m = L.items ? L.members[~item.x] : L.single;
      if (threadIdx.x == 0) {
        bool ok = true;
        for (int b = item.z; ok && b <= item.w; ++b) ok = ps_wait_geq(L.done + m.row_base + b, m.need, L.polls);
        if (!ok) atomicAdd(L.timeouts, 1u);
        s_ok = ok;
      }
      __syncthreads();
      if (s_ok) {
        const HV<S> p{(const S*)m.u, (const S*)m.v, (const S*)m.w, (const S*)m.coeff, (S*)m.uo, (S*)m.vo,
                      m.ni, m.nj, m.nk, m.sj, m.sk};
        hv_thomas_block<P, kPSCols, kPSDepth, false, Off, DISCARD>(p, (const C*)m.ud, (const C*)m.vd, L.dtr,
                                                                   (R*)m.scr, m.ncolp, item.y, ps_ring);
      }
    }
    __syncthreads();   // s_item, s_ok and the ring are free for the next item
  }
}

template <class P>
cudaError_t pstaged_dispatch(const PSLaunch& L, bool query, int* per_sm, cudaStream_t st) {
  const size_t smem = thomas_ring_bytes<P, kPSCols, kPSDepth>();
#define OEC_PS(U, OFF, D)                                                                            \
  {                                                                                                   \
    auto k = hv_pstaged_kernel<P, U, OFF, D>;                                                        \
    /* the ring and the item slots may pass 48 KB: opt in */                                          \
    cudaError_t ea = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
    if (ea != cudaSuccess) return ea;                                                                 \
    if (query) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, 2 * kPSCols, smem);   \
    k<<<L.grid, 2 * kPSCols, smem, st>>>(L);                                                          \
    return cudaGetLastError();                                                                        \
  }
#define OEC_PS_D(U, OFF) \
  if (L.discard) OEC_PS(U, OFF, true) else OEC_PS(U, OFF, false)
#define OEC_PS_O(U) \
  if (L.o32) { OEC_PS_D(U, int) } else { OEC_PS_D(U, int64_t) }
  if (L.unroll == 2) { OEC_PS_O(2) } else { OEC_PS_O(1) }
#undef OEC_PS_O
#undef OEC_PS_D
#undef OEC_PS
}

// The closed-form plan of one FP32 domain's persistent launch: levels per
// producer item, producer items per row block (tiles along i x 2 fields x
// level chunks), row blocks of 4 x unroll rows, 64-column groups and the
// ticket count; false when the tickets do not fit an int.
bool ps_single_plan(const oec_schedule& s, const Dom& d, PSLaunch& L) {
  PSMember& m = L.single;
  m.ni = d.ni; m.nj = d.nj; m.nk = d.nk;
  m.kchunk = (s.k_chunk <= 0 || s.k_chunk > d.nk) ? d.nk : s.k_chunk;
  m.nkz = ceil_div(d.nk, m.kchunk);
  m.row_base = 0;
  L.tiles_i = ceil_div(d.ni, 128);   // 32 lanes x 4 floats
  m.need = L.tiles_i * 2 * m.nkz;
  L.per_block = m.need;
  L.rows = 4 * s.unroll;
  L.blocks = ceil_div(d.nj, L.rows);
  const int64_t ncol = (int64_t)d.ni * d.nj;
  L.groups = (int)((ncol + kPSCols - 1) / kPSCols);
  const int64_t n_items = (int64_t)L.blocks * L.per_block + L.groups;
  if (n_items > INT32_MAX / 2) return false;
  L.n_items = (int)n_items;
  L.unroll = s.unroll;
  return true;
}

// the lag for `grid` resident CTAs: a group follows its last producers by
// about two resident CTAs' worth of items
int ps_single_lag(const PSLaunch& L, int grid) {
  const int64_t per_row_block = L.per_block + std::max<int64_t>(1, (int64_t)L.rows * L.single.ni / kPSCols);
  return (int)std::min<int64_t>(L.blocks, (2 * (int64_t)grid + per_row_block - 1) / per_row_block);
}

// One FP32 domain as a persistent staged launch (the closed-form ticket order
// of ps_decode, no tables): false in *ran when the fields' rows are not
// 16-byte aligned (the two kernels run then).
template <class P>
cudaError_t pstaged_single_launch(const oec_schedule& s, const Dom& d, const HV<float>& p, float* ud, float* vd,
                                  typename P::R* scr, int* counters, double dtr, cudaStream_t st, bool* ran) {
  *ran = false;
  const bool aligned = ((uintptr_t)p.u | (uintptr_t)p.v | (uintptr_t)p.coeff | (uintptr_t)ud | (uintptr_t)vd) % 16 == 0 &&
                       d.sj % 4 == 0 && d.sk % 4 == 0 && d.ni % 4 == 0;
  if (!aligned) return cudaSuccess;
  PSLaunch L{};
  PSMember& m = L.single;
  m.u = p.u; m.v = p.v; m.w = p.w; m.coeff = p.coeff; m.uo = p.uo; m.vo = p.vo;
  m.ud = ud; m.vd = vd; m.scr = scr;
  m.sj = d.sj; m.sk = d.sk;
  const int64_t ncol = (int64_t)d.ni * d.nj;
  m.ncolp = pair_pitch(ncol);
  if (!ps_single_plan(s, d, L)) return cudaSuccess;
  const int64_t n_items = L.n_items;
  L.timeouts = wait_timeout_counter();
  if (!L.timeouts) return cudaSuccess;
  L.o32 = use_int32(s, d) && 4 * m.ncolp * d.nk < INT32_MAX;
  L.discard = (uintptr_t)scr % 128 == 0 && size_t(24) * m.ncolp * d.nk > kDiscardAboveBytes;
  L.dtr = dtr;
  L.polls = 1u << 22;
  L.done = counters;
  L.ticket = counters + L.blocks;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // CTAs per SM of this kernel form, looked up once per device
  static std::atomic<int> cache[8][64];
  const int form = (L.unroll - 1) * 4 + (L.o32 ? 2 : 0) + (L.discard ? 1 : 0);
  int per_sm = dev < 64 ? cache[form][dev].load() : 0;
  if (per_sm <= 0) {
    e = pstaged_dispatch<P>(L, true, &per_sm, nullptr);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaSuccess;
    if (dev < 64) cache[form][dev].store(per_sm);
  }
  L.grid = (int)std::min<int64_t>(n_items, (int64_t)per_sm * sms);
  L.lag = ps_single_lag(L, L.grid);
  e = cudaMemsetAsync(counters, 0, sizeof(int) * (size_t)(L.blocks + 1), st);
  if (e == cudaSuccess) e = pstaged_dispatch<P>(L, false, nullptr, st);
  if (e == cudaSuccess) {
    *ran = true;
    launched(st);
  }
  return e;
}

// The staged form's slab streams and their events (one set per device, made
// on first use): with slabs > 1 the producer of every slab runs on the
// caller's stream and the column sweep of slab s on stream s once producer s
// has finished, so the sweeps run concurrently with each other and with the
// producers of the later slabs.
struct SlabStreams {
  cudaStream_t side[kMaxSlabs] = {};
  cudaEvent_t ev[kMaxSlabs + 1] = {};     // fork, then one per producer
  cudaEvent_t done[kMaxSlabs] = {};       // one per sweep
};
constexpr int kMaxDevices = 64;
SlabStreams g_slab[kMaxDevices];
std::mutex g_slab_mu;

cudaError_t slab_streams(SlabStreams** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_slab_mu);
  SlabStreams& ss = g_slab[dev];
  if (!ss.side[kMaxSlabs - 1]) {
    for (int x = 0; e == cudaSuccess && x < kMaxSlabs; ++x) {
      if (!ss.side[x]) e = cudaStreamCreateWithFlags(&ss.side[x], cudaStreamNonBlocking);
      if (e == cudaSuccess && !ss.done[x]) e = cudaEventCreateWithFlags(&ss.done[x], cudaEventDisableTiming);
    }
    for (int x = 0; e == cudaSuccess && x < kMaxSlabs + 1; ++x)
      if (!ss.ev[x]) e = cudaEventCreateWithFlags(&ss.ev[x], cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  *out = &ss;
  return cudaSuccess;
}

template <class P>
cudaError_t run(const oec_schedule& s, int dtype, const Dom& d, const HV<typename P::S>& p, double dtr, char* scratch,
                cudaStream_t st, bool batch_member) {
  typedef typename P::S S;
  typedef typename P::C C;
  typedef typename P::R R;
  Layout l = layout(s, dtype, d);
  if (s.fusion != OEC_FUSE_NONE) return dispatch_fused<P>(s, d, p, dtr, scratch + l.thomas, st);
  C* ud = (C*)(scratch + l.ud);
  C* vd = (C*)(scratch + l.vd);
  R* scr = (R*)(scratch + l.thomas);
  const int ns = std::min(std::max(s.slabs, 1), std::min(d.nj, kMaxSlabs));
  if (ns == 1) {
    if constexpr (std::is_same<typename P::S, float>::value) {
      // a large FP32 domain: producer and column sweep in one persistent launch
      if (!batch_member && pstaged_single_ok(s, dtype, d)) {
        bool ran = false;
        cudaError_t e = pstaged_single_launch<P>(s, d, p, (float*)ud, (float*)vd, scr, (int*)(scratch + l.counters),
                                                 dtr, st, &ran);
        if (e != cudaSuccess || ran) return e;
      }
    }
    cudaError_t e = hdiff_to_compute(s, dtype, d, p.u, p.v, p.coeff, ud, vd, st);
    if (e != cudaSuccess) return e;
    return launch_sweep<P>(s, d, p, ud, vd, scr, dtr, st, batch_member);
  }
  // slab pipeline: slab x holds the rows [j0, j1) with its own compact
  // hdiff(u), hdiff(v) and column scratch (the same bytes in total)
  SlabStreams* ss = nullptr;
  cudaError_t e = slab_streams(&ss);
  if (e != cudaSuccess) return e;
  const size_t plane = size_t(d.ni) * d.nk;                // points per row of the domain, all levels
  size_t soff = 0;                                         // this slab's column scratch (elements)
  // one thread at a time enqueues onto the shared slab streams and events
  // (an event is re-recorded by the next apply only after this one's waits)
  std::lock_guard<std::mutex> lock(g_slab_mu);
  launch_group_begin();
  e = cudaEventRecord(ss->ev[0], st);
  for (int x = 0; e == cudaSuccess && x < ns; ++x) e = cudaStreamWaitEvent(ss->side[x], ss->ev[0], 0);
  for (int x = 0; e == cudaSuccess && x < ns; ++x) {
    const int j0 = int(int64_t(d.nj) * x / ns), j1 = int(int64_t(d.nj) * (x + 1) / ns);
    const Dom ds{d.ni, j1 - j0, d.nk, d.sj, d.sk};
    const int64_t fo = (int64_t)j0 * d.sj;
    const HV<S> ps{p.u + fo, p.v + fo, p.w + fo, p.coeff + fo, p.uo + fo, p.vo + fo, ds.ni, ds.nj, ds.nk, ds.sj, ds.sk};
    const size_t before = plane * j0;
    e = hdiff_to_compute(s, dtype, ds, ps.u, ps.v, ps.coeff, ud + before, vd + before, st);
    if (e == cudaSuccess) e = cudaEventRecord(ss->ev[x + 1], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ss->side[x], ss->ev[x + 1], 0);
    if (e == cudaSuccess) e = launch_sweep<P>(s, ds, ps, ud + before, vd + before, scr + soff, dtr, ss->side[x]);
    soff += (sweep_scratch_elems(s, ds, ds.nj) + 15) / 16 * 16;   // next slab's lines start on 128 bytes
    if (e == cudaSuccess) e = cudaEventRecord(ss->done[x], ss->side[x]);
  }
  for (int x = 0; e == cudaSuccess && x < ns; ++x) e = cudaStreamWaitEvent(st, ss->done[x], 0);
  launch_group_end(st);
  return e;
}

}  // namespace

bool hdiff_vadvc_schedule_ok(const oec_schedule& s, std::string& why) {
  if (s.arith < 0 || s.arith > 2) { why = "arith must be 0 (native), 1 (double-float) or 2 (fixed point)"; return false; }
  if (s.arith == 2 && s.fusion != OEC_FUSE_NONE) {
    why = "fixed-point hdiff feeds the stage-by-stage (OEC_FUSE_NONE) form";
    return false;
  }
  if (s.fusion == OEC_FUSE_NONE) return true;
  if (s.fusion != OEC_FUSE_INLINE) { why = "fusion must be OEC_FUSE_INLINE or OEC_FUSE_NONE"; return false; }
#define X(a, b) if (s.tile_i == a && s.tile_j == b) return true;
  OEC_HV_TILES(X)
#undef X
  why = "hdiff+vadvc column tiles: 16x4, 32x2, 8x8, 32x4, 8x4, 16x2";
  return false;
}

size_t hdiff_vadvc_scratch_bytes(const oec_schedule& s, int dtype, const Dom& d) { return layout(s, dtype, d).total; }

cudaError_t hdiff_vadvc_launch(const oec_schedule& s, int dtype, const Dom& d, const void* u, const void* v,
                               const void* w, const void* coeff, void* u_out, void* v_out, double dtr, void* scratch,
                               cudaStream_t st, bool batch_member) {
  const bool df = s.arith >= 1;   // arith 2: fixed-point hdiff producer, double-float column
  if (dtype == OEC_F64) {
    HV<double> p{(const double*)u, (const double*)v, (const double*)w, (const double*)coeff,
                 (double*)u_out, (double*)v_out, d.ni, d.nj, d.nk, d.sj, d.sk};
    return df ? run<P64D>(s, dtype, d, p, dtr, (char*)scratch, st, batch_member)
              : run<P64>(s, dtype, d, p, dtr, (char*)scratch, st, batch_member);
  }
  HV<float> p{(const float*)u, (const float*)v, (const float*)w, (const float*)coeff,
              (float*)u_out, (float*)v_out, d.ni, d.nj, d.nk, d.sj, d.sk};
  return df ? run<P32D>(s, dtype, d, p, dtr, (char*)scratch, st, batch_member)
            : run<P32>(s, dtype, d, p, dtr, (char*)scratch, st, batch_member);
}

int64_t hdiff_vadvc_pstaged_order(const oec_schedule& s, const Dom& d, int grid, int32_t* items, int64_t cap) {
  PSLaunch L{};
  if (grid < 1 || !ps_single_plan(s, d, L)) return -1;
  L.lag = ps_single_lag(L, grid);
  if (items && cap >= 4 * (int64_t)L.n_items)
    for (int t = 0; t < L.n_items; ++t) {
      const PSItem it = ps_decode(L, t);
      items[4 * (int64_t)t] = it.x;
      items[4 * (int64_t)t + 1] = it.y;
      items[4 * (int64_t)t + 2] = it.z;
      items[4 * (int64_t)t + 3] = it.w;
    }
  return L.n_items;
}

bool hdiff_vadvc_pstaged_ok(const oec_schedule& s, int dtype) {
  return dtype == OEC_F32 && s.fusion == OEC_FUSE_NONE && s.staging == OEC_STAGE_WARP &&
         (s.unroll == 1 || s.unroll == 2) && s.sweep == OEC_SWEEP_PAIR && (s.arith == 0 || s.arith == 1);
}

void hdiff_vadvc_scratch_parts(const oec_schedule& s, int dtype, const Dom& d, size_t* ud, size_t* vd) {
  const Layout l = layout(s, dtype, d);
  *ud = l.ud;
  *vd = l.vd;
}

int64_t hdiff_vadvc_pair_pitch(int64_t ncol) { return pair_pitch(ncol); }

size_t hdiff_vadvc_discard_above_bytes() { return kDiscardAboveBytes; }

cudaError_t hdiff_vadvc_pstaged_blocks_per_sm(const oec_schedule& s, const PSLaunch& L, int* per_sm) {
  return s.arith == 1 ? pstaged_dispatch<P32D>(L, true, per_sm, nullptr)
                      : pstaged_dispatch<P32>(L, true, per_sm, nullptr);
}

cudaError_t hdiff_vadvc_pstaged_launch(const oec_schedule& s, const PSLaunch& L, cudaStream_t st) {
  cudaError_t e = s.arith == 1 ? pstaged_dispatch<P32D>(L, false, nullptr, st)
                               : pstaged_dispatch<P32>(L, false, nullptr, st);
  if (e == cudaSuccess) launched(st);
  return e;
}

// Give-up path of the persistent batch's wait: one sweep item whose row-block
// counter nothing releases (no producer items), so its wait gives up after
// `polls` polls, counts a timeout and skips the item. The buffers are valid
// for the 4-column domain the item names, though nothing reads them.
cudaError_t pstaged_wait_selftest_launch(unsigned polls, cudaStream_t st) {
  constexpr size_t kRegion = 256, kBytes = 16 * kRegion;
  char* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, kBytes);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(buf, 0, kBytes, st);
  PSMember m{};
  auto at = [&](int r) { return (void*)(buf + (r + 1) * kRegion); };   // a region, room before it
  m.u = at(0); m.v = at(1); m.w = at(2); m.coeff = at(3); m.uo = at(4); m.vo = at(5);
  m.ud = at(6); m.vd = at(7); m.scr = at(8);
  m.sj = 4; m.sk = 4; m.ncolp = 16;
  m.ni = 4; m.nj = 1; m.nk = 1; m.kchunk = 1; m.nkz = 1;
  m.row_base = 0;
  m.need = 1;
  const PSItem item{~0, 0, 0, 0};
  PSMember* dm = (PSMember*)(buf + 12 * kRegion);
  PSItem* di = (PSItem*)(buf + 13 * kRegion);
  int* ticket = (int*)(buf + 14 * kRegion);
  int* done = (int*)(buf + 15 * kRegion);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dm, &m, sizeof(m), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(di, &item, sizeof(item), cudaMemcpyHostToDevice, st);
  PSLaunch L{};
  L.members = dm;
  L.items = di;
  L.n_items = 1;
  L.ticket = ticket;
  L.done = done;
  L.timeouts = wait_timeout_counter();
  L.polls = polls;
  L.dtr = 2.0;
  L.grid = 1;
  L.unroll = 1;
  L.o32 = true;
  L.discard = false;
  if (e == cudaSuccess && !L.timeouts) e = cudaErrorInvalidSymbol;
  if (e == cudaSuccess) e = pstaged_dispatch<P32D>(L, false, nullptr, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);   // the host copies' sources and the buffer outlive the kernel
  cudaFree(buf);
  return e != cudaSuccess ? e : e2;
}

size_t hdiff_vadvc_batch_slot_elems(const oec_schedule& s, int nk_max) {
  return size_t(3) * nk_max * s.tile_i * s.tile_j;
}

int hdiff_vadvc_batch_blocks_per_sm(const oec_schedule& s, int dtype) {
  const bool df = s.arith == 1;
  if (dtype == OEC_F64) return df ? occupancy_of<P64D>(s) : occupancy_of<P64>(s);
  return df ? occupancy_of<P32D>(s) : occupancy_of<P32>(s);
}

cudaError_t hdiff_vadvc_batch_launch(const oec_schedule& s, int dtype, const HVBatchLaunch& b, cudaStream_t st) {
  const bool df = s.arith == 1;
  if (dtype == OEC_F64) return df ? dispatch_batch<P64D>(s, b, st) : dispatch_batch<P64>(s, b, st);
  return df ? dispatch_batch<P32D>(s, b, st) : dispatch_batch<P32>(s, b, st);
}

}  // namespace oec
