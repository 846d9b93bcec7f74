// df64.cuh - double-float arithmetic: a value is the unevaluated sum hi + lo of
// two floats (|lo| <= ulp(hi)/2), about 48 significant bits. Built from the
// error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2): TwoSum,
// FastTwoSum and the FMA form of TwoProduct. GB300 runs FP32 at ~70x the rate
// of FP64, so FP64 stencil programs evaluate in df64 on the FP32 pipes and
// convert to/from IEEE binary64 storage with integer operations only.
//
// Range: finite values with 2^-74 <= |x| < 2^128 keep ~48 bits; below that
// the low part is dropped (absolute error below 2^-98), below 2^-126 the
// value flushes to zero; |x| >= 2^128 overflows. Every operation is written with explicit-rounding intrinsics so
// that the compiler neither contracts nor reorders the error terms.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace oec {

// 8-byte aligned, so a pair moves with one 64-bit load or store
struct __align__(8) df64 {
  float hi, lo;
};

__device__ __forceinline__ df64 df_make(float hi, float lo) { return df64{hi, lo}; }

// s + e == a + b exactly (any a, b)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// s + e == a + b exactly when |a| >= |b| (or a == 0)
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df64 df_norm(float a, float b) {
  df64 r;
  fast_two_sum(a, b, r.hi, r.lo);
  return r;
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64{-a.hi, -a.lo}; }

// accurate addition: both parts summed error-free, two renormalisations
// (error about 2^-47 |a + b|, also under cancellation)
__device__ __forceinline__ df64 operator+(df64 a, df64 b) {
  float s, e, t, f;
  two_sum(a.hi, b.hi, s, e);
  two_sum(a.lo, b.lo, t, f);
  e = __fadd_rn(e, t);
  fast_two_sum(s, e, s, e);
  e = __fadd_rn(e, f);
  return df_norm(s, e);
}
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

// fast addition: the high parts summed error-free, the low parts added once
// (error about 3 * 2^-48 (|a| + |b|), bounded by the operands rather than the
// sum; for chains without catastrophic cancellation)
__device__ __forceinline__ df64 df_add_fast(df64 a, df64 b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return df_norm(s, e);
}
__device__ __forceinline__ df64 df_sub_fast(df64 a, df64 b) { return df_add_fast(a, -b); }

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_norm(p, e);
}
// a - b * c with the product left unnormalised (its low part carried into
// the low sum): one renormalisation fewer than a product and a fast
// subtraction. Error at most about 2^-46 (|a| + |b c|) (worst of 20,000
// random cases in exact arithmetic: 2^-46.2, against 2^-46.7 for the product
// and the fast subtraction).
__device__ __forceinline__ df64 df_fms(df64 a, df64 b, df64 c) {
  const float p = __fmul_rn(b.hi, c.hi);
  float pe = __fmaf_rn(b.hi, c.hi, -p);
  pe = __fmaf_rn(b.hi, c.lo, pe);
  pe = __fmaf_rn(b.lo, c.hi, pe);
  float s, e;
  two_sum(a.hi, -p, s, e);
  e = __fadd_rn(e, __fsub_rn(a.lo, pe));
  return df_norm(s, e);
}
// df times float
__device__ __forceinline__ df64 df_mulf(df64 a, float b) {
  const float p = __fmul_rn(a.hi, b);
  float e = __fmaf_rn(a.hi, b, -p);
  e = __fmaf_rn(a.lo, b, e);
  return df_norm(p, e);
}
// exact scaling by a power of two
__device__ __forceinline__ df64 df_scale(df64 a, float pow2) { return df64{__fmul_rn(a.hi, pow2), __fmul_rn(a.lo, pow2)}; }

// a / b: quotient estimate, two remainder corrections
__device__ __forceinline__ df64 operator/(df64 a, df64 b) {
  const float rb = __frcp_rn(b.hi);
  const float q1 = __fmul_rn(a.hi, rb);
  df64 r = a - df_mulf(b, q1);
  const float q2 = __fmul_rn(r.hi, rb);
  r = r - df_mulf(b, q2);
  const float q3 = __fmul_rn(r.hi, rb);
  df64 q = df_norm(q1, q2);
  return q + df64{q3, 0.0f};
}
// 1 / b: correctly rounded float seed x0 (relative error 2^-24), one Newton
// step x0 + x0 (1 - b x0) with the residual in double-float: error ~2^-47
__device__ __forceinline__ df64 df_rcp(df64 b) {
  const float x0 = __frcp_rn(b.hi);
  const df64 r = df_sub_fast(df64{1.0f, 0.0f}, df_mulf(b, x0));
  return df_norm(x0, __fmul_rn(r.hi, x0));
}

// 1 / b seeded by the hardware's approximate reciprocal (rcp.approx.ftz.f32,
// relative error about 2^-23), then one Newton step x0 + x0 r. The residual
// r = 1 - b x0 is of order 2^-23, so it is formed in single floats by two
// FMAs: 1 - b.hi x0 is exact before its one rounding, and b.lo x0 is added by
// the second. Error about 2^-44 (in exact arithmetic, with seeds one ulp off,
// the same as the residual formed as a double-float product and difference,
// in 7 float operations instead of 22). For b.hi normal and below 2^126 (the
// column recurrence's pivots).
__device__ __forceinline__ df64 df_rcp_approx_seed(df64 b) {
  float x0;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(x0) : "f"(b.hi));
  const float r = __fmaf_rn(-b.lo, x0, __fmaf_rn(-b.hi, x0, 1.0f));
  return df_norm(x0, __fmul_rn(x0, r));
}

__device__ __forceinline__ bool df_gt0(df64 a) { return a.hi > 0.0f; }   // sign of a normalised pair
__device__ __forceinline__ df64 df_abs(df64 a) { return a.hi < 0.0f ? -a : a; }

// float value of a non-negative integer below 2^30, without a conversion
// instruction: the two halves are placed in float significands by bit
// assembly (exact), then combined with one rounding.
__device__ __forceinline__ float u30_to_float(unsigned r) {
  const float fh = __fsub_rn(__uint_as_float(0x4B000000u | (r >> 12)), 8388608.0f);
  const float fl = __fsub_rn(__uint_as_float(0x4B000000u | (r & 0xFFFu)), 8388608.0f);
  return __fmaf_rn(fh, 4096.0f, fl);
}

// ---- conversion from IEEE binary64 (integer and FP32 operations only) ------
// hi = x rounded (half up) to a 24-bit significand by bit assembly; lo =
// (x - hi), an integer of at most 2^29 units of x's ulp, rounded to a float.
// Conversion error below 2^-48 |x|. Conversion instructions between float and
// double run on the FP64 pipe on this part, so none is used.
__device__ __forceinline__ df64 df_from_double(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned sign = hw & 0x80000000u;
  const unsigned ex = (hw >> 20) & 0x7FFu;                // biased binary64 exponent
  const unsigned rnd = (lw >> 28) & 1u;                   // first bit below the float significand
  unsigned hib = __funnelshift_l(lw, (hw & 0x7FFFFFFFu) - 0x38000000u, 3) + rnd;  // exponent and fraction
  hib = ex <= 896u ? 0u : hib;                            // below float range: zero
  hib = ex >= 1151u ? 0x7F800000u : hib;                  // above float range: infinity
  const int r = (int)(lw & 0x1FFFFFFFu) - (int)(rnd << 29);   // x - hi in units of x's ulp
  const float scale = __uint_as_float((ex - 948u) << 23);    // 2^(e - 52) as a float
  float lo = __fmul_rn(u30_to_float((unsigned)abs(r)), scale);
  lo = (ex >= 949u && ex <= 1150u) ? lo : 0.0f;          // tiny or huge x: lo dropped
  const unsigned lsign = sign ^ (r < 0 ? 0x80000000u : 0u);
  return df64{__uint_as_float(sign | hib), __uint_as_float(__float_as_uint(lo) | lsign)};
}

// ---- conversion to IEEE binary64 (integer operations only) -----------------
// hi's bits widened to binary64, plus lo expressed as an integer count of that
// binary64's ulp, added to the bit pattern (sign-magnitude, so magnitudes
// add); when hi is a power of two and lo lowers the magnitude the result sits
// one binade down and the count doubles. lo bits below the binary64 ulp are
// truncated (error below one ulp).
__device__ __forceinline__ double df_to_double(df64 a) {
  const unsigned hb = __float_as_uint(a.hi), lb = __float_as_uint(a.lo);
  const unsigned eh = (hb >> 23) & 0xFFu, el = (lb >> 23) & 0xFFu;
  if (eh == 0u) return 0.0;                               // zero (and float denormals)
  unsigned long long bits = ((unsigned long long)(hb & 0x80000000u) << 32) |
                            ((unsigned long long)(eh + 896u) << 52) | ((unsigned long long)(hb & 0x7FFFFFu) << 29);
  if (el != 0u) {                                         // lo zero or denormal: nothing to add
    const bool down = ((lb ^ hb) & 0x80000000u) != 0u;
    const bool pow2 = (hb & 0x7FFFFFu) == 0u;
    const int sh = 29 - (int)eh + (int)el + ((pow2 && down) ? 1 : 0);
    const unsigned ml = (lb & 0x7FFFFFu) | 0x800000u;
    const unsigned long long n = sh >= 0 ? ((unsigned long long)ml << min(sh, 31)) : (sh > -24 ? (ml >> -sh) : 0u);
    bits = down ? bits - n : bits + n;
  }
  return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ df64 df_from_float(float x) { return df64{x, 0.0f}; }

}  // namespace oec
