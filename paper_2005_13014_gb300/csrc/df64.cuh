// df64.cuh - double-float arithmetic: a value is the unevaluated sum hi + lo of
// two floats (|lo| <= ulp(hi)/2), about 48 significant bits. Built from the
// error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2): TwoSum,
// FastTwoSum and the FMA form of TwoProduct. GB300 runs FP32 at ~70x the rate
// of FP64, so FP64 stencil programs evaluate in df64 on the FP32 pipes and
// convert to/from IEEE binary64 storage with integer operations only.
//
// Range: finite values with 2^-74 <= |x| < 2^128 keep ~48 bits; below that
// the low part is dropped (absolute error below 2^-98); |x| >= 2^128
// overflows. Every operation is written with explicit-rounding intrinsics so
// that the compiler neither contracts nor reorders the error terms.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace oec {

struct df64 {
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

__device__ __forceinline__ df64 operator*(df64 a, df64 b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  return df_norm(p, e);
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
__device__ __forceinline__ df64 df_rcp(df64 b) { return df64{1.0f, 0.0f} / b; }

__device__ __forceinline__ bool df_gt0(df64 a) { return a.hi > 0.0f; }   // sign of a normalised pair
__device__ __forceinline__ df64 df_abs(df64 a) { return a.hi < 0.0f ? -a : a; }

// ---- conversion from IEEE binary64 -----------------------------------------
// hi = x rounded to float; lo = (x - hi) rounded to float, where x - hi is
// taken exactly as the difference of the two binary64 bit patterns (same sign,
// same or adjacent binade, at most 2^28 units of x's ulp), so no FP64
// arithmetic is issued. Conversion error below 2^-48 |x|.
__device__ __forceinline__ df64 df_from_double(double x) {
  const float hi = __double2float_rn(x);
  const long long bx = __double_as_longlong(x);
  const long long bh = __double_as_longlong((double)hi);
  const int d = (int)(bx - bh);                          // (|x| - |hi|) in units of x's ulp
  const unsigned ex = (unsigned)(bx >> 52) & 0x7FFu;     // biased exponent of x
  const float scale = __uint_as_float((ex - 948u) << 23);  // 2^(e-52) as a float
  float lo = __fmul_rn(__int2float_rn(d), scale);
  lo = (ex >= 949u && ex <= 1150u) ? lo : 0.0f;          // tiny or huge x: lo dropped
  lo = bx < 0 ? -lo : lo;
  return df64{hi, lo};
}

// ---- conversion to IEEE binary64 -------------------------------------------
// (double)hi plus lo expressed as an integer count of hi's binary64 ulp, added
// to the bit pattern (sign-magnitude, so magnitudes add); when hi is a power of
// two and lo lowers the magnitude, the result sits one binade down and the
// count doubles. Error below one binary64 ulp; no FP64 arithmetic.
__device__ __forceinline__ double df_to_double(df64 a) {
  const unsigned hb = __float_as_uint(a.hi);
  const unsigned eh = (hb >> 23) & 0xFFu;
  const double hd = (double)a.hi;
  if (eh < 52u || eh == 255u) return hd;                 // |hi| < 2^-75: lo dropped
  const bool down = ((__float_as_uint(a.lo) ^ hb) & 0x80000000u) != 0u;
  const bool pow2 = (hb & 0x7FFFFFu) == 0u;
  float t = __fmul_rn(fabsf(a.lo), __uint_as_float((306u - eh) << 23));  // |lo| / ulp(hi as binary64)
  t = (pow2 && down) ? __fmul_rn(t, 2.0f) : t;
  const long long n = (long long)__float2int_rn(t);
  return __longlong_as_double(__double_as_longlong(hd) + (down ? -n : n));
}

__device__ __forceinline__ df64 df_from_float(float x) { return df64{x, 0.0f}; }

}  // namespace oec
