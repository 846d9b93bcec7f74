// arith.cuh - arithmetic policies of the hand-written kernels and the few
// generic operations the stencil bodies need, for float, double and df64.
//
//   policy   storage S   stencil compute C   column recurrence R
//   P32      float       float               double  (FP64 recurrence)
//   P32D     float       float               df64    (FP64-class recurrence on FP32 pipes)
//   P64      double      double              double  (native FP64)
//   P64D     double      df64                df64    (FP64-class, FP32 pipes)
#pragma once

#include "df64.cuh"

namespace oec {

struct P32 { typedef float S; typedef float C; typedef double R; };
struct P32D { typedef float S; typedef float C; typedef df64 R; };
struct P64 { typedef double S; typedef double C; typedef double R; };
struct P64D { typedef double S; typedef df64 C; typedef df64 R; };

// ---- conversions -------------------------------------------------------------
template <class To> __device__ __forceinline__ To cvt(float x);
template <class To> __device__ __forceinline__ To cvt(double x);
template <class To> __device__ __forceinline__ To cvt(df64 x);
template <> __device__ __forceinline__ float cvt<float>(float x) { return x; }
template <> __device__ __forceinline__ double cvt<double>(float x) { return (double)x; }
template <> __device__ __forceinline__ df64 cvt<df64>(float x) { return df64{x, 0.0f}; }
template <> __device__ __forceinline__ float cvt<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ double cvt<double>(double x) { return x; }
template <> __device__ __forceinline__ df64 cvt<df64>(double x) { return df_from_double(x); }
template <> __device__ __forceinline__ float cvt<float>(df64 x) { return x.hi + x.lo; }
template <> __device__ __forceinline__ double cvt<double>(df64 x) { return df_to_double(x); }
template <> __device__ __forceinline__ df64 cvt<df64>(df64 x) { return x; }

// ---- constants and small operations ------------------------------------------
template <class T> __device__ __forceinline__ T kc(float v) { return cvt<T>(v); }

// multiplication by a constant that is a power of two (exact in every type)
__device__ __forceinline__ float mul_p2(float a, float c) { return a * c; }
__device__ __forceinline__ double mul_p2(double a, float c) { return a * (double)c; }
__device__ __forceinline__ df64 mul_p2(df64 a, float c) { return df_scale(a, c); }
// multiplication by any float constant
__device__ __forceinline__ float mul_c(float a, float c) { return a * c; }
__device__ __forceinline__ double mul_c(double a, float c) { return a * (double)c; }
__device__ __forceinline__ df64 mul_c(df64 a, float c) { return df_mulf(a, c); }

__device__ __forceinline__ float abs_(float a) { return fabsf(a); }
__device__ __forceinline__ double abs_(double a) { return fabs(a); }
__device__ __forceinline__ df64 abs_(df64 a) { return df_abs(a); }

__device__ __forceinline__ bool gt0(float a) { return a > 0.0f; }
__device__ __forceinline__ bool gt0(double a) { return a > 0.0; }
__device__ __forceinline__ bool gt0(df64 a) { return df_gt0(a); }

// a*b > 0 (the limiter's test): for df64 decided from the signs, which are
// exact for normalised pairs
__device__ __forceinline__ bool prod_gt0(float a, float b) { return a * b > 0.0f; }
__device__ __forceinline__ bool prod_gt0(double a, double b) { return a * b > 0.0; }
__device__ __forceinline__ bool prod_gt0(df64 a, df64 b) {
  return (a.hi > 0.0f && b.hi > 0.0f) || (a.hi < 0.0f && b.hi < 0.0f);
}

__device__ __forceinline__ float rcp_(float a) { return 1.0f / a; }
__device__ __forceinline__ double rcp_(double a) { return 1.0 / a; }
__device__ __forceinline__ df64 rcp_(df64 a) { return df_rcp(a); }
// reciprocal of a pivot bounded away from zero and overflow (diagonally
// dominant recurrences): double-float takes the approximate hardware seed
__device__ __forceinline__ float rcp_pivot(float a) { return 1.0f / a; }
__device__ __forceinline__ double rcp_pivot(double a) { return 1.0 / a; }
__device__ __forceinline__ df64 rcp_pivot(df64 a) { return df_rcp_approx_seed(a); }

template <class T> __device__ __forceinline__ T zero_() { return kc<T>(0.0f); }

// value of the lane d below / above (full warp; lanes at the edge get their own)
__device__ __forceinline__ float shfl_up_(float a, int d) { return __shfl_up_sync(0xFFFFFFFFu, a, d); }
__device__ __forceinline__ double shfl_up_(double a, int d) { return __shfl_up_sync(0xFFFFFFFFu, a, d); }
__device__ __forceinline__ df64 shfl_up_(df64 a, int d) {
  return df64{__shfl_up_sync(0xFFFFFFFFu, a.hi, d), __shfl_up_sync(0xFFFFFFFFu, a.lo, d)};
}
__device__ __forceinline__ float shfl_down_(float a, int d) { return __shfl_down_sync(0xFFFFFFFFu, a, d); }
__device__ __forceinline__ double shfl_down_(double a, int d) { return __shfl_down_sync(0xFFFFFFFFu, a, d); }
__device__ __forceinline__ df64 shfl_down_(df64 a, int d) {
  return df64{__shfl_down_sync(0xFFFFFFFFu, a.hi, d), __shfl_down_sync(0xFFFFFFFFu, a.lo, d)};
}
// exchange with the lane whose index differs in the bits of m (full warp)
__device__ __forceinline__ float shfl_xor_(float a, int m) { return __shfl_xor_sync(0xFFFFFFFFu, a, m); }
__device__ __forceinline__ double shfl_xor_(double a, int m) { return __shfl_xor_sync(0xFFFFFFFFu, a, m); }
__device__ __forceinline__ df64 shfl_xor_(df64 a, int m) {
  return df64{__shfl_xor_sync(0xFFFFFFFFu, a.hi, m), __shfl_xor_sync(0xFFFFFFFFu, a.lo, m)};
}

// addition/subtraction for chains without catastrophic cancellation (the
// column recurrence): the fast double-float add, plain IEEE otherwise
__device__ __forceinline__ float addf(float a, float b) { return a + b; }
__device__ __forceinline__ double addf(double a, double b) { return a + b; }
__device__ __forceinline__ df64 addf(df64 a, df64 b) { return df_add_fast(a, b); }
__device__ __forceinline__ float subf(float a, float b) { return a - b; }
__device__ __forceinline__ double subf(double a, double b) { return a - b; }
__device__ __forceinline__ df64 subf(df64 a, df64 b) { return df_sub_fast(a, b); }

// a - b * c for the column recurrence (chains without catastrophic
// cancellation): plain IEEE for float and double, the fused double-float form
// for df64
__device__ __forceinline__ float fms_(float a, float b, float c) { return a - b * c; }
__device__ __forceinline__ double fms_(double a, double b, double c) { return a - b * c; }
__device__ __forceinline__ df64 fms_(df64 a, df64 b, df64 c) { return df_fms(a, b, c); }

// a double-precision constant in the compute type
template <class T> __device__ __forceinline__ T kd(double v) { return cvt<T>(v); }

// a / b for the stencil bodies: FP32 by the hardware reciprocal and one
// multiply (within 2 ulp for |b| in [2^-126, 2^126]); FP64 IEEE division;
// df64 its estimate-and-correct quotient
__device__ __forceinline__ float fdiv_(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv_(double a, double b) { return a / b; }
__device__ __forceinline__ df64 fdiv_(df64 a, df64 b) { return a / b; }

// x / 12: FP32 multiplies by the rounded reciprocal (within 1 ulp of the
// quotient, far inside FP32's tolerance), FP64 divides (IEEE), df64
// multiplies by the double-float reciprocal
__device__ __forceinline__ float div12(float x) { return x * (1.0f / 12.0f); }
__device__ __forceinline__ double div12(double x) { return x / 12.0; }
__device__ __forceinline__ df64 div12(df64 x) { return x * df_from_double(1.0 / 12.0); }

// ---- stage bodies of horizontal diffusion (any compute type) ------------------
// Laplacian 4c - w - e - s - n; flux with the sign limiter; flux divergence.
template <class T> __device__ __forceinline__ T hlap(T c, T w, T e, T s, T n) {
  return mul_p2(c, 4.0f) - w - e - s - n;
}
template <class T> __device__ __forceinline__ T hflux(T lap_hi, T lap_lo, T in_hi, T in_lo) {
  const T f = lap_hi - lap_lo;
  return prod_gt0(f, in_hi - in_lo) ? zero_<T>() : f;
}
template <class T> __device__ __forceinline__ T hout(T in, T coeff, T flx, T flx_m, T fly, T fly_m) {
  return in - coeff * ((flx - flx_m) + (fly - fly_m));
}

}  // namespace oec
