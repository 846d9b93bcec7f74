// fixedpt.cuh - exact fixed-point evaluation of FP64 horizontal diffusion
// (OEC_ARITH_FIXED), used by the shared-memory tile kernel (k_hdiff.cu).
//
// hdiff is linear in `in` apart from the limiter's sign tests and the final
// product with coeff, so the Laplacian, fluxes and flux divergence of binary64
// inputs are evaluated exactly in 64-bit integers. Per window and level, E
// (the largest biased exponent of the window's values) fixes the scale: value
// x = m * 2^(e-1075) becomes X = (m << 3) >> (E - e) (truncated toward zero),
// an integer multiple of 2^(E-1078) with |X| < 2^56, so |lap| < 2^59,
// |flux| < 2^60, |divergence| < 2^62: no overflow. The limiter tests the sign
// of the flux (exact) against the sign of in_hi - in_lo taken exactly from the
// raw binary64 values (ordered integer keys). The output is one rounding of
// the exact divergence term: out = fma(-coeff, div * 2^(E - 1078), in). Only
// values more than 2^53 times smaller than the window's largest lose bits
// (absolute error below 2^(E-1078) per value). Windows whose values all lie
// below 2^-923 are treated as zero-diffusion (E is raised to 100, so every
// such value converts to 0). Inputs must be finite.
#pragma once

#include <cuda_runtime.h>

namespace oec {

// fixed-point value of x at scale E (E >= the biased exponent of x, E >= 100)
__device__ __forceinline__ long long fx_of(double x, unsigned E) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sh = E - ((unsigned)(b >> 52) & 0x7FFu);   // >= 0; zero and denormals: >= 100
  const unsigned long long m = ((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull) << 3;
  const long long X = sh < 64u ? (long long)(m >> sh) : 0ll;
  return (long long)b < 0 ? -X : X;
}

// biased binary64 exponent of x
__device__ __forceinline__ unsigned fx_exp(double x) {
  return (unsigned)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FFu;
}

// total order of finite binary64 values as signed integers (sign and
// magnitude to two's complement; -0 and +0 both map to 0)
__device__ __forceinline__ long long fx_key(double x) {
  const long long b = __double_as_longlong(x);
  const long long m = b & 0x7FFFFFFFFFFFFFFFll;
  return b < 0 ? -m : m;
}

// flux with the limiter: zero where the flux and in_hi - in_lo (given by
// their ordered keys) have the same strict sign
__device__ __forceinline__ long long fx_flux(long long lap_hi, long long lap_lo, long long key_hi, long long key_lo) {
  const long long f = lap_hi - lap_lo;
  const bool lim = (f > 0 && key_hi > key_lo) || (f < 0 && key_hi < key_lo);
  return lim ? 0ll : f;
}

// div * 2^(E - 1078) as a binary64 (div rounded to nearest once, then an
// exact exponent shift: |div| >= 1 and E >= 100 keep it normal). The
// conversion runs on the FP64 pipe, which these integer-bound kernels leave
// mostly idle (forming the bits with integer operations instead measured
// slower: it loads the busiest pipe).
__device__ __forceinline__ double fx_scaled(long long div, unsigned E) {
  const double dv = __ll2double_rn(div);
  return div == 0 ? 0.0 : __longlong_as_double(__double_as_longlong(dv) + ((long long)((int)E - 1078) << 52));
}

}  // namespace oec
