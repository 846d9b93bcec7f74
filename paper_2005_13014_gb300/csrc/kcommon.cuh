// kcommon.cuh - helpers shared by the hand-written stencil kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstring>

namespace oec {

// Read-only load through the non-coherent path (inputs never alias outputs,
// paper §IV, so the texture/L1 path is safe).
template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// Asynchronous global -> shared copy of one element (4, 8 or 16 bytes) that
// bypasses the registers; copies are grouped per commit and waited for by
// group count, so a thread can keep many levels of a column in flight.
template <typename T>
__device__ __forceinline__ void cp_async(T* smem, const T* gmem) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8 || sizeof(T) == 16, "cp.async copies 4, 8 or 16 bytes");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"((int)sizeof(T)) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

// L2 eviction priorities (createpolicy): values that are read again soon
// (a column sweep's own recurrence values) stay while streamed fields, read
// or written once, leave first.
__device__ __forceinline__ uint64_t l2_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
// cp_async with an L2 eviction priority
template <typename T>
__device__ __forceinline__ void cp_async_l2(T* smem, const T* gmem, uint64_t pol) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8 || sizeof(T) == 16, "cp.async copies 4, 8 or 16 bytes");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global.L2::cache_hint [%0], [%1], %2, %3;\n" ::"r"(s), "l"(gmem),
               "n"((int)sizeof(T)), "l"(pol)
               : "memory");
}
// store of a 4- or 8-byte value with an L2 eviction priority
template <typename T>
__device__ __forceinline__ void st_l2(T* gmem, const T& v, uint64_t pol) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte stores");
  const size_t g = __cvta_generic_to_global(gmem);
  if (sizeof(T) == 8) {
    unsigned long long b;
    memcpy(&b, &v, 8);
    asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;\n" ::"l"(g), "l"(b), "l"(pol) : "memory");
  } else {
    unsigned b;
    memcpy(&b, &v, 4);
    asm volatile("st.global.L2::cache_hint.b32 [%0], %1, %2;\n" ::"l"(g), "r"(b), "l"(pol) : "memory");
  }
}
// drop the 128-byte L2 line at p (128-byte aligned) without writing it back:
// for scratch that nothing reads again. Its contents become undefined.
__device__ __forceinline__ void l2_discard(const void* p) {
  asm volatile("discard.global.L2 [%0], 128;\n" ::"l"(__cvta_generic_to_global(p)) : "memory");
}
// wait until at most N of this thread's committed groups are still pending
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Stage bodies of the horizontal-diffusion program, written once and used by
// every kernel variant (fused, unfused, batched, and inside the column sweep).
// Laplacian: 4*c - w - e - s - n, in that order.
template <typename T>
__device__ __forceinline__ T hd_lap(T c, T w, T e, T s, T n) {
  return T(4) * c - w - e - s - n;
}
// Flux with the sign limiter: 0 where the flux points down the input gradient.
template <typename T>
__device__ __forceinline__ T hd_flux(T lap_hi, T lap_lo, T in_hi, T in_lo) {
  T f = lap_hi - lap_lo;
  return (f * (in_hi - in_lo) > T(0)) ? T(0) : f;
}
// Output: in - coeff*((flx - flx(i-1)) + (fly - fly(j-1))).
template <typename T>
__device__ __forceinline__ T hd_out(T in, T coeff, T flx, T flx_m, T fly, T fly_m) {
  return in - coeff * ((flx - flx_m) + (fly - fly_m));
}

__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

}  // namespace oec
