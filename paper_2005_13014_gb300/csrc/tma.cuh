// tma.cuh - tensor-memory-accelerator copies into shared memory: mbarrier
// helpers (bounded waits), the 3-D tiled cp.async.bulk.tensor load, and the
// host-side tensor-map encoding of a field (driver entry point looked up at
// run time). Shared by the TMA-staged kernels.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>

#include "kernels.h"

namespace oec {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
// bounded wait for the phase with the given parity to complete: at most
// `polls` polls; false when it gave up
__device__ __forceinline__ bool mbar_wait_n(unsigned bar, unsigned parity, unsigned polls) {
  for (unsigned it = 0; it < polls; ++it) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// the kernels' wait: about a second of polling
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) { return mbar_wait_n(bar, parity, 1u << 20); }
// 3-D tile load global -> shared, completion counted on bar; x must be a
// multiple of 16 bytes / element size and dst 128-byte aligned (the callers
// guarantee both)
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
      ::"r"(smem_u32(dst)), "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// cuTensorMapEncodeTiled from the CUDA driver API (null if unavailable)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();
// device address of the counter of bounded waits that gave up
unsigned* wait_timeout_counter();

// tensor map of a field's storage (3-D, element strides sj, sk) with a bx x
// by x 1 box; out-of-range elements read as zero
template <class S>
bool encode_map(CUtensorMap* m, const TmaField& f, int64_t sj, int64_t sk, int bx, int by) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)f.size[0], (cuuint64_t)f.size[1], (cuuint64_t)f.size[2]};
  const cuuint64_t strides[2] = {(cuuint64_t)(sj * sizeof(S)), (cuuint64_t)(sk * sizeof(S))};
  const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  return enc(m, sizeof(S) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
             const_cast<void*>(f.base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace oec
