// noalloc.cu - hdiff+vadvc for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they run the program: code
// that owns a fixed device-memory budget handed out by another allocator (a
// framework's caching allocator, a pool sized at start-up) and must not take
// memory behind its back, and latency-critical loops where an allocation or
// free may synchronise the whole device. oec_program_apply allocates its
// scratch on the first apply at a new size, so it does not suit them. The
// entry point below runs hdiff+vadvc with its scratch placed in a fixed array
// that is part of the library's device image: the staged form (hdiff of u and
// v, then the twisted column sweep of two threads per column, all on the
// caller's stream) when the domain's staged scratch fits, else the fused
// column sweep, which needs less.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/oec.h"
#include "api_internal.h"
#include "kernels.h"

namespace {

// 64 MiB. The staged form needs 40 bytes per grid point in FP64 (hdiff(u),
// hdiff(v) as double-float pairs, and g, e_u, e_v of the sweep, whose rows are
// padded to a multiple of 16 columns) and 32 in FP32 (each part rounded up to
// 256 bytes): up to 1,677,721 / 2,097,152 points. The
// fused form needs 24 * ceil16(ni) * ceil4(nj) * nk bytes (c', d'_u, d'_v per
// column of its 16 x 4 tiles).
constexpr size_t kNoallocScratchBytes = size_t(64) << 20;
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device. In host code
// the symbol name only stands for the array; it is never a device address.
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

int scratch_on_current_device(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return oec::cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return oec::fail(OEC_ERR_UNSUPPORTED, "device index %d above %d", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return oec::cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return OEC_OK;
}

bool holds(const oec_field_desc& f, const int64_t lo[3], const int64_t hi[3]) {
  for (int d = 0; d < 3; ++d)
    if (f.origin[d] + lo[d] < 0 || f.origin[d] + hi[d] > f.size[d]) return false;
  return true;
}

void span(const oec_field_desc& f, const int64_t lo[3], const int64_t hi[3], size_t es, uintptr_t& a, uintptr_t& b) {
  int64_t x = 0, y = 0;
  for (int d = 0; d < 3; ++d) {
    const int64_t p = (f.origin[d] + lo[d]) * f.stride[d], q = (f.origin[d] + hi[d] - 1) * f.stride[d];
    x += p < q ? p : q;
    y += p < q ? q : p;
  }
  a = (uintptr_t)f.data + x * (int64_t)es;
  b = (uintptr_t)f.data + y * (int64_t)es + es - 1;
}

}  // namespace

extern "C" OEC_API int oec_hdiff_vadvc_apply_noalloc(int32_t dtype, const oec_field_desc* in, const oec_field_desc* out,
                                                     const int64_t lb[3], const int64_t ub[3], double dtr,
                                                     void* cuda_stream) {
  using namespace oec;
  clear_error();
  if (!in || !out || !lb || !ub) return fail(OEC_ERR_INVALID_ARG, "null argument");
  if (dtype != OEC_F32 && dtype != OEC_F64) return fail(OEC_ERR_DTYPE, "dtype must be OEC_F32 or OEC_F64");
  for (int d = 0; d < 3; ++d) {
    if (ub[d] < lb[d]) return fail(OEC_ERR_INVALID_ARG, "inverted domain in dim %d", d);
    if (ub[d] - lb[d] > (1 << 30)) return fail(OEC_ERR_UNSUPPORTED, "domain extent above 2^30");
  }
  if (ub[0] == lb[0] || ub[1] == lb[1] || ub[2] == lb[2]) return OEC_OK;
  const oec_field_desc* f[6] = {&in[0], &in[1], &in[2], &in[3], &out[0], &out[1]};
  const int64_t sj = out[0].stride[1], sk = out[0].stride[2];
  for (int x = 0; x < 6; ++x) {
    if (!f[x]->data) return fail(OEC_ERR_INVALID_ARG, "field %d: null data pointer", x);
    if (f[x]->dtype != dtype) return fail(OEC_ERR_DTYPE, "field %d: dtype differs", x);
    if (f[x]->ndim != 3 || f[x]->stride[0] != 1 || f[x]->stride[1] != sj || f[x]->stride[2] != sk)
      return fail(OEC_ERR_UNSUPPORTED, "field %d: needs a 3-D field with stride[0] = 1 and the shared j/k strides", x);
  }
  // ranges the fused sweep reads: u, v at i/j +-2 (hdiff), w at i+1, coeff on the domain
  const int64_t uv_lo[3] = {lb[0] - 2, lb[1] - 2, lb[2]}, uv_hi[3] = {ub[0] + 2, ub[1] + 2, ub[2]};
  const int64_t w_hi[3] = {ub[0] + 1, ub[1], ub[2]};
  if (!holds(in[0], uv_lo, uv_hi) || !holds(in[1], uv_lo, uv_hi)) return fail(OEC_ERR_SHAPE, "u or v storage lacks the i/j halo of 2");
  if (!holds(in[2], lb, w_hi)) return fail(OEC_ERR_SHAPE, "w storage lacks the i+1 column");
  if (!holds(in[3], lb, ub) || !holds(out[0], lb, ub) || !holds(out[1], lb, ub))
    return fail(OEC_ERR_SHAPE, "a field's storage does not hold the domain");
  const size_t es = dtype == OEC_F64 ? 8 : 4;
  for (int o = 0; o < 2; ++o) {
    uintptr_t a, b;
    span(out[o], lb, ub, es, a, b);
    for (int x = 0; x < 4; ++x) {
      int64_t slo[3], shi[3];
      for (int d = 0; d < 3; ++d) { slo[d] = -in[x].origin[d]; shi[d] = in[x].size[d] - in[x].origin[d]; }
      uintptr_t c, e;
      span(in[x], slo, shi, es, c, e);
      if (a <= e && c <= b) return fail(OEC_ERR_ALIAS, "output %d overlaps input %d", o, x);
    }
    if (o == 1) {
      uintptr_t c, e;
      span(out[0], lb, ub, es, c, e);
      if (a <= e && c <= b) return fail(OEC_ERR_ALIAS, "the two outputs overlap");
    }
  }
  const Dom d{int(ub[0] - lb[0]), int(ub[1] - lb[1]), int(ub[2] - lb[2]), sj, sk};
  // the programs' default (staged) schedule; the fused column sweep (16x4
  // tiles, double-float) when its scratch does not fit
  oec_schedule s = default_schedule(OEC_KIND_HDIFF_VADVC, dtype);
  s.sweep = OEC_SWEEP_PAIR;   // the sweep with the smaller scratch
  s.slabs = 0;                // one stream: the caller's
  if (hdiff_vadvc_scratch_bytes(s, dtype, d) > kNoallocScratchBytes) {
    s = oec_schedule{};
    s.fusion = OEC_FUSE_INLINE;
    s.staging = OEC_STAGE_SMEM;
    s.tile_i = 16;
    s.tile_j = 4;
    s.unroll = 1;
    s.arith = OEC_ARITH_DOUBLE_FLOAT;
  }
  const size_t need = hdiff_vadvc_scratch_bytes(s, dtype, d);
  if (need > kNoallocScratchBytes)
    return fail(OEC_ERR_UNSUPPORTED, "domain needs %zu scratch bytes; the no-allocation entry point holds %zu",
                need, kNoallocScratchBytes);
  void* scratch = nullptr;
  int rc = scratch_on_current_device(&scratch);
  if (rc) return rc;
  auto at = [&](const oec_field_desc& g) {
    int64_t off = 0;
    for (int k = 0; k < 3; ++k) off += (g.origin[k] + lb[k]) * g.stride[k];
    return (char*)g.data + off * (int64_t)es;
  };
  cudaError_t e = hdiff_vadvc_launch(s, dtype, d, at(in[0]), at(in[1]), at(in[2]), at(in[3]), at(out[0]), at(out[1]),
                                     dtr, scratch, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return OEC_OK;
}
