// dispatch.cpp - turns a validated apply into launches of the hand-written
// kernels: base pointers at the domain's lower corner, shared strides, scratch.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/oec.h"
#include "api_internal.h"
#include "kernels.h"

namespace oec {

static char* base_at(const oec_field_desc& f, const int64_t lb[3], size_t es) {
  int64_t off = 0;
  for (int d = 0; d < 3; ++d) off += (f.origin[d] + lb[d]) * f.stride[d];
  return (char*)f.data + off * (int64_t)es;
}

int dispatch_apply(oec_program* p, const oec_field_desc* in, const oec_field_desc* out, const int64_t lb[3],
                   const int64_t ub[3], const double* params, cudaStream_t st) {
  if (p->kind == OEC_KIND_GENERIC) return generic_apply(p, in, out, lb, ub, params, st);
  const Program& ir = p->ir;
  const size_t es = elem_size(p->dtype);
  const int n_in = (int)ir.inputs.size(), n_out = (int)ir.outputs.size();
  // the hand-written kernels index every field with one pair of strides
  const int64_t sj = out[0].stride[1], sk = out[0].stride[2];
  for (int x = 0; x < n_in + n_out; ++x) {
    const oec_field_desc& f = x < n_in ? in[x] : out[x - n_in];
    if (f.ndim != 3 || f.stride[1] != sj || f.stride[2] != sk)
      return fail(OEC_ERR_UNSUPPORTED, "hand-written kernels need 3-D fields with equal j/k strides (field %d differs)", x);
  }
  Dom d{int(ub[0] - lb[0]), int(ub[1] - lb[1]), int(ub[2] - lb[2]), sj, sk};
  char* I[16];
  char* O[4];
  for (int x = 0; x < n_in; ++x) I[x] = base_at(in[x], lb, es);
  for (int x = 0; x < n_out; ++x) O[x] = base_at(out[x], lb, es);
  cudaError_t e = cudaSuccess;
  int rc = OEC_OK;
  switch (p->kind) {
    case OEC_KIND_HDIFF: {
      const bool vec = p->sched.fusion == OEC_FUSE_INLINE &&
                       (p->sched.staging == OEC_STAGE_WARP || p->sched.staging == OEC_STAGE_TMA);
      if (vec && ((((uintptr_t)I[0] | (uintptr_t)I[1] | (uintptr_t)O[0]) % 16 != 0) || (sj * (int64_t)es) % 16 != 0 ||
                  (sk * (int64_t)es) % 16 != 0))
        return fail(OEC_ERR_UNSUPPORTED,
                    "OEC_STAGE_WARP/TMA need 16-byte aligned rows: domain corner of every field and j/k strides");
      if (vec && p->sched.staging == OEC_STAGE_TMA) {
        TmaField t[2];
        for (int x = 0; x < 2; ++x) {
          if ((uintptr_t)in[x].data % 16 != 0) return fail(OEC_ERR_UNSUPPORTED, "TMA staging: storage not 16-byte aligned");
          t[x].base = in[x].data;
          for (int a = 0; a < 3; ++a) {
            t[x].size[a] = in[x].size[a];
            t[x].corner[a] = in[x].origin[a] + lb[a];
          }
        }
        e = hdiff_tma_launch(p->sched, p->dtype, d, t[0], t[1], O[0], st);
        if (e == cudaErrorNotSupported) return fail(OEC_ERR_UNSUPPORTED, "TMA staging: tensor maps unavailable");
        break;
      }
      rc = ensure_scratch(p, hdiff_scratch_bytes(p->sched, p->dtype, d));
      if (rc) return rc;
      e = hdiff_launch(p->sched, p->dtype, d, I[0], I[1], O[0], p->scratch, st);
      break;
    }
    case OEC_KIND_HDIFF_VADVC:
      rc = ensure_scratch(p, hdiff_vadvc_scratch_bytes(p->sched, p->dtype, d));
      if (rc) return rc;
      e = hdiff_vadvc_launch(p->sched, p->dtype, d, I[0], I[1], I[2], I[3], O[0], O[1], params[0], p->scratch, st);
      break;
    case OEC_KIND_FASTWAVES: {
      rc = ensure_scratch(p, fastwaves_scratch_bytes(p->sched, p->dtype, d));
      if (rc) return rc;
      FastwavesPtrs f{I[0], I[1], I[2], I[3], I[4], I[5], I[6], I[7], I[8], O[0], O[1]};
      if (p->sched.fusion == OEC_FUSE_INLINE && p->sched.staging == OEC_STAGE_TMA) {
        // tensor maps: 16-byte aligned storage and j/k strides
        if ((sj * (int64_t)es) % 16 != 0 || (sk * (int64_t)es) % 16 != 0)
          return fail(OEC_ERR_UNSUPPORTED, "TMA staging: j/k strides must be multiples of 16 bytes");
        TmaField t[9];
        for (int x = 0; x < 9; ++x) {
          if ((uintptr_t)in[x].data % 16 != 0) return fail(OEC_ERR_UNSUPPORTED, "TMA staging: storage not 16-byte aligned");
          t[x].base = in[x].data;
          for (int a = 0; a < 3; ++a) {
            t[x].size[a] = in[x].size[a];
            t[x].corner[a] = in[x].origin[a] + lb[a];
          }
        }
        e = fastwaves_launch(p->sched, p->dtype, d, f, params[0], params[1], p->scratch, st, t);
        if (e == cudaErrorNotSupported) return fail(OEC_ERR_UNSUPPORTED, "TMA staging: tensor maps unavailable");
        break;
      }
      e = fastwaves_launch(p->sched, p->dtype, d, f, params[0], params[1], p->scratch, st);
      break;
    }
    default:
      return fail(OEC_ERR_UNSUPPORTED, "unknown program kind");
  }
  if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
  return OEC_OK;
}

}  // namespace oec
