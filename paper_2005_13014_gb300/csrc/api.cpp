// api.cpp - the C ABI of liboec (include/oec.h): program handles, validation of
// field descriptors against the inferred ranges (paper §V-B), schedule
// selection and dispatch to the hand-written kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/oec.h"
#include "api_internal.h"
#include "builtin_programs.h"
#include "ir.h"
#include "kernels.h"

namespace oec {

namespace {
thread_local std::string g_err;
}

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

void clear_error() { g_err.clear(); }

int cuda_fail(cudaError_t e, const char* where) {
  return fail(OEC_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

static const std::string& builtin_canon(int kind) {
  static std::string c[4];
  static std::once_flag once;
  std::call_once(once, [] {
    const char* src[4] = {nullptr, kBuiltin_hdiff, kBuiltin_hdiff_vadvc, kBuiltin_fastwaves};
    for (int k = 1; k < 4; ++k) {
      Program p;
      std::string err;
      if (parse(src[k], p, err)) c[k] = canonical(p);
    }
  });
  return c[kind];
}

oec_schedule default_schedule(int kind, int dtype) {
  oec_schedule s{};
  s.fusion = OEC_FUSE_INLINE;
  s.unroll = 1;
  switch (kind) {
    case OEC_KIND_HDIFF:
      s.staging = OEC_STAGE_SMEM;
      s.tile_i = 64;
      s.tile_j = 4;
      s.k_chunk = 2;
      s.arith = OEC_ARITH_DOUBLE_FLOAT;
      break;
    case OEC_KIND_HDIFF_VADVC:
      // the staged form the autotuner picks at 128x128x80: FP64 fixed-point
      // producer 32x16 with 2 rows per thread, 2 levels per CTA; FP32
      // vector-row producer (REGS on unaligned fields), 20 levels per CTA;
      // double-float column sweep
      s.fusion = OEC_FUSE_NONE;
      s.staging = dtype == OEC_F64 ? OEC_STAGE_REGS : OEC_STAGE_WARP;
      s.tile_i = 32;
      s.tile_j = dtype == OEC_F64 ? 16 : 4;
      s.unroll = dtype == OEC_F64 ? 2 : 1;
      s.k_chunk = dtype == OEC_F64 ? 2 : 20;
      s.arith = dtype == OEC_F64 ? OEC_ARITH_FIXED : OEC_ARITH_DOUBLE_FLOAT;
      break;
    case OEC_KIND_FASTWAVES:
      s.staging = OEC_STAGE_REGS;
      s.tile_i = 64;
      s.tile_j = 4;
      s.unroll = 2;
      s.arith = OEC_ARITH_DOUBLE_FLOAT;
      break;
    default:
      s.staging = OEC_STAGE_REGS;
      s.tile_i = 64;
      s.tile_j = 4;
      break;
  }
  return s;
}

bool schedule_ok(int kind, const oec_schedule& s, std::string& why) {
  for (int r : s.reserved)
    if (r != 0) { why = "reserved schedule fields must be zero"; return false; }
  if (s.index_bits != OEC_INDEX_AUTO && s.index_bits != OEC_INDEX_64) {
    why = "index_bits must be OEC_INDEX_AUTO (0) or OEC_INDEX_64 (64)";
    return false;
  }
  const bool staged_hv = kind == OEC_KIND_HDIFF_VADVC && s.fusion == OEC_FUSE_NONE;
  const bool sweep_ok = s.sweep == OEC_SWEEP_SPLIT || s.sweep == OEC_SWEEP_SEGMENTS4 || s.sweep == OEC_SWEEP_SEGMENTS8;
  if (s.sweep != OEC_SWEEP_PAIR && !(staged_hv && sweep_ok)) {
    why = "sweep: OEC_SWEEP_PAIR (0), or OEC_SWEEP_SPLIT (1), OEC_SWEEP_SEGMENTS4 (4), OEC_SWEEP_SEGMENTS8 (8) for "
          "the stage-by-stage hdiff+vadvc form";
    return false;
  }
  if (s.slabs != 0 && !(staged_hv && s.slabs >= 1 && s.slabs <= 16)) {
    why = "slabs: 0, or 1..16 for the stage-by-stage hdiff+vadvc form";
    return false;
  }
  switch (kind) {
    case OEC_KIND_HDIFF: return hdiff_schedule_ok(s, why);
    case OEC_KIND_HDIFF_VADVC: return hdiff_vadvc_schedule_ok(s, why);
    case OEC_KIND_FASTWAVES: return fastwaves_schedule_ok(s, why);
    default: return generic_schedule_ok(s, why);
  }
}

size_t elem_size(int dtype) { return dtype == OEC_F64 ? 8 : 4; }

// Byte interval [lo, hi] touched by `f` over the box [blo, bhi) (non-empty).
static void byte_span(const oec_field_desc& f, const int64_t blo[3], const int64_t bhi[3], size_t es, uintptr_t& lo,
                      uintptr_t& hi) {
  int64_t a = 0, b = 0;
  for (int d = 0; d < 3; ++d) {
    const int64_t s = f.stride[d];
    const int64_t x0 = (f.origin[d] + blo[d]) * s, x1 = (f.origin[d] + bhi[d] - 1) * s;
    a += std::min(x0, x1);
    b += std::max(x0, x1);
  }
  lo = (uintptr_t)f.data + a * (int64_t)es;
  hi = (uintptr_t)f.data + b * (int64_t)es + es - 1;
}

int validate_fields(const oec_program* p, const oec_field_desc* in, int n_in, const oec_field_desc* out, int n_out,
                    const int64_t lb[3], const int64_t ub[3], const int64_t halo[3], std::vector<Box>& ranges) {
  const Program& ir = p->ir;
  const size_t es = elem_size(p->dtype);
  std::string err;
  if (!infer_ranges(ir, lb, ub, ranges, err)) return fail(OEC_ERR_SHAPE, "%s", err.c_str());
  auto check_desc = [&](const oec_field_desc& f, const char* role, int idx) -> int {
    if (!f.data) return fail(OEC_ERR_INVALID_ARG, "%s %d: null data pointer", role, idx);
    if (f.dtype != p->dtype) return fail(OEC_ERR_DTYPE, "%s %d: dtype %d, program dtype %d", role, idx, f.dtype, p->dtype);
    if (f.ndim < 1 || f.ndim > 3) return fail(OEC_ERR_INVALID_ARG, "%s %d: ndim must be 1..3", role, idx);
    if (f.stride[0] != 1) return fail(OEC_ERR_UNSUPPORTED, "%s %d: stride[0] must be 1", role, idx);
    for (int d = 0; d < 3; ++d)
      if (f.size[d] < 1) return fail(OEC_ERR_INVALID_ARG, "%s %d: size[%d] < 1", role, idx, d);
    return OEC_OK;
  };
  for (int x = 0; x < n_in; ++x) {
    int rc = check_desc(in[x], "input", x);
    if (rc) return rc;
    const Box& r = ranges[ir.inputs[x]];
    if (!r.valid) continue;
    for (int d = 0; d < 3; ++d) {
      if (r.lo[d] < lb[d] - halo[d] || r.hi[d] > ub[d] + halo[d])
        return fail(OEC_ERR_HALO, "input '%s': inferred range [%lld, %lld) in dim %d exceeds halo %lld around [%lld, %lld)",
                    ir.values[ir.inputs[x]].name.c_str(), (long long)r.lo[d], (long long)r.hi[d], d,
                    (long long)halo[d], (long long)lb[d], (long long)ub[d]);
      if (in[x].origin[d] + r.lo[d] < 0 || in[x].origin[d] + r.hi[d] > in[x].size[d])
        return fail(OEC_ERR_SHAPE, "input '%s': storage does not hold inferred range [%lld, %lld) in dim %d",
                    ir.values[ir.inputs[x]].name.c_str(), (long long)r.lo[d], (long long)r.hi[d], d);
    }
  }
  for (int x = 0; x < n_out; ++x) {
    int rc = check_desc(out[x], "output", x);
    if (rc) return rc;
    for (int d = 0; d < 3; ++d)
      if (out[x].origin[d] + lb[d] < 0 || out[x].origin[d] + ub[d] > out[x].size[d])
        return fail(OEC_ERR_SHAPE, "output %d: storage does not hold the domain in dim %d", x, d);
  }
  // alias: an output's written bytes may not meet any input's storage or another output
  for (int x = 0; x < n_out; ++x) {
    uintptr_t olo, ohi;
    byte_span(out[x], lb, ub, es, olo, ohi);
    for (int y = 0; y < n_in; ++y) {
      int64_t slo[3], shi[3];
      for (int d = 0; d < 3; ++d) { slo[d] = -in[y].origin[d]; shi[d] = in[y].size[d] - in[y].origin[d]; }
      uintptr_t ilo, ihi;
      byte_span(in[y], slo, shi, es, ilo, ihi);
      if (olo <= ihi && ilo <= ohi) return fail(OEC_ERR_ALIAS, "output %d overlaps input %d", x, y);
    }
    for (int y = 0; y < x; ++y) {
      uintptr_t plo, phi;
      byte_span(out[y], lb, ub, es, plo, phi);
      if (olo <= phi && plo <= ohi) return fail(OEC_ERR_ALIAS, "output %d overlaps output %d", x, y);
    }
  }
  return OEC_OK;
}

int ensure_scratch(oec_program* p, size_t bytes) {
  if (bytes == 0) return OEC_OK;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (p->scratch && p->scratch_bytes >= bytes && p->scratch_dev == dev) return OEC_OK;
  if (p->scratch && p->graphs > 0)
    return fail(OEC_ERR_UNSUPPORTED, "the program's scratch is used by %d captured apply graph(s): destroy them "
                "before applying at a larger domain", p->graphs);
  if (p->scratch) {
    int cur = dev;
    cudaSetDevice(p->scratch_dev);
    cudaFree(p->scratch);                    // waits for work that may still use it
    cudaSetDevice(cur);
    p->scratch = nullptr;
    p->scratch_bytes = 0;
  }
  if (fault_injected("alloc"))
    return fail(OEC_ERR_CUDA, "scratch allocation of %zu bytes failed (injected by OEC_FAULT=alloc)", bytes);
  e = cudaMalloc(&p->scratch, bytes);
  if (e != cudaSuccess) {
    p->scratch = nullptr;
    return cuda_fail(e, "cudaMalloc(scratch)");
  }
  p->scratch_bytes = bytes;
  p->scratch_dev = dev;
  return OEC_OK;
}

}  // namespace oec

using namespace oec;

namespace oec {
namespace {
// the program whose apply is running on this thread (launched() is a no-op
// outside an apply, e.g. for batches and the no-allocation entry point)
thread_local oec_program* t_applying = nullptr;

int record_event(oec_program* p, cudaStream_t st) {
  if (p->ev_used == (int)p->ev_pool.size()) {
    cudaEvent_t e;
    cudaError_t err = cudaEventCreate(&e);
    if (err != cudaSuccess) return cuda_fail(err, "cudaEventCreate");
    p->ev_pool.push_back(e);
  }
  cudaError_t err = cudaEventRecord(p->ev_pool[p->ev_used], st);
  if (err != cudaSuccess) return cuda_fail(err, "cudaEventRecord");
  ++p->ev_used;
  return OEC_OK;
}
}  // namespace

namespace {
thread_local bool t_group = false;   // inside launch_group_begin/end
}

void launched(cudaStream_t st) {
  oec_program* p = t_applying;
  if (!p) return;
  ++p->last_launches;
  if (p->timing && !t_group && record_event(p, st) == OEC_OK) ++p->last_timed;
}

void launch_group_begin() { t_group = true; }

void launch_group_end(cudaStream_t st) {
  t_group = false;
  oec_program* p = t_applying;
  if (p && p->timing && record_event(p, st) == OEC_OK) ++p->last_timed;
}
}  // namespace oec

extern "C" {

const char* oec_last_error(void) { return g_err.c_str(); }

int oec_program_create(const char* source, const oec_program_options* opts, oec_program_t* out) {
  clear_error();
  if (!source || !out) return fail(OEC_ERR_INVALID_ARG, "null source or output handle");
  *out = nullptr;
  const int dtype = opts ? opts->dtype : OEC_F64;
  if (dtype != OEC_F32 && dtype != OEC_F64) return fail(OEC_ERR_DTYPE, "dtype must be OEC_F32 or OEC_F64");
  oec_program* p = new (std::nothrow) oec_program();
  if (!p) return fail(OEC_ERR_INVALID_ARG, "out of host memory");
  std::string err;
  if (!parse(source, p->ir, err)) {
    delete p;
    return fail(OEC_ERR_PARSE, "%s", err.c_str());
  }
  p->dtype = dtype;
  p->kind = OEC_KIND_GENERIC;
  if (!(opts && (opts->flags & OEC_OPT_GENERIC))) {
    const std::string c = canonical(p->ir);
    for (int k = 1; k < 4; ++k)
      if (c == builtin_canon(k)) p->kind = k;
  }
  p->sched = default_schedule(p->kind, dtype);
  *out = p;
  return OEC_OK;
}

namespace {

// device staging of oec_program_apply_host: wait for the last use, free
void host_stage_release(oec_program* p) {
  auto& h = p->host;
  if (h.dev < 0) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(h.dev);
  for (cudaStream_t c : h.copy)
    if (c) cudaStreamSynchronize(c);
  for (int s = 0; s < 2; ++s) {
    if (h.released[s]) cudaEventSynchronize(h.released[s]);
    for (void* b : h.buf[s]) cudaFree(b);
    h.buf[s].clear();
    for (cudaEvent_t& ev : h.inputs_in[s]) {
      if (ev) cudaEventDestroy(ev);
      ev = nullptr;
    }
    if (h.released[s]) cudaEventDestroy(h.released[s]);
    h.released[s] = nullptr;
  }
  for (cudaStream_t& c : h.copy) {
    if (c) cudaStreamDestroy(c);
    c = nullptr;
  }
  h.bytes.clear();
  h.dev = -1;
  h.next = 0;
  cudaSetDevice(cur);
}

// bytes spanned by a field's storage (positive strides)
size_t span_bytes(const oec_field_desc& f, size_t es) {
  int64_t last = 0;
  for (int d = 0; d < 3; ++d) last += (f.size[d] - 1) * f.stride[d];
  return size_t(last + 1) * es;
}

}  // namespace

void oec_program_destroy(oec_program_t p) {
  if (!p) return;
  host_stage_release(p);
  if (p->scratch) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(p->scratch_dev);
    cudaFree(p->scratch);
    cudaSetDevice(cur);
  }
  generic_release(p);
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  delete p;
}

int oec_program_get_info(oec_program_t p, oec_program_info* info) {
  clear_error();
  if (!p || !info) return fail(OEC_ERR_INVALID_ARG, "null argument");
  info->kind = p->kind;
  info->n_inputs = (int)p->ir.inputs.size();
  info->n_outputs = (int)p->ir.outputs.size();
  info->n_params = (int)p->ir.params.size();
  info->n_stages = (int)p->ir.stmts.size();
  info->dtype = p->dtype;
  return OEC_OK;
}

int oec_program_input_name(oec_program_t p, int index, char* buf, int len) {
  clear_error();
  if (!p || !buf || len < 1) return fail(OEC_ERR_INVALID_ARG, "null argument");
  if (index < 0 || index >= (int)p->ir.inputs.size()) return fail(OEC_ERR_INVALID_ARG, "input index out of range");
  std::snprintf(buf, (size_t)len, "%s", p->ir.values[p->ir.inputs[index]].name.c_str());
  return OEC_OK;
}

int oec_program_input_range(oec_program_t p, int index, const int64_t lb[3], const int64_t ub[3], int64_t lo[3],
                            int64_t hi[3]) {
  clear_error();
  if (!p || !lb || !ub || !lo || !hi) return fail(OEC_ERR_INVALID_ARG, "null argument");
  if (index < 0 || index >= (int)p->ir.inputs.size()) return fail(OEC_ERR_INVALID_ARG, "input index out of range");
  std::vector<Box> r;
  std::string err;
  if (!infer_ranges(p->ir, lb, ub, r, err)) return fail(OEC_ERR_SHAPE, "%s", err.c_str());
  const Box& b = r[p->ir.inputs[index]];
  for (int d = 0; d < 3; ++d) {
    lo[d] = b.valid ? b.lo[d] : lb[d];
    hi[d] = b.valid ? b.hi[d] : lb[d];
  }
  return OEC_OK;
}

int oec_program_set_schedule(oec_program_t p, const oec_schedule* s) {
  clear_error();
  if (!p || !s) return fail(OEC_ERR_INVALID_ARG, "null argument");
  std::string why;
  if (!schedule_ok(p->kind, *s, why)) return fail(OEC_ERR_UNSUPPORTED, "schedule: %s", why.c_str());
  if (p->kind == OEC_KIND_GENERIC && s->arith == 1 && p->dtype != OEC_F64)
    return fail(OEC_ERR_UNSUPPORTED, "schedule: double-float generated kernels are for FP64 programs");
  p->sched = *s;
  return OEC_OK;
}

int oec_program_get_schedule(oec_program_t p, oec_schedule* s) {
  clear_error();
  if (!p || !s) return fail(OEC_ERR_INVALID_ARG, "null argument");
  *s = p->sched;
  return OEC_OK;
}

int oec_program_algorithmic_bytes(oec_program_t p, const int64_t lb[3], const int64_t ub[3], int64_t* bytes) {
  clear_error();
  if (!p || !lb || !ub || !bytes) return fail(OEC_ERR_INVALID_ARG, "null argument");
  std::vector<Box> r;
  std::string err;
  if (!infer_ranges(p->ir, lb, ub, r, err)) return fail(OEC_ERR_SHAPE, "%s", err.c_str());
  int64_t elems = 0;
  for (int v : p->ir.inputs) elems += r[v].volume();
  int64_t dom = 1;
  for (int d = 0; d < 3; ++d) dom *= std::max<int64_t>(0, ub[d] - lb[d]);
  elems += dom * (int64_t)p->ir.outputs.size();
  *bytes = elems * (int64_t)elem_size(p->dtype);
  return OEC_OK;
}

int oec_program_apply_host(oec_program_t p, const oec_field_desc* in, int n_in, const oec_field_desc* out,
                           int n_out, const int64_t lb[3], const int64_t ub[3], const int64_t halo[3],
                           const double* params, int n_params, void* cuda_stream) {
  clear_error();
  NvtxRange range("oec_program_apply_host");
  if (!p || !lb || !ub || !halo) return fail(OEC_ERR_INVALID_ARG, "null argument");
  const Program& ir = p->ir;
  if (n_in != (int)ir.inputs.size() || (n_in && !in))
    return fail(OEC_ERR_INVALID_ARG, "program has %zu inputs, got %d", ir.inputs.size(), n_in);
  if (n_out != (int)ir.outputs.size() || !out)
    return fail(OEC_ERR_INVALID_ARG, "program has %zu outputs, got %d", ir.outputs.size(), n_out);
  for (int d = 0; d < 3; ++d)
    if (ub[d] < lb[d]) return fail(OEC_ERR_INVALID_ARG, "inverted domain in dim %d", d);
  if (ub[0] == lb[0] || ub[1] == lb[1] || ub[2] == lb[2]) return OEC_OK;   // empty domain: nothing to do
  const size_t es = elem_size(p->dtype);
  const int nf = n_in + n_out;
  std::vector<size_t> bytes(nf);
  for (int x = 0; x < nf; ++x) {
    const oec_field_desc& f = x < n_in ? in[x] : out[x - n_in];
    if (!f.data) return fail(OEC_ERR_INVALID_ARG, "field %d: null data", x);
    if (f.ndim != 3 || f.stride[0] != 1 || f.stride[1] <= 0 || f.stride[2] <= 0 || f.size[0] < 1 || f.size[1] < 1 ||
        f.size[2] < 1)
      return fail(OEC_ERR_UNSUPPORTED, "host fields: 3-D, unit i stride, positive j/k strides (field %d)", x);
    bytes[x] = span_bytes(f, es);
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  auto& h = p->host;
  if (h.dev != dev || h.bytes != bytes) {
    host_stage_release(p);
    h.dev = dev;
    h.bytes = bytes;
    for (int c = 0; c < oec_program::kCopyStreams && e == cudaSuccess; ++c)
      e = cudaStreamCreateWithFlags(&h.copy[c], cudaStreamNonBlocking);
    for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
      for (int c = 0; c < oec_program::kCopyStreams && e == cudaSuccess; ++c)
        e = cudaEventCreateWithFlags(&h.inputs_in[s][c], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h.released[s], cudaEventDisableTiming);
      for (int x = 0; x < nf && e == cudaSuccess; ++x) {
        void* b = nullptr;
        e = cudaMalloc(&b, bytes[x]);
        if (e == cudaSuccess) h.buf[s].push_back(b);
      }
    }
    if (e != cudaSuccess) {
      host_stage_release(p);
      return cuda_fail(e, "host staging buffers");
    }
  }
  const int s = h.next;
  h.next ^= 1;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  // set s is free once the outputs of its previous call have left it. Each
  // input crosses as one contiguous copy of its storage from the first to
  // the last element of its access box (shape inference), widened to 4 KiB
  // boundaries of the host address: strided host-to-device copies of the box
  // itself ran at a sixth of the contiguous rate
  std::vector<Box> boxes;
  std::string err;
  if (!infer_ranges(ir, lb, ub, boxes, err)) return fail(OEC_ERR_SHAPE, "%s", err.c_str());
  constexpr int NC = oec_program::kCopyStreams;
  for (int c = 0; c < NC && e == cudaSuccess; ++c) e = cudaStreamWaitEvent(h.copy[c], h.released[s], 0);
  for (int x = 0; x < n_in && e == cudaSuccess; ++x) {
    const oec_field_desc& f = in[x];
    const Box& b = boxes[ir.inputs[x]];
    if (!b.valid) continue;
    int64_t first = 0, last = 0;
    for (int d = 0; d < 3; ++d) {
      first += std::max<int64_t>(0, f.origin[d] + b.lo[d]) * f.stride[d];
      last += std::min<int64_t>(f.size[d] - 1, f.origin[d] + b.hi[d] - 1) * f.stride[d];
    }
    const uintptr_t base = (uintptr_t)f.data;
    uintptr_t lo = (base + size_t(first) * es) & ~uintptr_t(4095), hi = (base + size_t(last + 1) * es + 4095) & ~uintptr_t(4095);
    lo = std::max(lo, base);
    hi = std::min(hi, base + bytes[x]);
    if (hi <= lo) continue;
    e = cudaMemcpyAsync((char*)h.buf[s][x] + (lo - base), (const void*)lo, hi - lo, cudaMemcpyHostToDevice,
                        h.copy[x % NC]);
  }
  for (int c = 0; c < NC && e == cudaSuccess; ++c) {
    e = cudaEventRecord(h.inputs_in[s][c], h.copy[c]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h.inputs_in[s][c], 0);
  }
  if (e != cudaSuccess) return cuda_fail(e, "host input copies");
  std::vector<oec_field_desc> dv(in, in + n_in), dw(out, out + n_out);
  for (int x = 0; x < n_in; ++x) dv[x].data = h.buf[s][x];
  for (int x = 0; x < n_out; ++x) dw[x].data = h.buf[s][n_in + x];
  int rc = oec_program_apply(p, dv.data(), n_in, dw.data(), n_out, lb, ub, halo, params, n_params, cuda_stream);
  if (rc == OEC_OK) {
    // each output's domain box back into the host storage
    for (int x = 0; x < n_out && e == cudaSuccess; ++x) {
      const oec_field_desc& f = out[x];
      const size_t pitch = size_t(f.stride[1]) * es;
      cudaMemcpy3DParms m = {};
      m.kind = cudaMemcpyDeviceToHost;
      m.extent = make_cudaExtent(size_t(ub[0] - lb[0]) * es, size_t(ub[1] - lb[1]), size_t(ub[2] - lb[2]));
      if (f.stride[2] % f.stride[1] == 0) {
        const size_t rows = size_t(f.stride[2] / f.stride[1]);   // rows per level (plane pitch)
        m.srcPtr = make_cudaPitchedPtr(h.buf[s][n_in + x], pitch, size_t(f.size[0]) * es, rows);
        m.dstPtr = make_cudaPitchedPtr(f.data, pitch, size_t(f.size[0]) * es, rows);
        m.srcPos = m.dstPos = make_cudaPos(size_t(f.origin[0] + lb[0]) * es, size_t(f.origin[1] + lb[1]),
                                           size_t(f.origin[2] + lb[2]));
        e = cudaMemcpy3DAsync(&m, st);
      } else {
        // plane pitch not a whole number of rows: one 2-D copy per level
        for (int64_t k = lb[2]; k < ub[2] && e == cudaSuccess; ++k) {
          const size_t off = (size_t((f.origin[2] + k) * f.stride[2] + (f.origin[1] + lb[1]) * f.stride[1]) +
                              size_t(f.origin[0] + lb[0])) * es;
          e = cudaMemcpy2DAsync((char*)f.data + off, pitch, (const char*)h.buf[s][n_in + x] + off, pitch,
                                size_t(ub[0] - lb[0]) * es, size_t(ub[1] - lb[1]), cudaMemcpyDeviceToHost, st);
        }
      }
    }
  }
  const cudaError_t er = cudaEventRecord(h.released[s], st);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "host output copies");
  if (er != cudaSuccess) return cuda_fail(er, "cudaEventRecord");
  return OEC_OK;
}

int oec_program_apply(oec_program_t p, const oec_field_desc* in, int n_in, const oec_field_desc* out, int n_out,
                      const int64_t lb[3], const int64_t ub[3], const int64_t halo[3], const double* params,
                      int n_params, void* cuda_stream) {
  clear_error();
  NvtxRange range("oec_program_apply");
  if (!p || !lb || !ub || !halo) return fail(OEC_ERR_INVALID_ARG, "null argument");
  p->last_launches = 0;
  p->last_timed = 0;
  const Program& ir = p->ir;
  if (n_in != (int)ir.inputs.size() || (n_in && !in))
    return fail(OEC_ERR_INVALID_ARG, "program has %zu inputs, got %d", ir.inputs.size(), n_in);
  if (n_out != (int)ir.outputs.size() || !out)
    return fail(OEC_ERR_INVALID_ARG, "program has %zu outputs, got %d", ir.outputs.size(), n_out);
  if (n_params != (int)ir.params.size() || (n_params && !params))
    return fail(OEC_ERR_INVALID_ARG, "program has %zu params, got %d", ir.params.size(), n_params);
  for (int d = 0; d < 3; ++d) {
    if (ub[d] < lb[d]) return fail(OEC_ERR_INVALID_ARG, "inverted domain in dim %d", d);
    if (halo[d] < 0) return fail(OEC_ERR_INVALID_ARG, "negative halo");
    if (ub[d] - lb[d] > (1 << 30)) return fail(OEC_ERR_UNSUPPORTED, "domain extent above 2^30");
  }
  if (ub[0] == lb[0] || ub[1] == lb[1] || ub[2] == lb[2]) return OEC_OK;   // empty domain: nothing to do
  std::vector<Box> ranges;
  int rc = validate_fields(p, in, n_in, out, n_out, lb, ub, halo, ranges);
  if (rc) return rc;
  const cudaStream_t st = (cudaStream_t)cuda_stream;
  const int first = p->ev_used;
  if (p->timing && (rc = record_event(p, st))) return rc;
  t_applying = p;
  rc = dispatch_apply(p, in, out, lb, ub, params, st);
  t_applying = nullptr;
  if (p->timing) {
    if (rc || p->ev_used != first + 1 + p->last_timed) {
      p->ev_used = first;   // drop a partly recorded apply
    } else {
      p->ev_first.push_back(first);
      p->ev_count.push_back(p->ev_used - first);
    }
  }
  return rc;
}

int oec_device_wait_selftest(int polls, void* cuda_stream) {
  clear_error();
  if (polls < 1 || polls > 65536) return fail(OEC_ERR_INVALID_ARG, "polls must be in 1..65536");
  const cudaError_t e = wait_selftest_launch((unsigned)polls, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "wait self-test launch");
  return OEC_OK;
}

int oec_batch_wait_selftest(int polls, void* cuda_stream) {
  clear_error();
  if (polls < 1 || polls > 65536) return fail(OEC_ERR_INVALID_ARG, "polls must be in 1..65536");
  const cudaError_t e = pstaged_wait_selftest_launch((unsigned)polls, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch wait self-test");
  return OEC_OK;
}

int oec_pstaged_ticket_order(int32_t ni, int32_t nj, int32_t nk, int32_t unroll, int32_t k_chunk, int32_t grid,
                             int32_t* items, int64_t cap, int64_t* n_items) {
  clear_error();
  if (!n_items) return fail(OEC_ERR_INVALID_ARG, "n_items is null");
  if (ni < 1 || nj < 1 || nk < 1) return fail(OEC_ERR_INVALID_ARG, "domain sizes must be at least 1");
  if (unroll != 1 && unroll != 2) return fail(OEC_ERR_INVALID_ARG, "unroll must be 1 or 2");
  if (grid < 1) return fail(OEC_ERR_INVALID_ARG, "grid must be at least 1");
  oec_schedule s{};
  s.unroll = unroll;
  s.k_chunk = k_chunk;
  const Dom d{ni, nj, nk, ni, (int64_t)ni * nj};
  const int64_t n = hdiff_vadvc_pstaged_order(s, d, grid, items, cap);
  if (n < 0) return fail(OEC_ERR_INVALID_ARG, "the launch would take more tickets than an int holds");
  *n_items = n;
  return OEC_OK;
}

int oec_device_status(void* cuda_stream) {
  clear_error();
  unsigned n = 0;
  const int e = device_wait_timeouts((cudaStream_t)cuda_stream, &n);
  if (e) return cuda_fail((cudaError_t)e, "oec_device_status");
  if (n) return fail(OEC_ERR_TIMEOUT, "%u bounded device waits gave up", n);
  return OEC_OK;
}

int oec_program_set_timing(oec_program_t p, int enable) {
  clear_error();
  if (!p) return fail(OEC_ERR_INVALID_ARG, "null program");
  p->timing = enable != 0;
  return OEC_OK;
}

int oec_program_launch_count(oec_program_t p) {
  clear_error();
  if (!p) return fail(OEC_ERR_INVALID_ARG, "null program");
  return p->last_launches;
}

int oec_program_kernel_times(oec_program_t p, float* ms, int cap, int* n_applies, int* n_kernels) {
  clear_error();
  if (!p || !n_applies || !n_kernels) return fail(OEC_ERR_INVALID_ARG, "null argument");
  const int na = (int)p->ev_first.size();
  const int nk = na ? p->ev_count[0] - 1 : 0;
  for (int a = 1; a < na; ++a)
    if (p->ev_count[a] - 1 != nk) return fail(OEC_ERR_INVALID_ARG, "recorded applies launched different kernel counts");
  *n_applies = na;
  *n_kernels = nk;
  if ((int64_t)na * nk > cap || (na && !ms)) return fail(OEC_ERR_INVALID_ARG, "need room for %d times", na * nk);
  for (int a = 0; a < na; ++a)
    for (int x = 0; x < nk; ++x) {
      cudaEvent_t e0 = p->ev_pool[p->ev_first[a] + x], e1 = p->ev_pool[p->ev_first[a] + x + 1];
      cudaError_t err = cudaEventSynchronize(e1);
      if (err == cudaSuccess) err = cudaEventElapsedTime(&ms[a * nk + x], e0, e1);
      if (err != cudaSuccess) return cuda_fail(err, "kernel timing events");
    }
  p->ev_first.clear();
  p->ev_count.clear();
  p->ev_used = 0;
  return OEC_OK;
}

}  // extern "C"

// ---- captured applies ----------------------------------------------------

struct oec_graph {
  oec_program* prog = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int kernels = 0;
};

extern "C" {

int oec_program_capture(oec_program_t p, const oec_field_desc* in, int n_in, const oec_field_desc* out, int n_out,
                        const int64_t lb[3], const int64_t ub[3], const int64_t halo[3], const double* params,
                        int n_params, oec_graph_t* graph) {
  clear_error();
  if (!p || !graph) return fail(OEC_ERR_INVALID_ARG, "null program or graph handle");
  *graph = nullptr;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamCreate");
  const bool timing = p->timing;
  p->timing = false;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  int rc = OEC_OK;
  cudaGraph_t g = nullptr;
  if (e == cudaSuccess) {
    rc = oec_program_apply(p, in, n_in, out, n_out, lb, ub, halo, params, n_params, cs);
    const std::string msg = rc ? oec_last_error() : "";
    e = cudaStreamEndCapture(cs, &g);
    if (rc) fail(rc, "%s", msg.c_str());   // the apply's error, not the capture's
  }
  p->timing = timing;
  cudaStreamDestroy(cs);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(e, "stream capture of the apply");
  }
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "cudaGraphInstantiate");
  }
  oec_graph* h = new (std::nothrow) oec_graph();
  if (!h) {
    cudaGraphExecDestroy(x);
    cudaGraphDestroy(g);
    return fail(OEC_ERR_INVALID_ARG, "out of host memory");
  }
  h->prog = p;
  h->graph = g;
  h->exec = x;
  h->kernels = p->last_launches;
  ++p->graphs;
  *graph = h;
  return OEC_OK;
}

int oec_graph_launch(oec_graph_t graph, void* cuda_stream) {
  clear_error();
  if (!graph) return fail(OEC_ERR_INVALID_ARG, "null graph");
  const cudaError_t e = cudaGraphLaunch(graph->exec, (cudaStream_t)cuda_stream);
  return e == cudaSuccess ? OEC_OK : cuda_fail(e, "cudaGraphLaunch");
}

int oec_graph_kernel_count(oec_graph_t graph) { return graph ? graph->kernels : 0; }

void oec_graph_destroy(oec_graph_t graph) {
  if (!graph) return;
  cudaGraphExecDestroy(graph->exec);
  cudaGraphDestroy(graph->graph);
  if (graph->prog) --graph->prog->graphs;
  delete graph;
}

}  // extern "C"
