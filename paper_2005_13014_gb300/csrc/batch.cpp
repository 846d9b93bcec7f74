// batch.cpp - ensembles of domains in one persistent launch, captured into a
// CUDA graph (include/oec.h, oec_batch_*).
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/oec.h"
#include "api_internal.h"
#include "kernels.h"

struct oec_batch {
  int dtype = OEC_F64;
  oec_schedule sched{};
  oec::HVBatchLaunch launch{};
  oec::HVMember* d_members = nullptr;
  int* d_counter = nullptr;
  void* d_scratch = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int dev = 0;
};

namespace {

void release(oec_batch* b) {
  if (!b) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(b->dev);
  if (b->exec || b->d_members) cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_members) cudaFree(b->d_members);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->d_scratch) cudaFree(b->d_scratch);
  cudaSetDevice(cur);
  delete b;
}

char* base_at(const oec_field_desc& f, const int64_t lb[3], size_t es) {
  int64_t off = 0;
  for (int d = 0; d < 3; ++d) off += (f.origin[d] + lb[d]) * f.stride[d];
  return (char*)f.data + off * (int64_t)es;
}

}  // namespace

using namespace oec;

extern "C" {

int oec_batch_create(oec_program_t p, const oec_batch_member* members, int n, const double* params, int n_params,
                     oec_batch_t* out) {
  clear_error();
  if (!p || !members || n < 1 || !out) return fail(OEC_ERR_INVALID_ARG, "null argument or no members");
  *out = nullptr;
  if (p->kind != OEC_KIND_HDIFF_VADVC) return fail(OEC_ERR_UNSUPPORTED, "batches run hdiff+vadvc programs");
  if (p->sched.fusion != OEC_FUSE_INLINE) return fail(OEC_ERR_UNSUPPORTED, "batches need a fused schedule");
  if (n_params != (int)p->ir.params.size() || (n_params && !params))
    return fail(OEC_ERR_INVALID_ARG, "program has %zu params, got %d", p->ir.params.size(), n_params);
  const size_t es = elem_size(p->dtype);
  const oec_schedule s = p->sched;
  std::vector<HVMember> tab;
  tab.reserve(n);
  int nk_max = 1;
  for (int m = 0; m < n; ++m) {
    const oec_batch_member& mb = members[m];
    if (!mb.in || !mb.out) return fail(OEC_ERR_INVALID_ARG, "member %d: null field array", m);
    bool empty = false;
    for (int d = 0; d < 3; ++d) {
      if (mb.ub[d] < mb.lb[d] || mb.halo[d] < 0) return fail(OEC_ERR_INVALID_ARG, "member %d: bad domain or halo", m);
      if (mb.ub[d] - mb.lb[d] > (1 << 30)) return fail(OEC_ERR_UNSUPPORTED, "member %d: extent above 2^30", m);
      empty |= mb.ub[d] == mb.lb[d];
    }
    if (empty) continue;
    std::vector<Box> ranges;
    int rc = validate_fields(p, mb.in, 4, mb.out, 2, mb.lb, mb.ub, mb.halo, ranges);
    if (rc) return fail(rc, "member %d: %s", m, oec_last_error());
    const int64_t sj = mb.out[0].stride[1], sk = mb.out[0].stride[2];
    for (int x = 0; x < 6; ++x) {
      const oec_field_desc& f = x < 4 ? mb.in[x] : mb.out[x - 4];
      if (f.ndim != 3 || f.stride[1] != sj || f.stride[2] != sk)
        return fail(OEC_ERR_UNSUPPORTED, "member %d: fields need equal j/k strides", m);
    }
    HVMember h{};
    h.u = base_at(mb.in[0], mb.lb, es);
    h.v = base_at(mb.in[1], mb.lb, es);
    h.w = base_at(mb.in[2], mb.lb, es);
    h.coeff = base_at(mb.in[3], mb.lb, es);
    h.uo = base_at(mb.out[0], mb.lb, es);
    h.vo = base_at(mb.out[1], mb.lb, es);
    h.ni = int(mb.ub[0] - mb.lb[0]);
    h.nj = int(mb.ub[1] - mb.lb[1]);
    h.nk = int(mb.ub[2] - mb.lb[2]);
    h.tiles_i = (h.ni + s.tile_i - 1) / s.tile_i;
    h.sj = sj;
    h.sk = sk;
    nk_max = std::max(nk_max, h.nk);
    tab.push_back(h);
  }
  if (tab.empty()) return fail(OEC_ERR_INVALID_ARG, "every member has an empty domain");
  // longest-processing-time order: tallest columns first, then larger domains
  std::stable_sort(tab.begin(), tab.end(), [](const HVMember& a, const HVMember& b) {
    if (a.nk != b.nk) return a.nk > b.nk;
    return (int64_t)a.ni * a.nj > (int64_t)b.ni * b.nj;
  });
  int64_t items = 0;
  for (auto& h : tab) {
    h.tile_begin = (int)items;
    items += (int64_t)h.tiles_i * ((h.nj + s.tile_j - 1) / s.tile_j);
  }
  if (items > (1 << 30)) return fail(OEC_ERR_UNSUPPORTED, "more than 2^30 tiles");

  oec_batch* b = new (std::nothrow) oec_batch();
  if (!b) return fail(OEC_ERR_INVALID_ARG, "out of host memory");
  b->dtype = p->dtype;
  b->sched = s;
  cudaGetDevice(&b->dev);
  int sms = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev);
  if (e != cudaSuccess) { release(b); return cuda_fail(e, "cudaDeviceGetAttribute"); }
  const int per_sm = hdiff_vadvc_batch_blocks_per_sm(s, p->dtype);
  const int grid = (int)std::min<int64_t>(items, (int64_t)sms * per_sm);
  const int64_t slot = (int64_t)hdiff_vadvc_batch_slot_elems(s, nk_max);
  e = cudaMalloc(&b->d_members, sizeof(HVMember) * tab.size());
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_scratch, (size_t)grid * slot * 8);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_members, tab.data(), sizeof(HVMember) * tab.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { release(b); return cuda_fail(e, "batch allocation"); }
  b->launch.members = b->d_members;
  b->launch.n_members = (int)tab.size();
  b->launch.total_items = (int)items;
  b->launch.counter = b->d_counter;
  b->launch.dtr = params[0];
  b->launch.scratch = b->d_scratch;
  b->launch.slot_elems = slot;
  b->launch.grid = grid;
  // capture: counter reset + persistent launch
  cudaStream_t cap = nullptr;
  e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = cudaMemsetAsync(b->d_counter, 0, sizeof(int), cap);
    cudaError_t e2 = e1 == cudaSuccess ? hdiff_vadvc_batch_launch(s, p->dtype, b->launch, cap) : e1;
    e = cudaStreamEndCapture(cap, &b->graph);
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (cap) cudaStreamDestroy(cap);
  if (e != cudaSuccess) { release(b); return cuda_fail(e, "graph capture"); }
  *out = b;
  return OEC_OK;
}

int oec_batch_apply(oec_batch_t b, void* stream) {
  clear_error();
  if (!b) return fail(OEC_ERR_INVALID_ARG, "null batch");
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  return e == cudaSuccess ? OEC_OK : cuda_fail(e, "cudaGraphLaunch");
}

int oec_batch_apply_direct(oec_batch_t b, void* stream) {
  clear_error();
  if (!b) return fail(OEC_ERR_INVALID_ARG, "null batch");
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), (cudaStream_t)stream);
  if (e == cudaSuccess) e = hdiff_vadvc_batch_launch(b->sched, b->dtype, b->launch, (cudaStream_t)stream);
  return e == cudaSuccess ? OEC_OK : cuda_fail(e, "batch launch");
}

int oec_batch_info(oec_batch_t b, int* n_items, int* n_ctas) {
  clear_error();
  if (!b || !n_items || !n_ctas) return fail(OEC_ERR_INVALID_ARG, "null argument");
  *n_items = b->launch.total_items;
  *n_ctas = b->launch.grid;
  return OEC_OK;
}

void oec_batch_destroy(oec_batch_t b) { release(b); }

}  // extern "C"
