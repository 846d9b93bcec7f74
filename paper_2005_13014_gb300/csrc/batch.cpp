// batch.cpp - ensembles of domains, captured into one CUDA graph
// (include/oec.h, oec_batch_*). Fused schedules: one persistent launch over
// the (member, tile) work items of every member. Staged schedules: every
// member's producer + column-sweep chain is an independent branch of the
// graph (members spread over up to 16 forked streams), so the members' column
// sweeps - latency-bound, with few warps each - run concurrently and fill the
// GPU together.
#include <cuda_runtime.h>

#include <algorithm>
#include <new>
#include <numeric>
#include <vector>

#include "../../include/oec.h"
#include "api_internal.h"
#include "kernels.h"

struct StagedMember {
  oec::Dom d{};
  const void *u = nullptr, *v = nullptr, *w = nullptr, *coeff = nullptr;
  void *uo = nullptr, *vo = nullptr;
  size_t scratch_off = 0;
  int stream = 0;
};

struct oec_batch {
  int dtype = OEC_F64;
  oec_schedule sched{};
  bool staged = false;
  std::vector<StagedMember> staged_members;
  double dtr = 0.0;
  int n_streams = 0;
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


// Staged batch: per member its own scratch; the chains are captured on up to
// 16 streams forked from (and joined back into) the capture stream, members
// assigned largest first to the least-loaded stream.
cudaError_t record_staged(const oec_batch* b, char* scratch, const std::vector<cudaStream_t>& streams) {
  cudaError_t e = cudaSuccess;
  for (const StagedMember& m : b->staged_members) {
    cudaError_t r = oec::hdiff_vadvc_launch(b->sched, b->dtype, m.d, m.u, m.v, m.w, m.coeff, m.uo, m.vo, b->dtr,
                                            scratch + m.scratch_off, streams[m.stream % streams.size()], true);
    if (e == cudaSuccess) e = r;
  }
  return e;
}

int create_staged(oec_program* p, const std::vector<oec::HVMember>& tab, double dtr, oec_batch_t* out) {
  using namespace oec;
  oec_batch* b = new (std::nothrow) oec_batch();
  if (!b) return fail(OEC_ERR_INVALID_ARG, "out of host memory");
  b->dtype = p->dtype;
  b->sched = p->sched;
  b->staged = true;
  b->dtr = dtr;
  cudaGetDevice(&b->dev);
  b->n_streams = (int)std::min<size_t>(tab.size(), 16);
  std::vector<int64_t> load(b->n_streams, 0);
  size_t off = 0;
  for (const HVMember& h : tab) {   // tab is sorted tallest / largest first
    StagedMember m;
    m.d = Dom{h.ni, h.nj, h.nk, h.sj, h.sk};
    m.u = h.u;
    m.v = h.v;
    m.w = h.w;
    m.coeff = h.coeff;
    m.uo = h.uo;
    m.vo = h.vo;
    m.scratch_off = off;
    off = align_up(off + hdiff_vadvc_scratch_bytes(b->sched, b->dtype, m.d), 256);
    m.stream = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[m.stream] += (int64_t)h.ni * h.nj * h.nk;
    b->staged_members.push_back(m);
  }
  cudaError_t e = cudaMalloc(&b->d_scratch, std::max<size_t>(off, 256));
  if (e != cudaSuccess) { release(b); return cuda_fail(e, "batch scratch"); }
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> streams(b->n_streams, nullptr);
  std::vector<cudaEvent_t> ev(b->n_streams + 1, nullptr);
  e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  for (auto& st : streams)
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  for (auto& x : ev)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t r = cudaEventRecord(ev[0], cap);
    for (auto& st : streams)
      if (r == cudaSuccess) r = cudaStreamWaitEvent(st, ev[0], 0);
    if (r == cudaSuccess) r = record_staged(b, (char*)b->d_scratch, streams);
    for (int x = 0; x < b->n_streams && r == cudaSuccess; ++x) {
      r = cudaEventRecord(ev[x + 1], streams[x]);
      if (r == cudaSuccess) r = cudaStreamWaitEvent(cap, ev[x + 1], 0);
    }
    e = cudaStreamEndCapture(cap, &b->graph);
    if (e == cudaSuccess) e = r;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  for (auto& x : ev)
    if (x) cudaEventDestroy(x);
  for (auto& st : streams)
    if (st) cudaStreamDestroy(st);
  if (cap) cudaStreamDestroy(cap);
  if (e != cudaSuccess) { release(b); return cuda_fail(e, "staged batch capture"); }
  *out = b;
  return OEC_OK;
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
  if (p->sched.fusion != OEC_FUSE_INLINE && p->sched.fusion != OEC_FUSE_NONE)
    return fail(OEC_ERR_UNSUPPORTED, "batches need a fused or a staged schedule");
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
  if (s.fusion == OEC_FUSE_NONE) return create_staged(p, tab, params[0], out);
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
  NvtxRange range("oec_batch_apply");
  if (!b) return fail(OEC_ERR_INVALID_ARG, "null batch");
  cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  return e == cudaSuccess ? OEC_OK : cuda_fail(e, "cudaGraphLaunch");
}

int oec_batch_apply_direct(oec_batch_t b, void* stream) {
  clear_error();
  NvtxRange range("oec_batch_apply_direct");
  if (!b) return fail(OEC_ERR_INVALID_ARG, "null batch");
  if (b->staged) {   // the same launches, one after another on the caller's stream
    cudaError_t e = record_staged(b, (char*)b->d_scratch, std::vector<cudaStream_t>{(cudaStream_t)stream});
    return e == cudaSuccess ? OEC_OK : cuda_fail(e, "batch launch");
  }
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), (cudaStream_t)stream);
  if (e == cudaSuccess) e = hdiff_vadvc_batch_launch(b->sched, b->dtype, b->launch, (cudaStream_t)stream);
  return e == cudaSuccess ? OEC_OK : cuda_fail(e, "batch launch");
}

int oec_batch_info(oec_batch_t b, int* n_items, int* n_ctas) {
  clear_error();
  if (!b || !n_items || !n_ctas) return fail(OEC_ERR_INVALID_ARG, "null argument");
  *n_items = b->staged ? (int)b->staged_members.size() : b->launch.total_items;
  *n_ctas = b->staged ? b->n_streams : b->launch.grid;
  return OEC_OK;
}

void oec_batch_destroy(oec_batch_t b) { release(b); }

}  // extern "C"
