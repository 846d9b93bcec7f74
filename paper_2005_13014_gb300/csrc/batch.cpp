// batch.cpp - ensembles of domains, captured into one CUDA graph
// (include/oec.h, oec_batch_*). Fused schedules: one persistent launch over
// the (member, tile) work items of every member. Staged schedules with FP32
// fields on the warp-row producer (rows 16-byte aligned): one persistent
// launch over producer and column-sweep items of every member, the sweeps
// waiting (bounded) on per-row-block counters. Other staged schedules: every
// member's producer + column-sweep chain is an independent branch of the
// graph (members spread over up to 16 forked streams), so the members' column
// sweeps - latency-bound, with few warps each - run concurrently and fill the
// GPU together.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <deque>
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
  // persistent staged form: one launch over every member's items
  bool persistent = false;
  oec::PSLaunch ps{};
  oec::PSMember* d_psm = nullptr;
  oec::PSItem* d_items = nullptr;
  int* d_done = nullptr;
  int n_done = 0;
};

namespace {

void release(oec_batch* b) {
  if (!b) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(b->dev);
  if (b->exec || b->d_members || b->d_items) cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->d_members) cudaFree(b->d_members);
  if (b->d_counter) cudaFree(b->d_counter);
  if (b->d_scratch) cudaFree(b->d_scratch);
  if (b->d_psm) cudaFree(b->d_psm);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_done) cudaFree(b->d_done);
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

// counters reset, then the persistent launch
cudaError_t record_pstaged(const oec_batch* b, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_done, 0, sizeof(int) * std::max(1, b->n_done), st);
  if (e == cudaSuccess) e = oec::hdiff_vadvc_pstaged_launch(b->sched, b->ps, st);
  return e;
}

// Members the persistent form can run: rows 16-byte aligned at the domain
// corner for the warp-row producer (pointers, j/k strides, and ni for its
// hdiff(u), hdiff(v) buffers).
bool pstaged_aligned(const oec_batch* b) {
  for (const StagedMember& m : b->staged_members) {
    const uintptr_t a = (uintptr_t)m.u | (uintptr_t)m.v | (uintptr_t)m.coeff;
    if (a % 16 != 0 || m.d.sj % 4 != 0 || m.d.sk % 4 != 0 || m.d.ni % 4 != 0) return false;
  }
  return true;
}

// The persistent staged form: the member table, the work items in ticket
// order, and a graph of (reset counters, one launch). Producer items go row
// block by row block, member after member; a sweep item (64 columns) follows
// once every row block it needs has its producer items at least `lag` tickets
// back (two per resident CTA), so that its rows are usually done and still in
// L2 when it starts.
// The items of a persistent staged batch in ticket order. Per member, row
// block by row block (4 x unroll rows): the block's producer items (level
// chunk and field, then tile of 128 columns along i), and every 64-column
// group whose columns all lie in the blocks placed so far becomes ready with
// the ticket of the block's last producer item; a ready group is placed once
// `lag` more items follow that ticket, the rest at the end. So every group
// comes after all producer items it waits for, and producer items wait for
// nothing.
std::vector<oec::PSItem> batch_ticket_order(const std::vector<oec::Dom>& doms, int unroll, int k_chunk,
                                            int64_t lag) {
  using oec::PSItem;
  constexpr int W = 128, COLS = 64;   // producer columns per CTA (32 lanes x 4 floats), sweep columns
  const int rows = 4 * unroll;
  std::vector<PSItem> items;
  struct Pending { int m, g, lo, hi; int64_t dep; };
  std::deque<Pending> ready;
  auto flush = [&](bool all) {
    while (!ready.empty() && (all || ready.front().dep + lag <= (int64_t)items.size())) {
      const Pending& q = ready.front();
      items.push_back(PSItem{~q.m, q.g, q.lo, q.hi});
      ready.pop_front();
    }
  };
  for (int mi = 0; mi < (int)doms.size(); ++mi) {
    const oec::Dom& d = doms[mi];
    const int kchunk = (k_chunk <= 0 || k_chunk > d.nk) ? d.nk : k_chunk;
    const int nkz = (d.nk + kchunk - 1) / kchunk;
    const int64_t ncol = (int64_t)d.ni * d.nj;
    const int tx = (d.ni + W - 1) / W, ty = (d.nj + rows - 1) / rows;
    int64_t g = 0;
    const int64_t groups = (ncol + COLS - 1) / COLS;
    for (int by = 0; by < ty; ++by) {
      for (int bz = 0; bz < 2 * nkz; ++bz)
        for (int bx = 0; bx < tx; ++bx) {
          items.push_back(PSItem{mi, bx, by, bz});
          flush(false);
        }
      // the sweep groups whose rows all lie in row blocks 0..by
      const int64_t dep = (int64_t)items.size() - 1;
      for (; g < groups; ++g) {
        const int64_t c0 = g * COLS, c1 = std::min(ncol, c0 + COLS) - 1;
        const int lo = int(c0 / d.ni) / rows, hi = int(c1 / d.ni) / rows;
        if (hi > by) break;
        ready.push_back(Pending{mi, (int)g, lo, hi, dep});
      }
    }
  }
  flush(true);
  return items;
}

int build_pstaged(oec_batch* b) {
  using namespace oec;
  const oec_schedule& s = b->sched;
  const int U = s.unroll, rows = 4 * U;
  constexpr int W = 128;   // producer columns per CTA (32 lanes x 4 floats)
  std::vector<PSMember> tab;
  bool o32 = true, discard = false;
  int row_base = 0;
  for (const StagedMember& sm : b->staged_members) {
    PSMember m{};
    const Dom& d = sm.d;
    size_t ud = 0, vd = 0;
    hdiff_vadvc_scratch_parts(s, b->dtype, d, &ud, &vd);
    char* scr = (char*)b->d_scratch + sm.scratch_off;
    m.u = sm.u; m.v = sm.v; m.w = sm.w; m.coeff = sm.coeff; m.uo = sm.uo; m.vo = sm.vo;
    m.ud = scr + ud; m.vd = scr + vd; m.scr = scr;
    m.sj = d.sj; m.sk = d.sk;
    const int64_t ncol = (int64_t)d.ni * d.nj;
    m.ncolp = hdiff_vadvc_pair_pitch(ncol);
    m.ni = d.ni; m.nj = d.nj; m.nk = d.nk;
    m.kchunk = (s.k_chunk <= 0 || s.k_chunk > d.nk) ? d.nk : s.k_chunk;
    m.nkz = (d.nk + m.kchunk - 1) / m.kchunk;
    m.row_base = row_base;
    row_base += (d.nj + rows - 1) / rows;
    m.need = ((d.ni + W - 1) / W) * 2 * m.nkz;
    o32 = o32 && use_int32(s, d) && 4 * m.ncolp * d.nk < INT32_MAX;
    discard = discard || size_t(24) * m.ncolp * d.nk > hdiff_vadvc_discard_above_bytes();
    tab.push_back(m);
  }
  PSLaunch& L = b->ps;
  L.unroll = U;
  L.o32 = o32;
  L.discard = discard;
  L.dtr = b->dtr;
  L.polls = 1u << 22;
  int sms = 0, per_sm = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev);
  if (e == cudaSuccess) e = hdiff_vadvc_pstaged_blocks_per_sm(s, L, &per_sm);
  if (e != cudaSuccess) return cuda_fail(e, "persistent batch occupancy");
  if (per_sm < 1) return fail(OEC_ERR_UNSUPPORTED, "persistent batch kernel does not fit on an SM");
  const int64_t lag = 2 * (int64_t)sms * per_sm;
  std::vector<Dom> doms;
  for (const StagedMember& sm : b->staged_members) doms.push_back(sm.d);
  const std::vector<PSItem> items = batch_ticket_order(doms, U, s.k_chunk, lag);
  if (items.size() > (size_t)INT32_MAX) return fail(OEC_ERR_UNSUPPORTED, "more than 2^31 batch items");
  L.n_items = (int)items.size();
  L.grid = (int)std::min<int64_t>(L.n_items, (int64_t)sms * per_sm);
  b->n_done = row_base;
  e = cudaMalloc(&b->d_psm, sizeof(PSMember) * tab.size());
  if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(PSItem) * items.size());
  if (e == cudaSuccess) e = cudaMalloc(&b->d_done, sizeof(int) * std::max(1, b->n_done));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_psm, tab.data(), sizeof(PSMember) * tab.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_items, items.data(), sizeof(PSItem) * items.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "persistent batch tables");
  L.members = b->d_psm;
  L.items = b->d_items;
  L.ticket = b->d_counter;
  L.done = b->d_done;
  L.timeouts = wait_timeout_counter();
  if (!L.timeouts) return fail(OEC_ERR_CUDA, "device wait counter not found");
  b->persistent = true;
  cudaStream_t cap = nullptr;
  e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t r = record_pstaged(b, cap);
    e = cudaStreamEndCapture(cap, &b->graph);
    if (e == cudaSuccess) e = r;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (cap) cudaStreamDestroy(cap);
  if (e != cudaSuccess) return cuda_fail(e, "persistent batch capture");
  return OEC_OK;
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
  if (hdiff_vadvc_pstaged_ok(b->sched, b->dtype) && pstaged_aligned(b)) {   // one persistent launch
    const int rc = build_pstaged(b);
    if (rc) { release(b); return rc; }
    *out = b;
    return OEC_OK;
  }
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
  if (b->persistent) {   // counters reset and the launch, on the caller's stream
    cudaError_t e = record_pstaged(b, (cudaStream_t)stream);
    return e == cudaSuccess ? OEC_OK : cuda_fail(e, "batch launch");
  }
  if (b->staged) {   // the same launches, one after another on the caller's stream
    cudaError_t e = record_staged(b, (char*)b->d_scratch, std::vector<cudaStream_t>{(cudaStream_t)stream});
    return e == cudaSuccess ? OEC_OK : cuda_fail(e, "batch launch");
  }
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), (cudaStream_t)stream);
  if (e == cudaSuccess) e = hdiff_vadvc_batch_launch(b->sched, b->dtype, b->launch, (cudaStream_t)stream);
  return e == cudaSuccess ? OEC_OK : cuda_fail(e, "batch launch");
}

int oec_batch_ticket_order(int32_t n_members, const int32_t* sizes, int32_t unroll, int32_t k_chunk, int64_t lag,
                           int32_t* items, int64_t cap, int64_t* n_items) {
  clear_error();
  if (!n_items || !sizes || n_members < 1) return fail(OEC_ERR_INVALID_ARG, "n_members, sizes or n_items invalid");
  if (unroll != 1 && unroll != 2) return fail(OEC_ERR_INVALID_ARG, "unroll must be 1 or 2");
  if (lag < 0) return fail(OEC_ERR_INVALID_ARG, "lag must be at least 0");
  std::vector<oec::Dom> doms;
  for (int m = 0; m < n_members; ++m) {
    const int32_t* z = sizes + 3 * (int64_t)m;
    if (z[0] < 1 || z[1] < 1 || z[2] < 1) return fail(OEC_ERR_INVALID_ARG, "member %d: sizes must be at least 1", m);
    doms.push_back(oec::Dom{z[0], z[1], z[2], z[0], (int64_t)z[0] * z[1]});
  }
  std::vector<oec::PSItem> order;
  try {
    order = batch_ticket_order(doms, unroll, k_chunk, lag);
  } catch (const std::bad_alloc&) {
    return fail(OEC_ERR_INVALID_ARG, "too many items");
  }
  *n_items = (int64_t)order.size();
  if (items && cap >= 4 * (int64_t)order.size())
    for (size_t t = 0; t < order.size(); ++t) {
      items[4 * t] = order[t].x;
      items[4 * t + 1] = order[t].y;
      items[4 * t + 2] = order[t].z;
      items[4 * t + 3] = order[t].w;
    }
  return OEC_OK;
}

int oec_batch_info(oec_batch_t b, int* n_items, int* n_ctas) {
  clear_error();
  if (!b || !n_items || !n_ctas) return fail(OEC_ERR_INVALID_ARG, "null argument");
  if (b->persistent) {
    *n_items = b->ps.n_items;
    *n_ctas = b->ps.grid;
    return OEC_OK;
  }
  *n_items = b->staged ? (int)b->staged_members.size() : b->launch.total_items;
  *n_ctas = b->staged ? b->n_streams : b->launch.grid;
  return OEC_OK;
}

void oec_batch_destroy(oec_batch_t b) { release(b); }

}  // extern "C"
