// tune.cpp - exhaustive autotuning: the candidate schedules of a program and
// their measured times. The paper picks unroll factors empirically and always
// fuses everything (§VII-C); here every fusion x staging x tile x unroll
// (x arithmetic) combination the kernels support is timed, which also
// produces the training data of the learned cost model.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <vector>

#include "../../include/oec.h"
#include "api_internal.h"

namespace oec {
namespace {

oec_schedule mk(int fusion, int staging, int ti, int tj, int unroll, int kc, int arith) {
  oec_schedule s{};
  s.fusion = fusion;
  s.staging = staging;
  s.tile_i = ti;
  s.tile_j = tj;
  s.unroll = unroll;
  s.k_chunk = kc;
  s.arith = arith;
  return s;
}

std::vector<oec_schedule> candidates(const oec_program* p) {
  std::vector<oec_schedule> c;
  const std::vector<int> ariths = p->dtype == OEC_F64 ? std::vector<int>{0, 1} : std::vector<int>{0};
  switch (p->kind) {
    case OEC_KIND_HDIFF:
      if (p->dtype == OEC_F64) {
        for (auto t : {std::pair<int, int>{32, 4}, {32, 8}, {64, 2}, {64, 4}, {64, 8}, {128, 2}, {128, 4}})
          for (int kc : {1, 2, 4, 8}) c.push_back(mk(OEC_FUSE_INLINE, OEC_STAGE_SMEM, t.first, t.second, 1, kc, 2));
        // fixed point, several rows per thread
        for (auto t : {std::array<int, 3>{32, 8, 2}, {32, 16, 1}, {32, 16, 2}, {32, 16, 4}, {64, 8, 2}})
          for (int kc : {2, 4, 8}) c.push_back(mk(OEC_FUSE_INLINE, OEC_STAGE_SMEM, t[0], t[1], t[2], kc, 2));
      }
      for (int a : ariths) {
        c.push_back(mk(OEC_FUSE_NONE, 0, 32, 8, 1, 0, a));
        for (auto t : {std::pair<int, int>{32, 4}, {32, 8}, {64, 2}, {64, 4}, {64, 8}, {128, 2}, {128, 4}})
          for (int kc : {1, 2, 4, 8}) c.push_back(mk(OEC_FUSE_INLINE, OEC_STAGE_SMEM, t.first, t.second, 1, kc, a));
        for (int ti : {32, 64, 128})
          for (int tj : {4, 8})
            for (int u : {1, 2, 4})
              for (int kc : {1, 4}) c.push_back(mk(OEC_FUSE_INLINE, OEC_STAGE_REGS, ti, tj, u, kc, a));
        for (auto t : {std::pair<int, int>{32, 4}, {32, 8}, {64, 4}, {64, 8}, {128, 2}, {128, 4}})
          for (int kc : {8, 16, 40}) c.push_back(mk(OEC_FUSE_INLINE, OEC_STAGE_STREAM, t.first, t.second, 1, kc, a));
        for (int u : {1, 2, 4})
          for (int kc : {4, 8, 16}) c.push_back(mk(OEC_FUSE_INLINE, OEC_STAGE_WARP, 32, 4 * u, u, kc, a));
        for (int u : {1, 2, 4}) c.push_back(mk(OEC_FUSE_INLINE, OEC_STAGE_TMA, 32, 4 * u, u, 0, a));
      }
      break;
    case OEC_KIND_HDIFF_VADVC:
      // staged: the tile is the hdiff producer's (FP64: the SMEM tile kernel,
      // staging unused; FP32: the REGS kernel, and the SMEM one at 64 x 4)
      if (p->dtype == OEC_F64) {
        // the fixed-point producer also with 2 and 3 levels per CTA: at
        // 128x128x80 its CTAs then fill the SMs in whole waves (32x16 tiles,
        // 2 rows per thread, 2 levels: 62.7 against 65.2 us per step at 4)
        for (int a : {2, 1, 0})
          for (auto t : {std::pair<int, int>{32, 4}, {32, 8}, {64, 4}, {64, 8}, {128, 4}})
            for (int kc : {2, 3, 4, 8})
              if (a == 2 || kc >= 4) c.push_back(mk(OEC_FUSE_NONE, 0, t.first, t.second, 1, kc, a));
        // the fixed-point producer with several rows per thread
        for (auto t : {std::array<int, 3>{32, 8, 2}, {32, 16, 1}, {32, 16, 2}, {32, 16, 4}, {64, 8, 2}})
          for (int kc : {2, 3, 4, 8}) c.push_back(mk(OEC_FUSE_NONE, 0, t[0], t[1], t[2], kc, 2));

      } else {
        for (int a : {1, 0}) {
          for (auto t : {std::pair<int, int>{32, 4}, {32, 8}, {64, 4}, {128, 2}})
            for (int u : {1, 2})
              for (int kc : {8, 20}) c.push_back(mk(OEC_FUSE_NONE, OEC_STAGE_REGS, t.first, t.second, u, kc, a));
          for (int u : {1, 2, 4})   // vector rows (aligned fields; else the REGS kernel)
            for (int kc : {8, 20}) c.push_back(mk(OEC_FUSE_NONE, OEC_STAGE_WARP, 32, 4 * u, u, kc, a));
          c.push_back(mk(OEC_FUSE_NONE, OEC_STAGE_SMEM, 64, 4, 1, 4, a));
        }
      }
      for (int a : {0, 1})
        for (auto t : {std::pair<int, int>{16, 4}, {32, 2}, {8, 8}, {32, 4}, {8, 4}, {16, 2}})
          c.push_back(mk(OEC_FUSE_INLINE, OEC_STAGE_SMEM, t.first, t.second, 1, 0, a));
      break;
    case OEC_KIND_FASTWAVES:
      for (int a : ariths) {
        c.push_back(mk(OEC_FUSE_NONE, 0, 32, 8, 1, 0, a));
        for (auto t : {std::pair<int, int>{32, 4}, {32, 8}, {64, 2}, {64, 4}, {128, 2}})
          for (int kc : {4, 16, 0}) c.push_back(mk(OEC_FUSE_INLINE, OEC_STAGE_SMEM, t.first, t.second, 1, kc, a));
        for (int ti : {32, 64, 128})
          for (int tj : {2, 4, 8})
            for (int u : {1, 2, 4})
              if (ti * tj <= 1024) c.push_back(mk(OEC_FUSE_INLINE, OEC_STAGE_REGS, ti, tj, u, 0, a));
        for (auto t : {std::pair<int, int>{32, 4}, {32, 8}, {64, 4}, {128, 2}})
          for (int u : {1, 2})   // 2: u/v windows through shared memory
            for (int kc : {8, 20, 40}) c.push_back(mk(OEC_FUSE_INLINE, OEC_STAGE_STREAM, t.first, t.second, u, kc, a));
        for (auto t : {std::pair<int, int>{32, 4}, {32, 8}, {64, 4}})   // aligned storage only
          for (int kc : {8, 20, 40}) c.push_back(mk(OEC_FUSE_INLINE, OEC_STAGE_TMA, t.first, t.second, 1, kc, a));
      }
      break;
    default:
      // generated kernels in the dtype's own arithmetic: double-float code
      // (arith 1) keeps ~48 bits, which a program that differences large,
      // nearly equal values can need, so it is the caller's choice (set the
      // schedule, or pass such candidates) and never an automatic pick
      for (int f : {OEC_FUSE_INLINE, OEC_FUSE_NONE, OEC_FUSE_PARTIAL})
        for (int u : {1, 2, 4})
          for (auto t : {std::pair<int, int>{32, 2}, {32, 4}, {32, 8}, {64, 1}, {64, 2}, {64, 4}, {128, 1},
                         {128, 2}, {128, 4}, {256, 1}, {256, 2}, {16, 8}})
            c.push_back(mk(f, OEC_STAGE_REGS, t.first, t.second, u, 0, 0));
      break;
  }
  return c;
}

}  // namespace
}  // namespace oec

using namespace oec;

extern "C" {

int oec_program_candidates(oec_program_t p, oec_schedule* out, int cap) {
  clear_error();
  if (!p) return fail(OEC_ERR_INVALID_ARG, "null program");
  std::vector<oec_schedule> c = candidates(p);
  if (out)
    for (int x = 0; x < (int)c.size() && x < cap; ++x) out[x] = c[x];
  return (int)c.size();
}

int oec_program_autotune(oec_program_t p, const oec_field_desc* in, int n_in, const oec_field_desc* out, int n_out,
                         const int64_t lb[3], const int64_t ub[3], const int64_t halo[3], const double* params,
                         int n_params, const oec_schedule* cand, int n_cand, int reps, void* cuda_stream,
                         double* times_ms, int* best) {
  clear_error();
  if (!p || !times_ms || reps < 1) return fail(OEC_ERR_INVALID_ARG, "null argument or reps < 1");
  std::vector<oec_schedule> own;
  if (!cand) {
    own = candidates(p);
    cand = own.data();
    n_cand = (int)own.size();
  }
  if (n_cand < 1) return fail(OEC_ERR_INVALID_ARG, "no candidates");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const oec_schedule saved = p->sched;
  std::vector<cudaEvent_t> ev(2 * reps);
  for (auto& e : ev)
    if (cudaEventCreate(&e) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaEventCreate");
  int best_i = -1;
  double best_t = 0;
  int rc_all = OEC_OK;
  std::vector<float> t(reps);
  for (int c = 0; c < n_cand; ++c) {
    times_ms[c] = -1.0;
    std::string why;
    if (!schedule_ok(p->kind, cand[c], why)) continue;
    p->sched = cand[c];
    int rc = oec_program_apply(p, in, n_in, out, n_out, lb, ub, halo, params, n_params, cuda_stream);   // warm-up
    if (rc == OEC_ERR_COMPILE || rc == OEC_ERR_UNSUPPORTED) continue;
    if (rc == OEC_ERR_CUDA && cudaStreamSynchronize(st) == cudaSuccess) {
      cudaGetLastError();   // a launch the hardware refuses (e.g. registers x threads): not a fault, skip it
      continue;
    }
    if (rc) { rc_all = rc; break; }
    for (int r = 0; r < reps && !rc; ++r) {
      cudaEventRecord(ev[2 * r], st);
      rc = oec_program_apply(p, in, n_in, out, n_out, lb, ub, halo, params, n_params, cuda_stream);
      cudaEventRecord(ev[2 * r + 1], st);
    }
    if (rc) { rc_all = rc; break; }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { rc_all = cuda_fail(e, "autotune"); break; }
    for (int r = 0; r < reps; ++r) cudaEventElapsedTime(&t[r], ev[2 * r], ev[2 * r + 1]);
    std::vector<float> sorted(t);
    std::sort(sorted.begin(), sorted.end());
    times_ms[c] = sorted[reps / 2];
    if (best_i < 0 || times_ms[c] < best_t) {
      best_i = c;
      best_t = times_ms[c];
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (rc_all) {
    p->sched = saved;
    return rc_all;
  }
  if (best_i < 0) {
    p->sched = saved;
    return fail(OEC_ERR_UNSUPPORTED, "no candidate schedule ran");
  }
  p->sched = cand[best_i];
  if (best) *best = best_i;
  return OEC_OK;
}

}  // extern "C"
