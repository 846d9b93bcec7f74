// kernels.h - host-side interface of the hand-written kernels. Every launcher
// takes pointers already offset to the domain's lower corner (logical lb), the
// domain extents, the fields' shared j/k strides (elements), a scratch buffer
// of at least *_scratch_bytes() bytes (may be null when that is 0) and the
// caller's stream, and returns the launch status.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/oec.h"
#include "k_vadvc.cuh"

namespace oec {

// Called after every kernel launch of an apply: counts the launches and, while
// the program's kernel timing is on, records an event after the kernel.
void launched(cudaStream_t st);
// Between these two calls launched() only counts the kernels; the end records
// one timing event on st (the kernels of a group run on several streams and
// overlap, so only the group as a whole has a duration).
void launch_group_begin();
void launch_group_end(cudaStream_t st);
// most j-slabs of the staged hdiff+vadvc pipeline (schedule field slabs)
constexpr int kMaxSlabs = 16;


struct Dom {
  int ni, nj, nk;        // domain extents
  int64_t sj, sk;        // element strides shared by all fields
};

// true when every element offset a kernel forms from the domain's base
// pointers (halo 2 around the domain) fits in a 32-bit int
inline bool offsets_fit_int32(const Dom& d) {
  const int64_t hi = (int64_t)(d.nk + 1) * d.sk + (int64_t)(d.nj + 2) * d.sj + d.ni + 2;
  const int64_t lo = -(2 * d.sj + 2);
  return hi < INT32_MAX && lo > INT32_MIN;
}

// the kernels with both offset widths take the 32-bit form unless the
// schedule asks for 64-bit offsets or the offsets do not fit
inline bool use_int32(const oec_schedule& s, const Dom& d) {
  return s.index_bits != OEC_INDEX_64 && offsets_fit_int32(d);
}

// ---- horizontal diffusion: in, coeff -> out --------------------------------
bool hdiff_schedule_ok(const oec_schedule& s, std::string& why);
size_t hdiff_scratch_bytes(const oec_schedule& s, int dtype, const Dom& d);
// vectorised warp rows (OEC_STAGE_WARP, k_hdiff_vec.cu); pointers and
// strides 16-byte aligned (checked by the caller)
cudaError_t hdiff_warp_launch(const oec_schedule& s, int dtype, const Dom& d, const void* in, const void* coeff,
                              void* out, cudaStream_t st);
// TMA-staged vectorised warp rows (OEC_STAGE_TMA): a field's storage (element
// 0, extents) and the storage coordinates of the domain's lower corner
struct TmaField {
  const void* base;
  int64_t size[3];
  int64_t corner[3];
};
// FP32 vector-row hdiff of two fields into the staged hdiff+vadvc compute
// buffers (domain layout osj, osk); every row 16-byte aligned (caller checks)
cudaError_t hdiff_warp_to_compute(const oec_schedule& s, const Dom& d, int64_t osj, int64_t osk, const float* in0,
                                  const float* in1, const float* coeff, float* out0, float* out1, cudaStream_t st);
cudaError_t hdiff_tma_launch(const oec_schedule& s, int dtype, const Dom& d, const TmaField& in,
                             const TmaField& coeff, void* out, cudaStream_t st);
// number of bounded device-side waits that gave up since the last call (the
// stream is synchronised first); clears the count
int device_wait_timeouts(cudaStream_t st, unsigned* count);
// launch a kernel whose mbarrier wait on a phase that never completes gives
// up after `polls` polls and counts a timeout (the give-up path, tested)
cudaError_t wait_selftest_launch(unsigned polls, cudaStream_t st);
cudaError_t hdiff_launch(const oec_schedule& s, int dtype, const Dom& d, const void* in, const void* coeff,
                         void* out, void* scratch, cudaStream_t st);

// ---- horizontal diffusion of u, v + vertical advection (Thomas) -------------
bool hdiff_vadvc_schedule_ok(const oec_schedule& s, std::string& why);
size_t hdiff_vadvc_scratch_bytes(const oec_schedule& s, int dtype, const Dom& d);
// batch_member: the apply runs concurrently with other members of a batch
// (they share DRAM bandwidth), so a large column sweep keeps its recurrence
// values in L2 and drops them once read (measured: a 32-member ensemble 10%
// faster; one large apply alone 3.6% slower, so single applies do not)
cudaError_t hdiff_vadvc_launch(const oec_schedule& s, int dtype, const Dom& d, const void* u, const void* v,
                               const void* w, const void* coeff, void* u_out, void* v_out, double dtr,
                               void* scratch, cudaStream_t st, bool batch_member = false);
// the partitioned column sweep (k_vadvc_seg.cu): nseg = 4 or 8 segments per
// column; ud, vd hdiff(u), hdiff(v) in the compute type over the domain
// layout; scr 4 recurrence values per point
cudaError_t hdiff_vadvc_segments_launch(int nseg, int dtype, int arith, const Dom& d, const void* u, const void* v,
                                        const void* w, const void* coeff, void* u_out, void* v_out,
                                        const void* ud, const void* vd, double dtr, void* scr, bool o32,
                                        cudaStream_t st);
// persistent staged batch (FP32 fields, vector-row producer; k_vadvc.cu):
// whether a schedule has it, a member's hdiff(u) / hdiff(v) offsets in its
// scratch, the column scratch row pitch, the scratch size above which the
// column sweep takes its L2 form, the CTAs per SM, and the launch
bool hdiff_vadvc_pstaged_ok(const oec_schedule& s, int dtype);
void hdiff_vadvc_scratch_parts(const oec_schedule& s, int dtype, const Dom& d, size_t* ud, size_t* vd);
int64_t hdiff_vadvc_pair_pitch(int64_t ncol);
size_t hdiff_vadvc_discard_above_bytes();
cudaError_t hdiff_vadvc_pstaged_blocks_per_sm(const oec_schedule& s, const PSLaunch& L, int* per_sm);
// The ticket order of one FP32 domain's persistent staged launch for `grid`
// resident CTAs, computed on the host: per ticket (x, y, z, w) as the kernel
// decodes it (x >= 0: producer item y, row block z, level chunk and field w;
// x < 0: column group y needing row blocks z..w). Returns the ticket count
// (items written when cap >= 4 x count), -1 when the plan does not fit.
int64_t hdiff_vadvc_pstaged_order(const oec_schedule& s, const Dom& d, int grid, int32_t* items, int64_t cap);
cudaError_t hdiff_vadvc_pstaged_launch(const oec_schedule& s, const PSLaunch& L, cudaStream_t st);
// the persistent batch's give-up path: one sweep item whose counter is never
// released; waits for the kernel before returning
cudaError_t pstaged_wait_selftest_launch(unsigned polls, cudaStream_t st);
// device counter of bounded waits that gave up (k_hdiff_vec.cu)
unsigned* wait_timeout_counter();
// batched persistent form (ensembles of domains)
size_t hdiff_vadvc_batch_slot_elems(const oec_schedule& s, int nk_max);
int hdiff_vadvc_batch_blocks_per_sm(const oec_schedule& s, int dtype);
cudaError_t hdiff_vadvc_batch_launch(const oec_schedule& s, int dtype, const HVBatchLaunch& b, cudaStream_t st);
// hdiff of two fields (one launch) written in the compute type of (s.arith,
// dtype) over the domain layout (pitch ni, plane ni*nj): the producer of the
// staged hdiff+vadvc form. s.tile_i x s.tile_j and s.k_chunk pick its tile
// when they name an SMEM hdiff tile, else 64 x 4 with 4 levels per CTA.
cudaError_t hdiff_to_compute(const oec_schedule& s, int dtype, const Dom& d, const void* in0, const void* in1,
                             const void* coeff, void* out0, void* out1, cudaStream_t st);

// ---- fastwaves-like program -------------------------------------------------
struct FastwavesPtrs {
  const void* u_in; const void* v_in; const void* utens; const void* vtens; const void* pp;
  const void* rho; const void* wgtfac; const void* hhl; const void* fx;
  void* u_out; void* v_out;
};
bool fastwaves_schedule_ok(const oec_schedule& s, std::string& why);
size_t fastwaves_scratch_bytes(const oec_schedule& s, int dtype, const Dom& d);
// tf: the nine inputs' storage (FASTWAVES input order), for OEC_STAGE_TMA
cudaError_t fastwaves_launch(const oec_schedule& s, int dtype, const Dom& d, const FastwavesPtrs& f, double dt,
                             double alpha, void* scratch, cudaStream_t st, const TmaField* tf = nullptr);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace oec
