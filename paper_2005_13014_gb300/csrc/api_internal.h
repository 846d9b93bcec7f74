// api_internal.h - the program handle and helpers shared by the ABI sources.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/oec.h"
#include "ir.h"

struct oec_generic_state;   // generic code generator state (codegen.cpp)

struct oec_program {
  oec::Program ir;
  int dtype = OEC_F64;
  int kind = OEC_KIND_GENERIC;
  oec_schedule sched{};
  void* scratch = nullptr;       // library-owned temporaries (device memory)
  size_t scratch_bytes = 0;
  int scratch_dev = -1;
  oec_generic_state* gen = nullptr;
  // kernel timing (oec_program_set_timing): events of the recorded applies,
  // apply a's events at ev_first[a] .. ev_first[a] + ev_count[a]
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  int ev_used = 0;
  std::vector<int> ev_first, ev_count;
  int last_launches = 0;
  int last_timed = 0;      // timing events recorded after the apply's first (kernels or groups)
  int graphs = 0;          // live captured applies (oec_program_capture) using the scratch
  // oec_program_apply_host: two sets of device staging buffers (inputs then
  // outputs, bytes[x] each), the input-copy streams and the sets' events
  static constexpr int kCopyStreams = 1;
  struct HostStage {
    cudaStream_t copy[kCopyStreams] = {};
    cudaEvent_t inputs_in[2][kCopyStreams] = {}, released[2] = {nullptr, nullptr};
    std::vector<void*> buf[2];
    std::vector<size_t> bytes;
    int dev = -1, next = 0;
  } host;
};

namespace oec {

// a named NVTX range over one ABI call, for profilers that filter or group
// by range (ncu --nvtx); costs a pointer test when no tool is attached
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// host-side fault injection: the environment variable OEC_FAULT names one
// failure to make ("compile": run-time compilation of generated kernels,
// "alloc": the program's scratch allocation)
inline bool fault_injected(const char* what) {
  const char* f = std::getenv("OEC_FAULT");
  return f && std::strcmp(f, what) == 0;
}

int fail(int code, const char* fmt, ...);
void clear_error();
int cuda_fail(cudaError_t e, const char* where);
size_t elem_size(int dtype);
oec_schedule default_schedule(int kind, int dtype);
bool schedule_ok(int kind, const oec_schedule& s, std::string& why);
int ensure_scratch(oec_program* p, size_t bytes);
int validate_fields(const oec_program* p, const oec_field_desc* in, int n_in, const oec_field_desc* out, int n_out,
                    const int64_t lb[3], const int64_t ub[3], const int64_t halo[3], std::vector<Box>& ranges);

// dispatch.cpp: run a validated apply
int dispatch_apply(oec_program* p, const oec_field_desc* in, const oec_field_desc* out, const int64_t lb[3],
                   const int64_t ub[3], const double* params, cudaStream_t st);

// codegen.cpp: generic programs
bool generic_schedule_ok(const oec_schedule& s, std::string& why);
void generic_release(oec_program* p);
int generic_apply(oec_program* p, const oec_field_desc* in, const oec_field_desc* out, const int64_t lb[3],
                  const int64_t ub[3], const double* params, cudaStream_t st);

}  // namespace oec
