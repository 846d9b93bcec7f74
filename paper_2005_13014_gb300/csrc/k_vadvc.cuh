// k_vadvc.cuh - argument blocks of the hdiff+vadvc kernels (plain C++).
#pragma once

#include <cstdint>

namespace oec {

// one domain: pointers at the domain's lower corner, extents, shared strides
template <typename S>
struct HV {
  const S *u, *v, *w, *coeff;
  S *uo, *vo;
  int ni, nj, nk;
  int64_t sj, sk;
};

// one ensemble member in the device-side work table of the batched kernel
struct HVMember {
  const void *u, *v, *w, *coeff;
  void *uo, *vo;
  int ni, nj, nk, tiles_i;
  int64_t sj, sk;
  int tile_begin, pad;     // first work item of this member
};

struct HVBatchLaunch {
  const HVMember* members;  // device memory, n_members entries
  int n_members;
  int total_items;          // sum of tiles over members
  int* counter;             // device int, zero before the launch
  double dtr;
  void* scratch;            // grid * slot_elems recurrence values
  int64_t slot_elems;
  int grid;                 // persistent CTAs
};

}  // namespace oec
