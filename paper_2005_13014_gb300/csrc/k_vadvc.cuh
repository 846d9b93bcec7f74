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

// Persistent staged batch (FP32 fields, vector-row producer): one member in
// the device-side table. Pointers at the domain's lower corner; ud, vd, scr
// are the member's hdiff(u), hdiff(v) buffers (domain layout) and column
// scratch (row pitch ncolp).
struct PSMember {
  const void *u, *v, *w, *coeff;
  void *uo, *vo;
  void *ud, *vd, *scr;
  int64_t sj, sk, ncolp;
  int ni, nj, nk, kchunk, nkz;
  int row_base;   // this member's first row-block counter
  int need;       // producer items per row block (tiles along i x 2 fields x nkz)
  int pad;
};

// One work item, in ticket order: x = member for a producer item (bx, by, bz
// = y, z, w: the warp-row kernel's block indices), or ~member for a sweep item
// (y = group of 64 columns, z..w = the row blocks it needs).
struct PSItem {
  int x, y, z, w;
};

struct PSLaunch {
  const PSMember* members;   // device memory (a batch), or null: one domain, `single`
  const PSItem* items;       // device memory, n_items entries, or null: one domain's closed-form order
  int n_items;
  int* ticket;               // device int, zero before the launch
  int* done;                 // device ints, one per (member, row block), zero before the launch
  unsigned* timeouts;        // device counter of waits that gave up
  unsigned polls;            // poll limit of one wait
  double dtr;
  int grid;
  int unroll;                // rows per warp of the producer (1 or 2)
  bool o32;                  // every member's offsets fit 32 bits
  bool discard;              // the column sweep's L2 form
  // one domain without tables: ticket order row block by row block, each
  // block's producer items followed by the column groups whose last row lies
  // `lag` row blocks back (the remaining groups after the last block)
  PSMember single;
  int tiles_i;               // producer CTAs along i
  int per_block;             // producer items per row block (tiles_i x 2 fields x chunks)
  int blocks;                // row blocks (rows each)
  int rows;                  // rows per row block (4 x unroll)
  int groups;                // column groups of 64
  int lag;                   // row blocks between a group's last producers and the group
};

}  // namespace oec
