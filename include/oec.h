/*
 * oec.h - C ABI of liboec, a GB300 (sm_103a) runtime for stencil programs.
 *
 * A stencil program (paper §IV, "Stencil Programs") loads input fields, applies
 * a chain of stencil operators (stencil.apply) that read their inputs at
 * constant offsets (stencil.access), and stores results to output fields over
 * a domain given as a range with an inclusive lower and an exclusive upper
 * bound (paper §IV, "Shapes & Domains"). The library parses a textual form of
 * such a program, infers the access range of every input (paper §V-B, shape
 * inference), and runs it on the GPU, fused into one kernel per program
 * (stencil inlining, paper §V-A) or stage by stage with temporaries in device
 * memory (the paper's "original" optimisation level, §VII-C).
 *
 * Conventions used by every call:
 *  - Coordinates are (i, j, k); i is the contiguous dimension.
 *  - Every pointer to device memory is owned by the caller; the library never
 *    frees it. Program and batch handles, compiled modules and scratch
 *    temporaries are owned by the library and freed by the matching destroy.
 *  - Functions return OEC_OK (0) or a negative OEC_ERR_* code; the message of
 *    the last error on the calling thread is returned by oec_last_error().
 *    No C++ exception crosses this interface.
 *  - Apply calls are asynchronous: they enqueue work on the caller's CUDA
 *    stream (a cudaStream_t passed as void*, NULL = legacy default stream)
 *    and never synchronise with the host.
 *  - Each apply call (oec_program_apply, oec_program_apply_host,
 *    oec_batch_apply, oec_batch_apply_direct) is an NVTX range of that name,
 *    for profilers that filter by range.
 *  - Host-side fault injection for tests: the environment variable OEC_FAULT
 *    set to "compile" makes run-time compilation of generated kernels fail
 *    (OEC_ERR_COMPILE); set to "alloc" it makes a program's scratch
 *    allocation fail (OEC_ERR_CUDA). Nothing is injected on the device.
 */
#ifndef OEC_H
#define OEC_H

#include <stdint.h>

#if defined(__GNUC__)
#define OEC_API __attribute__((visibility("default")))
#else
#define OEC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------- */
#define OEC_OK 0
#define OEC_ERR_INVALID_ARG (-1)   /* null pointer, bad count, empty or inverted domain  */
#define OEC_ERR_PARSE (-2)         /* program text does not parse or verify              */
#define OEC_ERR_SHAPE (-3)         /* a field's storage does not hold its inferred range  */
#define OEC_ERR_HALO (-4)          /* inferred input range exceeds the caller's halo      */
#define OEC_ERR_ALIAS (-5)         /* an output range overlaps an input or other output   */
#define OEC_ERR_DTYPE (-6)         /* field element type differs from the program's       */
#define OEC_ERR_UNSUPPORTED (-7)   /* valid request the library cannot run                */
#define OEC_ERR_COMPILE (-8)       /* run-time compilation of a generated kernel failed    */
#define OEC_ERR_CUDA (-9)          /* a CUDA runtime call failed                          */
#define OEC_ERR_TIMEOUT (-10)      /* a bounded device-side wait gave up                  */

/* ---- element types (paper §IV: fields hold f32 or f64) ------------------ */
typedef enum { OEC_F32 = 0, OEC_F64 = 1 } oec_dtype;

/*
 * A field: caller-owned storage of a 1-, 2- or 3-D grid (paper §IV,
 * !stencil.field). Element (i, j, k) of the logical grid lives at
 *   data + ((origin[0]+i)*stride[0] + (origin[1]+j)*stride[1] + (origin[2]+k)*stride[2]) elements,
 * valid for 0 <= origin[d] + x_d < size[d]. Logical (0,0,0) is the origin of
 * the computation domain (paper §IV, range notation). stride[0] must be 1.
 * Unused trailing dimensions of 1-/2-D fields have size 1 and stride 0.
 */
typedef struct oec_field_desc {
  void* data;          /* device pointer to element (0,0,0) of the storage    */
  int32_t dtype;       /* oec_dtype                                           */
  int32_t ndim;        /* 1..3                                                */
  int64_t size[3];     /* storage extents (halo and padding included), i,j,k  */
  int64_t stride[3];   /* element strides                                     */
  int64_t origin[3];   /* storage index of logical point (0,0,0)              */
} oec_field_desc;

/* ---- schedules (paper §V-A: inlining and unrolling; §VI: grid mapping) --- */
typedef enum {
  OEC_FUSE_INLINE = 0,   /* all producers inlined into one kernel (paper §V-A)          */
  OEC_FUSE_NONE = 1,     /* one kernel per stage, temporaries in device memory; for
                            hdiff+vadvc: hdiff of u and v in one kernel, then the
                            column sweep. The hdiff kernel: FP32 fields with
                            OEC_STAGE_WARP staging and 16-byte aligned rows (ni a
                            multiple of 4) run the vector-row kernel (unroll rows
                            per warp); with OEC_STAGE_REGS staging, or WARP on
                            unaligned fields, the REGS kernel (tile_i x
                            tile_j/unroll threads, k_chunk levels per CTA; else
                            64 x 4, unroll 1); otherwise the SMEM tile kernel (tile_i
                            x tile_j, k_chunk levels when they name an SMEM hdiff
                            tile, else 64 x 4, 4 levels; FP64 arith 2: fixed point) */
  OEC_FUSE_PARTIAL = 2   /* generated programs: stages read at more than two offsets are
                            materialised, the rest inlined                              */
} oec_fusion;

typedef enum {
  OEC_STAGE_REGS = 0,    /* every thread recomputes what it reads (paper's model)      */
  OEC_STAGE_SMEM = 1,    /* overlapped tile in shared memory, no redundant compute     */
  OEC_STAGE_STREAM = 2,  /* k-streaming. hdiff: overlapped tile walked up k, the next
                            levels' windows copied asynchronously into a shared-memory
                            ring while the current level is computed. fastwaves: a
                            thread walks its column, carrying the k-shared values from
                            level to level, next level's loads in flight; with unroll
                            2 (tiles 32x4, 32x8, 64x4, 128x2) the CTA's u/v windows
                            come through a shared-memory ring                       */
  OEC_STAGE_WARP = 3,    /* horizontal diffusion: a warp owns `unroll` (1, 2, 4) rows of
                            32 x 16-byte vectors of columns; neighbours across vectors by
                            warp shuffles; the next level loaded ahead. Needs 16-byte
                            aligned rows (base at the domain corner and j/k strides),
                            else OEC_ERR_UNSUPPORTED; tile_i/tile_j unused             */
  OEC_STAGE_TMA = 4      /* horizontal diffusion: as OEC_STAGE_WARP, computed by a
                            persistent grid whose CTAs stream (tile, level) units; the
                            windows of the next 4 units are copied by the tensor memory
                            accelerator (cp.async.bulk.tensor) into a shared-memory ring.
                            Same alignment needs, and 16-byte aligned storage; k_chunk
                            unused. fastwaves: k-streaming CTA tiles (32x4, 32x8, 64x4)
                            whose nine input boxes per level are copied by TMA into a
                            4-stage ring; needs 16-byte aligned storage and j/k strides
                            (any domain corner), else OEC_ERR_UNSUPPORTED            */
} oec_staging;

typedef struct oec_schedule {
  int32_t fusion;        /* oec_fusion                                                   */
  int32_t staging;       /* oec_staging (fused kernels; and the FP32 hdiff+vadvc
                            producer of OEC_FUSE_NONE)                                  */
  int32_t tile_i;        /* CTA tile extent along i, in points (16..256)                 */
  int32_t tile_j;        /* CTA tile extent along j, in points (1..16)                   */
  int32_t unroll;        /* points per thread along the unroll dimension (1, 2 or 4)     */
  int32_t k_chunk;       /* levels per CTA for horizontal programs (0 = whole column)    */
  int32_t arith;         /* OEC_ARITH_*                                                   */
  int32_t index_bits;    /* OEC_INDEX_AUTO (0) or OEC_INDEX_64 (64)                       */
  int32_t sweep;         /* column sweep of the stage-by-stage hdiff+vadvc form:
                            OEC_SWEEP_PAIR (0), OEC_SWEEP_SPLIT (1), OEC_SWEEP_SEGMENTS4
                            (4) or OEC_SWEEP_SEGMENTS8 (8); 0 elsewhere                  */
  int32_t slabs;         /* stage-by-stage hdiff+vadvc: the domain's j-rows in this many
                            slabs (0 or 1: one), each slab's column sweep on a stream of
                            its own once that slab's hdiff is done, overlapping the
                            later slabs' hdiff (1..16); 0 elsewhere                      */
  int32_t reserved[2];   /* zero                                                          */
} oec_schedule;

/* Column sweep of the stage-by-stage hdiff+vadvc form (the twisted Thomas
 * factorisation: every column solved from both ends at once by two threads).
 * OEC_SWEEP_PAIR: the two threads carry both right-hand sides (u and v);
 * OEC_SWEEP_SPLIT: four threads per column, one field each (the matrix part of
 * the recurrence is then computed twice, but each thread's dependent chain
 * is shorter and twice as many warps hide its latency). Same results up to
 * rounding (the same operations per field). */
#define OEC_SWEEP_PAIR 0
#define OEC_SWEEP_SPLIT 1
/* With FP32 fields, the warp-row producer (OEC_STAGE_WARP, unroll 1 or 2,
 * rows 16-byte aligned), OEC_SWEEP_PAIR, slabs 0 or 1 and at least 65,536
 * columns, oec_program_apply runs the stage-by-stage form as one persistent
 * launch: CTAs take producer items (a block of 4 x unroll rows) and column
 * sweep items (64 columns) in a fixed ticket order, a sweep item waiting
 * (bounded, see oec_device_status) until the producer items of its rows are
 * done. Same results as the two kernels bit for bit. */
/* OEC_SWEEP_SEGMENTS4 / 8: the partitioned Thomas solve. Each column is cut
 * into 4 or 8 segments of consecutive levels, one thread each; a segment
 * eliminates downwards carrying its coupling to the level below it, then
 * substitutes upwards; the first and last rows of the column's segments form
 * a small reduced system, solved by every thread of the column; then every
 * thread forms its rows' solution. More threads per column, each with a
 * shorter dependent chain, for about a quarter more operations. Same results
 * up to rounding. */
#define OEC_SWEEP_SEGMENTS4 4
#define OEC_SWEEP_SEGMENTS8 8

/* Width of the element offsets that kernels form from their fields' base
 * pointers (the paper's index type, §V-B and §VII-C). OEC_INDEX_AUTO: the
 * kernels that have a 32-bit form (fused horizontal diffusion with OEC_STAGE_REGS
 * or OEC_STAGE_WARP or OEC_ARITH_FIXED, the hdiff producers and the column
 * sweep of the stage-by-stage hdiff+vadvc form, and generated kernels) use
 * 32-bit offsets
 * when every offset they form fits in an int32, else 64-bit; all other kernels
 * use 64-bit offsets. OEC_INDEX_64: 64-bit offsets in every kernel. Both give
 * the same results bit for bit: only address arithmetic differs. */
#define OEC_INDEX_AUTO 0
#define OEC_INDEX_64 64

/* Arithmetic of a schedule. OEC_ARITH_NATIVE evaluates in the dtype's own
 * IEEE arithmetic (FP32 programs keep their column recurrence in native FP64).
 * OEC_ARITH_DOUBLE_FLOAT evaluates FP64 values as pairs of floats (~48
 * significant bits, Dekker/Knuth error-free transformations) on the FP32 pipes,
 * which GB300 runs ~70x faster than its FP64 pipe: for FP64 programs every
 * operation, for FP32 programs the column recurrence. Results stay within the
 * FP64 tolerance (normwise 1e-13) for values of magnitude 2^-74..2^128. */
#define OEC_ARITH_NATIVE 0
#define OEC_ARITH_DOUBLE_FLOAT 1
/* OEC_ARITH_FIXED (FP64 horizontal diffusion only, fused SMEM schedules, and
 * the stage-by-stage hdiff+vadvc form): the linear part of the stencil
 * (Laplacian, fluxes, divergence) is evaluated exactly in 64-bit integers on a
 * per-tile scale, the limiter's signs are taken exactly from the binary64
 * inputs, and the output is one fused multiply-add in FP64. Inputs must be
 * finite. */
#define OEC_ARITH_FIXED 2

/* ---- programs ----------------------------------------------------------- */
typedef struct oec_program* oec_program_t;

#define OEC_OPT_GENERIC 1      /* never use a hand-written kernel for this program */

typedef struct oec_program_options {
  int32_t dtype;         /* oec_dtype of every field of the program             */
  int32_t flags;         /* OEC_OPT_* bits                                      */
  int32_t reserved[6];   /* zero                                                */
} oec_program_options;

/* What kind of kernel runs a program (oec_program_info.kind). */
#define OEC_KIND_GENERIC 0
#define OEC_KIND_HDIFF 1
#define OEC_KIND_HDIFF_VADVC 2
#define OEC_KIND_FASTWAVES 3

typedef struct oec_program_info {
  int32_t kind;          /* OEC_KIND_*                                           */
  int32_t n_inputs;      /* fields named by `input`, in order                    */
  int32_t n_outputs;     /* values named by `output`, in order                   */
  int32_t n_params;      /* scalars named by `param`, in order                   */
  int32_t n_stages;      /* stencil.apply statements (+ column solves)           */
  int32_t dtype;         /* oec_dtype                                            */
} oec_program_info;

/*
 * Parse and verify a program in the textual stencil form (paper §IV):
 *   input a, b            loaded fields          (stencil.load)
 *   param p               scalar parameters
 *   stage x = expr        one stencil.apply; reads name[di,dj,dk] (stencil.access)
 *   stage x, y = { let t = expr; return e1, e2 }   multi-result apply
 *   column x = thomas(a, b, c, d)                  tridiagonal solve along k
 *   output x              stored values           (stencil.store)
 * Expressions: + - * / unary -, min, max, abs, select(x > y, a, b) (also <, >=,
 * <=), numbers, params, `kpos` (k minus the domain's lower k) and `ksize`,
 * and control flow inside an apply (paper §IV-C, scf.if / scf.yield):
 *   if (x > y) { let t = expr; yield e1 } else { yield e2 }
 * whose value is the yield of the region the condition picks; a region's lets
 * are visible in it only. Regions are pure, so the library evaluates the if
 * as select(x > y, e1, e2) with the regions' lets bound in the stage.
 * On success *out receives a handle. No GPU work happens here.
 * Errors: OEC_ERR_INVALID_ARG, OEC_ERR_PARSE (message gives the position).
 */
OEC_API int oec_program_create(const char* source, const oec_program_options* opts, oec_program_t* out);

/* Free a program, its scratch temporaries and compiled modules (NULL is a no-op).
 * The caller must ensure no apply of this program is still running. */
OEC_API void oec_program_destroy(oec_program_t p);

/* Counts and kind of a program. Errors: OEC_ERR_INVALID_ARG. */
OEC_API int oec_program_get_info(oec_program_t p, oec_program_info* info);

/* Name of input `index` (0-based, declaration order) copied into buf (NUL
 * terminated, truncated to len). Errors: OEC_ERR_INVALID_ARG. */
OEC_API int oec_program_input_name(oec_program_t p, int index, char* buf, int len);

/*
 * Inferred access range of input `index` for the domain [lb, ub) (paper §V-B:
 * the bounding box of all extents its consumers read), returned as the
 * half-open box [range_lo, range_hi) in logical coordinates. An input that
 * no output depends on gets an empty box (range_lo == range_hi == lb).
 * Errors: OEC_ERR_INVALID_ARG.
 */
OEC_API int oec_program_input_range(oec_program_t p, int index, const int64_t lb[3], const int64_t ub[3],
                            int64_t range_lo[3], int64_t range_hi[3]);

/*
 * Select the schedule used by later applies (fusion, staging, tile, unroll,
 * k-chunk). Values outside the supported set give OEC_ERR_UNSUPPORTED and
 * leave the schedule unchanged. A new program starts with the library's
 * default schedule for its kind and dtype (hdiff+vadvc: the staged form the
 * autotuner picks at 128x128x80 - FP64 fixed-point producer 32x16 with 2
 * rows per thread and 2 levels per CTA, FP32 vector-row producer with 20
 * levels per CTA, both with the double-float column sweep).
 */
OEC_API int oec_program_set_schedule(oec_program_t p, const oec_schedule* s);
OEC_API int oec_program_get_schedule(oec_program_t p, oec_schedule* s);

/*
 * Run the program over the domain [lb, ub) (paper §IV range notation, logical
 * coordinates).
 *   in[n_in]    input fields in `input` order (device memory, caller-owned)
 *   out[n_out]  output fields in `output` order; written over [lb, ub) only
 *   halo[3]     cells around [lb, ub) (per side, per dimension) that hold valid
 *               input data; the inferred range of every input must stay inside
 *               [lb - halo, ub + halo) (OEC_ERR_HALO) and inside the field's
 *               storage (OEC_ERR_SHAPE)
 *   params      the program's scalars in `param` order (n_params of them)
 *   cuda_stream cudaStream_t (void*); NULL = legacy default stream
 * Inputs may alias each other; an output's written range may overlap no
 * input's storage and no other output's range (OEC_ERR_ALIAS; paper §IV
 * requires alias-free program arguments). All fields of one program must
 * share the program's dtype (OEC_ERR_DTYPE) and the same j and k strides
 * (OEC_ERR_UNSUPPORTED). The first apply at a new domain size may allocate
 * scratch temporaries (unfused schedules, column solves); later applies at
 * that size reuse them. Asynchronous: returns after enqueueing.
 * Errors: OEC_ERR_INVALID_ARG, OEC_ERR_SHAPE, OEC_ERR_HALO, OEC_ERR_ALIAS,
 * OEC_ERR_DTYPE, OEC_ERR_UNSUPPORTED, OEC_ERR_COMPILE, OEC_ERR_CUDA.
 */
OEC_API int oec_program_apply(oec_program_t p, const oec_field_desc* in, int n_in, const oec_field_desc* out,
                      int n_out, const int64_t lb[3], const int64_t ub[3], const int64_t halo[3],
                      const double* params, int n_params, void* cuda_stream);

/*
 * oec_program_apply with every field in HOST memory: `data` of each
 * descriptor is a host pointer (page-locked memory keeps the call
 * asynchronous; pageable memory works, with the copies synchronous). The
 * library copies each input's storage from the first to the last element of
 * its access box (the range shape inference gives it for [lb, ub), paper
 * §IV), widened to 4 KiB boundaries of the host address, into device staging
 * buffers laid out like the host storage, applies the program there, and
 * copies back each output's domain box [lb, ub) only: host output storage
 * outside the domain is left as it was. Staging buffers come in two sets used
 * in turn, allocated at the first call and again when field shapes change;
 * the input copies run on a library stream, so the next call's inputs cross
 * while this call computes and its outputs cross on `cuda_stream`.
 * Ordered on `cuda_stream`: the host outputs are complete once it has been
 * synchronised. Fields need a unit i stride and positive j/k strides
 * (OEC_ERR_UNSUPPORTED). Not for stream capture.
 * Errors: those of oec_program_apply, and OEC_ERR_CUDA for allocations and
 * copies.
 */
OEC_API int oec_program_apply_host(oec_program_t p, const oec_field_desc* in, int n_in, const oec_field_desc* out,
                                   int n_out, const int64_t lb[3], const int64_t ub[3], const int64_t halo[3],
                                   const double* params, int n_params, void* cuda_stream);

/*
 * Captured applies (no counterpart in the paper, which times kernels launched
 * one by one): oec_program_capture records one oec_program_apply with these
 * arguments into a CUDA graph and instantiates it; oec_graph_launch enqueues
 * that graph on a stream, one launch per apply, so a loop of applies with
 * fixed fields pays one launch instead of one per kernel and no argument
 * marshalling. The graph reads and writes the fields' memory at the addresses
 * given at capture (their contents may change between launches) and the
 * program's scratch as it was then: while a program has live graphs, an apply
 * that would need a larger scratch fails with OEC_ERR_UNSUPPORTED; destroy
 * the graphs first (and before destroying the program). The capture runs on
 * a private stream in relaxed capture mode, so the program's scratch and, for
 * generated programs, its module are set up eagerly during the call (call
 * oec_program_prepare first to compile outside it); kernel timing is off
 * inside the capture. Argument errors are those of oec_program_apply; the
 * capture itself: OEC_ERR_CUDA. Synchronous with respect to the host (returns
 * once the graph is instantiated); nothing runs on the GPU.
 */
typedef struct oec_graph* oec_graph_t;
OEC_API int oec_program_capture(oec_program_t p, const oec_field_desc* in, int n_in, const oec_field_desc* out,
                                int n_out, const int64_t lb[3], const int64_t ub[3], const int64_t halo[3],
                                const double* params, int n_params, oec_graph_t* graph);
/* Enqueue one launch of a captured apply on cuda_stream (asynchronous).
 * Errors: OEC_ERR_INVALID_ARG, OEC_ERR_CUDA. */
OEC_API int oec_graph_launch(oec_graph_t graph, void* cuda_stream);
/* Kernels one launch of the graph runs. */
OEC_API int oec_graph_kernel_count(oec_graph_t graph);
OEC_API void oec_graph_destroy(oec_graph_t graph);

/*
 * Compile and load the generated kernels of a program without a hand-written
 * kernel for a domain extent and field j/k strides (what the first apply at
 * that shape would do), so that applies and stream capture that follow
 * compile nothing. Safe to call for different programs from different host
 * threads. No-op for programs with hand-written kernels.
 * Errors: OEC_ERR_INVALID_ARG, OEC_ERR_SHAPE, OEC_ERR_UNSUPPORTED,
 * OEC_ERR_COMPILE, OEC_ERR_CUDA.
 */
OEC_API int oec_program_prepare(oec_program_t p, const int64_t extent[3], int64_t sj, int64_t sk);

/*
 * The CUDA C++ that liboec generates for a program without a hand-written
 * kernel (paper §V-C/§VI lowering: inlined stages, k-unrolled bodies,
 * temporaries for materialised stages), for a domain extent and the fields' j/k
 * strides: all fusion x unroll variants in one translation unit. The source is
 * copied into buf (NUL-terminated, truncated to cap; buf may be NULL) and its
 * full length stored in *len. With compile != 0 it is also compiled with NVRTC
 * for sm_103a (no GPU needed; nothing is loaded). Errors: OEC_ERR_INVALID_ARG,
 * OEC_ERR_SHAPE, OEC_ERR_UNSUPPORTED (column solves), OEC_ERR_COMPILE.
 */
OEC_API int oec_program_codegen(oec_program_t p, const int64_t extent[3], int64_t sj, int64_t sk, int compile, char* buf,
                                int64_t cap, int64_t* len);

/* ---- autotuning (paper §VII-C tunes unroll factors empirically; here every
 * supported schedule is timed) -------------------------------------------- */

/* The candidate schedules the autotuner tries for this program (every fusion,
 * staging, tile, unroll, k-chunk and arithmetic choice its kernels support).
 * Returns their number; copies up to cap of them into out (out may be NULL). */
OEC_API int oec_program_candidates(oec_program_t p, oec_schedule* out, int cap);

/*
 * Time candidate schedules on the given fields and keep the fastest as the
 * program's schedule. For each candidate (candidates = NULL: the program's own
 * set from oec_program_candidates): one untimed apply (it compiles generated
 * kernels and allocates scratch), then `reps` applies timed one by one with
 * CUDA events on cuda_stream; times_ms[c] = the median in milliseconds, or -1
 * for a candidate that cannot run. *best (may be NULL) receives the index of
 * the fastest. Synchronises the stream; fields as for oec_program_apply
 * (outputs are overwritten). Repeated applies reuse the same data, so domains
 * that fit in L2 are timed cache-warm.
 */
OEC_API int oec_program_autotune(oec_program_t p, const oec_field_desc* in, int n_in, const oec_field_desc* out,
                                 int n_out, const int64_t lb[3], const int64_t ub[3], const int64_t halo[3],
                                 const double* params, int n_params, const oec_schedule* candidates, int n_candidates,
                                 int reps, void* cuda_stream, double* times_ms, int* best);

/* ---- tuning database (the autotuner's results kept across runs) ---------- */
typedef struct oec_tunedb* oec_tunedb_t;

/*
 * Open a tuning database: entries map a key - the program (hash of its
 * canonical text, recognised kind, dtype), the domain extent, the fields'
 * shared j/k strides, whether every field's domain corner and the strides
 * are 16-byte aligned, and the device (name, SM count, compute capability) -
 * to a schedule and its time in milliseconds. path: a text file ("oec-tunedb
 * 1" then one tab-separated entry per line), loaded if it exists, else the
 * database starts empty; NULL keeps it in memory. Errors: OEC_ERR_INVALID_ARG
 * (the file exists but is not a database, with the line in the message).
 */
OEC_API int oec_tunedb_open(const char* path, oec_tunedb_t* out);
/* Write every entry to path (NULL: the path given at open) through a
 * temporary file renamed over it. Errors: OEC_ERR_INVALID_ARG (no path, not
 * writable). */
OEC_API int oec_tunedb_save(oec_tunedb_t db, const char* path);
/* Number of entries (>= 0), or OEC_ERR_INVALID_ARG. */
OEC_API int oec_tunedb_count(oec_tunedb_t db);
OEC_API void oec_tunedb_close(oec_tunedb_t db);
/* Look up the key of an apply (fields and domain as for oec_program_apply;
 * nothing is read from the fields' memory). *found = 1 and *s, *ms (each may
 * be NULL) set when present, else *found = 0. No GPU work. */
OEC_API int oec_tunedb_find(oec_tunedb_t db, oec_program_t p, const oec_field_desc* in, int n_in,
                            const oec_field_desc* out, int n_out, const int64_t lb[3], const int64_t ub[3],
                            oec_schedule* s, double* ms, int* found);
/* Record (or replace) the entry of an apply's key. Errors: OEC_ERR_INVALID_ARG,
 * OEC_ERR_UNSUPPORTED (a schedule the program cannot run). */
OEC_API int oec_tunedb_record(oec_tunedb_t db, oec_program_t p, const oec_field_desc* in, int n_in,
                              const oec_field_desc* out, int n_out, const int64_t lb[3], const int64_t ub[3],
                              const oec_schedule* s, double ms);
/*
 * Autotune through the database: when the key of this apply is recorded (and
 * its schedule still valid) the program takes that schedule and *from_db = 1,
 * with no GPU work; otherwise oec_program_autotune times every candidate,
 * the fastest becomes the schedule and is recorded, *from_db = 0. The
 * database is not saved. Errors: as oec_program_autotune.
 */
OEC_API int oec_program_autotune_db(oec_program_t p, oec_tunedb_t db, const oec_field_desc* in, int n_in,
                                    const oec_field_desc* out, int n_out, const int64_t lb[3], const int64_t ub[3],
                                    const int64_t halo[3], const double* params, int n_params, int reps,
                                    void* cuda_stream, int* from_db);

/*
 * Features of (program, domain extent, field strides, schedule) for the learned
 * cost model (no counterpart in the paper): 42 floats - program structure
 * (stages, inputs, outputs, accesses, operations by kind, maximal offsets, DAG
 * depth, inferred halos, read amplification), domain size, schedule (fusion
 * one-hot, unroll, tile, threads), and the per-point loads, operations, stores
 * and temporary bytes of the code generated for that schedule. Returns the
 * number of features (out = NULL to query), or a negative error; programs with
 * column solves are OEC_ERR_UNSUPPORTED. Host only.
 */
OEC_API int oec_program_features(oec_program_t p, const int64_t extent[3], int64_t sj, int64_t sk,
                                 const oec_schedule* s, float* out, int cap);

/*
 * Algorithmic device-memory bytes of one apply over [lb, ub): the sum over
 * inputs of the inferred range volume plus the sum over outputs of the domain
 * volume, times the element size. Temporaries are not counted (a fused
 * kernel keeps them on chip). Errors: OEC_ERR_INVALID_ARG.
 */
OEC_API int oec_program_algorithmic_bytes(oec_program_t p, const int64_t lb[3], const int64_t ub[3], int64_t* bytes);

/*
 * Kernel launches and per-kernel timing of applies (measurement support; the
 * paper times whole programs, §VII, and a staged schedule runs several kernels
 * per apply).
 *
 * oec_program_launch_count: the number of kernels the program's most recent
 * successful or failed oec_program_apply launched (0 before any apply, and for
 * an empty domain).
 *
 * oec_program_set_timing(p, 1): from now on every oec_program_apply records a
 * CUDA event on its stream before its first kernel and one after each kernel
 * (events owned by the program, created on first use on the current device);
 * an apply that fails records nothing. 0 stops recording; recorded applies
 * are kept. The staged hdiff+vadvc pipeline (schedule field slabs > 1) runs
 * its kernels on two streams, overlapped: it records one event after all of
 * them, so its applies report one duration (the whole pipeline).
 *
 * oec_program_kernel_times: waits for the recorded events, writes the
 * duration of kernel x of recorded apply a to ms[a * *n_kernels + x] (in
 * milliseconds), sets *n_applies and *n_kernels, and forgets the recorded
 * applies. Errors: OEC_ERR_INVALID_ARG (null argument, fewer than
 * n_applies * n_kernels entries in cap - nothing is forgotten then -, or
 * recorded applies with different kernel counts), OEC_ERR_CUDA.
 */
/*
 * Status of the library's bounded device-side waits (the TMA-staged kernels
 * wait on mbarriers for their own copies, for about a second at most).
 * Synchronises cuda_stream, then returns OEC_ERR_TIMEOUT if any wait gave up
 * since the previous call (the affected outputs are incomplete), OEC_OK
 * otherwise, and clears the record. Errors: OEC_ERR_CUDA.
 */
OEC_API int oec_device_status(void* cuda_stream);
/* Exercise the give-up path of the bounded waits: enqueue a one-thread kernel
 * whose mbarrier wait on a phase that never completes gives up after `polls`
 * polls (1..65536) and records a timeout, so the next oec_device_status
 * reports OEC_ERR_TIMEOUT. No copies are involved; the GPU context stays
 * usable. Errors: OEC_ERR_INVALID_ARG, OEC_ERR_CUDA. */
OEC_API int oec_device_wait_selftest(int polls, void* cuda_stream);
/* The same for the persistent staged batch's wait on its per-row-block
 * counters (see oec_batch_create): launch the batch kernel on one column-sweep
 * item whose counter nothing releases; its wait gives up after `polls` polls
 * (1..65536), records a timeout and skips the item, so the next
 * oec_device_status reports OEC_ERR_TIMEOUT. Synchronises cuda_stream before
 * returning. Errors: OEC_ERR_INVALID_ARG, OEC_ERR_CUDA. */
OEC_API int oec_batch_wait_selftest(int polls, void* cuda_stream);
/* The ticket order of the persistent launch that runs one FP32 domain of
 * ni x nj x nk points (warp-row producer with `unroll` rows per warp, 1 or 2;
 * `k_chunk` levels per producer item, 0 or more than nk: all) when `grid`
 * CTAs are resident, computed on the host exactly as the kernel's CTAs
 * decode their tickets. No GPU is used. For ticket t, items[4t..4t+3] hold
 * (x, y, z, w): x = 0 for a producer item (y its tile along i, z its row
 * block, w its level chunk, plus the number of chunks for the second field),
 * x = -1 for a column-sweep item (y its group of 64 columns, z..w the row
 * blocks whose producer items it waits for). The order is what keeps every
 * bounded wait of the launch finite without assuming which CTAs are
 * resident: each sweep item comes after all the producer items it waits for,
 * and producer items never wait. *n_items receives the ticket count; items
 * is written only when cap >= 4 x that count (items may be null to query).
 * Errors: OEC_ERR_INVALID_ARG (a size or grid below 1, unroll not 1 or 2,
 * more tickets than an int holds). The paper has no counterpart: this is a
 * diagnostic of the library's own scheduling. */
OEC_API int oec_pstaged_ticket_order(int32_t ni, int32_t nj, int32_t nk, int32_t unroll, int32_t k_chunk,
                                     int32_t grid, int32_t* items, int64_t cap, int64_t* n_items);
/* The same for a persistent staged batch (see oec_batch_create) of
 * n_members FP32 domains, sizes[3m..3m+2] = (ni, nj, nk) of member m in
 * order, when a column group is placed `lag` tickets after the last producer
 * item it waits for (the batch uses twice the resident CTAs). Host only, no
 * GPU. For ticket t, items[4t..4t+3] hold (x, y, z, w): x = m >= 0 for a
 * producer item of member m (y its tile along i, z its row block, w its
 * level chunk, plus the number of chunks for the second field), x = -1 - m
 * for a column group y of member m waiting for its row blocks z..w.
 * *n_items receives the ticket count; items is written only when cap >= 4 x
 * that count. Errors: OEC_ERR_INVALID_ARG (no members, a size below 1,
 * unroll not 1 or 2, lag below 0). The paper has no counterpart. */
OEC_API int oec_batch_ticket_order(int32_t n_members, const int32_t* sizes, int32_t unroll, int32_t k_chunk,
                                   int64_t lag, int32_t* items, int64_t cap, int64_t* n_items);
OEC_API int oec_program_launch_count(oec_program_t p);
OEC_API int oec_program_set_timing(oec_program_t p, int enable);
OEC_API int oec_program_kernel_times(oec_program_t p, float* ms, int cap, int* n_applies, int* n_kernels);

/* ---- batched ensembles (no counterpart in the paper's compiler; the paper's
 * programs run one domain per launch) ------------------------------------- */
typedef struct oec_batch* oec_batch_t;

typedef struct oec_batch_member {
  const oec_field_desc* in;    /* the program's inputs for this member (device memory)  */
  const oec_field_desc* out;   /* its outputs                                           */
  int64_t lb[3], ub[3];        /* the member's domain [lb, ub)                          */
  int64_t halo[3];             /* valid cells around the domain (as oec_program_apply)  */
} oec_batch_member;

/*
 * Prepare one graph over an ensemble of domains of different sizes (currently
 * hdiff+vadvc programs); every member is validated as oec_program_apply would
 * validate it. With a fused schedule (OEC_FUSE_INLINE) the members' column
 * tiles become one work list (tallest columns first), and a persistent kernel
 * - one CTA per resident slot on every SM - pulls (member, tile) items from an
 * atomic counter and runs the fused column sweep with the program's tile
 * shape and arithmetic; the counter reset and the launch are captured into
 * the graph. With a staged schedule (OEC_FUSE_NONE) on FP32 fields with the
 * warp-row producer (OEC_STAGE_WARP, unroll 1 or 2, the pair column sweep)
 * and every member's rows 16-byte aligned (u, v, coeff at the domain corner,
 * j/k strides, ni a multiple of 4): one persistent kernel takes, in ticket
 * order, producer items (a block of 4 x unroll rows of one member: hdiff of
 * u and v into the member's buffers) and column-sweep items (64 columns of
 * one member), a sweep item waiting - bounded, see oec_batch_wait_selftest -
 * on counters of the row blocks it needs; the counters' reset and the launch
 * are captured into the graph. Other staged schedules: every member's
 * producer and column-sweep launches form an independent branch of the graph
 * (members on up to 16 forked streams, largest first to the least-loaded
 * one), so the members' sweeps run concurrently. Device memory: the work
 * table, the counters and per-CTA or per-member scratch, owned by the batch.
 * The program and every member's fields must outlive the batch.
 * params: the program's scalars. Errors: as oec_program_apply, and
 * OEC_ERR_UNSUPPORTED for other program kinds.
 */
OEC_API int oec_batch_create(oec_program_t p, const oec_batch_member* members, int n_members, const double* params,
                             int n_params, oec_batch_t* out);
/* Launch the captured graph on cuda_stream (asynchronous). */
OEC_API int oec_batch_apply(oec_batch_t b, void* cuda_stream);
/* The same work without the graph on cuda_stream: the persistent kernel(s)
 * launched directly, or the staged members' launches one after another. */
OEC_API int oec_batch_apply_direct(oec_batch_t b, void* cuda_stream);
/* Work items (tiles, or producer and sweep items; staged chains: members) and
 * persistent CTAs (staged chains: streams) of a batch. */
OEC_API int oec_batch_info(oec_batch_t b, int* n_items, int* n_ctas);
/* Free the batch (NULL is a no-op); waits for its device work to finish. */
OEC_API void oec_batch_destroy(oec_batch_t b);

/* ---- learned cost model (no counterpart in the paper, which tunes
 * empirically and always fuses, §VII-C) ----------------------------------- */
typedef struct oec_costmodel* oec_costmodel_t;

/*
 * An FP32 MLP: features -> hidden -> hidden -> 1 with ReLU, predicting a
 * log cost of a (program, domain, schedule) - the project trains it on
 * log(t / t_best) within each program, and selection only ranks predictions
 * of one program's candidates. Parameters are
 * one flat array W1 [H][F], b1 [H], W2 [H][H], b2 [H], W3 [1][H], b3 [1]
 * (params_host may be NULL: all zero). Training uses mean squared error and
 * Adam; all compute runs in liboec's kernels, and every reduction has a fixed
 * order, so results are reproducible run to run. Device buffers for a batch
 * grow on the first call with a larger n. All pointers other than the
 * parameter copies are device memory; calls enqueue on cuda_stream.
 */
OEC_API int oec_costmodel_create(int n_features, int hidden, const float* params_host, oec_costmodel_t* out);
OEC_API int oec_costmodel_param_count(oec_costmodel_t m);
/* Copy the parameters to/from host memory (checkpoint and resume; setting
 * them also resets Adam's moments and step count). Synchronous. */
OEC_API int oec_costmodel_get_params(oec_costmodel_t m, float* params_host, int count);
OEC_API int oec_costmodel_set_params(oec_costmodel_t m, const float* params_host, int count);
/* Features are standardised as (x - mu[f]) / sigma[f] before the first layer
 * (default mu = 0, sigma = 1; sigma <= 0 counts as 1). Host arrays of F floats. */
OEC_API int oec_costmodel_set_normalization(oec_costmodel_t m, const float* mu, const float* sigma);
/* y[n] = model(X[n][F]) */
OEC_API int oec_costmodel_predict(oec_costmodel_t m, const float* X, int n, float* y, void* cuda_stream);
/* grad[param_count] = d loss / d params and *loss = mean (y - t)^2 over n rows */
OEC_API int oec_costmodel_gradient(oec_costmodel_t m, const float* X, const float* t, int n, float* grad, float* loss,
                                   void* cuda_stream);
/* One Adam step on the batch (X, t): *loss receives the batch loss before it. */
OEC_API int oec_costmodel_train_step(oec_costmodel_t m, const float* X, const float* t, int n, float lr, float beta1,
                                     float beta2, float eps, float* loss, void* cuda_stream);
OEC_API void oec_costmodel_destroy(oec_costmodel_t m);

/* Checkpoint file: dimensions, parameters and standardisation (binary, little
 * endian as written). save errors: OEC_ERR_INVALID_ARG (path unwritable);
 * load: OEC_ERR_INVALID_ARG (unreadable, or not a checkpoint), and
 * oec_costmodel_create's errors. Synchronous. */
OEC_API int oec_costmodel_save(oec_costmodel_t m, const char* path);
OEC_API int oec_costmodel_load(const char* path, oec_costmodel_t* out);

/*
 * Model-guided schedule selection: the features of every candidate schedule
 * (oec_program_candidates, oec_program_features) are predicted by m; top_k <= 0
 * takes the best-ranked valid candidate untimed, top_k > 0 times the top_k
 * best-ranked as oec_program_autotune does (reps applies each; fields as for
 * oec_program_apply, outputs overwritten) and takes the fastest, with
 * exhaustive oec_program_autotune as the reference its choices are measured
 * against.
 * Sets the program's schedule; *best = the pick's index in the candidate
 * list; pred (may be NULL) receives the n_cand predictions. Synchronises
 * cuda_stream. Errors: as oec_program_features and oec_program_autotune, and
 * OEC_ERR_INVALID_ARG when the model's feature count differs.
 */
OEC_API int oec_program_autotune_model(oec_program_t p, oec_costmodel_t m, const oec_field_desc* in, int n_in,
                                       const oec_field_desc* out, int n_out, const int64_t lb[3], const int64_t ub[3],
                                       const int64_t halo[3], const double* params, int n_params, int top_k, int reps,
                                       void* cuda_stream, float* pred, int* best);

/*
 * hdiff+vadvc without any device allocation. There is no counterpart in the
 * paper; this entry point exists for callers that cannot allocate device
 * memory while they run the program: code that must stay inside a
 * device-memory budget owned by another allocator (a framework's caching
 * allocator, a pool sized at start-up) and latency-critical loops where
 * cudaMalloc/cudaFree may synchronise the device. oec_program_apply allocates
 * scratch on its first apply at a new size; this call never does: its scratch
 * is a fixed 64 MiB array inside the library's device image (held on every
 * GPU where the library's device code is loaded, until the process exits).
 * It runs the staged form (hdiff of u and v, then the twisted column sweep,
 * two threads per column; FP64: fixed-point producer and double-float sweep,
 * FP32: vector-row or REGS producer and double-float sweep) on the caller's
 * stream when its scratch fits, else the fused column sweep.
 *   dtype   OEC_F32 or OEC_F64 (all six fields)
 *   in[4]   u, v, w, coeff; u and v must hold [lb-2, ub+2) in i and j, w must
 *           hold [lb, ub+1) in i, coeff the domain
 *   out[2]  u_out, v_out, written over [lb, ub)
 *   dtr     the scalar parameter of the vertical advection
 * Limit, for a domain of ni x nj x nk points: the staged form needs
 * 24 * ceil16(ni * nj) * nk + 16 * ni * nj * nk bytes in FP64 and
 * 24 * ceil16(ni * nj) * nk + 8 * ni * nj * nk in FP32, each of its two parts
 * rounded up to 256 bytes (40 and 32 bytes per point when ni * nj is a
 * multiple of 16; FP32 domains of at least 65,536 columns add
 * 4 * (ceil(nj / 4) + 1) bytes of counters, rounded up to 256); beyond 64 MiB
 * the fused form needs
 * 24 * ceil16(ni) * ceil4(nj) * nk bytes (ceilN: rounded up to a multiple of
 * N); a domain whose fused form needs more than 64 MiB is rejected with
 * OEC_ERR_UNSUPPORTED before anything is enqueued. The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current and keeps it for the life of the process; make that first
 * call before any stream capture. A device reset (cudaDeviceReset) after that
 * first call is not supported: the kept address would be stale. All calls
 * share the one array and it keeps the last call's contents (nothing in it
 * needs to start at zero: every value is written before it is read): calls
 * whose kernels overlap on the GPU race and corrupt each other's results, so
 * serialise them (one stream, or events). Returns as oec_program_apply does.
 */
OEC_API int oec_hdiff_vadvc_apply_noalloc(int32_t dtype, const oec_field_desc* in, const oec_field_desc* out,
                                          const int64_t lb[3], const int64_t ub[3], double dtr, void* cuda_stream);

/* Message of the last error on the calling thread ("" if none). The pointer
 * stays valid until the thread's next liboec call. */
OEC_API const char* oec_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
