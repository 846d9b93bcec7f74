"""ctypes declarations of liboec's C ABI (include/oec.h). Marshalling only."""

from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboec.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "oec.h")

OEC_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "PARSE", -3: "SHAPE", -4: "HALO", -5: "ALIAS", -6: "DTYPE",
          -7: "UNSUPPORTED", -8: "COMPILE", -9: "CUDA", -10: "TIMEOUT"}
F32, F64 = 0, 1
FUSE_INLINE, FUSE_NONE = 0, 1
ARITH_NATIVE, ARITH_DOUBLE_FLOAT = 0, 1
STAGE_REGS, STAGE_SMEM = 0, 1
KIND_NAMES = {0: "generic", 1: "hdiff", 2: "hdiff_vadvc", 3: "fastwaves"}

I64x3 = C.c_int64 * 3


class FieldDesc(C.Structure):
    _fields_ = [("data", C.c_void_p), ("dtype", C.c_int32), ("ndim", C.c_int32),
                ("size", I64x3), ("stride", I64x3), ("origin", I64x3)]


class Schedule(C.Structure):
    _fields_ = [("fusion", C.c_int32), ("staging", C.c_int32), ("tile_i", C.c_int32), ("tile_j", C.c_int32),
                ("unroll", C.c_int32), ("k_chunk", C.c_int32), ("arith", C.c_int32), ("index_bits", C.c_int32),
                ("sweep", C.c_int32), ("slabs", C.c_int32), ("reserved", C.c_int32 * 2)]


class ProgramOptions(C.Structure):
    _fields_ = [("dtype", C.c_int32), ("flags", C.c_int32), ("reserved", C.c_int32 * 6)]


class ProgramInfo(C.Structure):
    _fields_ = [("kind", C.c_int32), ("n_inputs", C.c_int32), ("n_outputs", C.c_int32),
                ("n_params", C.c_int32), ("n_stages", C.c_int32), ("dtype", C.c_int32)]


class BatchMember(C.Structure):
    _fields_ = [("in_", C.POINTER(FieldDesc)), ("out", C.POINTER(FieldDesc)), ("lb", I64x3), ("ub", I64x3),
                ("halo", I64x3)]


class OecError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"oec error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code
        self.name = ERRORS.get(code, "?")


_lib = None


def declared_symbols():
    """Names of every function include/oec.h declares."""
    with open(HEADER) as f:
        return re.findall(r"^OEC_API\s+[\w\s\*]+?\b(oec_\w+)\s*\(", f.read(), flags=re.M)


def lib():
    """Load liboec.so (built in-tree by build.py); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError(f"{LIB_PATH} is not built; run paper_2005_13014_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    sig = {
        "oec_last_error": (C.c_char_p, []),
        "oec_program_create": (C.c_int, [C.c_char_p, C.POINTER(ProgramOptions), C.POINTER(P)]),
        "oec_program_destroy": (None, [P]),
        "oec_program_get_info": (C.c_int, [P, C.POINTER(ProgramInfo)]),
        "oec_program_input_name": (C.c_int, [P, C.c_int, C.c_char_p, C.c_int]),
        "oec_program_input_range": (C.c_int, [P, C.c_int, I64x3, I64x3, I64x3, I64x3]),
        "oec_program_set_schedule": (C.c_int, [P, C.POINTER(Schedule)]),
        "oec_program_get_schedule": (C.c_int, [P, C.POINTER(Schedule)]),
        "oec_program_apply": (C.c_int, [P, C.POINTER(FieldDesc), C.c_int, C.POINTER(FieldDesc), C.c_int,
                                        I64x3, I64x3, I64x3, C.POINTER(C.c_double), C.c_int, P]),
        "oec_program_apply_host": (C.c_int, [P, C.POINTER(FieldDesc), C.c_int, C.POINTER(FieldDesc), C.c_int,
                                             I64x3, I64x3, I64x3, C.POINTER(C.c_double), C.c_int, P]),
        "oec_program_capture": (C.c_int, [P, C.POINTER(FieldDesc), C.c_int, C.POINTER(FieldDesc), C.c_int,
                                          I64x3, I64x3, I64x3, C.POINTER(C.c_double), C.c_int, C.POINTER(P)]),
        "oec_graph_launch": (C.c_int, [P, P]),
        "oec_graph_kernel_count": (C.c_int, [P]),
        "oec_graph_destroy": (None, [P]),
        "oec_tunedb_open": (C.c_int, [C.c_char_p, C.POINTER(P)]),
        "oec_tunedb_save": (C.c_int, [P, C.c_char_p]),
        "oec_tunedb_count": (C.c_int, [P]),
        "oec_tunedb_close": (None, [P]),
        "oec_tunedb_find": (C.c_int, [P, P, C.POINTER(FieldDesc), C.c_int, C.POINTER(FieldDesc), C.c_int, I64x3,
                                      I64x3, C.POINTER(Schedule), C.POINTER(C.c_double), C.POINTER(C.c_int)]),
        "oec_tunedb_record": (C.c_int, [P, P, C.POINTER(FieldDesc), C.c_int, C.POINTER(FieldDesc), C.c_int, I64x3,
                                        I64x3, C.POINTER(Schedule), C.c_double]),
        "oec_program_autotune_db": (C.c_int, [P, P, C.POINTER(FieldDesc), C.c_int, C.POINTER(FieldDesc), C.c_int,
                                              I64x3, I64x3, I64x3, C.POINTER(C.c_double), C.c_int, C.c_int, P,
                                              C.POINTER(C.c_int)]),
        "oec_program_algorithmic_bytes": (C.c_int, [P, I64x3, I64x3, C.POINTER(C.c_int64)]),
        "oec_device_status": (C.c_int, [P]),
        "oec_device_wait_selftest": (C.c_int, [C.c_int, P]),
        "oec_batch_wait_selftest": (C.c_int, [C.c_int, P]),
        "oec_pstaged_ticket_order": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                               C.POINTER(C.c_int32), C.c_int64, C.POINTER(C.c_int64)]),
        "oec_batch_ticket_order": (C.c_int, [C.c_int32, C.POINTER(C.c_int32), C.c_int32, C.c_int32, C.c_int64,
                                             C.POINTER(C.c_int32), C.c_int64, C.POINTER(C.c_int64)]),
        "oec_costmodel_save": (C.c_int, [P, C.c_char_p]),
        "oec_costmodel_load": (C.c_int, [C.c_char_p, C.POINTER(P)]),
        "oec_program_autotune_model": (C.c_int, [P, P, C.POINTER(FieldDesc), C.c_int, C.POINTER(FieldDesc), C.c_int,
                                                 I64x3, I64x3, I64x3, C.POINTER(C.c_double), C.c_int, C.c_int,
                                                 C.c_int, P, C.POINTER(C.c_float), C.POINTER(C.c_int)]),
        "oec_program_launch_count": (C.c_int, [P]),
        "oec_program_set_timing": (C.c_int, [P, C.c_int]),
        "oec_program_kernel_times": (C.c_int, [P, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int),
                                               C.POINTER(C.c_int)]),
        "oec_hdiff_vadvc_apply_noalloc": (C.c_int, [C.c_int32, C.POINTER(FieldDesc), C.POINTER(FieldDesc), I64x3,
                                                    I64x3, C.c_double, P]),
        "oec_batch_create": (C.c_int, [P, C.POINTER(BatchMember), C.c_int, C.POINTER(C.c_double), C.c_int,
                                       C.POINTER(P)]),
        "oec_batch_apply": (C.c_int, [P, P]),
        "oec_batch_apply_direct": (C.c_int, [P, P]),
        "oec_batch_info": (C.c_int, [P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "oec_batch_destroy": (None, [P]),
        "oec_program_candidates": (C.c_int, [P, C.POINTER(Schedule), C.c_int]),
        "oec_program_autotune": (C.c_int, [P, C.POINTER(FieldDesc), C.c_int, C.POINTER(FieldDesc), C.c_int, I64x3,
                                           I64x3, I64x3, C.POINTER(C.c_double), C.c_int, C.POINTER(Schedule),
                                           C.c_int, C.c_int, P, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
        "oec_program_features": (C.c_int, [P, I64x3, C.c_int64, C.c_int64, C.POINTER(Schedule),
                                           C.POINTER(C.c_float), C.c_int]),
        "oec_costmodel_create": (C.c_int, [C.c_int, C.c_int, C.POINTER(C.c_float), C.POINTER(P)]),
        "oec_costmodel_param_count": (C.c_int, [P]),
        "oec_costmodel_get_params": (C.c_int, [P, C.POINTER(C.c_float), C.c_int]),
        "oec_costmodel_set_params": (C.c_int, [P, C.POINTER(C.c_float), C.c_int]),
        "oec_costmodel_set_normalization": (C.c_int, [P, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
        "oec_costmodel_predict": (C.c_int, [P, P, C.c_int, P, P]),
        "oec_costmodel_gradient": (C.c_int, [P, P, P, C.c_int, P, P, P]),
        "oec_costmodel_train_step": (C.c_int, [P, P, P, C.c_int, C.c_float, C.c_float, C.c_float, C.c_float, P, P]),
        "oec_costmodel_destroy": (None, [P]),
        "oec_program_prepare": (C.c_int, [P, I64x3, C.c_int64, C.c_int64]),
        "oec_program_codegen": (C.c_int, [P, I64x3, C.c_int64, C.c_int64, C.c_int, C.c_char_p, C.c_int64,
                                          C.POINTER(C.c_int64)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(code):
    if code != OEC_OK:
        raise OecError(code, lib().oec_last_error().decode(errors="replace"))
    return code
