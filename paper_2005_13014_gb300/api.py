"""Python face of liboec: argument marshalling between torch tensors and the C
ABI. Every step of a stencil program runs in liboec's CUDA kernels; there is no
Python or CPU execution path. torch provides device memory and streams only.
"""

from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L

_DTYPES = {"f32": L.F32, "f64": L.F64}


def _torch():
    import torch
    return torch


SCHEDULE_KEYS = ("fusion", "staging", "tile_i", "tile_j", "unroll", "k_chunk", "arith", "index_bits", "sweep",
                 "slabs")


def schedule_struct(d: dict) -> L.Schedule:
    s = L.Schedule()
    for k in SCHEDULE_KEYS:
        setattr(s, k, int(d.get(k, 0)))
    return s


def schedule_dict(s: L.Schedule) -> dict:
    return {k: int(getattr(s, k)) for k in SCHEDULE_KEYS}


class Field:
    """A device field: a torch tensor indexed [k, j, i] plus the storage index
    (i, j, k) of the logical origin (paper §IV range notation)."""

    def __init__(self, tensor, origin):
        torch = _torch()
        if tensor.dim() != 3:
            raise ValueError("fields are 3-D tensors indexed [k, j, i]")
        if tensor.dtype not in (torch.float32, torch.float64):
            raise ValueError("fields hold float32 or float64")
        self.tensor = tensor
        self.origin = tuple(int(x) for x in origin)

    @property
    def dtype_code(self):
        return L.F64 if self.tensor.dtype == _torch().float64 else L.F32

    def desc(self) -> L.FieldDesc:
        t = self.tensor
        d = L.FieldDesc()
        d.data = t.data_ptr()
        d.dtype = self.dtype_code
        d.ndim = 3
        d.size = L.I64x3(t.shape[2], t.shape[1], t.shape[0])
        d.stride = L.I64x3(t.stride(2), t.stride(1), t.stride(0))
        d.origin = L.I64x3(*self.origin)
        return d

    def interior(self, lb, ub):
        """View of the tensor over the logical box [lb, ub)."""
        oi, oj, ok = self.origin
        return self.tensor[ok + lb[2]:ok + ub[2], oj + lb[1]:oj + ub[1], oi + lb[0]:oi + ub[0]]


def device_field(arr: np.ndarray, h, dtype="f64", device="cuda", align_bytes=0, pad_i=0, pad_value=0.0):
    """Copy a host storage array [k, j, i] with halo ``h`` (int or (hi, hj, hk))
    to the device. With ``align_bytes`` > 0 the i-rows are padded in front so
    that the first interior point of every row starts on that boundary; ``pad_i``
    extra elements are appended to every row; padding holds ``pad_value``."""
    torch = _torch()
    hi = h if np.isscalar(h) else h[0]
    hj = h if np.isscalar(h) else h[1]
    hk = h if np.isscalar(h) else h[2]
    tdt = torch.float64 if dtype == "f64" else torch.float32
    es = 8 if dtype == "f64" else 4
    front = 0
    if align_bytes:
        a = align_bytes // es
        front = (-hi) % a
    nk, nj, ni = arr.shape
    row = front + ni + pad_i
    if align_bytes:
        row = -(-row // (align_bytes // es)) * (align_bytes // es)
    host = np.full((nk, nj, row), pad_value, dtype=np.float64 if dtype == "f64" else np.float32)
    host[:, :, front:front + ni] = arr
    t = torch.from_numpy(host).to(device)
    return Field(t, (front + hi, hj, hk))


class TuneDB:
    """The tuning database (oec_tunedb_*): best schedules by (program, dtype,
    domain, strides, alignment, device), loaded from and saved to ``path``
    (None: memory only)."""

    def __init__(self, path=None):
        h = C.c_void_p()
        L.check(L.lib().oec_tunedb_open(path.encode() if path else None, C.byref(h)))
        self._h = h

    def __len__(self):
        n = L.lib().oec_tunedb_count(self._h)
        L.check(min(n, 0))
        return n

    def save(self, path=None):
        L.check(L.lib().oec_tunedb_save(self._h, path.encode() if path else None))

    def _fields(self, inputs, outputs):
        ins = (L.FieldDesc * max(1, len(inputs)))(*[f.desc() for f in inputs])
        outs = (L.FieldDesc * max(1, len(outputs)))(*[f.desc() for f in outputs])
        return ins, outs

    def find(self, prog, inputs, outputs, lb, ub):
        """(schedule dict, ms) recorded for this apply, or None."""
        ins, outs = self._fields(inputs, outputs)
        s, ms, found = L.Schedule(), C.c_double(), C.c_int()
        L.check(L.lib().oec_tunedb_find(self._h, prog.handle, ins, len(inputs), outs, len(outputs), L.I64x3(*lb),
                                        L.I64x3(*ub), C.byref(s), C.byref(ms), C.byref(found)))
        return (schedule_dict(s), ms.value) if found.value else None

    def record(self, prog, inputs, outputs, lb, ub, schedule, ms):
        ins, outs = self._fields(inputs, outputs)
        s = schedule_struct(schedule)
        L.check(L.lib().oec_tunedb_record(self._h, prog.handle, ins, len(inputs), outs, len(outputs), L.I64x3(*lb),
                                          L.I64x3(*ub), C.byref(s), float(ms)))

    def close(self):
        if getattr(self, "_h", None) is not None:
            L.lib().oec_tunedb_close(self._h)
            self._h = None

    def __del__(self):
        self.close()


def host_field(arr: np.ndarray, h, dtype="f64", pinned=True, align_bytes=0, pad_i=0, pad_value=0.0):
    """``device_field``'s layout in host memory (page-locked unless
    ``pinned`` is false), for ``Program.apply_host``."""
    f = device_field(arr, h, dtype, device="cpu", align_bytes=align_bytes, pad_i=pad_i, pad_value=pad_value)
    if pinned:
        f.tensor = f.tensor.pin_memory()
    return f


class BoundApply:
    """One program apply with its arguments marshalled once (Program.bind)."""

    def __init__(self, prog, inputs, outputs, lb, ub, halo, params, stream):
        if stream is None:
            stream = _torch().cuda.current_stream().cuda_stream
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self._keep = (prog, list(inputs), list(outputs))   # the fields must outlive the binding
        ins = (L.FieldDesc * max(1, len(inputs)))(*[f.desc() for f in inputs])
        outs = (L.FieldDesc * max(1, len(outputs)))(*[f.desc() for f in outputs])
        par = (C.c_double * max(1, len(params)))(*params)
        self._args = (prog._h, ins, len(inputs), outs, len(outputs), L.I64x3(*lb), L.I64x3(*ub), L.I64x3(*halo),
                      par, len(params), C.c_void_p(stream))
        self._fn = L.lib().oec_program_apply

    def __call__(self):
        rc = self._fn(*self._args)
        if rc:
            L.check(rc)


class CapturedApply:
    """One program apply captured into a CUDA graph (Program.capture): each
    call launches it on a stream. The fields must outlive it; destroy it
    (close, or drop it) before the program."""

    def __init__(self, prog, inputs, outputs, lb, ub, halo, params):
        self._h = None
        self._keep = (prog, list(inputs), list(outputs))
        ins = (L.FieldDesc * max(1, len(inputs)))(*[f.desc() for f in inputs])
        outs = (L.FieldDesc * max(1, len(outputs)))(*[f.desc() for f in outputs])
        par = (C.c_double * max(1, len(params)))(*params)
        h = C.c_void_p()
        L.check(L.lib().oec_program_capture(prog._h, ins, len(inputs), outs, len(outputs), L.I64x3(*lb), L.I64x3(*ub),
                                            L.I64x3(*halo), par, len(params), C.byref(h)))
        self._h = h
        self.kernel_count = L.lib().oec_graph_kernel_count(h)

    def __call__(self, stream=None):
        if stream is None:
            stream = _torch().cuda.current_stream().cuda_stream
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        rc = L.lib().oec_graph_launch(self._h, C.c_void_p(stream))
        if rc:
            L.check(rc)

    def close(self):
        if self._h is not None:
            L.lib().oec_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


class Program:
    """A compiled stencil program (liboec handle)."""

    def __init__(self, source: str, dtype: str = "f64", generic: bool = False):
        self._h = None
        opts = L.ProgramOptions()
        opts.dtype = _DTYPES[dtype]
        opts.flags = 1 if generic else 0
        h = C.c_void_p()
        L.check(L.lib().oec_program_create(source.encode(), C.byref(opts), C.byref(h)))
        self._h = h
        self.dtype = dtype
        info = L.ProgramInfo()
        L.check(L.lib().oec_program_get_info(h, C.byref(info)))
        self.kind = L.KIND_NAMES.get(info.kind, "?")
        self.n_inputs, self.n_outputs, self.n_params = info.n_inputs, info.n_outputs, info.n_params
        self.n_stages = info.n_stages
        buf = C.create_string_buffer(256)
        names = []
        for x in range(self.n_inputs):
            L.check(L.lib().oec_program_input_name(h, x, buf, 256))
            names.append(buf.value.decode())
        self.input_names = names

    def __del__(self):
        if getattr(self, "_h", None) is not None:
            L.lib().oec_program_destroy(self._h)
            self._h = None

    @property
    def handle(self):
        return self._h

    @property
    def schedule(self) -> dict:
        s = L.Schedule()
        L.check(L.lib().oec_program_get_schedule(self._h, C.byref(s)))
        return schedule_dict(s)

    def set_schedule(self, fusion=0, staging=0, tile_i=64, tile_j=4, unroll=1, k_chunk=0, arith=0, index_bits=0,
                     sweep=0, slabs=0):
        s = L.Schedule(fusion, staging, tile_i, tile_j, unroll, k_chunk, arith, index_bits, sweep, slabs)
        L.check(L.lib().oec_program_set_schedule(self._h, C.byref(s)))

    def input_range(self, index, lb, ub):
        lo, hi = L.I64x3(), L.I64x3()
        L.check(L.lib().oec_program_input_range(self._h, index, L.I64x3(*lb), L.I64x3(*ub), lo, hi))
        return tuple(lo), tuple(hi)

    def algorithmic_bytes(self, lb, ub) -> int:
        b = C.c_int64()
        L.check(L.lib().oec_program_algorithmic_bytes(self._h, L.I64x3(*lb), L.I64x3(*ub), C.byref(b)))
        return b.value

    def autotune_model(self, model, inputs, outputs, lb, ub, halo, params=(), top_k=3, reps=3, stream=None):
        """Model-guided selection in liboec: rank every candidate by the cost
        model's prediction, time the top_k (top_k=0: take the best-ranked
        untimed), set the schedule. Returns (index of the pick in
        candidates(), predictions)."""
        n = len(self.candidates())
        ins = (L.FieldDesc * max(1, len(inputs)))(*[f.desc() for f in inputs])
        outs = (L.FieldDesc * max(1, len(outputs)))(*[f.desc() for f in outputs])
        par = (C.c_double * max(1, len(params)))(*params)
        pred = np.zeros(max(1, n), np.float32)
        best = C.c_int(-1)
        L.check(L.lib().oec_program_autotune_model(
            self._h, model._h, ins, len(inputs), outs, len(outputs), L.I64x3(*lb), L.I64x3(*ub), L.I64x3(*halo),
            par, len(params), top_k, reps, C.c_void_p(_stream_handle(stream)),
            pred.ctypes.data_as(C.POINTER(C.c_float)), C.byref(best)))
        return best.value, pred[:n]

    def bind(self, inputs, outputs, lb, ub, halo, params=(), stream=None):
        """Prepare repeated applies of the same fields: the ctypes arguments
        are built once, and calling the result enqueues one apply (a single
        foreign call, for loops where the per-call marshalling of ``apply``
        would cost more than a short kernel)."""
        return BoundApply(self, inputs, outputs, lb, ub, halo, params, stream)

    def capture(self, inputs, outputs, lb, ub, halo, params=()):
        """Capture one apply with these fields into a CUDA graph; calling the
        result launches it (one launch per apply, no argument marshalling)."""
        return CapturedApply(self, inputs, outputs, lb, ub, halo, params)

    def launch_count(self) -> int:
        """Kernels launched by the most recent apply."""
        n = L.lib().oec_program_launch_count(self._h)
        if n < 0:
            L.check(n)
        return n

    def set_timing(self, enable: bool):
        """Record an event before and after every kernel of the following applies."""
        L.check(L.lib().oec_program_set_timing(self._h, 1 if enable else 0))

    def kernel_times(self, cap=1 << 20):
        """Durations (ms) of the recorded applies' kernels: numpy [n_applies, n_kernels]."""
        ms = np.zeros(cap, np.float32)
        na, nk = C.c_int(), C.c_int()
        L.check(L.lib().oec_program_kernel_times(self._h, ms.ctypes.data_as(C.POINTER(C.c_float)), cap,
                                                 C.byref(na), C.byref(nk)))
        return ms[:na.value * nk.value].reshape(na.value, nk.value).copy()

    def prepare(self, extent, sj, sk):
        """Compile and load generated kernels for this shape ahead of time."""
        L.check(L.lib().oec_program_prepare(self._h, L.I64x3(*extent), sj, sk))

    def candidates(self):
        """The schedules the autotuner tries for this program (list of dicts)."""
        n = L.lib().oec_program_candidates(self._h, None, 0)
        L.check(min(n, 0))
        arr = (L.Schedule * n)()
        L.lib().oec_program_candidates(self._h, arr, n)
        return [schedule_dict(x) for x in arr]

    def autotune(self, inputs, outputs, lb, ub, halo, params=(), candidates=None, reps=5, stream=None):
        """Time candidate schedules (default: all) on these fields; the fastest
        becomes the program's schedule. Returns (times_ms list, best index)."""
        cands = candidates if candidates is not None else self.candidates()
        arr = (L.Schedule * len(cands))(*[schedule_struct(c) for c in cands])
        times = (C.c_double * len(cands))()
        best = C.c_int(-1)
        ins = (L.FieldDesc * max(1, len(inputs)))(*[f.desc() for f in inputs])
        outs = (L.FieldDesc * max(1, len(outputs)))(*[f.desc() for f in outputs])
        par = (C.c_double * max(1, len(params)))(*params)
        L.check(L.lib().oec_program_autotune(self._h, ins, len(inputs), outs, len(outputs), L.I64x3(*lb),
                                             L.I64x3(*ub), L.I64x3(*halo), par, len(params), arr, len(cands), reps,
                                             C.c_void_p(_stream_handle(stream)), times, C.byref(best)))
        return list(times), best.value

    def features(self, extent, sj, sk, schedule: dict):
        """Cost-model features of this program on a domain extent with the given
        field strides and schedule (numpy float32 array)."""
        n = L.lib().oec_program_features(self._h, L.I64x3(*extent), sj, sk, C.byref(schedule_struct(schedule)), None, 0)
        L.check(min(n, 0))
        out = (C.c_float * n)()
        L.check(min(0, L.lib().oec_program_features(self._h, L.I64x3(*extent), sj, sk,
                                                    C.byref(schedule_struct(schedule)), out, n)))
        return np.frombuffer(out, dtype=np.float32).copy()

    def generated_source(self, extent, sj, sk, compile=False) -> str:
        """CUDA C++ generated for this program (all fusion x unroll variants);
        with compile=True it is also compiled by NVRTC (no GPU needed)."""
        n = C.c_int64()
        L.check(L.lib().oec_program_codegen(self._h, L.I64x3(*extent), sj, sk, 0, None, 0, C.byref(n)))
        buf = C.create_string_buffer(n.value + 1)
        L.check(L.lib().oec_program_codegen(self._h, L.I64x3(*extent), sj, sk, 1 if compile else 0, buf,
                                            n.value + 1, C.byref(n)))
        return buf.value.decode()

    def apply(self, inputs, outputs, lb, ub, halo, params=(), stream=None):
        """Enqueue the program on ``stream`` (torch.cuda.Stream or raw handle;
        default: torch's current stream). Fields are ``Field`` objects."""
        ins = (L.FieldDesc * max(1, len(inputs)))(*[f.desc() for f in inputs])
        outs = (L.FieldDesc * max(1, len(outputs)))(*[f.desc() for f in outputs])
        par = (C.c_double * max(1, len(params)))(*params)
        if stream is None:
            stream = _torch().cuda.current_stream().cuda_stream
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        L.check(L.lib().oec_program_apply(self._h, ins, len(inputs), outs, len(outputs), L.I64x3(*lb),
                                          L.I64x3(*ub), L.I64x3(*halo), par, len(params), C.c_void_p(stream)))

    def autotune_db(self, db, inputs, outputs, lb, ub, halo, params=(), reps=5, stream=None):
        """Autotune through a ``TuneDB``: a recorded case takes its schedule
        without timing; otherwise every candidate is timed and the fastest
        recorded. Returns True when the schedule came from the database."""
        ins = (L.FieldDesc * max(1, len(inputs)))(*[f.desc() for f in inputs])
        outs = (L.FieldDesc * max(1, len(outputs)))(*[f.desc() for f in outputs])
        par = (C.c_double * max(1, len(params)))(*params)
        hit = C.c_int()
        L.check(L.lib().oec_program_autotune_db(self._h, db._h, ins, len(inputs), outs, len(outputs), L.I64x3(*lb),
                                                L.I64x3(*ub), L.I64x3(*halo), par, len(params), reps,
                                                C.c_void_p(_stream_handle(stream)), C.byref(hit)))
        return bool(hit.value)

    def apply_host(self, inputs, outputs, lb, ub, halo, params=(), stream=None):
        """``apply`` with fields in host memory (``host_field``): the library
        copies the inputs in and the outputs' domain back, ordered on
        ``stream``; the host outputs are complete after it is synchronised."""
        ins = (L.FieldDesc * max(1, len(inputs)))(*[f.desc() for f in inputs])
        outs = (L.FieldDesc * max(1, len(outputs)))(*[f.desc() for f in outputs])
        par = (C.c_double * max(1, len(params)))(*params)
        L.check(L.lib().oec_program_apply_host(self._h, ins, len(inputs), outs, len(outputs), L.I64x3(*lb),
                                               L.I64x3(*ub), L.I64x3(*halo), par, len(params),
                                               C.c_void_p(_stream_handle(stream))))


def _stream_handle(stream):
    if stream is None:
        return _torch().cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else stream


class Batch:
    """An ensemble of domains run by one persistent launch (replayed from a
    CUDA graph). ``members``: list of (inputs, outputs, lb, ub, halo)."""

    def __init__(self, program: Program, members, params=()):
        self._h = None
        self.program = program
        self._keep = []
        arr = (L.BatchMember * len(members))()
        for x, (ins, outs, lb, ub, halo) in enumerate(members):
            di = (L.FieldDesc * len(ins))(*[f.desc() for f in ins])
            do = (L.FieldDesc * len(outs))(*[f.desc() for f in outs])
            self._keep += [di, do, ins, outs]
            arr[x].in_ = C.cast(di, C.POINTER(L.FieldDesc))
            arr[x].out = C.cast(do, C.POINTER(L.FieldDesc))
            arr[x].lb = L.I64x3(*lb)
            arr[x].ub = L.I64x3(*ub)
            arr[x].halo = L.I64x3(*halo)
        par = (C.c_double * max(1, len(params)))(*params)
        h = C.c_void_p()
        L.check(L.lib().oec_batch_create(program.handle, arr, len(members), par, len(params), C.byref(h)))
        self._h = h
        ni, nc = C.c_int(), C.c_int()
        L.check(L.lib().oec_batch_info(h, C.byref(ni), C.byref(nc)))
        self.n_items, self.n_ctas = ni.value, nc.value

    def apply(self, stream=None, graph=True):
        fn = L.lib().oec_batch_apply if graph else L.lib().oec_batch_apply_direct
        L.check(fn(self._h, C.c_void_p(_stream_handle(stream))))

    def __del__(self):
        if getattr(self, "_h", None) is not None:
            L.lib().oec_batch_destroy(self._h)
            self._h = None
