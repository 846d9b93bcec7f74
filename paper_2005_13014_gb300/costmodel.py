"""Learned cost model for schedule selection (no counterpart in the paper,
which tunes unroll factors empirically and always fuses everything, §VII-C).

An FP32 MLP (42 features -> 64 -> 64 -> 1, ReLU) predicts, for a (stencil
program, domain, schedule) triple, log(t / t_best): how much slower the
schedule is than the program's fastest one (selection only ranks the schedules
of one program, so the program's absolute cost level need not be learned). Features come from
liboec (oec_program_features: program structure, domain, schedule, and the
per-point loads/operations/stores of the code generated for that schedule);
timings come from liboec's exhaustive autotuner (oec_program_autotune); the
network is trained and evaluated by liboec's CUDA kernels (oec_costmodel_*).
This module only moves arrays between those calls.

Selection ("model top-k"): rank a program's candidate schedules by predicted
time, measure the k best-ranked (k = 0: take the first unmeasured), keep the
fastest. Exhaustive autotuning (every candidate timed) is the fallback and the
ground truth against which the model's regret is reported.
"""

from __future__ import annotations

import ctypes as C
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import _lib as L
from .api import Program, device_field

N_FEATURES = 42

# the features oec_program_features writes, in order (per point: of the
# generated code for the schedule; l2_*: log2)
FEATURE_NAMES = (
    "stages", "inputs", "outputs", "accesses", "arith_ops", "selects", "min_max", "divisions",
    "max_offset_i", "max_offset_j", "max_offset_k", "depth", "halo_i", "halo_j", "halo_k", "input_amplification",
    "l2_ni", "l2_nj", "l2_nk", "l2_points", "element_bytes", "fuse_inline", "fuse_none", "fuse_partial",
    "l2_unroll", "l2_tile_i", "l2_tile_j", "l2_tile_threads", "kernels", "loads_per_point", "ops_per_point",
    "stores_per_point", "temp_bytes_per_point", "l2_max_blocks", "tile_efficiency_i", "tile_efficiency_j",
    "bytes_per_point", "inline_ops_per_point", "ops_over_unfused_ops", "materialised_stages", "waves",
    "l2_total_ops")
F = {name: x for x, name in enumerate(FEATURE_NAMES)}
assert len(FEATURE_NAMES) == N_FEATURES


def _torch():
    import torch
    return torch


def _ptr(t):
    return C.c_void_p(t.data_ptr())


class CostModel:
    def __init__(self, n_features=N_FEATURES, hidden=64, params=None):
        self._h = None
        self.n_features, self.hidden = n_features, hidden
        arr = None
        if params is not None:
            flat = np.ascontiguousarray(params, dtype=np.float32)
            arr = flat.ctypes.data_as(C.POINTER(C.c_float))
        h = C.c_void_p()
        L.check(L.lib().oec_costmodel_create(n_features, hidden, arr, C.byref(h)))
        self._h = h
        self.param_count = L.lib().oec_costmodel_param_count(h)
        self._loss = _torch().zeros(1, dtype=_torch().float32, device="cuda")

    @staticmethod
    def flatten(p: dict) -> np.ndarray:
        """Flat parameter vector W1, b1, W2, b2, W3, b3 (float32)."""
        return np.concatenate([np.asarray(p[k], np.float32).ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])

    def get_params(self) -> np.ndarray:
        out = np.empty(self.param_count, np.float32)
        L.check(L.lib().oec_costmodel_get_params(self._h, out.ctypes.data_as(C.POINTER(C.c_float)), self.param_count))
        return out

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, dtype=np.float32)
        L.check(L.lib().oec_costmodel_set_params(self._h, flat.ctypes.data_as(C.POINTER(C.c_float)), self.param_count))

    def set_normalization(self, mu, sigma):
        mu = np.ascontiguousarray(mu, dtype=np.float32)
        sigma = np.ascontiguousarray(sigma, dtype=np.float32)
        self.mu, self.sigma = mu, sigma
        L.check(L.lib().oec_costmodel_set_normalization(self._h, mu.ctypes.data_as(C.POINTER(C.c_float)),
                                                         sigma.ctypes.data_as(C.POINTER(C.c_float))))

    def save(self, path):
        """Checkpoint file (liboec's format: dimensions, parameters, standardisation)."""
        L.check(L.lib().oec_costmodel_save(self._h, str(path).encode()))

    @classmethod
    def load(cls, path):
        h = C.c_void_p()
        L.check(L.lib().oec_costmodel_load(str(path).encode(), C.byref(h)))
        m = cls.__new__(cls)
        m._h = h
        m.param_count = L.lib().oec_costmodel_param_count(h)
        m.hidden = None
        m.n_features = None
        m._loss = _torch().zeros(1, dtype=_torch().float32, device="cuda")
        return m

    def predict(self, X):
        """X: device float32 tensor [n, F] -> device tensor [n]."""
        torch = _torch()
        y = torch.empty(X.shape[0], dtype=torch.float32, device=X.device)
        L.check(L.lib().oec_costmodel_predict(self._h, _ptr(X), X.shape[0], _ptr(y),
                                              C.c_void_p(torch.cuda.current_stream().cuda_stream)))
        return y

    def gradient(self, X, t):
        torch = _torch()
        g = torch.empty(self.param_count, dtype=torch.float32, device=X.device)
        L.check(L.lib().oec_costmodel_gradient(self._h, _ptr(X), _ptr(t), X.shape[0], _ptr(g), _ptr(self._loss),
                                               C.c_void_p(torch.cuda.current_stream().cuda_stream)))
        return g, self._loss

    def train_step(self, X, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        L.check(L.lib().oec_costmodel_train_step(self._h, _ptr(X), _ptr(t), X.shape[0], lr, beta1, beta2, eps,
                                                 _ptr(self._loss),
                                                 C.c_void_p(_torch().cuda.current_stream().cuda_stream)))
        return self._loss

    def fit(self, X, t, epochs=200, batch=512, lr=1e-3, seed=0):
        """Mini-batch Adam over (X, t) (device tensors); returns per-epoch mean loss."""
        torch = _torch()
        n = X.shape[0]
        rng = np.random.default_rng(seed)
        losses = []
        for _ in range(epochs):
            perm = torch.from_numpy(rng.permutation(n)).to(X.device)
            acc = torch.zeros(1, device=X.device)
            nb = 0
            for s in range(0, n, batch):
                idx = perm[s:s + batch]
                acc += self.train_step(X[idx].contiguous(), t[idx].contiguous(), lr=lr)
                nb += 1
            losses.append(float(acc.item()) / nb)
        return losses

    def __del__(self):
        if getattr(self, "_h", None) is not None:
            L.lib().oec_costmodel_destroy(self._h)
            self._h = None


# ---------------------------------------------------------------- measurement

class DagCase:
    """A generated program with device fields on a domain, ready to time."""

    def __init__(self, src, shape, dtype="f32", halo=(8, 8, 4), seed=0):
        from . import inputs
        self.src, self.shape, self.dtype, self.halo = src, tuple(shape), dtype, tuple(halo)
        self.program = Program(src, dtype, generic=True)
        n, h = self.shape, self.halo
        self.inputs = []
        for x in range(self.program.n_inputs):
            arr = inputs.field_uniform(n, h, -1.0, 1.0, seed * 16 + x)
            self.inputs.append(device_field(arr, h, dtype))
        self.outputs = [device_field(np.zeros_like(arr), h, dtype) for _ in range(self.program.n_outputs)]
        t = self.inputs[0].tensor
        self.sj, self.sk = t.stride(1), t.stride(0)

    def prepare(self):
        self.program.prepare(self.shape, self.sj, self.sk)

    def features(self, candidates):
        return np.stack([self.program.features(self.shape, self.sj, self.sk, c) for c in candidates])

    def time(self, candidates, reps=3):
        times, _ = self.program.autotune(self.inputs, self.outputs, (0, 0, 0), self.shape, self.halo,
                                         candidates=candidates, reps=reps)
        return np.array(times)


def measure_dags(seeds, shape, dtype="f32", reps=3, threads=8, log=None):
    """For each DAG seed: candidate features and exhaustive timings. shape: one
    domain for every program, or a function of the seed (e.g.
    inputs.dag_shape)."""
    from . import inputs
    cases = [DagCase(inputs.random_dag(s), shape(s) if callable(shape) else shape, dtype, seed=s) for s in seeds]
    t0 = time.time()
    with ThreadPoolExecutor(max_workers=threads) as ex:       # NVRTC compiles in parallel
        list(ex.map(lambda c: c.prepare(), cases))
    t_compile = time.time() - t0
    cands = cases[0].program.candidates()
    out = []
    t0 = time.time()
    for c in cases:
        out.append((c.features(cands), c.time(cands, reps)))
    if log is not None:
        log["compile_s"] = t_compile
        log["timing_s"] = time.time() - t0
    return cands, out, cases


def targets(times_ms, points):
    """Absolute target: log of milliseconds per grid point."""
    return np.log(np.maximum(times_ms, 1e-6) / points)


def relative_targets(times_ms):
    """Per-program target: log(t / t_best) over the program's candidates
    (selection only ranks schedules of one program, so the program's own cost
    level need not be learned). Non-positive times (candidates that cannot
    run) are dropped by the caller."""
    t = np.asarray(times_ms, np.float64)
    return np.log(t / t[t > 0].min())


def training_set(features, times):
    """Stack (features, relative target) over programs; features [P, C, F],
    times [P, C]."""
    X, y = [], []
    for f, t in zip(features, times):
        ok = t > 0
        X.append(f[ok])
        y.append(relative_targets(t)[ok])
    return np.concatenate(X).astype(np.float32), np.concatenate(y).astype(np.float32)


def best_fixed(times, ok_mask=None):
    """Index of the single schedule with the lowest geometric-mean relative
    time over the given programs (a data-driven fixed schedule)."""
    t = np.where(times > 0, times, np.inf)
    rel = np.log(t / t.min(axis=1, keepdims=True))
    return int(np.argmin(np.mean(rel, axis=0)))


def select(model, feats_dev, k=1):
    """Indices of the k candidates with the lowest predicted time."""
    pred = model.predict(feats_dev).cpu().numpy()
    return np.argsort(pred, kind="stable")[:k], pred


def regret_stats(r):
    r = np.asarray(r)
    return {"mean": float(np.mean(r)), "median": float(np.median(r)), "p90": float(np.percentile(r, 90)),
            "max": float(np.max(r)), "frac_within_5pct": float(np.mean(r <= 0.05))}


def roofline_seconds_per_point(features, hbm_bytes_per_s, ops_per_s):
    """Roofline estimate per grid point of each candidate (rows of a feature
    matrix): max(bytes per point / HBM bandwidth, operations per point /
    operation rate)."""
    f = np.asarray(features, np.float64)
    return np.maximum(f[:, F["bytes_per_point"]] / hbm_bytes_per_s, f[:, F["ops_per_point"]] / ops_per_s)


def greedy_fusion(features, candidates, hbm_bytes_per_s, ops_per_s, tile=(64, 4), unroll=1, usable=None):
    """Non-learned baseline between inlining everything and the learned model
    (the paper inlines every stage, §V-A): among the candidates at the given
    tile and unroll, the fusion choice (inline, none, partial) whose roofline
    estimate is lowest. Returns that candidate's index (ties: the first in
    candidate order). usable (optional boolean mask): candidates that can run."""
    est = roofline_seconds_per_point(features, hbm_bytes_per_s, ops_per_s)
    pool = [x for x, c in enumerate(candidates)
            if c["tile_i"] == tile[0] and c["tile_j"] == tile[1] and c["unroll"] == unroll
            and (usable is None or usable[x])]
    if not pool:
        raise ValueError("no candidate at the given tile and unroll")
    return min(pool, key=lambda x: (est[x], x))
