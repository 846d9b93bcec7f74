"""Mixed precision against the FP64 oracle, per output field: hdiff and the
fastwaves-like program at 256x256x80 (halo 3), and hdiff+vadvc at 128x128x80
with FP32 fields and an FP64 or double-float column recurrence. Every variant
reads the same seeded FP64 inputs (FP32 storage rounds them on the way in, as
a program that stores its fields in FP32 would), and each output field is
compared with the oracle's FP64 result on the unrounded inputs by two
measures:

  normwise   max|x - r| / max|r|
  pointwise  max |x - r| / max(|r|, 1e-3 max|r|)

Bounds: the normwise error within the FP64 (1e-13) and FP32 (1e-5)
tolerances; the pointwise one within 1e3 times those, the most the floor of
1e-3 max|r| allows for a result within the normwise bound.

hdiff's flux limiter is discontinuous: where two neighbouring inputs agree to
within FP32 rounding, rounding them can flip its sign test, and the flux there
is kept instead of zeroed (or the reverse), an O(coeff * flux) change that no
arithmetic precision undoes. For FP32 storage the test therefore also runs the
oracle on the FP32-rounded inputs: the kernels must match that result at every
point (within 1e-5), and the unrounded oracle at every point where rounding
the inputs alone moves the oracle's own FP64 result by less than the
tolerance. The points where it moves more (limiter flips and, through the
column solve, the rest of their columns) are counted and reported with the
error over all points. The measured figures print one JSON line per variant
(run with -s to see them)."""

import json

import numpy as np
import pytest

from conftest import TOL, rel_err
from oracle import stencils as S
from paper_2005_13014_gb300 import inputs, programs

torch = pytest.importorskip("torch")

N3, N_HV, H = (256, 256, 80), (128, 128, 80), 3


def pointwise_err(x, r):
    x = np.asarray(x, np.float64)
    r = np.asarray(r, np.float64)
    m = np.max(np.abs(r))
    den = np.maximum(np.abs(r), 1e-3 * m if m > 0 else 1.0)
    return float(np.max(np.abs(x - r) / den))


def _run(src, names, f, n, params, dtype, sched, n_out):
    from paper_2005_13014_gb300.api import Program, device_field
    p = Program(src, dtype)
    p.set_schedule(**sched)
    d = [device_field(f[k], H, dtype, align_bytes=16) for k in names]
    o = [device_field(np.zeros_like(f[names[0]]), H, dtype, align_bytes=16) for _ in range(n_out)]
    p.apply(d, o, (0, 0, 0), n, (H, H, H), params)
    torch.cuda.synchronize()
    return [x.interior((0, 0, 0), n).cpu().numpy().astype(np.float64) for x in o]


def _check(label, dtype, arith, sched, outs, refs, refs32, fields):
    """refs: the oracle on the FP64 inputs; refs32: on the FP32-rounded inputs."""
    rec = {"case": label, "dtype": dtype, "arith": arith, "schedule": sched,
           "normwise": {}, "pointwise": {}}
    for f_, x, r, r32 in zip(fields, outs, refs, refs32):
        m = np.max(np.abs(r))
        rec["normwise"][f_] = rel_err(x, r)
        rec["pointwise"][f_] = pointwise_err(x, r)
        if dtype == "f64":
            assert rec["normwise"][f_] <= TOL[dtype], (label, f_, rec["normwise"][f_])
            assert rec["pointwise"][f_] <= 1e3 * TOL[dtype], (label, f_, rec["pointwise"][f_])
            continue
        assert rel_err(x, r32) <= TOL[dtype], (label, f_, "vs the oracle on rounded inputs")
        moved = np.abs(r32 - r) > TOL[dtype] * m        # the oracle itself moves there
        keep = ~moved
        away = float(np.max(np.abs(x - r)[keep]) / m) if keep.any() else 0.0
        away_p = pointwise_err(x[keep], r[keep]) if keep.any() else 0.0
        rec.setdefault("points_moved_by_input_rounding", {})[f_] = int(moved.sum())
        rec.setdefault("normwise_elsewhere", {})[f_] = away
        rec.setdefault("pointwise_elsewhere", {})[f_] = away_p
        assert away <= TOL[dtype], (label, f_, away)
        assert away_p <= 1e3 * TOL[dtype], (label, f_, away_p)
    print(json.dumps(rec))


# (dtype, arith, schedule): the schedules the autotuner picks for each form
HDIFF_VARIANTS = [
    ("f32", 0, dict(fusion=0, staging=3, tile_i=32, tile_j=8, unroll=2, k_chunk=4)),
    ("f64", 0, dict(fusion=0, staging=1, tile_i=64, tile_j=8, k_chunk=1)),
    ("f64", 1, dict(fusion=0, staging=1, tile_i=32, tile_j=8, k_chunk=2)),
    ("f64", 2, dict(fusion=0, staging=1, tile_i=32, tile_j=8, unroll=2, k_chunk=2)),
]
FW_VARIANTS = [
    ("f32", 0, dict(fusion=0, staging=4, tile_i=32, tile_j=4, k_chunk=8)),
    ("f64", 0, dict(fusion=0, staging=1, tile_i=32, tile_j=8, k_chunk=4)),
    ("f64", 1, dict(fusion=0, staging=1, tile_i=32, tile_j=8, k_chunk=4)),
]
HV_VARIANTS = [
    ("f32", 0, dict(fusion=1, staging=3, tile_i=32, tile_j=4, k_chunk=8)),
    ("f32", 1, dict(fusion=1, staging=3, tile_i=32, tile_j=8, unroll=2, k_chunk=8)),
    ("f64", 2, dict(fusion=1, staging=0, tile_i=32, tile_j=8, k_chunk=4)),
    ("f64", 0, dict(fusion=1, staging=0, tile_i=32, tile_j=8, k_chunk=4)),
]


def _rounded(f):
    return {k: v.astype(np.float32).astype(np.float64) for k, v in f.items()}


def _hdiff_oracle(f):
    return [S.hdiff(S.Grid.storage(f["in"], H), S.Grid.storage(f["coeff"], H), (0, 0, 0), N3)]


def _fastwaves_oracle(f):
    G = {k: S.Grid.storage(v, H) for k, v in f.items()}
    return list(S.fastwaves(G, (0, 0, 0), N3, 0.5, 0.0625))


def _hv_oracle(f):
    G = {k: S.Grid.storage(v, H) for k, v in f.items()}
    return list(S.hdiff_vadvc(G["u"], G["v"], G["w"], G["coeff"], (0, 0, 0), N_HV, 2.0))


# (fields, oracle on them, oracle on the FP32-rounded fields); seed 41 has a
# pair of neighbouring inputs that FP32 rounding reorders for the limiter
@pytest.fixture(scope="module")
def hdiff_case():
    f = inputs.hdiff_fields(*N3, H, seed=41)
    return f, _hdiff_oracle(f), _hdiff_oracle(_rounded(f))


@pytest.fixture(scope="module")
def fastwaves_case():
    f = inputs.fastwaves_fields(*N3, H, seed=42)
    return f, _fastwaves_oracle(f), _fastwaves_oracle(_rounded(f))


@pytest.fixture(scope="module")
def hv_case():
    f = inputs.hdiff_vadvc_fields(*N_HV, H, seed=43)
    return f, _hv_oracle(f), _hv_oracle(_rounded(f))


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,arith,sched", HDIFF_VARIANTS, ids=str)
def test_hdiff_256x256x80_per_field(hdiff_case, dtype, arith, sched):
    f, refs, refs32 = hdiff_case
    s = dict(sched, arith=arith)
    outs = _run(programs.HDIFF, ("in", "coeff"), f, N3, [], dtype, s, 1)
    _check("hdiff 256x256x80", dtype, arith, s, outs, refs, refs32, ["out"])


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,arith,sched", FW_VARIANTS, ids=str)
def test_fastwaves_256x256x80_per_field(fastwaves_case, dtype, arith, sched):
    f, refs, refs32 = fastwaves_case
    s = dict(sched, arith=arith)
    outs = _run(programs.FASTWAVES, inputs.FASTWAVES_NAMES, f, N3, [0.5, 0.0625], dtype, s, 2)
    _check("fastwaves 256x256x80", dtype, arith, s, outs, refs, refs32, ["u_out", "v_out"])


@pytest.mark.gpu
@pytest.mark.parametrize("dtype,arith,sched", HV_VARIANTS, ids=str)
def test_hdiff_vadvc_128x128x80_per_field(hv_case, dtype, arith, sched):
    f, refs, refs32 = hv_case
    s = dict(sched, arith=arith)
    outs = _run(programs.HDIFF_VADVC, ("u", "v", "w", "coeff"), f, N_HV, [2.0], dtype, s, 2)
    _check("hdiff+vadvc 128x128x80", dtype, arith, s, outs, refs, refs32, ["u_out", "v_out"])


def test_pointwise_measure_on_a_constructed_case():
    """The pointwise measure divides by the floor where |r| is small: an
    error of 1e-6 at a point where r = 0, in a field whose largest value is 2,
    gives 1e-6 / 2e-3 = 5e-4, and 1e-6 / 1.5 where r = 1.5."""
    r = np.array([0.0, 1.5, -2.0])
    assert pointwise_err(r + np.array([1e-6, 0, 0]), r) == pytest.approx(5e-4)
    assert pointwise_err(r + np.array([0, 1e-6, 0]), r) == pytest.approx(1e-6 / 1.5)
