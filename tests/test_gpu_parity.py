"""GPU parity: every hand-written kernel variant against the FP64 oracle,
element by element, through the C ABI. Sizes span several tiles with ragged
tails, and the full workload sizes; tolerances are the normwise relative
errors 1e-13 (FP64) and 1e-5 (FP32 fields, oracle fed the FP32-rounded inputs).
Poisoned halos check that no kernel reads outside the inferred input ranges or
writes outside the domain."""

import numpy as np
import pytest

from conftest import TOL, rel_err
from oracle import stencils as S
from paper_2005_13014_gb300 import inputs, programs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _round(arr, dtype):
    return arr.astype(np.float32).astype(np.float64) if dtype == "f32" else arr


def _dev(arr, h, dtype, align=0, pad_value=0.0):
    from paper_2005_13014_gb300.api import device_field
    return device_field(arr, h, dtype, align_bytes=align, pad_value=pad_value)


def _prog(src, dtype, sched=None):
    from paper_2005_13014_gb300.api import Program
    p = Program(src, dtype)
    if sched:
        p.set_schedule(**sched)
    return p


HDIFF_SCHEDS = (
    [dict(fusion=1)]
    + [dict(fusion=0, staging=1, tile_i=a, tile_j=b, k_chunk=kc)
       for (a, b) in [(32, 4), (32, 8), (64, 2), (64, 4), (64, 8), (128, 2), (128, 4)] for kc in (0, 3)]
    + [dict(fusion=0, staging=0, tile_i=a, tile_j=b, unroll=u, k_chunk=kc)
       for (a, b, u) in [(32, 4, 1), (64, 4, 2), (32, 8, 4), (128, 4, 4), (64, 1, 1)] for kc in (0, 2)]
    + [dict(fusion=0, staging=2, tile_i=a, tile_j=b, k_chunk=kc)
       for (a, b) in [(32, 4), (32, 8), (64, 4), (64, 8), (128, 2), (128, 4)] for kc in (0, 3)]
)

# vectorised warp rows: need 16-byte aligned rows
WARP_SCHEDS = [dict(fusion=0, staging=st, tile_i=32, tile_j=4 * u, unroll=u, k_chunk=kc) for st in (3, 4)
               for u in (1, 2, 4) for kc in (0, 3)]


def _hdiff_case(n, h, dtype, sched, align=0, lb=None, ub=None, poison=True):
    f = inputs.hdiff_fields(*n, h, seed=31)
    fin = _round(f["in"], dtype)
    fco = _round(f["coeff"], dtype)
    lb = lb or (0, 0, 0)
    ub = ub or n
    if poison:
        # NaN outside the inferred input range: [lb-2, ub+2) in i/j for in, [lb, ub) for coeff
        pin = np.full_like(fin, np.nan)
        sl = (slice(h + lb[2], h + ub[2]), slice(h + lb[1] - 2, h + ub[1] + 2), slice(h + lb[0] - 2, h + ub[0] + 2))
        pin[sl] = fin[sl]
        pco = np.full_like(fco, np.nan)
        sl2 = (slice(h + lb[2], h + ub[2]), slice(h + lb[1], h + ub[1]), slice(h + lb[0], h + ub[0]))
        pco[sl2] = fco[sl2]
    else:
        pin, pco = fin, fco
    p = _prog(programs.HDIFF, dtype, sched)
    din, dco = _dev(pin, h, dtype, align), _dev(pco, h, dtype, align)
    sentinel = 12345.0
    dout = _dev(np.full_like(fin, sentinel), h, dtype, align, pad_value=sentinel)
    p.apply([din, dco], [dout], lb, ub, (h, h, h))
    torch.cuda.synchronize()
    full = dout.tensor.cpu().numpy().astype(np.float64)
    oi, oj, ok = dout.origin
    got = full[ok + lb[2]:ok + ub[2], oj + lb[1]:oj + ub[1], oi + lb[0]:oi + ub[0]]
    ref = S.hdiff(S.Grid.storage(fin, h), S.Grid.storage(fco, h), lb, ub)
    assert np.all(np.isfinite(got))
    mask = np.ones(full.shape, bool)
    mask[ok + lb[2]:ok + ub[2], oj + lb[1]:oj + ub[1], oi + lb[0]:oi + ub[0]] = False
    assert np.all(full[mask] == sentinel), "write outside the domain"
    return rel_err(got, ref)


# (dtype, arith): FP64 programs in native FP64 and in double-float; FP32 native
PRECISIONS = [("f64", 0), ("f64", 1), ("f32", 0)]
HV_PRECISIONS = [("f64", 0), ("f64", 1), ("f32", 0), ("f32", 1)]


def _with(sched, arith):
    s = dict(sched)
    s["arith"] = arith
    return s


@pytest.mark.parametrize("sched", HDIFF_SCHEDS, ids=str)
@pytest.mark.parametrize("dtype,arith", PRECISIONS)
def test_hdiff_ragged(sched, dtype, arith):
    assert _hdiff_case((37, 29, 5), 2, dtype, _with(sched, arith)) <= TOL[dtype]


@pytest.mark.parametrize("n", [(37, 29, 5), (130, 9, 3), (257, 6, 2), (3, 40, 2)], ids=str)
@pytest.mark.parametrize("sched", WARP_SCHEDS, ids=str)
@pytest.mark.parametrize("dtype,arith", PRECISIONS)
def test_hdiff_vector_rows(sched, dtype, arith, n):
    """Vectorised warp rows, loaded directly (staging 3) or by TMA into a
    shared-memory ring (staging 4): ragged warps (partial vectors at the end
    of the input range and of the domain), edge lanes inside and outside the
    range, poisoned halos; no bounded wait gives up."""
    from paper_2005_13014_gb300 import _lib as L
    assert _hdiff_case(n, 2, dtype, _with(sched, arith), align=16) <= TOL[dtype]
    assert L.lib().oec_device_status(None) == 0


def test_hdiff_vector_rows_need_alignment():
    from paper_2005_13014_gb300._lib import OecError
    with pytest.raises(OecError, match="16-byte aligned"):
        _hdiff_case((37, 29, 5), 3, "f32", WARP_SCHEDS[0], align=0)


@pytest.mark.parametrize("sched", [dict(fusion=1), dict(fusion=0, staging=1, tile_i=64, tile_j=4, k_chunk=2),
                                   dict(fusion=0, staging=0, tile_i=64, tile_j=4, unroll=2)], ids=str)
@pytest.mark.parametrize("arith", [0, 1])
def test_hdiff_config_64x64x60_f64(sched, arith):
    assert _hdiff_case((64, 64, 60), 2, "f64", _with(sched, arith)) <= TOL["f64"]


@pytest.mark.parametrize("dtype,arith", PRECISIONS)
def test_hdiff_256x256x80_halo3(dtype, arith):
    sched = dict(fusion=0, staging=1, tile_i=64, tile_j=4, k_chunk=2, arith=arith)
    assert _hdiff_case((256, 256, 80), 3, dtype, sched, poison=False) <= TOL[dtype]


def test_hdiff_subdomain_and_aligned_rows():
    assert _hdiff_case((40, 30, 6), 3, "f64", None, lb=(5, 3, 1), ub=(33, 27, 5)) <= TOL["f64"]
    assert _hdiff_case((40, 30, 6), 2, "f32", dict(fusion=0, staging=0, tile_i=32, tile_j=4, unroll=4),
                       align=128) <= TOL["f32"]


def test_hdiff_single_point_and_line():
    assert _hdiff_case((1, 1, 1), 2, "f64", None) <= TOL["f64"]
    assert _hdiff_case((130, 1, 2), 2, "f64", dict(fusion=0, staging=0, tile_i=64, tile_j=4, unroll=4)) <= TOL["f64"]


# ---------------------------------------------------------------- hdiff+vadvc

HV_SCHEDS = [dict(fusion=1)] + [dict(fusion=0, staging=1, tile_i=a, tile_j=b)
                                for a, b in [(16, 4), (32, 2), (8, 8), (32, 4), (8, 4), (16, 2)]]


def _hv_case(n, h, dtype, sched, dtr=2.0):
    f = inputs.hdiff_vadvc_fields(*n, h, seed=32)
    g = {k: _round(v, dtype) for k, v in f.items()}
    p = _prog(programs.HDIFF_VADVC, dtype, sched)
    d = {k: _dev(v, h, dtype) for k, v in g.items()}
    uo = _dev(np.full_like(g["u"], 777.0), h, dtype)
    vo = _dev(np.full_like(g["u"], 777.0), h, dtype)
    p.apply([d["u"], d["v"], d["w"], d["coeff"]], [uo, vo], (0, 0, 0), n, (h, h, h), [dtr])
    torch.cuda.synchronize()
    G = {k: S.Grid.storage(v, h) for k, v in g.items()}
    ru, rv = S.hdiff_vadvc(G["u"], G["v"], G["w"], G["coeff"], (0, 0, 0), n, dtr)
    gu = uo.interior((0, 0, 0), n).cpu().numpy().astype(np.float64)
    gv = vo.interior((0, 0, 0), n).cpu().numpy().astype(np.float64)
    full = uo.tensor.cpu().numpy()
    oi, oj, ok = uo.origin
    mask = np.ones(full.shape, bool)
    mask[ok:ok + n[2], oj:oj + n[1], oi:oi + n[0]] = False
    assert np.all(full[mask] == 777.0)
    return max(rel_err(gu, ru), rel_err(gv, rv))


@pytest.mark.parametrize("sched", HV_SCHEDS, ids=str)
@pytest.mark.parametrize("dtype,arith", HV_PRECISIONS)
def test_hdiff_vadvc_ragged(sched, dtype, arith):
    assert _hv_case((37, 23, 11), 3, dtype, _with(sched, arith)) <= TOL[dtype]


@pytest.mark.parametrize("nk", [1, 2, 3, 4, 5, 9])
@pytest.mark.parametrize("arith", [0, 1])
def test_hdiff_vadvc_short_columns(nk, arith):
    for sched in HV_SCHEDS:
        assert _hv_case((33, 5, nk), 3, "f64", _with(sched, arith)) <= TOL["f64"]


@pytest.mark.parametrize("sched", HV_SCHEDS[:3], ids=str)
@pytest.mark.parametrize("arith", [0, 1])
def test_hdiff_vadvc_config_128x128x80_f64(sched, arith):
    assert _hv_case((128, 128, 80), 3, "f64", _with(sched, arith)) <= TOL["f64"]


@pytest.mark.parametrize("n", [(33, 5, 1001), (16, 16, 137), (20, 12, 256), (1, 1, 80), (1, 1, 1)], ids=str)
@pytest.mark.parametrize("dtype,arith", [("f64", 2), ("f64", 1), ("f32", 1)])
def test_hdiff_vadvc_staged_long_columns(n, dtype, arith):
    """The twisted column sweep on long columns (odd and even level counts):
    the two halves of up to 501 rows each meet in the middle."""
    sched = dict(fusion=1, tile_i=32, tile_j=8, k_chunk=4, arith=arith)
    assert _hv_case(n, 3, dtype, sched) <= TOL[dtype]
    if arith == 2:   # the split sweep and the slab pipeline
        sched = dict(fusion=1, tile_i=32, tile_j=8, k_chunk=4, arith=2, sweep=1, slabs=3)
        assert _hv_case(n, 3, dtype, sched) <= TOL[dtype]


@pytest.mark.parametrize("arith", [0, 1])
def test_hdiff_vadvc_config_128x128x137_f32(arith):
    assert _hv_case((128, 128, 137), 3, "f32", dict(fusion=0, staging=1, tile_i=16, tile_j=4, arith=arith)) <= TOL["f32"]


# ------------------------------------------------------------------ fastwaves

FW_SCHEDS = ([dict(fusion=1)]
             + [dict(fusion=0, staging=1, tile_i=a, tile_j=b, k_chunk=kc)
                for (a, b) in [(32, 4), (32, 8), (64, 2), (64, 4), (128, 2)] for kc in (0, 3)]
             + [dict(fusion=0, staging=0, tile_i=a, tile_j=b, unroll=u)
                for (a, b, u) in [(32, 4, 1), (64, 4, 2), (32, 8, 4), (128, 2, 4)]]
             + [dict(fusion=0, staging=2, tile_i=a, tile_j=b, k_chunk=kc)
                for (a, b) in [(32, 4), (64, 4), (128, 2)] for kc in (0, 3, 4)]
             + [dict(fusion=0, staging=2, tile_i=a, tile_j=b, unroll=2, k_chunk=kc)
                for (a, b) in [(32, 4), (32, 8), (64, 4), (128, 2)] for kc in (0, 3, 4)])


def _fw_case(n, h, dtype, sched, dt=0.5, alpha=0.0625, align=0, pad_i=0):
    f = inputs.fastwaves_fields(*n, h, seed=33)
    g = {k: _round(v, dtype) for k, v in f.items()}
    p = _prog(programs.FASTWAVES, dtype, sched)
    from paper_2005_13014_gb300.api import device_field
    d = [device_field(g[name], h, dtype, align_bytes=align, pad_i=pad_i) for name in inputs.FASTWAVES_NAMES]
    uo = device_field(np.full_like(g["pp"], 555.0), h, dtype, align_bytes=align, pad_i=pad_i)
    vo = device_field(np.full_like(g["pp"], 555.0), h, dtype, align_bytes=align, pad_i=pad_i)
    p.apply(d, [uo, vo], (0, 0, 0), n, (h, h, h), [dt, alpha])
    torch.cuda.synchronize()
    G = {k: S.Grid.storage(v, h) for k, v in g.items()}
    ru, rv = S.fastwaves(G, (0, 0, 0), n, dt, alpha)
    gu = uo.interior((0, 0, 0), n).cpu().numpy().astype(np.float64)
    gv = vo.interior((0, 0, 0), n).cpu().numpy().astype(np.float64)
    return max(rel_err(gu, ru), rel_err(gv, rv))


@pytest.mark.parametrize("sched", FW_SCHEDS, ids=str)
@pytest.mark.parametrize("dtype,arith", PRECISIONS)
def test_fastwaves_ragged(sched, dtype, arith):
    assert _fw_case((37, 29, 7), 3, dtype, _with(sched, arith)) <= TOL[dtype]


FW_TMA_SCHEDS = [dict(fusion=0, staging=4, tile_i=a, tile_j=b, k_chunk=kc)
                 for (a, b) in [(32, 4), (32, 8), (64, 4)] for kc in (0, 3)]


@pytest.mark.parametrize("sched", FW_TMA_SCHEDS, ids=str)
@pytest.mark.parametrize("dtype,arith", PRECISIONS)
def test_fastwaves_tma(sched, dtype, arith):
    """TMA-staged boxes: rows aligned at the domain corner (align 16: box
    offsets 2 and 0 elements for FP32), and rows of 44 elements with the
    corner at column 3 (offsets 1 and 3)."""
    s = _with(sched, arith)
    assert _fw_case((37, 29, 7), 3, dtype, s, align=16) <= TOL[dtype]
    assert _fw_case((37, 29, 7), 3, dtype, s, pad_i=1) <= TOL[dtype]


@pytest.mark.parametrize("dtype,arith", PRECISIONS)
@pytest.mark.parametrize("lb,ub", [((3, 2, 1), (33, 27, 7)), ((1, 5, 2), (70, 9, 3))], ids=str)
def test_fastwaves_tma_subdomain(dtype, arith, lb, ub):
    """TMA boxes for a domain that starts inside the storage at an odd column:
    box corners round down from origin + lb; nothing is written outside the
    domain."""
    from paper_2005_13014_gb300.api import device_field
    n_st, h = (72, 32, 9), 3
    f = inputs.fastwaves_fields(*n_st, h, seed=36)
    g = {k: _round(v, dtype) for k, v in f.items()}
    p = _prog(programs.FASTWAVES, dtype, dict(fusion=0, staging=4, tile_i=32, tile_j=4, k_chunk=3, arith=arith))
    d = [device_field(g[name], h, dtype, align_bytes=16) for name in inputs.FASTWAVES_NAMES]
    o = [device_field(np.full_like(g["pp"], 555.0), h, dtype, align_bytes=16, pad_value=555.0) for _ in range(2)]
    p.apply(d, o, lb, ub, (h, h, h), [0.5, 0.0625])
    torch.cuda.synchronize()
    G = {k: S.Grid.storage(v, h) for k, v in g.items()}
    ru, rv = S.fastwaves(G, lb, ub, 0.5, 0.0625)
    gu = o[0].interior(lb, ub).cpu().numpy().astype(np.float64)
    gv = o[1].interior(lb, ub).cpu().numpy().astype(np.float64)
    assert max(rel_err(gu, ru), rel_err(gv, rv)) <= TOL[dtype]
    full = o[0].tensor.cpu().numpy()
    oi, oj, ok = o[0].origin
    mask = np.ones(full.shape, bool)
    mask[ok + lb[2]:ok + ub[2], oj + lb[1]:oj + ub[1], oi + lb[0]:oi + ub[0]] = False
    assert np.all(full[mask] == 555.0)
    from paper_2005_13014_gb300 import _lib as L
    assert L.lib().oec_device_status(None) == 0


def test_fastwaves_tma_needs_aligned_pitch():
    from paper_2005_13014_gb300._lib import OecError
    with pytest.raises(OecError, match="16 bytes"):
        _fw_case((37, 29, 7), 3, "f32", FW_TMA_SCHEDS[0])   # rows of 43 floats


@pytest.mark.parametrize("n", [(37, 29, 7), (130, 9, 5), (256, 256, 80)], ids=str)
@pytest.mark.parametrize("dtype,arith", PRECISIONS)
def test_fastwaves_tma_bitwise(n, dtype, arith):
    """Every input through TMA boxes against the k-streaming kernel that
    loads per point: the same arithmetic, so the same bits."""
    from paper_2005_13014_gb300 import _lib as L
    from paper_2005_13014_gb300.api import device_field
    h = 3
    f = inputs.fastwaves_fields(*n, h, seed=35)
    g = {k: _round(v, dtype) for k, v in f.items()}
    outs = []
    for sched in (dict(fusion=0, staging=2, tile_i=32, tile_j=8, k_chunk=8, arith=arith),
                  dict(fusion=0, staging=4, tile_i=32, tile_j=4, k_chunk=8, arith=arith)):
        p = _prog(programs.FASTWAVES, dtype, sched)
        d = [device_field(g[name], h, dtype, align_bytes=16) for name in inputs.FASTWAVES_NAMES]
        o = [device_field(np.zeros_like(g["pp"]), h, dtype, align_bytes=16) for _ in range(2)]
        p.apply(d, o, (0, 0, 0), n, (h, h, h), [0.5, 0.0625])
        torch.cuda.synchronize()
        outs.append([x.tensor.cpu().numpy() for x in o])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)
    assert L.lib().oec_device_status(None) == 0


@pytest.mark.parametrize("n", [(37, 29, 7), (130, 9, 5), (256, 256, 80)], ids=str)
@pytest.mark.parametrize("dtype,arith", PRECISIONS)
def test_fastwaves_stream_smem_windows_bitwise(n, dtype, arith):
    """k-streaming with shared-memory u/v windows against the k-streaming
    kernel that loads them per point: the same arithmetic, so the same bits."""
    h = 3
    f = inputs.fastwaves_fields(*n, h, seed=34)
    g = {k: _round(v, dtype) for k, v in f.items()}
    outs = []
    for unroll in (1, 2):
        p = _prog(programs.FASTWAVES, dtype, dict(fusion=0, staging=2, tile_i=32, tile_j=8, unroll=unroll,
                                                  k_chunk=8, arith=arith))
        d = [_dev(g[name], h, dtype) for name in inputs.FASTWAVES_NAMES]
        o = [_dev(np.zeros_like(g["pp"]), h, dtype) for _ in range(2)]
        p.apply(d, o, (0, 0, 0), n, (h, h, h), [0.5, 0.0625])
        torch.cuda.synchronize()
        outs.append([x.tensor.cpu().numpy() for x in o])
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("dtype,arith", PRECISIONS)
def test_fastwaves_config_256x256x80(dtype, arith):
    sched = dict(fusion=0, staging=0, tile_i=64, tile_j=4, unroll=2, arith=arith)
    assert _fw_case((256, 256, 80), 3, dtype, sched) <= TOL[dtype]


@pytest.mark.parametrize("arith", [0, 1])
def test_hdiff_f64_identity_on_edge_values(arith):
    """coeff = 0 makes out = in: exercises the binary64 <-> double-float
    conversions on powers of two, values next to binade boundaries, both signs
    and magnitudes from 2^-70 to 2^110, inside the double-float range that
    starts at 2^-74 (relative error within 2^-47)."""
    from paper_2005_13014_gb300.api import Program, device_field
    n, h = (40, 9, 3), 2
    rng = np.random.default_rng(5)
    base = np.array([1.0, -1.0, 2.0, 0.5, 1 - 2.0**-53, 1 + 2.0**-52, 2.0**-60, -(2.0**100), 3.0, 1 / 3,
                     1 - 2.0**-25, 1 - 2.0**-24, 16777215.0, 16777217.0, 0.1, -7.25e-12, 123456.789])
    inp = rng.choice(base, size=(n[2] + 2 * h, n[1] + 2 * h, n[0] + 2 * h)) * rng.choice([1.0, -1.0], size=1)
    inp = inp * 10.0 ** rng.integers(-3, 4, size=inp.shape)
    p = Program(programs.HDIFF, "f64")
    p.set_schedule(fusion=0, staging=1, tile_i=32, tile_j=4, k_chunk=0, arith=arith)
    din = device_field(inp, h, "f64")
    dco = device_field(np.zeros_like(inp), h, "f64")
    dout = device_field(np.zeros_like(inp), h, "f64")
    p.apply([din, dco], [dout], (0, 0, 0), n, (h, h, h))
    torch.cuda.synchronize()
    got = dout.interior((0, 0, 0), n).cpu().numpy()
    ref = inp[h:-h, h:-h, h:-h]
    assert np.max(np.abs(got - ref) / np.abs(ref)) <= 2.0**-47


# ----------------------------------------------------- FP64 fixed-point hdiff

FIXED_SCHEDS = ([dict(fusion=0, staging=1, tile_i=a, tile_j=b, k_chunk=kc, arith=2)
                 for (a, b) in [(32, 4), (32, 8), (64, 2), (64, 4), (64, 8), (128, 2), (128, 4)] for kc in (0, 3)]
                + [dict(fusion=0, staging=1, tile_i=a, tile_j=b, unroll=u, k_chunk=3, arith=2)
                   for (a, b, u) in [(32, 8, 2), (32, 16, 1), (32, 16, 2), (32, 16, 4), (64, 8, 2)]])


@pytest.mark.parametrize("sched", FIXED_SCHEDS, ids=str)
def test_hdiff_fixed_point_ragged(sched):
    assert _hdiff_case((37, 29, 5), 2, "f64", sched) <= TOL["f64"]


@pytest.mark.parametrize("n", [(37, 29, 5), (33, 18, 3), (64, 64, 4)], ids=str)
def test_hdiff_fixed_point_rows_per_thread_bitwise(n):
    """Several rows per thread share the flux across the edges between their
    points; the integer arithmetic is the same, so the bits are."""
    from paper_2005_13014_gb300.api import Program, device_field
    h = 2
    f = inputs.hdiff_fields(*n, h, seed=41)
    outs = []
    for u in (1, 2, 4):
        p = Program(programs.HDIFF, "f64")
        p.set_schedule(fusion=0, staging=1, tile_i=32, tile_j=16, unroll=u, k_chunk=2, arith=2)
        o = device_field(np.zeros_like(f["in"]), h, "f64")
        p.apply([device_field(f["in"], h, "f64"), device_field(f["coeff"], h, "f64")], [o], (0, 0, 0), n, (h, h, h))
        torch.cuda.synchronize()
        outs.append(o.tensor.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_hdiff_fixed_point_config_sizes():
    assert _hdiff_case((64, 64, 60), 2, "f64", FIXED_SCHEDS[6]) <= TOL["f64"]
    assert _hdiff_case((256, 256, 80), 3, "f64", FIXED_SCHEDS[7], poison=False) <= TOL["f64"]
    assert _hdiff_case((40, 30, 6), 3, "f64", FIXED_SCHEDS[0], lb=(5, 3, 1), ub=(33, 27, 5)) <= TOL["f64"]


def test_hdiff_fixed_point_identity_is_exact():
    """coeff = 0: out = fma(-0, div, in) = in bit for bit, whatever the values."""
    from paper_2005_13014_gb300.api import Program, device_field
    n, h = (40, 9, 3), 2
    rng = np.random.default_rng(9)
    inp = rng.choice([1.0, -3.5, 2.0**-60, 2.0**100, 1 - 2.0**-53, 0.1], size=(n[2] + 4, n[1] + 4, n[0] + 4))
    inp = inp * 10.0 ** rng.integers(-3, 4, size=inp.shape)
    p = Program(programs.HDIFF, "f64")
    p.set_schedule(**FIXED_SCHEDS[0])
    out = device_field(np.zeros_like(inp), h, "f64")
    p.apply([device_field(inp, h, "f64"), device_field(np.zeros_like(inp), h, "f64")], [out], (0, 0, 0), n, (h, h, h))
    torch.cuda.synchronize()
    assert np.array_equal(out.interior((0, 0, 0), n).cpu().numpy(), inp[h:-h, h:-h, h:-h])


def test_hdiff_fixed_point_mixed_magnitudes():
    """Tiles holding 1e10 next to tiny values with near-equal neighbours: the
    limiter's sign decisions come from the exact inputs, so the result still
    matches the oracle normwise."""
    from paper_2005_13014_gb300.api import Program, device_field
    n, h = (37, 21, 4), 2
    rng = np.random.default_rng(10)
    shape = (n[2] + 4, n[1] + 4, n[0] + 4)
    inp = 1e-10 * (1.0 + 1e-12 * rng.integers(-3, 4, size=shape))
    inp[:, ::7, ::5] = 1e10 * rng.uniform(-1, 1, size=inp[:, ::7, ::5].shape)
    coeff = rng.uniform(0, 0.1, size=shape)
    p = Program(programs.HDIFF, "f64")
    p.set_schedule(**FIXED_SCHEDS[2])
    out = device_field(np.zeros_like(inp), h, "f64")
    p.apply([device_field(inp, h, "f64"), device_field(coeff, h, "f64")], [out], (0, 0, 0), n, (h, h, h))
    torch.cuda.synchronize()
    ref = S.hdiff(S.Grid.storage(inp, h), S.Grid.storage(coeff, h), (0, 0, 0), n)
    assert rel_err(out.interior((0, 0, 0), n).cpu().numpy(), ref) <= TOL["f64"]


# column sweep variants of the staged form: the fields split over warps, and
# the j-slab pipeline (each slab's sweep on a second stream, overlapping the
# next slab's hdiff)
@pytest.mark.parametrize("n", [(37, 23, 11), (33, 5, 1), (33, 5, 2), (16, 16, 137), (1, 1, 80)], ids=str)
@pytest.mark.parametrize("dtype,arith", [("f64", 2), ("f64", 1), ("f64", 0), ("f32", 0), ("f32", 1)])
def test_hdiff_vadvc_split_sweep(n, dtype, arith):
    sched = dict(fusion=1, tile_i=32, tile_j=8, k_chunk=4, arith=arith, sweep=1)
    assert _hv_case(n, 3, dtype, sched) <= TOL[dtype]


@pytest.mark.parametrize("nseg", [4, 8])
@pytest.mark.parametrize("n", [(37, 23, 11), (33, 5, 1), (33, 5, 2), (33, 5, 3), (31, 7, 5), (30, 9, 9),
                               (16, 16, 137), (20, 12, 256), (33, 5, 1001), (1, 1, 80), (128, 128, 80)], ids=str)
@pytest.mark.parametrize("dtype,arith", [("f64", 2), ("f64", 1), ("f64", 0), ("f32", 0), ("f32", 1)])
def test_hdiff_vadvc_partitioned_sweep(n, dtype, arith, nseg):
    """The partitioned column solve (4 or 8 segments per column, a reduced
    system over the segments' first and last rows), including columns with
    fewer levels than segments (empty segments) and long columns."""
    if (dtype, arith) != ("f64", 2) and n[2] in (1001, 256):
        pytest.skip("long columns: the fixed-point producer case covers them")
    sched = dict(fusion=1, tile_i=32, tile_j=8, k_chunk=4, arith=arith, sweep=nseg)
    assert _hv_case(n, 3, dtype, sched) <= TOL[dtype]


@pytest.mark.parametrize("nseg", [4, 8])
@pytest.mark.parametrize("dtr", [2.0, 0.5, 3.0, 1.0 / 3.0])
def test_hdiff_vadvc_partitioned_sweep_dtr_and_slabs(nseg, dtr):
    sched = dict(fusion=1, tile_i=32, tile_j=8, k_chunk=4, arith=2, sweep=nseg)
    assert _hv_case((37, 23, 11), 3, "f64", sched, dtr=dtr) <= TOL["f64"]
    sched["slabs"] = 3
    assert _hv_case((37, 23, 11), 3, "f64", sched, dtr=dtr) <= TOL["f64"]


@pytest.mark.parametrize("sweep", [0, 1])
@pytest.mark.parametrize("slabs", [2, 3, 4, 8, 16])
@pytest.mark.parametrize("n", [(37, 23, 11), (33, 5, 2), (40, 17, 9)], ids=str)
def test_hdiff_vadvc_slab_pipeline(n, slabs, sweep):
    sched = dict(fusion=1, tile_i=32, tile_j=8, k_chunk=4, arith=2, sweep=sweep, slabs=slabs)
    assert _hv_case(n, 3, "f64", sched) <= TOL["f64"]


@pytest.mark.parametrize("dtype,arith,producer", [("f64", 2, dict(staging=0, tile_i=32, tile_j=8, unroll=1)),
                                                  ("f64", 2, dict(staging=0, tile_i=32, tile_j=16, unroll=2)),
                                                  ("f32", 1, dict(staging=3, tile_i=32, tile_j=8, unroll=2))],
                         ids=str)
def test_hdiff_vadvc_sweep_forms_bitwise(dtype, arith, producer):
    """The split sweep does each field's operations of the pair sweep, and the
    slab pipeline runs the same kernels on slabs whose rows are whole tiles:
    every form gives the bits of the plain staged form (128x128x80)."""
    from paper_2005_13014_gb300.api import Program, device_field
    n, h = (128, 128, 80), 3
    f = inputs.hdiff_vadvc_fields(*n, h, seed=51)
    g = {k: _round(v, dtype) for k, v in f.items()}
    d = [device_field(g[k], h, dtype, align_bytes=16) for k in ("u", "v", "w", "coeff")]
    outs = []
    for sweep, slabs in ((0, 0), (1, 0), (0, 4), (1, 4), (0, 2), (1, 16)):
        p = Program(programs.HDIFF_VADVC, dtype)
        p.set_schedule(fusion=1, k_chunk=4, arith=arith, sweep=sweep, slabs=slabs, **producer)
        o = [device_field(np.zeros_like(g["u"]), h, dtype, align_bytes=16) for _ in range(2)]
        p.apply(d, o, (0, 0, 0), n, (h, h, h), [2.0])
        p.apply(d, o, (0, 0, 0), n, (h, h, h), [2.0])   # twice: the pipeline's events and stream reused
        torch.cuda.synchronize()
        outs.append([x.tensor.clone() for x in o])
    for o in outs[1:]:
        assert torch.equal(o[0], outs[0][0]) and torch.equal(o[1], outs[0][1])


def test_schedule_fields_sweep_and_slabs_are_validated():
    from paper_2005_13014_gb300.api import Program
    from paper_2005_13014_gb300._lib import OecError
    p = Program(programs.HDIFF_VADVC, "f64")
    for bad in (dict(fusion=0, tile_i=16, tile_j=4, sweep=1), dict(fusion=1, slabs=17), dict(fusion=1, sweep=2),
                dict(fusion=1, slabs=-1), dict(fusion=1, sweep=16), dict(fusion=0, tile_i=16, tile_j=4, sweep=4)):
        with pytest.raises(OecError):
            p.set_schedule(**bad)
    q = Program(programs.HDIFF, "f64")
    with pytest.raises(OecError):
        q.set_schedule(fusion=0, staging=1, tile_i=32, tile_j=8, slabs=2)


@pytest.mark.parametrize("n", [(37, 23, 11), (33, 5, 1), (33, 5, 2), (128, 128, 80)], ids=str)
def test_hdiff_vadvc_fixed_point_staged(n):
    assert _hv_case(n, 3, "f64", dict(fusion=1, arith=2)) <= TOL["f64"]


@pytest.mark.parametrize("kc", [4, 8])
@pytest.mark.parametrize("tile", [(32, 4), (32, 8), (64, 4), (64, 8), (128, 4)], ids=str)
@pytest.mark.parametrize("dtype,arith", [("f64", 0), ("f64", 1), ("f64", 2), ("f32", 0), ("f32", 1)])
def test_hdiff_vadvc_staged_producer_tiles(dtype, arith, tile, kc):
    """The staged form's hdiff producer on each tile the tuner may pick, with
    the twisted column sweep behind it (ragged tiles, odd column count)."""
    sched = dict(fusion=1, tile_i=tile[0], tile_j=tile[1], k_chunk=kc, arith=arith)
    assert _hv_case((37, 23, 11), 3, dtype, sched) <= TOL[dtype]


@pytest.mark.parametrize("kc", [2, 3, 4])
@pytest.mark.parametrize("tile", [(32, 8, 2), (32, 16, 1), (32, 16, 2), (32, 16, 4), (64, 8, 2)], ids=str)
def test_hdiff_vadvc_staged_fixed_rows_per_thread(tile, kc):
    sched = dict(fusion=1, tile_i=tile[0], tile_j=tile[1], unroll=tile[2], k_chunk=kc, arith=2)
    assert _hv_case((37, 23, 11), 3, "f64", sched) <= TOL["f64"]
    assert _hv_case((128, 128, 80), 3, "f64", sched) <= TOL["f64"]


@pytest.mark.parametrize("kc", [2, 3])
@pytest.mark.parametrize("tile", [(32, 4), (32, 8), (64, 4), (64, 8), (128, 4)], ids=str)
def test_hdiff_vadvc_staged_fixed_short_chunks(tile, kc):
    """The fixed-point producer with 2 or 3 levels per CTA (the tuner's
    shortest chunks; 11 levels leave a partial last chunk), one row per
    thread."""
    sched = dict(fusion=1, tile_i=tile[0], tile_j=tile[1], k_chunk=kc, arith=2)
    assert _hv_case((37, 23, 11), 3, "f64", sched) <= TOL["f64"]


@pytest.mark.parametrize("unroll", [1, 2, 4])
@pytest.mark.parametrize("tile", [(32, 4), (32, 8), (64, 4), (128, 2), (16, 8)], ids=str)
@pytest.mark.parametrize("arith", [0, 1])
def test_hdiff_vadvc_f32_regs_producer(arith, tile, unroll):
    """FP32 staged form with the REGS hdiff producer writing both fields in one
    launch (tiles it cannot run, e.g. 128x2 at unroll 4, fall back to 64x4)."""
    sched = dict(fusion=1, staging=0, tile_i=tile[0], tile_j=tile[1], unroll=unroll, k_chunk=3, arith=arith)
    assert _hv_case((37, 23, 11), 3, "f32", sched) <= TOL["f32"]
    assert _hv_case((33, 5, 2), 3, "f32", sched) <= TOL["f32"]


@pytest.mark.parametrize("unroll", [1, 2, 4])
@pytest.mark.parametrize("arith", [0, 1])
@pytest.mark.parametrize("n,align", [((36, 23, 11), 16), ((128, 128, 80), 16), ((37, 23, 11), 16),
                                     ((36, 23, 11), 0)], ids=str)
def test_hdiff_vadvc_f32_vector_producer(n, align, arith, unroll):
    """FP32 staged form with the vector-row producer (aligned rows, ni a
    multiple of 4) and its REGS fallback (ni = 37, or unaligned storage)."""
    h = 3
    f = inputs.hdiff_vadvc_fields(*n, h, seed=37)
    g = {k: _round(v, "f32") for k, v in f.items()}
    p = _prog(programs.HDIFF_VADVC, "f32", dict(fusion=1, staging=3, tile_i=32, tile_j=4 * unroll, unroll=unroll,
                                                 k_chunk=8, arith=arith))
    d = {k: _dev(v, h, "f32", align) for k, v in g.items()}
    o = [_dev(np.full_like(g["u"], 777.0), h, "f32", align, pad_value=777.0) for _ in range(2)]
    p.apply([d["u"], d["v"], d["w"], d["coeff"]], o, (0, 0, 0), n, (h, h, h), [2.0])
    torch.cuda.synchronize()
    G = {k: S.Grid.storage(v, h) for k, v in g.items()}
    ru, rv = S.hdiff_vadvc(G["u"], G["v"], G["w"], G["coeff"], (0, 0, 0), n, 2.0)
    gu = o[0].interior((0, 0, 0), n).cpu().numpy().astype(np.float64)
    gv = o[1].interior((0, 0, 0), n).cpu().numpy().astype(np.float64)
    assert max(rel_err(gu, ru), rel_err(gv, rv)) <= TOL["f32"]
    full = o[0].tensor.cpu().numpy()
    oi, oj, ok = o[0].origin
    mask = np.ones(full.shape, bool)
    mask[ok:ok + n[2], oj:oj + n[1], oi:oi + n[0]] = False
    assert np.all(full[mask] == 777.0)


@pytest.mark.parametrize("arith", [0, 1])
def test_hdiff_vadvc_f32_smem_producer(arith):
    sched = dict(fusion=1, staging=1, tile_i=64, tile_j=4, k_chunk=4, arith=arith)
    assert _hv_case((37, 23, 11), 3, "f32", sched) <= TOL["f32"]


@pytest.mark.parametrize("dtr", [2.0, 0.5, 64.0, 3.0, 1.0 / 3.0])
@pytest.mark.parametrize("dtype,arith", [("f64", 1), ("f64", 2), ("f64", 0), ("f32", 1)])
def test_hdiff_vadvc_staged_dtr(dtype, arith, dtr):
    """dtr a power of two (the double-float column sweep scales exactly) and
    not a power of two (the pair product)."""
    sched = dict(fusion=1, tile_i=32, tile_j=8, k_chunk=4, arith=arith)
    assert _hv_case((37, 23, 11), 3, dtype, sched, dtr=dtr) <= TOL[dtype]
    if arith == 2:   # the split sweep and the slab pipeline
        sched = dict(fusion=1, tile_i=32, tile_j=8, k_chunk=4, arith=2, sweep=1, slabs=4)
        assert _hv_case((37, 23, 11), 3, dtype, sched, dtr=dtr) <= TOL[dtype]


@pytest.mark.parametrize("n", [(256, 256, 8), (268, 250, 5), (512, 128, 3), (1024, 64, 2), (256, 257, 1)], ids=str)
@pytest.mark.parametrize("unroll,k_chunk,arith", [(1, 4, 1), (2, 0, 1), (1, 20, 0), (2, 3, 0)])
def test_hdiff_vadvc_f32_persistent_single_domain(n, unroll, k_chunk, arith):
    """FP32 fields on the warp-row producer with at least 65,536 columns: the
    producer and the column sweep run as one persistent launch whose tickets
    follow a closed-form order (producer items of a row block, then the
    column groups a lag of row blocks back). Partial row blocks, partial
    column groups, 1-level columns, the threshold itself (1024x64): the bits
    of the two-kernel form with the one-field-per-thread sweep (the same
    operations per field), sampled blocks within tolerance of the oracle, no
    bounded wait given up, also when replayed from a captured graph."""
    from paper_2005_13014_gb300 import _lib as L
    from paper_2005_13014_gb300.api import Program, device_field
    h = 3
    f = inputs.hdiff_vadvc_fields(*n, h, seed=91)
    g = {k: _round(v, "f32") for k, v in f.items()}
    d = [device_field(g[k], h, "f32", align_bytes=16) for k in ("u", "v", "w", "coeff")]
    res = []
    for sweep in (0, 1):
        p = Program(programs.HDIFF_VADVC, "f32")
        p.set_schedule(fusion=1, staging=3, tile_i=32, tile_j=4 * unroll, unroll=unroll, k_chunk=k_chunk, arith=arith,
                       sweep=sweep)
        o = [device_field(np.full_like(g["u"], 5.0), h, "f32", align_bytes=16) for _ in range(2)]
        p.apply(d, o, (0, 0, 0), n, (h, h, h), [2.0])
        if sweep == 0:
            assert p.launch_count() == 1   # one persistent launch
            cg = [device_field(np.full_like(g["u"], 5.0), h, "f32", align_bytes=16) for _ in range(2)]
            gr = p.capture(d, cg, (0, 0, 0), n, (h, h, h), [2.0])
            gr()
            gr()
            torch.cuda.synchronize()
            gr.close()
            for a, b in zip(o, cg):
                assert torch.equal(a.tensor, b.tensor)
        torch.cuda.synchronize()
        res.append(o)
    for a, b in zip(*res):
        assert torch.equal(a.tensor, b.tensor)
    assert L.lib().oec_device_status(None) == 0
    rng = np.random.default_rng(3)
    i0, j0 = int(rng.integers(0, n[0] - 8)), int(rng.integers(0, n[1] - 8))
    lb, ub = (i0, j0, 0), (i0 + 8, j0 + 8, n[2])
    G = {k: S.Grid.storage(v, h) for k, v in g.items()}
    ru, rv = S.hdiff_vadvc(G["u"], G["v"], G["w"], G["coeff"], lb, ub, 2.0)
    gu = res[0][0].interior(lb, ub).cpu().numpy().astype(np.float64)
    gv = res[0][1].interior(lb, ub).cpu().numpy().astype(np.float64)
    assert max(rel_err(gu, ru), rel_err(gv, rv)) <= TOL["f32"]
