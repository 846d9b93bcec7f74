"""Offset width (the schedule's index_bits, the paper's index type of §V-B
and §VII-C): every kernel that has a 32-bit-offset form gives, with 64-bit
offsets forced (OEC_INDEX_64), the same outputs bit for bit as with the
automatic choice, and both agree with the FP64 oracle. Covered: fused
horizontal diffusion with REGS, WARP and fixed-point schedules, the staged
hdiff+vadvc producers, and generated kernels of random stage DAGs."""

import numpy as np
import pytest

from conftest import TOL, rel_err
from oracle import program as OP
from oracle import stencils as S
from paper_2005_13014_gb300 import inputs, programs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _round(arr, dtype):
    return arr.astype(np.float32).astype(np.float64) if dtype == "f32" else arr


def _both_widths(src, dtype, sched, fields, names, n, h, params=(), align=0, generic=False, n_out=1):
    """Outputs (interior, float64) for index_bits 0 and 64 on the same fields."""
    from paper_2005_13014_gb300.api import Program, device_field
    p = Program(src, dtype, generic=generic)
    din = [device_field(fields[k], h, dtype, align_bytes=align) for k in names]
    res = []
    for bits in (0, 64):
        p.set_schedule(**dict(sched, index_bits=bits))
        outs = [device_field(np.full_like(fields[names[0]], 7.0), h, dtype, align_bytes=align, pad_value=7.0)
                for _ in range(n_out)]
        p.apply(din, outs, (0, 0, 0), n, (h, h, h) if np.isscalar(h) else h, list(params))
        torch.cuda.synchronize()
        res.append([o.interior((0, 0, 0), n).cpu().numpy().astype(np.float64) for o in outs])
    return res


@pytest.mark.parametrize("dtype,sched,align", [
    ("f32", dict(fusion=0, staging=0, tile_i=64, tile_j=4, unroll=2, k_chunk=3), 0),
    ("f32", dict(fusion=0, staging=0, tile_i=32, tile_j=8, unroll=4), 0),
    ("f64", dict(fusion=0, staging=0, tile_i=64, tile_j=4, unroll=1, k_chunk=3), 0),
    ("f32", dict(fusion=0, staging=3, tile_i=32, tile_j=8, unroll=2, k_chunk=3), 16),
    ("f64", dict(fusion=0, staging=3, tile_i=32, tile_j=4, unroll=1), 16),
    ("f64", dict(fusion=0, staging=1, tile_i=64, tile_j=4, k_chunk=3, arith=2), 0),
    ("f64", dict(fusion=0, staging=1, tile_i=32, tile_j=16, unroll=2, arith=2), 0),
], ids=str)
def test_hdiff_offset_widths_agree(dtype, sched, align):
    n, h = ((36, 23, 11) if align else (37, 23, 11)), 2
    f = inputs.hdiff_fields(*n, h, seed=41)
    g = {k: _round(v, dtype) for k, v in f.items()}
    (a,), (b,) = _both_widths(programs.HDIFF, dtype, sched, g, ["in", "coeff"], n, h, align=align)
    assert np.array_equal(a, b)
    ref = S.hdiff(S.Grid.storage(g["in"], h), S.Grid.storage(g["coeff"], h), (0, 0, 0), n)
    assert rel_err(a, ref) <= TOL[dtype]


@pytest.mark.parametrize("dtype,sched,align,n", [
    ("f64", dict(fusion=1, staging=0, tile_i=32, tile_j=8, k_chunk=4, arith=2), 0, (37, 23, 11)),
    ("f64", dict(fusion=1, staging=0, tile_i=32, tile_j=8, k_chunk=4, arith=2), 0, (128, 128, 80)),
    ("f32", dict(fusion=1, staging=0, tile_i=64, tile_j=4, unroll=2, k_chunk=3, arith=1), 0, (37, 23, 11)),
    ("f32", dict(fusion=1, staging=3, tile_i=32, tile_j=8, unroll=2, k_chunk=8, arith=1), 16, (36, 23, 11)),
], ids=str)
def test_hdiff_vadvc_staged_offset_widths_agree(dtype, sched, align, n):
    h = 3
    f = inputs.hdiff_vadvc_fields(*n, h, seed=42)
    g = {k: _round(v, dtype) for k, v in f.items()}
    (au, av), (bu, bv) = _both_widths(programs.HDIFF_VADVC, dtype, sched, g, ["u", "v", "w", "coeff"], n, h,
                                      params=[2.0], align=align, n_out=2)
    assert np.array_equal(au, bu) and np.array_equal(av, bv)
    G = {k: S.Grid.storage(v, h) for k, v in g.items()}
    ru, rv = S.hdiff_vadvc(G["u"], G["v"], G["w"], G["coeff"], (0, 0, 0), n, 2.0)
    assert max(rel_err(au, ru), rel_err(av, rv)) <= TOL[dtype]


@pytest.mark.parametrize("seed", [10000, 10004, 10009])
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_generated_offset_widths_agree(seed, dtype):
    n, h = (37, 21, 7), (8, 8, 4)
    src = inputs.random_dag(seed)
    prog = OP.parse(src)
    fields = {}
    for idx, name in enumerate(prog.inputs):
        arr = np.random.default_rng(seed * 10 + idx).uniform(-1, 1, (n[2] + 2 * h[2], n[1] + 2 * h[1],
                                                                      n[0] + 2 * h[0]))
        fields[name] = _round(arr, dtype)
    ref = OP.run_staged(prog, {k: S.Grid.storage(v, h) for k, v in fields.items()}, (0, 0, 0), n)
    for fusion in (0, 1, 2):
        sched = dict(fusion=fusion, unroll=2, tile_i=32, tile_j=4)
        a, b = _both_widths(src, dtype, sched, fields, list(prog.inputs), n, h, generic=True,
                            n_out=len(prog.outputs))
        for x, y, name in zip(a, b, prog.outputs):
            assert np.array_equal(x, y)
            assert rel_err(x, ref[name]) <= TOL[dtype]


@pytest.mark.parametrize("dtype,arith", [("f64", 0), ("f64", 1), ("f32", 0)])
@pytest.mark.parametrize("sched", [dict(fusion=0, staging=1, tile_i=32, tile_j=8, k_chunk=4),
                                   dict(fusion=0, staging=2, tile_i=64, tile_j=4, k_chunk=8),
                                   dict(fusion=0, staging=2, tile_i=32, tile_j=8, unroll=2, k_chunk=4),
                                   dict(fusion=0, staging=4, tile_i=32, tile_j=4, k_chunk=8)], ids=str)
def test_fastwaves_offset_widths_agree(dtype, arith, sched):
    """The fastwaves kernels (shared-memory tile, k-streaming, k-streaming with
    shared u/v windows, TMA boxes): 64-bit offsets forced give the bits of
    the automatic (32-bit) form, within tolerance of the oracle."""
    n, h = (37, 29, 7), 3
    f = inputs.fastwaves_fields(*n, h, seed=71)
    g = {k: _round(v, dtype) for k, v in f.items()}
    s = dict(sched, arith=arith)
    a, b = _both_widths(programs.FASTWAVES, dtype, s, g, inputs.FASTWAVES_NAMES, n, h, params=(0.5, 0.0625),
                        align=16, n_out=2)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    G = {k: S.Grid.storage(v, h) for k, v in g.items()}
    ru, rv = S.fastwaves(G, (0, 0, 0), n, 0.5, 0.0625)
    assert max(rel_err(a[0], ru), rel_err(a[1], rv)) <= TOL[dtype]
