"""GPU parity of the Table II stand-in programs (programs.TESTSET) through the
generic code generator: every fusion x unroll x tile variant against the
oracle's staged interpreter, with NaN outside each input's inferred range
and a sentinel outside the domain."""

import numpy as np
import pytest

from conftest import TOL, rel_err
from oracle import program as OP
from oracle import stencils as S
from paper_2005_13014_gb300 import inputs, programs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

VARIANTS = [dict(fusion=f, unroll=u, tile_i=ti, tile_j=tj)
            for f in (0, 1, 2) for u in (1, 2, 4) for (ti, tj) in ((32, 4), (64, 2))]


def _case(name, n, dtype, h=3, arith=0):
    from paper_2005_13014_gb300.api import Program, device_field
    src, params, _ = programs.TESTSET[name]
    prog = OP.parse(src)
    f = inputs.testset_fields(name, *n, h)
    if dtype == "f32":
        f = {k: v.astype(np.float32).astype(np.float64) for k, v in f.items()}
    G = {k: S.Grid.storage(v, h) for k, v in f.items()}
    ref = OP.run_staged(prog, G, (0, 0, 0), n, dict(zip(prog.params, params)))
    halo = OP.input_halo(prog, (0, 0, 0), n)
    poisoned = {}
    for k, v in f.items():   # NaN outside the range the program may read
        (il, iu), (jl, ju), (kl, ku) = halo[k]
        q = np.full_like(v, np.nan)
        sl = (slice(h - kl, h + n[2] + ku), slice(h - jl, h + n[1] + ju), slice(h - il, h + n[0] + iu))
        q[sl] = v[sl]
        poisoned[k] = q
    p = Program(src, dtype, generic=True)
    din = [device_field(poisoned[nm], h, dtype) for nm in prog.inputs]
    errs = []
    for sched in VARIANTS:
        p.set_schedule(**sched, arith=arith)
        outs = [device_field(np.full_like(f[prog.inputs[0]], 7.0), h, dtype) for _ in prog.outputs]
        p.apply(din, outs, (0, 0, 0), n, (h, h, h), params)
        torch.cuda.synchronize()
        for o, nm in zip(outs, prog.outputs):
            got = o.interior((0, 0, 0), n).cpu().numpy().astype(np.float64)
            assert np.all(np.isfinite(got)), (name, sched)
            errs.append(rel_err(got, ref[nm]))
            full = o.tensor.cpu().numpy()
            oi, oj, ok = o.origin
            mask = np.ones(full.shape, bool)
            mask[ok:ok + n[2], oj:oj + n[1], oi:oi + n[0]] = False
            assert np.all(full[mask] == 7.0), "write outside the domain"
    return max(errs)


@pytest.mark.parametrize("dtype,arith", [("f32", 0), ("f64", 0), ("f64", 1)])
@pytest.mark.parametrize("name", list(programs.TESTSET))
def test_testset_ragged(name, dtype, arith):
    """arith 1: the FP64 program evaluated in generated double-float code."""
    assert _case(name, (37, 29, 7), dtype, arith=arith) <= TOL[dtype]


@pytest.mark.parametrize("name", list(programs.TESTSET))
def test_testset_paper_size_f32(name):
    assert _case(name, (128, 128, 60), "f32") <= TOL["f32"]
