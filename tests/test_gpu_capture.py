"""Captured applies (oec_program_capture / oec_graph_launch): one apply
recorded into a CUDA graph gives the bits of the same apply launched
directly, also after the fields' contents change between launches; the
program's scratch stays put while graphs use it."""

import numpy as np
import pytest

from paper_2005_13014_gb300 import inputs, programs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _fields(n, h, dtype, seed):
    from paper_2005_13014_gb300.api import device_field
    f = inputs.hdiff_vadvc_fields(*n, h, seed=seed)
    return f, [device_field(f[k], h, dtype) for k in ("u", "v", "w", "coeff")]


@pytest.mark.parametrize("dtype,sched", [
    ("f64", None),
    ("f64", dict(fusion=1, tile_i=32, tile_j=8, k_chunk=4, arith=2, slabs=3)),
    ("f64", dict(fusion=0, staging=1, tile_i=16, tile_j=4, arith=1)),
    ("f32", None)], ids=str)
def test_captured_apply_matches_direct_apply(dtype, sched):
    from paper_2005_13014_gb300.api import Program, device_field
    n, h = (37, 23, 11), 3
    p = Program(programs.HDIFF_VADVC, dtype)
    if sched:
        p.set_schedule(**sched)
    f, d = _fields(n, h, dtype, 61)
    got = [device_field(np.zeros_like(f["u"]), h, dtype) for _ in range(2)]
    ref = [device_field(np.zeros_like(f["u"]), h, dtype) for _ in range(2)]
    g = p.capture(d, got, (0, 0, 0), n, (h, h, h), [2.0])
    p.apply(d, ref, (0, 0, 0), n, (h, h, h), [2.0])
    assert g.kernel_count == p.launch_count() >= 1
    torch.cuda.synchronize()
    assert all(float(x.tensor.abs().max()) == 0.0 for x in got)   # capturing ran nothing
    g()
    torch.cuda.synchronize()
    for a, b in zip(got, ref):
        assert torch.equal(a.tensor, b.tensor)
    # new contents in the same storage: the next launch reads them
    f2, d2 = _fields(n, h, dtype, 62)
    for x, y in zip(d, d2):
        x.tensor.copy_(y.tensor)
    g()
    p.apply(d, ref, (0, 0, 0), n, (h, h, h), [2.0])
    torch.cuda.synchronize()
    for a, b in zip(got, ref):
        assert torch.equal(a.tensor, b.tensor)
    g.close()


def test_scratch_is_kept_while_graphs_use_it():
    from paper_2005_13014_gb300._lib import OecError
    from paper_2005_13014_gb300.api import Program, device_field
    h = 3
    p = Program(programs.HDIFF_VADVC, "f64")
    p.set_schedule(fusion=1, tile_i=32, tile_j=8, k_chunk=4, arith=2)
    small, big = (20, 12, 6), (40, 30, 20)
    fs, ds = _fields(small, h, "f64", 63)
    fb, db = _fields(big, h, "f64", 64)
    os_ = [device_field(np.zeros_like(fs["u"]), h, "f64") for _ in range(2)]
    ob = [device_field(np.zeros_like(fb["u"]), h, "f64") for _ in range(2)]
    g = p.capture(ds, os_, (0, 0, 0), small, (h, h, h), [2.0])
    with pytest.raises(OecError, match="captured"):
        p.apply(db, ob, (0, 0, 0), big, (h, h, h), [2.0])
    p.apply(ds, os_, (0, 0, 0), small, (h, h, h), [2.0])   # the same size still runs
    g.close()
    p.apply(db, ob, (0, 0, 0), big, (h, h, h), [2.0])
    torch.cuda.synchronize()


def test_captured_generated_program():
    from paper_2005_13014_gb300.api import Program, device_field
    name = "uvbke"
    src, params, shape = programs.TESTSET[name]
    n, h = (40, 20, 6), 3
    f = inputs.testset_fields(name, *n, h)
    names = list(inputs.TESTSET_INPUTS[name])
    p = Program(src, "f32", generic=True)
    d = [device_field(f[k], h, "f32") for k in names]
    got = [device_field(np.zeros_like(f[names[0]]), h, "f32") for _ in range(shape[2])]
    ref = [device_field(np.zeros_like(f[names[0]]), h, "f32") for _ in range(shape[2])]
    p.prepare(n, d[0].tensor.stride(1), d[0].tensor.stride(0))
    g = p.capture(d, got, (0, 0, 0), n, (h, h, h), params)
    g()
    p.apply(d, ref, (0, 0, 0), n, (h, h, h), params)
    torch.cuda.synchronize()
    for a, b in zip(got, ref):
        assert torch.equal(a.tensor, b.tensor)
    g.close()
