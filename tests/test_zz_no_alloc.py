"""The allocation-free hdiff+vadvc entry point (for callers that cannot call
cudaMalloc while they run, e.g. during stream capture or under a fixed memory
budget) must give the same results as oec_program_apply, call after call,
although every call reuses the same fixed scratch array. Kept in its own file
so that pytest collects it last."""

import ctypes as C

import numpy as np
import pytest

from conftest import TOL, rel_err
from paper_2005_13014_gb300 import _lib as L
from paper_2005_13014_gb300 import inputs, programs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_matches_program_apply_on_two_calls(liboec, dtype):
    from paper_2005_13014_gb300.api import Program, device_field
    n, h = (128, 96, 40), 3
    prog = Program(programs.HDIFF_VADVC, dtype)
    for call, seed in enumerate((2005, 4242)):
        f = inputs.hdiff_vadvc_fields(*n, h, seed=seed)
        d = [device_field(f[k], h, dtype) for k in ("u", "v", "w", "coeff")]
        ref = [device_field(np.zeros_like(f["u"]), h, dtype) for _ in range(2)]
        got = [device_field(np.full_like(f["u"], 9.0), h, dtype) for _ in range(2)]
        prog.apply(d, ref, (0, 0, 0), n, (h, h, h), [2.0])
        ins = (L.FieldDesc * 4)(*[x.desc() for x in d])
        outs = (L.FieldDesc * 2)(*[x.desc() for x in got])
        stream = torch.cuda.current_stream().cuda_stream
        rc = liboec.oec_hdiff_vadvc_apply_noalloc(L.F64 if dtype == "f64" else L.F32, ins, outs, L.I64x3(0, 0, 0),
                                                  L.I64x3(*n), 2.0, C.c_void_p(stream))
        assert rc == 0, liboec.oec_last_error()
        torch.cuda.synchronize()
        for g, r in zip(got, ref):
            a = g.interior((0, 0, 0), n).cpu().numpy().astype(np.float64)
            b = r.interior((0, 0, 0), n).cpu().numpy().astype(np.float64)
            assert rel_err(a, b) <= TOL[dtype], f"call {call}"


@pytest.mark.parametrize("dtype,n,sched", [
    ("f64", (128, 128, 80), dict(fusion=1, staging=0, tile_i=32, tile_j=8, unroll=1, k_chunk=4, arith=2)),
    ("f32", (128, 128, 80), dict(fusion=1, staging=3, tile_i=32, tile_j=4, unroll=1, k_chunk=20, arith=1)),
    ("f64", (128, 128, 120), dict(fusion=0, staging=1, tile_i=16, tile_j=4, arith=1))], ids=str)
def test_noalloc_bits_of_the_schedule_it_runs(liboec, dtype, n, sched):
    """Staged where its scratch fits (128x128x80), fused beyond (128x128x120,
    1.97 M points in FP64): bit for bit the apply with that schedule."""
    from paper_2005_13014_gb300.api import Program, device_field
    h = 3
    prog = Program(programs.HDIFF_VADVC, dtype)
    if sched:
        prog.set_schedule(**sched)
    f = inputs.hdiff_vadvc_fields(*n, h, seed=77)
    d = [device_field(f[k], h, dtype) for k in ("u", "v", "w", "coeff")]
    ref = [device_field(np.zeros_like(f["u"]), h, dtype) for _ in range(2)]
    got = [device_field(np.zeros_like(f["u"]), h, dtype) for _ in range(2)]
    prog.apply(d, ref, (0, 0, 0), n, (h, h, h), [2.0])
    ins = (L.FieldDesc * 4)(*[x.desc() for x in d])
    outs = (L.FieldDesc * 2)(*[x.desc() for x in got])
    rc = liboec.oec_hdiff_vadvc_apply_noalloc(L.F64 if dtype == "f64" else L.F32, ins, outs, L.I64x3(0, 0, 0),
                                              L.I64x3(*n), 2.0, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, liboec.oec_last_error()
    torch.cuda.synchronize()
    for g, r in zip(got, ref):
        assert torch.equal(g.tensor, r.tensor)


def test_noalloc_rejects_oversized_domain(liboec):
    # 2,796,203 points need more than the fixed 64 MiB even in the fused
    # form; rejected before any launch
    d = L.FieldDesc()
    d.data, d.dtype, d.ndim = 1 << 30, L.F64, 3
    n = (2796203, 1, 1)
    d.size = L.I64x3(n[0] + 6, 7, 7)
    d.stride = L.I64x3(1, n[0] + 6, (n[0] + 6) * 7)
    d.origin = L.I64x3(3, 3, 3)
    ins = (L.FieldDesc * 4)(*[d for _ in range(4)])
    fields = []
    for x in range(2):
        o = L.FieldDesc()
        C.memmove(C.byref(o), C.byref(d), C.sizeof(d))
        o.data = (x + 2) << 34
        fields.append(o)
    outs = (L.FieldDesc * 2)(*fields)
    rc = liboec.oec_hdiff_vadvc_apply_noalloc(L.F64, ins, outs, L.I64x3(0, 0, 0), L.I64x3(*n), 2.0, None)
    assert rc == -7
    assert b"scratch" in liboec.oec_last_error()
