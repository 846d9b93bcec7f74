"""The allocation-free hdiff+vadvc entry point (for callers that cannot call
cudaMalloc while they run, e.g. under a device-memory budget owned by another
allocator) must give the same results as oec_program_apply, call after call,
although every call reuses the same fixed scratch array, and must take no
device memory. Kept in its own file so that pytest collects it last."""

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


FUSED_DF = dict(fusion=0, staging=1, tile_i=16, tile_j=4, arith=1)


@pytest.mark.parametrize("dtype,n,sched", [
    ("f64", (128, 128, 80), None),
    ("f32", (128, 128, 80), None),
    ("f64", (128, 128, 102), None),
    ("f64", (128, 128, 103), FUSED_DF),
    ("f64", (128, 128, 120), FUSED_DF),
    ("f64", (128, 128, 170), FUSED_DF),
    ("f32", (160, 128, 110), FUSED_DF)], ids=str)
def test_noalloc_bits_of_the_schedule_it_runs(liboec, dtype, n, sched):
    """Staged (the program's default schedule, two threads per column, one
    stream) where 40 B (FP64) / 32 B (FP32) per point fit in 64 MiB: at
    128x128x80 and just below the limit (128x128x102); the fused 16x4
    double-float sweep beyond it: just above (128x128x103), at 128x128x120,
    at the fused form's own limit (128x128x170: 24*128*128*170 bytes), and in
    FP32 (160x128x110, 2.25 M points). Bit for bit the apply with that
    schedule."""
    from paper_2005_13014_gb300.api import Program, device_field
    h = 3
    prog = Program(programs.HDIFF_VADVC, dtype)
    if sched:
        prog.set_schedule(**sched)
    else:
        prog.set_schedule(**dict(prog.schedule, sweep=0, slabs=0))
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


@pytest.mark.parametrize("n", [(256, 256, 24), (260, 256, 7)], ids=str)
def test_noalloc_f32_persistent_single_domain(liboec, n):
    """FP32 fields with 16-byte aligned rows and at least 65,536 columns: the
    default schedule (warp-row producer) runs as one persistent launch whose
    row-block counters and ticket sit in the fixed scratch after the column
    scratch and the hdiff planes (50.3 MB at 256x256x24). Bit for bit the
    apply with that schedule, twice in a row (the counters are reset by
    every call), and no bounded wait given up."""
    from paper_2005_13014_gb300.api import Program, device_field
    h = 3
    prog = Program(programs.HDIFF_VADVC, "f32")
    prog.set_schedule(**dict(prog.schedule, sweep=0, slabs=0))
    f = inputs.hdiff_vadvc_fields(*n, h, seed=78)
    d = [device_field(f[k], h, "f32", align_bytes=16) for k in ("u", "v", "w", "coeff")]
    ref = [device_field(np.zeros_like(f["u"]), h, "f32", align_bytes=16) for _ in range(2)]
    prog.apply(d, ref, (0, 0, 0), n, (h, h, h), [2.0])
    assert prog.launch_count() == 1   # the persistent form
    for call in range(2):
        got = [device_field(np.full_like(f["u"], 7.0), h, "f32", align_bytes=16) for _ in range(2)]
        assert _noalloc(liboec, "f32", d, got, n) == 0, liboec.oec_last_error()
        torch.cuda.synchronize()
        for g, r in zip(got, ref):
            assert torch.equal(g.interior((0, 0, 0), n), r.interior((0, 0, 0), n)), f"call {call}"
    assert liboec.oec_device_status(None) == 0


@pytest.mark.parametrize("n", [(2796203, 1, 1), (128, 128, 171)], ids=str)
def test_noalloc_rejects_oversized_domain(liboec, n):
    # more than the fixed 64 MiB even in the fused form (24 * ceil16(ni) *
    # ceil4(nj) * nk bytes): rejected before any launch (the pointers are
    # never dereferenced)
    d = L.FieldDesc()
    d.data, d.dtype, d.ndim = 1 << 30, L.F64, 3
    d.size = L.I64x3(n[0] + 6, n[1] + 6, n[2] + 6)
    d.stride = L.I64x3(1, n[0] + 6, (n[0] + 6) * (n[1] + 6))
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


def _noalloc(liboec, dtype, d, got, n):
    ins = (L.FieldDesc * 4)(*[x.desc() for x in d])
    outs = (L.FieldDesc * 2)(*[x.desc() for x in got])
    return liboec.oec_hdiff_vadvc_apply_noalloc(L.F64 if dtype == "f64" else L.F32, ins, outs, L.I64x3(0, 0, 0),
                                                L.I64x3(*n), 2.0, C.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_takes_no_device_memory_at_a_new_size(liboec):
    """A first call at a new domain size leaves the device's free memory as it
    was (every field is allocated beforehand); the same first apply through
    oec_program_apply allocates its scratch, which the same measurement sees."""
    from paper_2005_13014_gb300.api import Program, device_field
    h = 3
    fields = {}
    for n in ((64, 64, 20), (128, 96, 40)):
        f = inputs.hdiff_vadvc_fields(*n, h, seed=5)
        fields[n] = ([device_field(f[k], h, "f64") for k in ("u", "v", "w", "coeff")],
                     [device_field(np.zeros_like(f["u"]), h, "f64") for _ in range(2)],
                     [device_field(np.zeros_like(f["u"]), h, "f64") for _ in range(2)])
    a, b = (64, 64, 20), (128, 96, 40)
    assert _noalloc(liboec, "f64", fields[a][0], fields[a][1], a) == 0   # device code loaded, address looked up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    assert _noalloc(liboec, "f64", fields[b][0], fields[b][1], b) == 0, liboec.oec_last_error()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free1 == free0
    prog = Program(programs.HDIFF_VADVC, "f64")
    prog.set_schedule(**dict(prog.schedule, sweep=0, slabs=0))
    prog.apply(fields[b][0], fields[b][2], (0, 0, 0), b, (h, h, h), [2.0])
    torch.cuda.synchronize()
    free2 = torch.cuda.mem_get_info()[0]
    assert free2 < free1   # 40 B per point of scratch: about 20 MB
    for g, r in zip(fields[b][1], fields[b][2]):
        assert torch.equal(g.tensor, r.tensor)
