"""Fields in host memory (oec_program_apply_host): the library copies the
inputs to its device staging, applies, and copies each output's domain box
back. The bits must equal a device apply with the same schedule, the host
outputs outside the domain must stay as they were, and calls issued back to
back (staging sets used in turn, input copies on the library's stream) must
each produce their own result."""

import numpy as np
import pytest

from conftest import TOL, rel_err
from oracle import stencils as S
from paper_2005_13014_gb300 import inputs, programs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SENTINEL = 7.0


def _hv(dtype, sched, n, h, seed):
    from paper_2005_13014_gb300.api import Program
    f = inputs.hdiff_vadvc_fields(*n, h, seed=seed)
    if dtype == "f32":
        f = {k: v.astype(np.float32).astype(np.float64) for k, v in f.items()}
    p = Program(programs.HDIFF_VADVC, dtype)
    p.set_schedule(**sched)
    return f, p


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("dtype,sched", [("f64", dict(fusion=1, tile_i=32, tile_j=8, k_chunk=4, arith=2)),
                                         ("f64", dict(fusion=0, staging=1, tile_i=32, tile_j=4, arith=1)),
                                         ("f32", dict(fusion=1, tile_i=32, tile_j=4, unroll=2, k_chunk=8, arith=1))],
                         ids=str)
def test_apply_host_equals_device_apply(dtype, sched, pinned):
    from paper_2005_13014_gb300.api import device_field, host_field
    n, h = (37, 23, 11), 3
    f, p = _hv(dtype, sched, n, h, seed=61)
    hin = [host_field(f[k], h, dtype, pinned=pinned) for k in ("u", "v", "w", "coeff")]
    hout = [host_field(np.full_like(f["u"], SENTINEL), h, dtype, pinned=pinned) for _ in range(2)]
    p.apply_host(hin, hout, (0, 0, 0), n, (h, h, h), [2.0])
    torch.cuda.synchronize()
    din = [device_field(f[k], h, dtype) for k in ("u", "v", "w", "coeff")]
    dout = [device_field(np.full_like(f["u"], SENTINEL), h, dtype) for _ in range(2)]
    p.apply(din, dout, (0, 0, 0), n, (h, h, h), [2.0])
    torch.cuda.synchronize()
    for a, b in zip(hout, dout):
        assert np.array_equal(a.tensor.numpy(), b.tensor.cpu().numpy())   # domain equal, outside untouched
    G = {k: S.Grid.storage(v, h) for k, v in f.items()}
    ru, _ = S.hdiff_vadvc(G["u"], G["v"], G["w"], G["coeff"], (0, 0, 0), n, 2.0)
    assert rel_err(hout[0].interior((0, 0, 0), n).numpy().astype(np.float64), ru) <= TOL[dtype]


def test_apply_host_back_to_back_calls():
    """Five calls issued without synchronising, each with its own inputs and
    outputs: sets alternate, the next call's inputs cross while this one
    computes; every call's outputs are its own."""
    from paper_2005_13014_gb300.api import device_field, host_field
    n, h, dtype = (64, 40, 17), 3, "f64"
    sched = dict(fusion=1, tile_i=32, tile_j=8, k_chunk=4, arith=2)
    runs = []
    for c in range(5):
        f, p = _hv(dtype, sched, n, h, seed=70 + c)
        runs.append(f)
    hins = [[host_field(f[k], h, dtype) for k in ("u", "v", "w", "coeff")] for f in runs]
    houts = [[host_field(np.full_like(f["u"], SENTINEL), h, dtype) for _ in range(2)] for f in runs]
    for hi, ho in zip(hins, houts):
        p.apply_host(hi, ho, (0, 0, 0), n, (h, h, h), [2.0])
    torch.cuda.synchronize()
    for f, ho in zip(runs, houts):
        din = [device_field(f[k], h, dtype) for k in ("u", "v", "w", "coeff")]
        dout = [device_field(np.full_like(f["u"], SENTINEL), h, dtype) for _ in range(2)]
        p.apply(din, dout, (0, 0, 0), n, (h, h, h), [2.0])
        torch.cuda.synchronize()
        for a, b in zip(ho, dout):
            assert np.array_equal(a.tensor.numpy(), b.tensor.cpu().numpy())


def test_apply_host_plane_pitch_not_whole_rows():
    """Fields whose k stride is not a multiple of the j stride: the outputs
    come back level by level."""
    from paper_2005_13014_gb300.api import Field, Program, device_field
    n, h = (30, 12, 6), 2
    f = inputs.hdiff_fields(*n, h, seed=62)
    nk, nj, ni = f["in"].shape
    plane = nj * ni + 3

    def strided(arr):
        buf = torch.full((nk * plane,), SENTINEL, dtype=torch.float64).pin_memory()
        t = buf.as_strided((nk, nj, ni), (plane, ni, 1))
        t.copy_(torch.from_numpy(arr))
        return Field(t, (h, h, h))

    hin = [strided(f["in"]), strided(f["coeff"])]
    hout = strided(np.full_like(f["in"], SENTINEL))
    p = Program(programs.HDIFF, "f64")
    p.set_schedule(fusion=0, staging=1, tile_i=32, tile_j=4, k_chunk=2, arith=2)
    p.apply_host(hin, [hout], (0, 0, 0), n, (h, h, h))
    torch.cuda.synchronize()
    dout = device_field(np.full_like(f["in"], SENTINEL), h, "f64")
    p.apply([device_field(f["in"], h, "f64"), device_field(f["coeff"], h, "f64")], [dout], (0, 0, 0), n,
            (h, h, h))
    torch.cuda.synchronize()
    assert np.array_equal(hout.tensor.numpy(), dout.tensor.cpu().numpy())
