"""Launch counts and per-kernel timing of applies (oec_program_launch_count,
oec_program_set_timing, oec_program_kernel_times): every schedule reports the
kernels it launches, and the recorded per-kernel durations tile the apply."""

import numpy as np
import pytest

from paper_2005_13014_gb300 import inputs, programs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _fields(names, n, h, dtype, seed=7):
    from paper_2005_13014_gb300.api import device_field
    return [device_field(inputs.field_uniform(n, h, -1.0, 1.0, seed + x), h, dtype) for x, _ in enumerate(names)]


CASES = [
    # (program, dtype, schedule, kernels per apply)
    ("HDIFF", "f64", dict(fusion=0, staging=1, tile_i=64, tile_j=4), 1),
    ("HDIFF", "f64", dict(fusion=0, staging=1, tile_i=64, tile_j=4, arith=2), 1),
    ("HDIFF", "f32", dict(fusion=0, staging=0, tile_i=32, tile_j=4, unroll=2), 1),
    ("HDIFF", "f32", dict(fusion=1), 4),
    ("HDIFF_VADVC", "f64", dict(fusion=0, staging=1, tile_i=16, tile_j=4), 1),
    ("HDIFF_VADVC", "f64", dict(fusion=1, arith=2), 2),
    ("HDIFF_VADVC", "f32", dict(fusion=1), 2),
    ("FASTWAVES", "f32", dict(fusion=1), 6),
    ("FASTWAVES", "f64", dict(fusion=0, staging=0, tile_i=32, tile_j=4, unroll=2), 1),
]


@pytest.mark.parametrize("name,dtype,sched,nk", CASES)
def test_launch_count_and_kernel_times(name, dtype, sched, nk):
    from paper_2005_13014_gb300.api import Program
    p = Program(getattr(programs, name), dtype)
    p.set_schedule(**sched)
    n, h = (70, 37, 9), 3
    din = _fields(range(p.n_inputs), n, h, dtype)
    dout = _fields(range(p.n_outputs), n, h, dtype, seed=100)
    params = programs.PARAMS[name.lower()]
    assert p.launch_count() == 0
    p.apply(din, dout, (0, 0, 0), n, (h, h, h), params)
    assert p.launch_count() == nk
    # empty domain: nothing launched
    p.apply(din, dout, (0, 0, 0), (0, n[1], n[2]), (h, h, h), params)
    assert p.launch_count() == 0
    stream = torch.cuda.Stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p.set_timing(True)
    with torch.cuda.stream(stream):
        e0.record(stream)
        for _ in range(3):
            p.apply(din, dout, (0, 0, 0), n, (h, h, h), params, stream=stream)
        e1.record(stream)
    p.set_timing(False)
    p.apply(din, dout, (0, 0, 0), n, (h, h, h), params, stream=stream)   # not recorded
    t = p.kernel_times()
    torch.cuda.synchronize()
    assert t.shape == (3, nk)
    assert np.all(t > 0)
    assert t.sum() <= e0.elapsed_time(e1) * 1.01 + 1e-3
    assert p.kernel_times().shape == (0, 0)   # forgotten after reading


def test_bound_apply_matches_apply():
    """Program.bind marshals once; its call enqueues the same apply."""
    from paper_2005_13014_gb300.api import Program
    p = Program(programs.HDIFF, "f32")
    n, h = (70, 37, 9), 3
    din = _fields(range(2), n, h, "f32")
    a, b = _fields(range(1), n, h, "f32", seed=100), _fields(range(1), n, h, "f32", seed=200)
    p.apply(din, a, (0, 0, 0), n, (h, h, h))
    call = p.bind(din, b, (0, 0, 0), n, (h, h, h))
    call()
    call()
    torch.cuda.synchronize()
    assert torch.equal(a[0].interior((0, 0, 0), n), b[0].interior((0, 0, 0), n))
    assert p.launch_count() == 1


def test_captured_generated_launch_keeps_its_parameters():
    """A generated program's scalar parameters travel with each launch: a
    CUDA graph captured with one value replays that value after the host
    array is gone and after applies with other values."""
    import gc
    from paper_2005_13014_gb300.api import Program
    src = programs.TESTSET["p_grad_c"][0]
    p = Program(src, "f64", generic=True)
    p.set_schedule(fusion=0)
    n, h = (40, 24, 6), 3
    f = inputs.testset_fields("p_grad_c", *n, h)
    from paper_2005_13014_gb300.api import device_field
    din = [device_field(f[k], h, "f64") for k in inputs.TESTSET_INPUTS["p_grad_c"]]
    outs = {x: [device_field(np.zeros_like(f["uc"]), h, "f64") for _ in range(2)] for x in "abc"}
    p.apply(din, outs["a"], (0, 0, 0), n, (h, h, h), [0.01])
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        p.apply(din, outs["b"], (0, 0, 0), n, (h, h, h), [0.01], stream=s)
    p.apply(din, outs["c"], (0, 0, 0), n, (h, h, h), [0.5])
    gc.collect()
    junk = [np.full(1024, 7.0) for _ in range(64)]   # reuse freed host memory
    with torch.cuda.stream(s):
        g.replay()
    torch.cuda.synchronize()
    for x in range(2):
        a, b, c = (outs[y][x].interior((0, 0, 0), n) for y in "abc")
        assert torch.equal(a, b)
        assert not torch.equal(a, c)
    del junk


def test_bounded_wait_gives_up_and_is_reported():
    """The give-up path of the kernels' bounded mbarrier waits: a wait on a
    phase that never completes stops after its poll limit, the timeout is
    reported once by oec_device_status, and the context keeps working."""
    from paper_2005_13014_gb300 import _lib as L
    lib = L.lib()
    assert lib.oec_device_status(None) == 0
    assert lib.oec_device_wait_selftest(64, None) == 0
    assert lib.oec_device_status(None) == -10   # OEC_ERR_TIMEOUT
    assert "gave up" in lib.oec_last_error().decode()
    assert lib.oec_device_status(None) == 0     # cleared
    t = torch.ones(1024, device="cuda")
    assert float((t * 2).sum()) == 2048.0
    assert lib.oec_device_wait_selftest(0, None) == -1


def test_batch_counter_wait_gives_up_and_is_reported():
    """The persistent staged batch's bounded wait on its row-block counters: a
    sweep item whose counter nothing releases gives up after its poll limit,
    skips the item, is reported once by oec_device_status, and the context
    keeps working."""
    from paper_2005_13014_gb300 import _lib as L
    lib = L.lib()
    assert lib.oec_device_status(None) == 0
    assert lib.oec_batch_wait_selftest(64, None) == 0
    assert lib.oec_device_status(None) == -10   # OEC_ERR_TIMEOUT
    assert "gave up" in lib.oec_last_error().decode()
    assert lib.oec_device_status(None) == 0
    t = torch.ones(1024, device="cuda")
    assert float((t * 3).sum()) == 3072.0


def test_injected_scratch_allocation_failure(monkeypatch):
    """OEC_FAULT=alloc: an apply that needs scratch returns OEC_ERR_CUDA with
    the reason and enqueues nothing; without it the same program runs and
    agrees with the library's native-FP64 unfused kernels."""
    from paper_2005_13014_gb300 import _lib as L
    from paper_2005_13014_gb300.api import Program, device_field
    n, h = (40, 24, 9), 3
    f = inputs.hdiff_vadvc_fields(*n, h, seed=5)
    din = [device_field(f[k], h, "f64") for k in ("u", "v", "w", "coeff")]
    outs = [device_field(np.full_like(f["u"], 3.0), h, "f64") for _ in range(2)]
    p = Program(programs.HDIFF_VADVC, "f64")
    p.set_schedule(fusion=1, staging=0, tile_i=32, tile_j=8, k_chunk=4, arith=2)
    monkeypatch.setenv("OEC_FAULT", "alloc")
    with pytest.raises(L.OecError) as e:
        p.apply(din, outs, (0, 0, 0), n, (h, h, h), [2.0])
    assert e.value.name == "CUDA" and "OEC_FAULT=alloc" in str(e.value)
    assert p.launch_count() == 0
    torch.cuda.synchronize()
    assert bool((outs[0].tensor == 3.0).all())
    monkeypatch.delenv("OEC_FAULT")
    p.apply(din, outs, (0, 0, 0), n, (h, h, h), [2.0])
    r = Program(programs.HDIFF_VADVC, "f64")
    r.set_schedule(fusion=1, arith=0)
    ref = [device_field(np.zeros_like(f["u"]), h, "f64") for _ in range(2)]
    r.apply(din, ref, (0, 0, 0), n, (h, h, h), [2.0])
    torch.cuda.synchronize()
    for o, q in zip(outs, ref):
        a = o.interior((0, 0, 0), n).cpu().numpy()
        b = q.interior((0, 0, 0), n).cpu().numpy()
        assert np.max(np.abs(a - b)) <= 1e-13 * np.max(np.abs(b))
