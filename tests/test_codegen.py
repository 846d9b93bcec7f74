"""The generic code generator: CUDA C++ generated from program IR for every
fusion x unroll variant compiles with NVRTC for sm_103a (host only), and the
generated kernels agree with the oracle's interpreter on the GPU."""

import numpy as np
import pytest

from conftest import TOL, rel_err
from oracle import program as OP
from oracle import stencils as S
from paper_2005_13014_gb300 import inputs, programs


def _prog(src, dtype="f32", generic=True):
    from paper_2005_13014_gb300.api import Program
    return Program(src, dtype, generic=generic)


@pytest.mark.parametrize("seed", [10000, 10001, 10002, 10050, 20007])
def test_generated_source_compiles(liboec, seed):
    p = _prog(inputs.random_dag(seed))
    src = p.generated_source((40, 24, 9), 60, 60 * 44, compile=True)
    # one output kernel per fusion x unroll variant, plus materialised stages
    assert src.count("__global__") >= 9
    assert "k_f1_u2_" in src and "k_f2_u4_" in src


def test_builtin_texts_compile_generically(liboec):
    for src in (programs.HDIFF, programs.FASTWAVES):
        for dt in ("f32", "f64"):
            _prog(src, dt).generated_source((33, 17, 5), 41, 41 * 25, compile=True)
    from paper_2005_13014_gb300 import _lib as L
    with pytest.raises(L.OecError) as e:
        _prog(programs.HDIFF_VADVC).generated_source((8, 8, 8), 16, 256)
    assert e.value.name == "UNSUPPORTED"


def test_offset_width_of_generated_kernels(liboec):
    """Generated kernels form the thread's element offset in 32-bit ints
    when every offset of the inferred ranges fits (OEC_INDEX_AUTO), in
    64-bit when the schedule asks for it (OEC_INDEX_64) or when the offsets
    do not fit; both compile."""
    p = _prog(inputs.random_dag(10003))
    src = p.generated_source((40, 24, 9), 60, 60 * 44, compile=True)
    assert "const int fo = " in src and "long long fo" not in src
    sched = p.schedule
    sched["index_bits"] = 64
    p.set_schedule(**sched)
    src = p.generated_source((40, 24, 9), 60, 60 * 44, compile=True)
    assert "const long long fo = " in src and "const int fo" not in src
    sched["index_bits"] = 0
    p.set_schedule(**sched)
    big = 1 << 28   # a plane stride of 2^28 elements: k offsets up to 9 * 2^28 > 2^31
    src = p.generated_source((40, 24, 9), 60, big, compile=False)
    assert "const long long fo = " in src and "const int fo" not in src


IF_SRC = """
input a, b
stage s = { let q = a[1,0,0] - a; return if (q > 0.0) { let t = q * b; yield t + 1.0 } else { yield b[0,1,0] - q } }
stage r = if (s <= 0.5) { yield s * 2.0 } else { let u = s - b[0,0,1]; yield min(u, s) }
output s, r
"""
# the same program with select and the regions' lets bound in the stage
SEL_SRC = """
input a, b
stage s = { let q = a[1,0,0] - a; let t = q * b; return select(q > 0.0, t + 1.0, b[0,1,0] - q) }
stage r = { let u = s - b[0,0,1]; return select(s <= 0.5, s * 2.0, min(u, s)) }
output s, r
"""


def test_if_regions_lower_to_select(liboec):
    """Region control flow (§IV-C, scf.if): the library reads an if whose
    regions are pure as the select of their yields, with each region's lets
    bound in the stage, so the program's inferred ranges, generated kernels
    and tuning-database key are those of the select form. Written with if,
    hdiff is still recognised and runs its hand-written kernels."""
    from paper_2005_13014_gb300 import _lib as L
    for dt in ("f32", "f64"):
        a, b = _prog(IF_SRC, dt), _prog(SEL_SRC, dt)
        assert a.generated_source((33, 17, 5), 41, 41 * 25, compile=True) == \
            b.generated_source((33, 17, 5), 41, 41 * 25)
        for x in range(2):
            assert a.input_range(x, (0, 0, 0), (8, 8, 4)) == b.input_range(x, (0, 0, 0), (8, 8, 4))
    assert _prog(IF_SRC).input_range(1, (0, 0, 0), (8, 8, 4)) == ((0, 0, 0), (8, 9, 5))
    hd = programs.HDIFF.replace("return select(f*(in[1,0,0] - in) > 0.0, 0.0, f)",
                                "return if (f*(in[1,0,0] - in) > 0.0) { yield 0.0 } else { yield f }")
    assert hd != programs.HDIFF
    assert _prog(hd, "f64", generic=False).kind == "hdiff"
    for bad in ("input a\nstage s = if (a > 0.0) { let t = a; yield t } else { yield t }\noutput s\n",
                "input a\nstage s = if (a > 0.0) { yield a }\noutput s\n",
                "input a\nstage s = if (a) { yield a } else { yield a }\noutput s\n",
                "input a\nstage yield = a\noutput yield\n"):
        with pytest.raises(L.OecError) as e:
            _prog(bad)
        assert e.value.name == "PARSE"


def test_double_float_generated_source_compiles(liboec):
    """FP64 programs with arith 1: the generated module carries the
    double-float arithmetic and compiles with NVRTC for sm_103a."""
    for src in (programs.TESTSET["hadvuv"][0], programs.TESTSET["p_grad_c"][0], inputs.random_dag(10001)):
        p = _prog(src, "f64")
        p.set_schedule(fusion=0, arith=1)
        gen = p.generated_source((33, 17, 5), 41, 41 * 25, compile=True)
        assert "struct __align__(8) df64" in gen and "cvt_in(__ldg(" in gen and "df_to_double" in gen
    from paper_2005_13014_gb300 import _lib as L
    with pytest.raises(L.OecError) as e:
        _prog(inputs.random_dag(10001), "f32").set_schedule(fusion=0, arith=1)
    assert e.value.name == "UNSUPPORTED"


def test_injected_compile_failure(liboec, monkeypatch):
    from paper_2005_13014_gb300 import _lib as L
    monkeypatch.setenv("OEC_FAULT", "compile")
    with pytest.raises(L.OecError) as e:
        _prog(inputs.random_dag(10001)).generated_source((8, 8, 4), 20, 400, compile=True)
    assert e.value.name == "COMPILE"


# ------------------------------------------------------------------ GPU parity

def _dag_case(seed, n, dtype, schedules, h=(8, 8, 4)):
    torch = pytest.importorskip("torch")
    from paper_2005_13014_gb300.api import device_field
    src = inputs.random_dag(seed)
    prog = OP.parse(src)
    fields = {}
    for idx, name in enumerate(prog.inputs):
        arr = np.random.default_rng(seed * 10 + idx).uniform(-1, 1, (n[2] + 2 * h[2], n[1] + 2 * h[1], n[0] + 2 * h[0]))
        if dtype == "f32":
            arr = arr.astype(np.float32).astype(np.float64)
        fields[name] = arr
    ref = OP.run_staged(prog, {k: S.Grid.storage(v, h) for k, v in fields.items()}, (0, 0, 0), n)
    p = _prog(src, dtype)
    din = [device_field(fields[nm], h, dtype) for nm in prog.inputs]
    errs = []
    for sched in schedules:
        p.set_schedule(**sched)
        outs = [device_field(np.full_like(fields[prog.inputs[0]], 7.0), h, dtype) for _ in prog.outputs]
        p.apply(din, outs, (0, 0, 0), n, h)
        torch.cuda.synchronize()
        for o, name in zip(outs, prog.outputs):
            got = o.interior((0, 0, 0), n).cpu().numpy().astype(np.float64)
            errs.append(rel_err(got, ref[name]))
            full = o.tensor.cpu().numpy()
            oi, oj, ok = o.origin
            mask = np.ones(full.shape, bool)
            mask[ok:ok + n[2], oj:oj + n[1], oi:oi + n[0]] = False
            assert np.all(full[mask] == 7.0), "write outside the domain"
    return max(errs)


ALL_VARIANTS = [dict(fusion=f, unroll=u, tile_i=ti, tile_j=tj)
                for f in (0, 1, 2) for u in (1, 2, 4) for (ti, tj) in ((32, 4), (64, 2))]


@pytest.mark.gpu
@pytest.mark.parametrize("seed", list(range(10000, 10012)))
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_generated_kernels_match_oracle(seed, dtype):
    assert _dag_case(seed, (37, 21, 7), dtype, ALL_VARIANTS) <= TOL[dtype]


@pytest.mark.gpu
def test_generated_kernels_short_columns_and_config_size():
    assert _dag_case(10005, (19, 5, 3), "f64", ALL_VARIANTS) <= TOL["f64"]
    big = [dict(fusion=0, unroll=2, tile_i=64, tile_j=4), dict(fusion=1, unroll=1, tile_i=128, tile_j=2),
           dict(fusion=2, unroll=4, tile_i=32, tile_j=8)]
    assert _dag_case(10100, (256, 256, 80), "f32", big) <= TOL["f32"]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_builtin_programs_through_the_generator(dtype):
    """hdiff and fastwaves forced through the code generator agree with the
    hand-written oracle functions."""
    torch = pytest.importorskip("torch")
    from paper_2005_13014_gb300.api import device_field
    n, h = (45, 19, 6), 3
    rnd = (lambda a: a.astype(np.float32).astype(np.float64)) if dtype == "f32" else (lambda a: a)
    f = {k: rnd(v) for k, v in inputs.hdiff_fields(*n, h).items()}
    p = _prog(programs.HDIFF, dtype)
    for sched in ALL_VARIANTS[::3]:
        p.set_schedule(**sched)
        out = device_field(np.zeros_like(f["in"]), h, dtype)
        p.apply([device_field(f["in"], h, dtype), device_field(f["coeff"], h, dtype)], [out], (0, 0, 0), n, (h, h, h))
        torch.cuda.synchronize()
        ref = S.hdiff(S.Grid.storage(f["in"], h), S.Grid.storage(f["coeff"], h), (0, 0, 0), n)
        assert rel_err(out.interior((0, 0, 0), n).cpu().numpy(), ref) <= TOL[dtype]
    fw = {k: rnd(v) for k, v in inputs.fastwaves_fields(*n, h).items()}
    p = _prog(programs.FASTWAVES, dtype)
    G = {k: S.Grid.storage(v, h) for k, v in fw.items()}
    ru, rv = S.fastwaves(G, (0, 0, 0), n, 0.5, 0.0625)
    for sched in ALL_VARIANTS[1::3]:
        p.set_schedule(**sched)
        outs = [device_field(np.zeros_like(fw["pp"]), h, dtype) for _ in range(2)]
        p.apply([device_field(fw[k], h, dtype) for k in inputs.FASTWAVES_NAMES], outs, (0, 0, 0), n, (h, h, h),
                [0.5, 0.0625])
        torch.cuda.synchronize()
        assert rel_err(outs[0].interior((0, 0, 0), n).cpu().numpy(), ru) <= TOL[dtype]
        assert rel_err(outs[1].interior((0, 0, 0), n).cpu().numpy(), rv) <= TOL[dtype]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_if_program_matches_oracle(dtype):
    """A program with region control flow, through the generated kernels
    (inlined and stage by stage), against the oracle, which runs only the
    region each point's condition picks."""
    torch = pytest.importorskip("torch")
    from paper_2005_13014_gb300.api import device_field
    n, h = (37, 21, 7), (2, 2, 2)
    prog = OP.parse(IF_SRC)
    fields = {}
    for x, name in enumerate(prog.inputs):
        arr = np.random.default_rng(90 + x).uniform(-1, 1, (n[2] + 4, n[1] + 4, n[0] + 4))
        fields[name] = arr.astype(np.float32).astype(np.float64) if dtype == "f32" else arr
    ref = OP.run_staged(prog, {k: S.Grid.storage(v, h) for k, v in fields.items()}, (0, 0, 0), n)
    p = _prog(IF_SRC, dtype)
    din = [device_field(fields[nm], h, dtype) for nm in prog.inputs]
    for sched in (dict(fusion=0, unroll=1, tile_i=32, tile_j=4), dict(fusion=1, unroll=2, tile_i=64, tile_j=2)):
        p.set_schedule(**sched)
        outs = [device_field(np.zeros_like(fields["a"]), h, dtype) for _ in prog.outputs]
        p.apply(din, outs, (0, 0, 0), n, h)
        torch.cuda.synchronize()
        for o, name in zip(outs, prog.outputs):
            got = o.interior((0, 0, 0), n).cpu().numpy().astype(np.float64)
            assert rel_err(got, ref[name]) <= TOL[dtype]


def _as_select(text):
    """The textual lowering of region ifs without lets to selects:
    if (c) { yield a } else { yield b }  ->  select(c, a, b)."""
    out, i = [], 0
    while True:
        j = text.find("if (", i)
        if j < 0:
            return "".join(out) + text[i:]
        out.append(text[i:j])
        pos, parts = j + 3, []
        for open_, close in (("(", ")"), ("{", "}"), ("{", "}")):
            pos = text.index(open_, pos)
            depth, m = 1, pos + 1
            while depth:
                depth += {open_: 1, close: -1}.get(text[m], 0)
                m += 1
            body = text[pos + 1:m - 1].strip()
            parts.append(_as_select(body[len("yield"):].strip() if body.startswith("yield") else body))
            pos = m
        out.append(f"select({parts[0]}, {parts[1]}, {parts[2]})")
        i = pos


@pytest.mark.parametrize("name", ["hadvuv", "hadvuv5th", "fvtp2d_qi", "fvtp2d_qj", "fvtp2d_flux"])
def test_testset_if_regions_generate_the_select_kernels(liboec, name):
    src = programs.TESTSET[name][0]
    sel = _as_select(src)
    assert "if (" in src and "if (" not in sel and "select(" in sel
    for dt in ("f32", "f64"):
        assert _prog(src, dt).generated_source((33, 17, 5), 41, 41 * 25) == \
            _prog(sel, dt).generated_source((33, 17, 5), 41, 41 * 25)
