"""The Python front end (dsl.py): traced programs print the textual form,
programs written like the library's own are recognised as them (and get the
hand-written kernels), and the oracle computes the same bits from the traced
text as from the hand-written text. No GPU."""

import numpy as np
import pytest

from oracle import program as OP
from oracle import stencils as S
from paper_2005_13014_gb300 import dsl, inputs, programs


def _hdiff_body(x, coeff, tag):
    lap = dsl.stage(4.0 * x - x[-1, 0, 0] - x[1, 0, 0] - x[0, -1, 0] - x[0, 1, 0], "lap" + tag)
    f = dsl.let(lap[1, 0, 0] - lap)
    flx = dsl.stage(dsl.select(f * (x[1, 0, 0] - x) > 0.0, 0.0, f), "flx" + tag)
    f = dsl.let(lap[0, 1, 0] - lap)
    fly = dsl.stage(dsl.select(f * (x[0, 1, 0] - x) > 0.0, 0.0, f), "fly" + tag)
    return x - coeff * ((flx - flx[-1, 0, 0]) + (fly - fly[0, -1, 0]))


@dsl.program
def HDIFF(inp: dsl.Field, coeff: dsl.Field):
    return {"out": _hdiff_body(inp, coeff, "")}


@dsl.program
def HDIFF_VADVC(u: dsl.Field, v: dsl.Field, w: dsl.Field, coeff: dsl.Field, dtr: dsl.Param):
    ud = dsl.stage(_hdiff_body(u, coeff, "u"), "ud")
    vd = dsl.stage(_hdiff_body(v, coeff, "v"), "vd")
    wf = dsl.stage(0.5 * (w + w[1, 0, 0]), "wf")
    a = dsl.stage(dsl.select(dsl.kpos > 0.0, -0.25 * wf, 0.0), "a")
    c = dsl.stage(dsl.select(dsl.kpos < dsl.ksize - 1.0, 0.25 * wf[0, 0, 1], 0.0), "c")
    b = dsl.stage(dtr + dsl.absolute(a) + dsl.absolute(c), "b")

    def rhs(x):
        return dtr * x - 0.5 * (dsl.select(dsl.kpos > 0.0, a * (x[0, 0, -1] - x), 0.0)
                                + dsl.select(dsl.kpos < dsl.ksize - 1.0, c * (x[0, 0, 1] - x), 0.0))
    du = dsl.stage(rhs(ud), "du")
    dv = dsl.stage(rhs(vd), "dv")
    return dsl.thomas(a, b, c, du, dv)


@dsl.program
def UVBKE(uc: dsl.Field, vc: dsl.Field, cosa: dsl.Field, rsina: dsl.Field, dt5: dsl.Param):
    ub = dt5 * (uc[0, -1, 0] + uc - (vc[-1, 0, 0] + vc) * cosa) * rsina
    vb = dt5 * (vc[-1, 0, 0] + vc - (uc[0, -1, 0] + uc) * cosa) * rsina
    return {"ub": ub, "vb": vb}


def _same_results(text_a, text_b, fields, n, h, params=()):
    pa, pb = OP.parse(text_a), OP.parse(text_b)
    G = {k: S.Grid.storage(v, h) for k, v in fields.items()}
    ga = [G[x] for x in fields]
    ra = OP.run_staged(pa, dict(zip(pa.inputs, ga)), (0, 0, 0), n, dict(zip(pa.params, params)))
    rb = OP.run_staged(pb, dict(zip(pb.inputs, ga)), (0, 0, 0), n, dict(zip(pb.params, params)))
    for oa, ob in zip(pa.outputs, pb.outputs):
        assert np.array_equal(ra[oa], rb[ob])


def test_hdiff_text_and_bits():
    assert HDIFF.inputs == ["inp", "coeff"] and HDIFF.outputs == ["out"] and HDIFF.params == []
    assert "let l0 = lap[1,0,0] - lap" in HDIFF.text
    f = inputs.hdiff_fields(13, 9, 3, 2, seed=5)
    _same_results(HDIFF.text, programs.HDIFF, {"in": f["in"], "coeff": f["coeff"]}, (13, 9, 3), 2)


def test_hdiff_vadvc_text_and_bits():
    assert "column x" in HDIFF_VADVC.text and HDIFF_VADVC.params == ["dtr"] and len(HDIFF_VADVC.outputs) == 2
    f = inputs.hdiff_vadvc_fields(11, 7, 6, 3, seed=6)
    _same_results(HDIFF_VADVC.text, programs.HDIFF_VADVC, {k: f[k] for k in ("u", "v", "w", "coeff")},
                  (11, 7, 6), 3, params=(2.0,))


def test_generic_program_bits():
    f = inputs.testset_fields("uvbke", 10, 8, 3, 2)
    _same_results(UVBKE.text, programs.UVBKE, f, (10, 8, 3), 2, params=(0.5,))


def test_recognised_as_hand_written_programs(liboec):
    assert HDIFF.compile("f64").kind == "hdiff"
    assert HDIFF_VADVC.compile("f32").kind == "hdiff_vadvc"
    assert UVBKE.compile("f32").kind == "generic"


def test_if_regions(liboec):
    """dsl.if_ prints a region if; hdiff written with it is still hdiff, and
    the oracle gives the same bits as for the select form."""
    @dsl.program
    def hd_if(inp: dsl.Field, coeff: dsl.Field):
        lap = dsl.stage(4.0 * inp - inp[-1, 0, 0] - inp[1, 0, 0] - inp[0, -1, 0] - inp[0, 1, 0], "lap")
        f = dsl.let(lap[1, 0, 0] - lap)
        flx = dsl.stage(dsl.if_(f * (inp[1, 0, 0] - inp) > 0.0, 0.0, f), "flx")
        f = dsl.let(lap[0, 1, 0] - lap)
        fly = dsl.stage(dsl.if_(f * (inp[0, 1, 0] - inp) > 0.0, 0.0, f), "fly")
        return {"out": inp - coeff * ((flx - flx[-1, 0, 0]) + (fly - fly[0, -1, 0]))}
    assert "return if (l0*(inp[1,0,0] - inp) > 0.0) { yield 0.0 } else { yield l0 }" in hd_if.text
    assert hd_if.compile("f64").kind == "hdiff"
    f = inputs.hdiff_fields(9, 7, 3, 2, seed=4)
    _same_results(hd_if.text, programs.HDIFF, {"inp": f["in"], "coeff": f["coeff"]}, (9, 7, 3), 2)
    with pytest.raises(TypeError, match="comparison"):
        @dsl.program
        def bad(a: dsl.Field):
            return dsl.if_(a, a, a)


def test_indexing_an_expression_makes_a_stage():
    @dsl.program
    def p(a: dsl.Field):
        return (a + 1.0)[1, 0, 0] * -2.0
    assert p.text.splitlines()[1] == "stage s0 = a + 1.0"
    assert p.text.splitlines()[2] == "stage s1 = s0[1,0,0]*-2.0"
    # a is read over i in [1, 5): one column inside the domain below, one above
    assert OP.input_halo(OP.parse(p.text), (0, 0, 0), (4, 4, 4))["a"] == ((-1, 1), (0, 0), (0, 0))


def test_misuse_is_reported():
    with pytest.raises(TypeError, match="select"):
        @dsl.program
        def p1(a: dsl.Field):
            return a if a > 0.0 else -a
    with pytest.raises(TypeError, match="three integers"):
        @dsl.program
        def p2(a: dsl.Field):
            return a[1, 0]
    with pytest.raises(ValueError, match="let"):
        @dsl.program
        def p3(a: dsl.Field):
            dsl.let(a * 2.0)
            return a
    with pytest.raises(RuntimeError, match="traced"):
        dsl.stage(1.0)


@pytest.mark.gpu
def test_traced_programs_on_the_gpu():
    """The traced hdiff+vadvc runs the hand-written kernels and the traced
    uvbke the generated ones, with the bits of the library's own texts."""
    torch = pytest.importorskip("torch")
    from paper_2005_13014_gb300.api import Program, device_field
    n, h = (37, 23, 11), 3
    f = inputs.hdiff_vadvc_fields(*n, h, seed=7)
    res = []
    for p in (HDIFF_VADVC.compile("f64"), Program(programs.HDIFF_VADVC, "f64")):
        p.set_schedule(fusion=1, tile_i=32, tile_j=8, k_chunk=4, arith=2)
        o = [device_field(np.zeros_like(f["u"]), h, "f64") for _ in range(2)]
        p.apply([device_field(f[k], h, "f64") for k in ("u", "v", "w", "coeff")], o, (0, 0, 0), n, (h, h, h), [2.0])
        torch.cuda.synchronize()
        res.append([x.tensor.cpu().numpy() for x in o])
    assert all(np.array_equal(a, b) for a, b in zip(*res))
    g = inputs.testset_fields("uvbke", *n, h)
    res = []
    for p in (UVBKE.compile("f32"), Program(programs.UVBKE, "f32")):
        o = [device_field(np.zeros_like(g["uc"]), h, "f32") for _ in range(2)]
        p.apply([device_field(g[k], h, "f32") for k in ("uc", "vc", "cosa", "rsina")], o, (0, 0, 0), n, (h, h, h),
                [0.5])
        torch.cuda.synchronize()
        res.append([x.tensor.cpu().numpy() for x in o])
    assert all(np.array_equal(a, b) for a, b in zip(*res))
