"""Host-side tests of liboec's C ABI: every declared symbol is exported, the
builtin programs are recognised by structure, shape inference agrees with the
oracle's independent implementation (paper §V-B), and validation rejects bad
calls before any GPU work (fake device pointers are never dereferenced)."""

import ctypes as C

import numpy as np
import pytest

from oracle import program as OP
from paper_2005_13014_gb300 import _lib as L
from paper_2005_13014_gb300 import inputs, programs


def test_every_declared_symbol_is_exported(liboec):
    names = L.declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(liboec, n), n


def _prog(src, dtype="f64", generic=False):
    from paper_2005_13014_gb300.api import Program
    return Program(src, dtype=dtype, generic=generic)


def test_builtin_programs_recognised(liboec):
    assert _prog(programs.HDIFF).kind == "hdiff"
    assert _prog(programs.HDIFF_VADVC).kind == "hdiff_vadvc"
    assert _prog(programs.FASTWAVES, "f32").kind == "fastwaves"
    assert _prog(programs.HDIFF, generic=True).kind == "generic"
    renamed = (programs.HDIFF.replace("lap", "L0").replace("coeff", "kappa").replace("flx", "fx")
               .replace(" in", " phi").replace("(in", "(phi").replace("*in", "*phi").replace(",in", ",phi"))
    assert _prog("# renamed\n" + renamed).kind == "hdiff"
    changed = programs.HDIFF.replace("4.0*in", "4.5*in")
    assert _prog(changed).kind == "generic"


def test_parse_errors_are_reported(liboec):
    for bad in ["input a\nstage b = a[1,0]\noutput b", "input a\nstage b = c\noutput b", "input a\nstage b = a\n",
                "input a\nstage b = a\nstage b = a\noutput b", "input a\nstage b = a $\noutput b"]:
        with pytest.raises(L.OecError) as e:
            _prog(bad)
        assert e.value.name == "PARSE"
        assert "line" in str(e.value)


def _oracle_ranges(src, lb, ub):
    prog = OP.parse(src)
    r = OP.infer_ranges(prog, lb, ub)
    out = []
    for n in prog.inputs:
        if n in r:
            out.append((tuple(x[0] for x in r[n]), tuple(x[1] for x in r[n])))
        else:
            out.append((tuple(lb), tuple(lb)))
    return out


@pytest.mark.parametrize("src", [programs.HDIFF, programs.HDIFF_VADVC, programs.FASTWAVES]
                         + [t[0] for t in programs.TESTSET.values()]
                         + [inputs.random_dag(s) for s in range(10000, 10030)])
def test_input_ranges_match_oracle_shape_inference(liboec, src):
    p = _prog(src)
    lb, ub = (3, -2, 1), (40, 17, 9)
    want = _oracle_ranges(src, lb, ub)
    for x in range(p.n_inputs):
        assert p.input_range(x, lb, ub) == want[x]


def test_algorithmic_bytes_hdiff_64():
    p = _prog(programs.HDIFF)
    # in over [-2,66)^2 x 60, coeff and out over the 64x64x60 interior
    assert p.algorithmic_bytes((0, 0, 0), (64, 64, 60)) == 8 * (68 * 68 * 60 + 2 * 64 * 64 * 60)


def _fake(addr, shape, origin, dtype=L.F64):
    d = L.FieldDesc()
    d.data = addr
    d.dtype = dtype
    d.ndim = 3
    ni, nj, nk = shape
    d.size = L.I64x3(ni, nj, nk)
    d.stride = L.I64x3(1, ni, ni * nj)
    d.origin = L.I64x3(*origin)
    return d


def _apply(p, ins, outs, lb, ub, halo, params=()):
    a = (L.FieldDesc * len(ins))(*ins)
    b = (L.FieldDesc * len(outs))(*outs)
    par = (C.c_double * max(1, len(params)))(*params)
    return L.lib().oec_program_apply(p.handle, a, len(ins), b, len(outs), L.I64x3(*lb), L.I64x3(*ub),
                                     L.I64x3(*halo), par, len(params), None)


def test_validation_errors_without_gpu(liboec):
    p = _prog(programs.HDIFF)
    n, h = (16, 12, 5), 2
    shp = (n[0] + 2 * h, n[1] + 2 * h, n[2] + 2 * h)
    GB = 1 << 30
    fin, fco, fout = _fake(1 * GB, shp, (h, h, h)), _fake(2 * GB, shp, (h, h, h)), _fake(3 * GB, shp, (h, h, h))
    lb, ub = (0, 0, 0), n
    assert _apply(p, [fin, fco], [fout], lb, ub, (1, 1, 0)) == -4            # HALO: needs 2
    small = _fake(1 * GB, (n[0] + 2, n[1] + 4, n[2] + 4), (1, 2, 2))
    assert _apply(p, [small, fco], [fout], lb, ub, (2, 2, 0)) == -3          # SHAPE
    assert _apply(p, [fin, fco], [_fake(1 * GB, shp, (h, h, h))], lb, ub, (2, 2, 0)) == -5   # ALIAS
    assert _apply(p, [fin, fco], [_fake(3 * GB, shp, (h, h, h), L.F32)], lb, ub, (2, 2, 0)) == -6   # DTYPE
    assert _apply(p, [fin], [fout], lb, ub, (2, 2, 0)) == -1                 # wrong input count
    assert _apply(p, [fin, fco], [fout], (0, 0, 0), (16, 12, 0), (2, 2, 0)) == 0   # empty domain: no work
    assert _apply(p, [fin, fco], [fout], (0, 5, 0), (16, 4, 5), (2, 2, 0)) == -1   # inverted
    msg = L.lib().oec_last_error().decode()
    assert "inverted" in msg


def test_apply_host_validation_without_gpu(liboec):
    """Host-memory apply: shape errors and empty domains are settled before
    any device call."""
    p = _prog(programs.HDIFF)
    n, h = (16, 12, 5), 2
    shp = (n[0] + 2 * h, n[1] + 2 * h, n[2] + 2 * h)
    fin, fco, fout = (_fake(a, shp, (h, h, h)) for a in (1 << 20, 2 << 20, 3 << 20))
    bad = _fake(4 << 20, shp, (h, h, h))
    bad.stride = L.I64x3(2, 2 * shp[0], 2 * shp[0] * shp[1])

    def host(ins, outs, ub):
        a = (L.FieldDesc * len(ins))(*ins)
        b = (L.FieldDesc * len(outs))(*outs)
        return L.lib().oec_program_apply_host(p.handle, a, len(ins), b, len(outs), L.I64x3(0, 0, 0), L.I64x3(*ub),
                                              L.I64x3(h, h, h), (C.c_double * 1)(), 0, None)
    assert host([fin, fco], [bad], n) == -7                        # UNSUPPORTED: i stride 2
    assert "unit i stride" in L.lib().oec_last_error().decode()
    assert host([fin], [fout], n) == -1                            # wrong input count
    assert host([fin, fco], [fout], (16, 12, 0)) == 0              # empty domain: nothing to do


def test_wait_selftest_validation_without_gpu(liboec):
    assert L.lib().oec_device_wait_selftest(0, None) == -1
    assert L.lib().oec_device_wait_selftest(70000, None) == -1
    assert L.lib().oec_batch_wait_selftest(0, None) == -1
    assert L.lib().oec_batch_wait_selftest(70000, None) == -1


def test_bad_schedule_rejected(liboec):
    p = _prog(programs.HDIFF)
    with pytest.raises(L.OecError):
        p.set_schedule(fusion=0, staging=1, tile_i=48, tile_j=4)
    with pytest.raises(L.OecError):
        p.set_schedule(fusion=0, staging=0, tile_i=64, tile_j=3, unroll=2)
    p.set_schedule(fusion=0, staging=0, tile_i=64, tile_j=4, unroll=2)
    assert p.schedule["unroll"] == 2


def test_index_bits_values(liboec):
    """index_bits is OEC_INDEX_AUTO (0) or OEC_INDEX_64 (64); anything else
    is refused with the reason, and the accepted value reads back."""
    p = _prog(programs.HDIFF)
    for bad in (32, 1, -64):
        with pytest.raises(L.OecError) as e:
            p.set_schedule(fusion=0, staging=0, tile_i=64, tile_j=4, index_bits=bad)
        assert "index_bits" in str(e.value)
    p.set_schedule(fusion=0, staging=0, tile_i=64, tile_j=4, index_bits=64)
    assert p.schedule["index_bits"] == 64
    p.set_schedule(fusion=0, staging=0, tile_i=64, tile_j=4)
    assert p.schedule["index_bits"] == 0


def test_timing_calls_without_gpu(liboec):
    """Launch counting and kernel timing need no GPU until an apply runs."""
    import ctypes as C
    from paper_2005_13014_gb300 import _lib as L
    p = C.c_void_p()
    L.check(liboec.oec_program_create(programs.HDIFF.encode(), None, C.byref(p)))
    try:
        assert liboec.oec_program_launch_count(p) == 0
        assert liboec.oec_program_set_timing(p, 1) == 0
        na, nk = C.c_int(-1), C.c_int(-1)
        assert liboec.oec_program_kernel_times(p, None, 0, C.byref(na), C.byref(nk)) == 0
        assert (na.value, nk.value) == (0, 0)
        assert liboec.oec_program_kernel_times(p, None, 0, None, C.byref(nk)) == -1   # OEC_ERR_INVALID_ARG
        assert liboec.oec_program_launch_count(None) == -1   # OEC_ERR_INVALID_ARG
    finally:
        liboec.oec_program_destroy(p)


def test_library_and_oracle_parsers_agree():
    """The library's parser and the oracle's (written separately) accept and
    reject the same texts: every program of the package, random stage DAGs,
    and a set of malformed texts."""
    good = [programs.HDIFF, programs.HDIFF_VADVC, programs.FASTWAVES]
    good += [src for src, _, _ in programs.TESTSET.values()]
    good += [inputs.random_dag(s) for s in range(10000, 10040)]
    good += ["input a\nstage s = if (a > 0.0) { let t = a*a; yield t } else { let t = -a; yield t }\noutput s\n"]
    bad = [
        "input a\nstage b = a[1,0]\noutput b\n",
        "input a\nstage b = c\noutput b\n",
        "input a\nstage b = a\n",
        "input a\nstage a = a\noutput a\n",
        "input a\nstage b = { let t = a; return t, t }\noutput b\n",
        "input a\nstage b = select(a, a, a)\noutput b\n",
        "input a\nstage b = if (a > 0.0) { yield a }\noutput b\n",
        "input a\nstage b = if (a > 0.0) { let t = a; yield t } else { yield t }\noutput b\n",
        "input a\nstage let = a\noutput let\n",
        "input a\nstage b = a\noutput a\n",
        "input a\nparam p\nstage b = p[1,0,0]\noutput b\n",
        "input a\nstage b = { let t = a; let t = a; return t }\noutput b\n",
    ]
    for src in good:
        OP.parse(src)
        _prog(src)
    for src in bad:
        with pytest.raises(OP.ParseError):
            OP.parse(src)
        with pytest.raises(L.OecError) as e:
            _prog(src)
        assert e.value.name == "PARSE", src
