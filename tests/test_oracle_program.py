"""Pins of the oracle's program interpreter: the staged and inlined evaluations
agree bit for bit on random programs; interpreting the library's program texts
reproduces the hand-written oracle stencils bit for bit; shape inference gives
the halos derived by hand from the access offsets (paper §V-B)."""

import numpy as np
import pytest

from oracle import program as P
from oracle import stencils as S
from paper_2005_13014_gb300 import inputs, programs


def _g(arr, h):
    return S.Grid.storage(arr, h)


def test_interpreted_hdiff_equals_oracle_hdiff():
    h, n = 2, (9, 8, 3)
    f = inputs.hdiff_fields(*n, h, seed=21)
    out = P.run_staged(programs.HDIFF, {k: _g(v, h) for k, v in f.items()}, (0, 0, 0), n)["out"]
    ref = S.hdiff(_g(f["in"], h), _g(f["coeff"], h), (0, 0, 0), n)
    np.testing.assert_array_equal(out, ref)


def test_interpreted_hdiff_vadvc_equals_oracle():
    h, n = 3, (6, 5, 7)
    f = inputs.hdiff_vadvc_fields(*n, h, seed=22)
    g = {k: _g(v, h) for k, v in f.items()}
    out = P.run_staged(programs.HDIFF_VADVC, g, (0, 0, 0), n, {"dtr": 2.0})
    uo, vo = S.hdiff_vadvc(g["u"], g["v"], g["w"], g["coeff"], (0, 0, 0), n, 2.0)
    np.testing.assert_array_equal(out["u_out"], uo)
    np.testing.assert_array_equal(out["v_out"], vo)


def test_interpreted_fastwaves_equals_oracle():
    h, n = 3, (7, 6, 4)
    f = inputs.fastwaves_fields(*n, h, seed=23)
    g = {k: _g(v, h) for k, v in f.items()}
    out = P.run_staged(programs.FASTWAVES, g, (0, 0, 0), n, {"dt": 0.5, "alpha": 0.0625})
    uo, vo = S.fastwaves(g, (0, 0, 0), n, 0.5, 0.0625)
    np.testing.assert_array_equal(out["u_out"], uo)
    np.testing.assert_array_equal(out["v_out"], vo)


def test_shape_inference_halos():
    # hand-derived from the offsets: hdiff reads in at +-2 in i and j (lap at +-1,
    # itself reading +-1); fastwaves reads u_in at i-2..i+3 (div at i+1 reads
    # u_in(i+3)), pp at k-1..k+1 (ppgk(k+1) reads pp(k)), hhl up to k+1 and i+1.
    hp = P.input_halo(P.parse(programs.HDIFF), (0, 0, 0), (10, 10, 5))
    assert hp["in"] == ((2, 2), (2, 2), (0, 0))
    assert hp["coeff"] == ((0, 0), (0, 0), (0, 0))
    fw = P.input_halo(P.parse(programs.FASTWAVES), (0, 0, 0), (10, 10, 5))
    assert fw["u_in"] == ((2, 3), (0, 1), (0, 0))
    assert fw["v_in"] == ((0, 1), (2, 3), (0, 0))
    assert fw["pp"] == ((0, 1), (0, 1), (1, 1))
    assert fw["hhl"] == ((0, 1), (0, 1), (0, 1))
    assert fw["wgtfac"] == ((0, 1), (0, 1), (0, 1))
    assert fw["rho"] == ((0, 1), (0, 1), (0, 0))
    assert fw["fx"] == ((0, 0), (0, 0), (0, 0))
    hv = P.input_halo(P.parse(programs.HDIFF_VADVC), (0, 0, 0), (10, 10, 5))
    assert hv["u"] == ((2, 2), (2, 2), (1, 1))      # ud read at k-1, k+1 under select
    assert hv["w"] == ((0, 1), (0, 0), (0, 1))


@pytest.mark.parametrize("seed", list(range(10000, 10012)))
def test_random_dag_staged_equals_inlined(seed):
    src = inputs.random_dag(seed)
    prog = P.parse(src)
    n = (5, 4, 3)
    h = (8, 8, 4)
    fields = {}
    for idx, name in enumerate(prog.inputs):
        arr = np.random.default_rng(seed * 10 + idx).uniform(-1, 1, (n[2] + 2 * h[2], n[1] + 2 * h[1], n[0] + 2 * h[0]))
        fields[name] = _g(arr, h)
    staged = P.run_staged(prog, fields, (0, 0, 0), n)
    pts = [(i, j, k) for k in range(n[2]) for j in range(n[1]) for i in range(n[0])]
    inl = P.run_inlined(prog, fields, (0, 0, 0), n, points=pts)
    for name in prog.outputs:
        for (i, j, k), val in inl[name].items():
            assert staged[name][k, j, i] == val
    halos = P.input_halo(prog, (0, 0, 0), n)
    for name, hh in halos.items():
        assert hh is not None
        assert max(hh[0]) <= 8 and max(hh[1]) <= 8 and max(hh[2]) <= 4


def test_parse_errors():
    with pytest.raises(P.ParseError):
        P.parse("input a\nstage b = a[1,0]\noutput b\n")
    with pytest.raises(P.ParseError):
        P.parse("input a\nstage b = c\noutput b\n")
    with pytest.raises(P.ParseError):
        P.parse("input a\nstage b = a\n")


# region control flow (§IV-C: scf.if runs the region its condition picks and
# yields that region's value; each region binds its own lets)
IF_SRC = """
input a, b
stage s = { let q = a[1,0,0] - a; return if (q > 0.0) { let t = q * b; yield t + 1.0 } else { yield b[0,1,0] - q } }
stage r = if (s <= 0.5) { yield s * 2.0 } else { let u = s - b[0,0,1]; yield min(u, s) }
output s, r
"""


def test_if_regions_match_their_definition():
    """Each point takes the value of the region its condition picks, computed
    here from the definition with whole-array numpy; the staged and the
    point-by-point interpreters both agree bit for bit, and the inferred
    ranges cover the accesses of both regions."""
    h, n = (2, 2, 2), (6, 5, 4)
    rng = np.random.default_rng(77)
    a = rng.uniform(-1, 1, (n[2] + 4, n[1] + 4, n[0] + 4))
    b = rng.uniform(-1, 1, a.shape)
    fields = {"a": _g(a, h), "b": _g(b, h)}
    prog = P.parse(IF_SRC)
    staged = P.run_staged(prog, fields, (0, 0, 0), n)
    # reference: interior slices of the storage (origin at h)
    K, J, I = slice(2, 2 + n[2]), slice(2, 2 + n[1]), slice(2, 2 + n[0])
    a0 = a[K, J, I]
    a_ip = a[K, J, slice(3, 3 + n[0])]
    b0 = b[K, J, I]
    b_jp = b[K, slice(3, 3 + n[1]), I]
    b_kp = b[slice(3, 3 + n[2]), J, I]
    q = a_ip - a0
    s = np.where(q > 0.0, q * b0 + 1.0, b_jp - q)
    r = np.where(s <= 0.5, s * 2.0, np.minimum(s - b_kp, s))
    np.testing.assert_array_equal(staged["s"], s)
    np.testing.assert_array_equal(staged["r"], r)
    pts = [(i, j, k) for k in range(n[2]) for j in range(n[1]) for i in range(n[0])]
    inl = P.run_inlined(prog, fields, (0, 0, 0), n, points=pts)
    for name, ref in (("s", s), ("r", r)):
        for (i, j, k), val in inl[name].items():
            assert val == ref[k, j, i]
    halos = P.input_halo(prog, (0, 0, 0), n)
    assert halos["a"] == ((0, 1), (0, 0), (0, 0))
    assert halos["b"] == ((0, 0), (0, 1), (0, 1))


def test_if_region_lets_are_local():
    bad = [
        "input a\nstage s = if (a > 0.0) { let t = a; yield t } else { yield t }\noutput s\n",
        "input a\nstage s = if (a > 0.0) { yield a }\noutput s\n",
        "input a\nstage s = if (a > 0.0) { a } else { yield a }\noutput s\n",
        "input a\nstage s = if (a) { yield a } else { yield a }\noutput s\n",
        "input a\nstage s = { let t = a; return if (a > 0.0) { let t = a; yield t } else { yield a } }\noutput s\n",
    ]
    for src in bad:
        with pytest.raises(P.ParseError):
            P.parse(src)
    # the same name in both regions is fine: each region has its own
    P.parse("input a\nstage s = if (a > 0.0) { let t = a; yield t } else { let t = -a; yield t }\noutput s\n")
