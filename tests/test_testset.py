"""The Table II stand-in programs (programs.TESTSET): their shapes are the
ones the paper lists, the oracle's shape inference gives the halos read off
their stencils by hand, and the oracle's staged and inlined interpreters
agree on them bit for bit."""

import numpy as np
import pytest

from oracle import program as OP
from oracle import stencils as S
from paper_2005_13014_gb300 import inputs, programs

# (lower, upper) halo per dimension (i, j, k), derived by reading the offsets
HALOS = {
    "uvbke": {"uc": ((0, 0), (1, 0), (0, 0)), "vc": ((1, 0), (0, 0), (0, 0)),
              "cosa": ((0, 0), (0, 0), (0, 0)), "rsina": ((0, 0), (0, 0), (0, 0))},
    "p_grad_c": {"uc": ((0, 0),) * 3, "vc": ((0, 0),) * 3, "delpc": ((1, 0), (1, 0), (0, 0)),
                 "pkc": ((1, 0), (1, 0), (0, 1)), "gz": ((1, 0), (1, 0), (0, 1)),
                 "rdxc": ((0, 0),) * 3, "rdyc": ((0, 0),) * 3},
    "hadvuv": {"uin": ((2, 2), (2, 2), (0, 0)), "vin": ((2, 2), (2, 2), (0, 0)),
               **{n: ((0, 0),) * 3 for n in ("uatupos", "vatupos", "uatvpos", "vatvpos")}},
    "fvtp2d_flux": {"q": ((1, 1), (1, 0), (0, 0)),
                    **{n: ((0, 0),) * 3 for n in ("crx", "cry", "xfx", "yfx", "al", "bl")}},
}


@pytest.mark.parametrize("name", list(programs.TESTSET))
def test_shape_matches_table_ii(name):
    src, params, (applies, n_in, n_out) = programs.TESTSET[name]
    p = OP.parse(src)
    assert len(p.stmts) == applies and len(p.inputs) == n_in and len(p.outputs) == n_out
    assert len(params) == len(p.params)
    if name in ("hadvuv", "fvtp2d_flux"):
        assert "select(" in src   # the table's `if`


@pytest.mark.parametrize("name", list(programs.TESTSET))
def test_shape_inference_halos(name):
    p = OP.parse(programs.TESTSET[name][0])
    assert OP.input_halo(p, (2, 3, 1), (30, 21, 7)) == HALOS[name]


@pytest.mark.parametrize("name", list(programs.TESTSET))
def test_staged_equals_inlined(name):
    src, params, _ = programs.TESTSET[name]
    prog = OP.parse(src)
    par = dict(zip(prog.params, params))
    n, h = (11, 9, 4), 3
    f = inputs.testset_fields(name, *n, h)
    G = {k: S.Grid.storage(v, h) for k, v in f.items()}
    staged = OP.run_staged(prog, G, (0, 0, 0), n, par)
    inlined = OP.run_inlined(prog, G, (0, 0, 0), n, par)
    for name_ in prog.outputs:
        arr = staged[name_]
        assert np.all(np.isfinite(arr))
        for (i, j, k), v in inlined[name_].items():
            assert arr[k, j, i] == v
