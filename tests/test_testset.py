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
    # t at (0,0),(0,1); s at (0,-1),(-1,0); updates at +-1 in i and j
    "hdiffsmag": {"u": ((1, 1), (1, 1), (0, 0)), "v": ((1, 1), (1, 1), (0, 0)), "crlavo": ((1, 0), (1, 0), (0, 0)),
                  "acrlat0": ((0, 0), (0, 1), (0, 0)),
                  **{n: ((0, 0),) * 3 for n in ("hdmask", "crlavu", "crlato", "crlatu")}},
    "hadvuv5th": {"uin": ((3, 3), (3, 3), (0, 0)), "vin": ((3, 3), (3, 3), (0, 0)),
                  **{n: ((0, 0),) * 3 for n in ("uatupos", "vatupos", "uatvpos", "vatvpos")}},
    # wk at (0,0),(1,0),(0,1), each spanning k and k+1
    "nh_p_grad": {"gz": ((0, 1), (0, 1), (0, 1)), "pk3": ((0, 1), (0, 1), (0, 1)), "pp": ((0, 1), (0, 1), (0, 0)),
                  "delp": ((0, 1), (0, 1), (0, 0)), **{n: ((0, 0),) * 3 for n in ("u", "v", "rdx", "rdy")}},
    # fx1 at i and i+1 reads al at i-1 .. i+2, al reads q at -2 .. +1
    "fvtp2d_qi": {"q": ((3, 3), (0, 0), (0, 0)), "crx": ((0, 1), (0, 0), (0, 0)), "xfx": ((0, 1), (0, 0), (0, 0)),
                  "area": ((0, 0),) * 3, "ra_x": ((0, 0),) * 3},
    "fvtp2d_qj": {"q": ((0, 0), (3, 3), (0, 0)), "cry": ((0, 0), (0, 1), (0, 0)), "yfx": ((0, 0), (0, 1), (0, 0)),
                  **{n: ((0, 0),) * 3 for n in ("area", "ra_y", "mfy")}},
}


@pytest.mark.parametrize("name", list(programs.TESTSET))
def test_shape_matches_table_ii(name):
    src, params, (applies, n_in, n_out) = programs.TESTSET[name]
    p = OP.parse(src)
    assert len(p.stmts) == applies and len(p.inputs) == n_in and len(p.outputs) == n_out
    assert len(params) == len(p.params)
    if name in ("hadvuv", "hadvuv5th", "fvtp2d_flux", "fvtp2d_qi", "fvtp2d_qj"):
        # the table's `if`: region control flow whose regions are upwind choices
        assert "if (" in src and "yield" in src
        assert any(e[0] == "if" for st in p.stmts for e in st.rets + [x for _, x in st.lets])
    if name == "hdiffsmag":
        assert "min(" in src and "max(" in src


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
