"""Pins of the FP64 oracle for hdiff, vadvc and fastwaves against facts that do
not come from the oracle itself: exact results on constant and linear fields,
hand-derived worked examples (tests/golden), a dense linear solve, symmetry
under swapping i and j, and agreement of the staged and inlined evaluations."""

import os

import numpy as np
import pytest

from oracle import stencils as S
from paper_2005_13014_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def _grid(arr, h):
    return S.Grid.storage(arr, h)


# --------------------------------------------------------------------- hdiff

def test_hdiff_constant_field_unchanged():
    h, n = 2, (9, 7, 3)
    inp = np.full(inputs.storage_shape(*n, h), 0.375)
    coeff = inputs.hdiff_fields(*n, h)["coeff"]
    st = S.hdiff_stages(_grid(inp, h), _grid(coeff, h), (0, 0, 0), n)
    assert np.all(st["lap"].arr == 0.0)
    assert np.array_equal(st["out"].arr, inp[h:-h, h:-h, h:-h])


def test_hdiff_linear_field_has_zero_laplacian():
    h, (ni, nj, nk) = 2, (10, 6, 4)
    k, j, i = np.meshgrid(np.arange(nk + 2 * h), np.arange(nj + 2 * h), np.arange(ni + 2 * h), indexing="ij")
    inp = (3.0 * i - 5.0 * j + 7.0 * k + 11.0)
    coeff = inputs.hdiff_fields(ni, nj, nk, h)["coeff"]
    st = S.hdiff_stages(_grid(inp, h), _grid(coeff, h), (0, 0, 0), (ni, nj, nk))
    assert np.all(st["lap"].arr == 0.0)
    assert np.array_equal(st["out"].arr, inp[h:-h, h:-h, h:-h])


def test_hdiff_impulse_matches_hand_derivation():
    rows = _read_golden("hdiff_delta.txt")
    c = float(rows[0][1])
    expect = {(int(r[0]), int(r[1])): float(r[2]) for r in rows[1:]}
    h, (ni, nj, nk) = 2, (9, 9, 2)
    inp = np.zeros(inputs.storage_shape(ni, nj, nk, h))
    p = (4, 4)
    inp[:, p[1] + h, p[0] + h] = 1.0
    coeff = np.full_like(inp, c)
    out = S.hdiff(_grid(inp, h), _grid(coeff, h), (0, 0, 0), (ni, nj, nk))
    for kk in range(nk):
        for jj in range(nj):
            for ii in range(ni):
                want = expect.get((ii - p[0], jj - p[1]), 0.0)
                assert out[kk, jj, ii] == want, (ii, jj, kk)
    assert np.sum(out - inp[h:-h, h:-h, h:-h]) == 0.0


def test_hdiff_flux_form_telescopes():
    """With a constant coeff c the interior sum of out - in is -c times the net
    flux through the domain's boundary (flux form: interior fluxes cancel);
    random data, so the sums agree to rounding."""
    h, n, c = 2, (12, 9, 3), 0.0625
    f = inputs.hdiff_fields(*n, h, seed=17)
    coeff = np.full_like(f["in"], c)
    st = S.hdiff_stages(_grid(f["in"], h), _grid(coeff, h), (0, 0, 0), n)
    flx, fly = st["flx"], st["fly"]
    net = 0.0
    for k in range(n[2]):
        for j in range(n[1]):
            net += flx.value(n[0] - 1, j, k) - flx.value(-1, j, k)
        for i in range(n[0]):
            net += fly.value(i, n[1] - 1, k) - fly.value(i, -1, k)
    lhs = float(np.sum(st["out"].arr - f["in"][h:-h, h:-h, h:-h]))
    assert abs(lhs - (-c * net)) <= 1e-12 * max(1.0, abs(c * net))
    assert abs(net) > 1e-3   # a case where the boundary flux is not zero


def test_hdiff_transpose_symmetry():
    h, n = 2, (8, 8, 3)
    f = inputs.hdiff_fields(*n, h)
    a = S.hdiff(_grid(f["in"], h), _grid(f["coeff"], h), (0, 0, 0), n)
    t = lambda x: np.ascontiguousarray(np.swapaxes(x, 1, 2))
    b = S.hdiff(_grid(t(f["in"]), h), _grid(t(f["coeff"]), h), (0, 0, 0), n)
    # the Laplacian sums its i and j neighbours in a fixed order, so swapping
    # the axes changes rounding only
    np.testing.assert_allclose(t(b), a, rtol=0, atol=1e-15)


def test_hdiff_staged_equals_inlined():
    h, n = 2, (6, 5, 2)
    f = inputs.hdiff_fields(*n, h, seed=7)
    gi, gc = _grid(f["in"], h), _grid(f["coeff"], h)
    out = S.hdiff(gi, gc, (0, 0, 0), n)
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                assert S.hdiff_point(gi, gc, i, j, k) == out[k, j, i]


def test_hdiff_subdomain_is_restriction():
    h, n = 2, (12, 10, 3)
    f = inputs.hdiff_fields(*n, h, seed=3)
    gi, gc = _grid(f["in"], h), _grid(f["coeff"], h)
    full = S.hdiff(gi, gc, (0, 0, 0), n)
    sub = S.hdiff(gi, gc, (3, 2, 1), (9, 7, 3))
    np.testing.assert_array_equal(sub, full[1:3, 2:7, 3:9])


# --------------------------------------------------------------------- vadvc

def test_vadvc_zero_wind_is_identity():
    h, n = 1, (5, 4, 9)
    phi = inputs.hdiff_fields(*n, h)["in"][h:-h, h:-h, h:-h]
    w = np.zeros(inputs.storage_shape(*n, h))
    x = S.vadvc_solve(phi, _grid(w, h), (0, 0, 0), n, 2.0)
    np.testing.assert_array_equal(x, phi)


def test_vadvc_two_level_hand_solution():
    rows = {r[0]: [float(v) for v in r[1:]] for r in _read_golden("vadvc_two_level.txt")}
    h = 1
    w = np.zeros(inputs.storage_shape(1, 1, 2, h))
    w[h + 0, h, h:h + 2] = rows["w_k0"]
    w[h + 1, h, h:h + 2] = rows["w_k1"]
    phi = np.array(rows["phi"]).reshape(2, 1, 1)
    x = S.vadvc_solve(phi, _grid(w, h), (0, 0, 0), (1, 1, 2), rows["dtr"][0])
    np.testing.assert_allclose(x.reshape(-1), rows["x"], rtol=1e-15, atol=0)


@pytest.mark.parametrize("K", [1, 2, 3, 5, 8])
def test_thomas_matches_dense_solve(K):
    h, n = 1, (3, 2, K)
    f = inputs.hdiff_vadvc_fields(*n, h, seed=11 + K)
    phi = f["u"][h:-h, h:-h, h:-h]
    gw = _grid(f["w"], h)
    x = S.vadvc_solve(phi, gw, (0, 0, 0), n, 2.0)
    a, c = S.vadvc_matrix(gw, (0, 0, 0), n)
    b = (2.0 + np.abs(a)) + np.abs(c)
    d = S.vadvc_rhs(phi, a, c, 2.0)
    for j in range(n[1]):
        for i in range(n[0]):
            A = np.diag(b[:, j, i]) + np.diag(a[1:, j, i], -1) + np.diag(c[:-1, j, i], 1)
            ref = np.linalg.solve(A, d[:, j, i])
            np.testing.assert_allclose(x[:, j, i], ref, rtol=0, atol=1e-14 * np.max(np.abs(ref)))
            # strict diagonal dominance by construction
            assert np.all(b[:, j, i] > np.abs(a[:, j, i]) + np.abs(c[:, j, i]))


def test_thomas_manufactured_solution_and_residual():
    rng = np.random.default_rng(5)
    K, m = 80, 64
    a = rng.uniform(-0.5, 0.5, (K, 1, m))
    c = rng.uniform(-0.5, 0.5, (K, 1, m))
    a[0] = 0.0
    c[-1] = 0.0
    b = 2.0 + np.abs(a) + np.abs(c)
    xs = rng.uniform(-1, 1, (K, 1, m))
    d = b * xs
    d[1:] += a[1:] * xs[:-1]
    d[:-1] += c[:-1] * xs[1:]
    x = S.thomas(a, b, c, d)
    assert np.max(np.abs(x - xs)) <= 1e-13 * np.max(np.abs(xs))
    r = b * x
    r[1:] += a[1:] * x[:-1]
    r[:-1] += c[:-1] * x[1:]
    assert np.max(np.abs(r - d)) <= 1e-14 * np.max(np.abs(d)) * 4


def test_hdiff_vadvc_staged_equals_inlined_per_column():
    h, n = 3, (5, 4, 6)
    f = inputs.hdiff_vadvc_fields(*n, h, seed=9)
    g = {k: _grid(v, h) for k, v in f.items()}
    uo, vo = S.hdiff_vadvc(g["u"], g["v"], g["w"], g["coeff"], (0, 0, 0), n, 2.0)
    # recompute with the per-point inlined hdiff feeding the same column solve
    ud = np.array([[[S.hdiff_point(g["u"], g["coeff"], i, j, k) for i in range(n[0])]
                    for j in range(n[1])] for k in range(n[2])])
    np.testing.assert_array_equal(S.vadvc_solve(ud, g["w"], (0, 0, 0), n, 2.0), uo)
    assert vo.shape == uo.shape


# ----------------------------------------------------------------- fastwaves

def _fw_grids(f, h):
    return {k: _grid(v, h) for k, v in f.items()}


def test_fastwaves_zero_pressure_linear_wind():
    h, (ni, nj, nk) = 3, (7, 6, 4)
    f = inputs.fastwaves_fields(ni, nj, nk, h, seed=4)
    k, j, i = np.meshgrid(np.arange(nk + 2 * h), np.arange(nj + 2 * h), np.arange(ni + 2 * h), indexing="ij")
    f["pp"] = np.zeros_like(f["pp"])
    f["u_in"] = 2.0 * i + 3.0 * j - k + 1.0
    f["v_in"] = -1.0 * i + 4.0 * j + 2.0 * k
    uo, vo = S.fastwaves(_fw_grids(f, h), (0, 0, 0), (ni, nj, nk), 0.5, 0.0625)
    inner = (slice(h, -h),) * 3
    np.testing.assert_array_equal(uo, f["u_in"][inner] + 0.5 * f["utens"][inner])
    np.testing.assert_array_equal(vo, f["v_in"][inner] + 0.5 * f["vtens"][inner])


def test_fastwaves_flat_levels_linear_pressure():
    h, (ni, nj, nk) = 3, (6, 5, 3)
    f = inputs.fastwaves_fields(ni, nj, nk, h, seed=8)
    k, j, i = np.meshgrid(np.arange(nk + 2 * h), np.arange(nj + 2 * h), np.arange(ni + 2 * h), indexing="ij")
    f["hhl"] = np.broadcast_to(f["hhl"][:, :1, :1], f["hhl"].shape).copy()
    f["pp"] = 2.0 * i + 3.0 * j + 5.0 * k
    st = S.fastwaves_stages(_fw_grids(f, h), (0, 0, 0), (ni, nj, nk), 0.5, 0.0625)
    assert np.all(st["ppgu"].arr == 2.0)
    assert np.all(st["ppgv"].arr == 3.0)


def test_fastwaves_transpose_symmetry():
    h, n = 3, (6, 6, 3)
    f = inputs.fastwaves_fields(*n, h, seed=2)
    a_u, a_v = S.fastwaves(_fw_grids(f, h), (0, 0, 0), n, 0.5, 0.0625)
    t = lambda x: np.ascontiguousarray(np.swapaxes(x, 1, 2))
    g = {k: t(v) for k, v in f.items()}
    g["u_in"], g["v_in"] = t(f["v_in"]), t(f["u_in"])
    g["utens"], g["vtens"] = t(f["vtens"]), t(f["utens"])
    b_u, b_v = S.fastwaves(_fw_grids(g, h), (0, 0, 0), n, 0.5, 0.0625)
    np.testing.assert_allclose(t(b_v), a_u, rtol=0, atol=1e-15)
    np.testing.assert_allclose(t(b_u), a_v, rtol=0, atol=1e-15)


def test_fastwaves_staged_equals_inlined():
    h, n = 3, (4, 3, 2)
    f = _fw_grids(inputs.fastwaves_fields(*n, h, seed=6), h)
    uo, vo = S.fastwaves(f, (0, 0, 0), n, 0.5, 0.0625)
    for k in range(n[2]):
        for j in range(n[1]):
            for i in range(n[0]):
                pu, pv = S.fastwaves_point(f, i, j, k, 0.5, 0.0625)
                assert pu == uo[k, j, i] and pv == vo[k, j, i]


def test_fastwaves_every_term_matches_hand_derivation():
    """tests/golden/fastwaves_point.txt: fields chosen so that S1's k-1
    weighting, S2's difference, the terrain term of S3/S4, S5's fourth-order
    coefficients and S6's density/fx term are all non-zero at one point, with
    the stage values and both outputs derived by hand (dyadic, so exact)."""
    h, n = 3, (1, 1, 1)
    shape = inputs.storage_shape(*n, h)
    k, j, i = np.meshgrid(*(np.arange(s_) - h for s_ in shape), indexing="ij")
    i, j, k = i.astype(np.float64), j.astype(np.float64), k.astype(np.float64)
    f = {"pp": (1 + i + 2 * j) * k ** 2 + 2 * k + 3 * i - 2 * j,
         "wgtfac": 0.75 - 0.25 * k,
         "hhl": 100 - 10 * k + (2 + 4 * k) * i + (1 + 12 * k) * j,
         "u_in": i ** 3 + 5 * j ** 2 + 1, "v_in": j ** 2 - 3 * i ** 2 + 2,
         "utens": 0.5 + 0.125 * i, "vtens": -0.25 + 0.125 * j,
         "rho": 1.5 - i + j, "fx": 0.75 + 0.25 * i}
    g = _fw_grids(f, h)
    st = S.fastwaves_stages(g, (0, 0, 0), n, 0.5, 0.0625)
    rows = _read_golden("fastwaves_point.txt")
    assert len(rows) == 16
    for name, a, b, c, want in rows:
        got = st[name].value(int(a), int(b), int(c))
        assert got == float(want), (name, a, b, c, got, want)
    pu, pv = S.fastwaves_point(g, 0, 0, 0, 0.5, 0.0625)
    assert pu == st["u_out"].value(0, 0, 0) and pv == st["v_out"].value(0, 0, 0)
