"""FP64 oracle for the three fixed stencil programs (test infrastructure only).

Arrays are numpy float64 indexed [k, j, i] (i contiguous). A ``Grid`` pairs an
array with the logical (i, j, k) coordinates of its first element; the logical
origin (0, 0, 0) is the lower corner of the computation domain and ranges are
half-open [lower, upper) boxes (paper §IV, "Shapes & Domains").

Staged evaluation: every stage is evaluated over its inferred bounding box
(paper §V-B) into a full array, then consumed. Inlined evaluation: every output
point recomputes its producers at the offsets it reads (paper §V-A). Both give
the same bits because every expression is evaluated in the same written order.

The paper prints no formulas for its benchmark kernels (Table II lists only
their shapes), so the formulas below follow the readings recorded in the
project's design notes:
  hdiff     - 5-point Laplacian, i/j fluxes with a sign limiter, flux divergence
              (Table II, "hdiffsa" shape: Laplacian -> fluxes -> output).
  vadvc     - implicit vertical advection, a tridiagonal system per (i, j)
              column solved by the Thomas algorithm (§VII-B mentions Thomas for
              vertical implicit integration).
  fastwaves - six stages, nine inputs, two outputs, no control flow (Table II,
              "fastwavesuv" shape).
"""

from __future__ import annotations

import numpy as np


class Grid:
    """A float64 array plus the logical (i, j, k) coordinates of arr[0, 0, 0]."""

    def __init__(self, arr: np.ndarray, lo):
        self.arr = np.asarray(arr, dtype=np.float64)
        self.lo = tuple(int(x) for x in lo)

    @staticmethod
    def storage(arr: np.ndarray, halo) -> "Grid":
        """A field stored with ``halo`` cells (int or (hi, hj, hk)) before the origin."""
        if np.isscalar(halo):
            halo = (halo, halo, halo)
        return Grid(arr, (-halo[0], -halo[1], -halo[2]))

    def box(self):
        nk, nj, ni = self.arr.shape
        li, lj, lk = self.lo
        return ((li, li + ni), (lj, lj + nj), (lk, lk + nk))

    def at(self, box, di=0, dj=0, dk=0) -> np.ndarray:
        """The values at logical points p + (di, dj, dk) for p in ``box``."""
        (i0, i1), (j0, j1), (k0, k1) = box
        li, lj, lk = self.lo
        nk, nj, ni = self.arr.shape
        a0, a1 = i0 + di - li, i1 + di - li
        b0, b1 = j0 + dj - lj, j1 + dj - lj
        c0, c1 = k0 + dk - lk, k1 + dk - lk
        if a0 < 0 or b0 < 0 or c0 < 0 or a1 > ni or b1 > nj or c1 > nk:
            raise IndexError(f"access {box}+({di},{dj},{dk}) outside grid {self.box()}")
        return self.arr[c0:c1, b0:b1, a0:a1]

    def value(self, i, j, k) -> float:
        li, lj, lk = self.lo
        if i < li or j < lj or k < lk:
            raise IndexError((i, j, k))
        return float(self.arr[k - lk, j - lj, i - li])


def _box(lb, ub):
    return ((lb[0], ub[0]), (lb[1], ub[1]), (lb[2], ub[2]))


# ----------------------------------------------------------------------------
# hdiff (Table II "hdiffsa" shape; formulas per the design-note reading D1)
# ----------------------------------------------------------------------------

def hdiff_stages(inp: Grid, coeff: Grid, lb, ub):
    """Staged horizontal diffusion; returns dict of Grids lap, flx, fly, out.

    lap = 4*in - in(i-1) - in(i+1) - in(j-1) - in(j+1)       (left to right)
    flx = lap(i+1) - lap;  flx = 0 where flx*(in(i+1) - in) > 0
    fly = lap(j+1) - lap;  fly = 0 where fly*(in(j+1) - in) > 0
    out = in - coeff*((flx - flx(i-1)) + (fly - fly(j-1)))
    Each temp lives on the bounding box of the points its consumers read
    (paper §V-B): flx on [lb_i-1, ub_i), fly on [lb_j-1, ub_j), lap on the
    box grown by one in i and j.
    """
    (i0, i1), (j0, j1), (k0, k1) = _box(lb, ub)
    lap_box = ((i0 - 1, i1 + 1), (j0 - 1, j1 + 1), (k0, k1))
    lap = Grid(4.0 * inp.at(lap_box) - inp.at(lap_box, -1, 0) - inp.at(lap_box, 1, 0)
               - inp.at(lap_box, 0, -1) - inp.at(lap_box, 0, 1), (i0 - 1, j0 - 1, k0))

    fx_box = ((i0 - 1, i1), (j0, j1), (k0, k1))
    f = lap.at(fx_box, 1, 0) - lap.at(fx_box)
    flx = Grid(np.where(f * (inp.at(fx_box, 1, 0) - inp.at(fx_box)) > 0, 0.0, f), (i0 - 1, j0, k0))

    fy_box = ((i0, i1), (j0 - 1, j1), (k0, k1))
    g = lap.at(fy_box, 0, 1) - lap.at(fy_box)
    fly = Grid(np.where(g * (inp.at(fy_box, 0, 1) - inp.at(fy_box)) > 0, 0.0, g), (i0, j0 - 1, k0))

    box = _box(lb, ub)
    out = inp.at(box) - coeff.at(box) * ((flx.at(box) - flx.at(box, -1, 0))
                                         + (fly.at(box) - fly.at(box, 0, -1)))
    return {"lap": lap, "flx": flx, "fly": fly, "out": Grid(out, lb)}


def hdiff(inp: Grid, coeff: Grid, lb, ub) -> np.ndarray:
    """Horizontal diffusion output over [lb, ub), staged evaluation."""
    return hdiff_stages(inp, coeff, lb, ub)["out"].arr


def hdiff_point(inp: Grid, coeff: Grid, i, j, k) -> float:
    """Inlined (paper §V-A) evaluation of one hdiff output point: every access
    to a producer recomputes it at that offset; pure Python floats (binary64)."""
    v = lambda a, b: inp.value(a, b, k)

    def lap(a, b):
        return 4.0 * v(a, b) - v(a - 1, b) - v(a + 1, b) - v(a, b - 1) - v(a, b + 1)

    def flx(a, b):
        f = lap(a + 1, b) - lap(a, b)
        return 0.0 if f * (v(a + 1, b) - v(a, b)) > 0 else f

    def fly(a, b):
        g = lap(a, b + 1) - lap(a, b)
        return 0.0 if g * (v(a, b + 1) - v(a, b)) > 0 else g

    return v(i, j) - coeff.value(i, j, k) * ((flx(i, j) - flx(i - 1, j)) + (fly(i, j) - fly(i, j - 1)))


# ----------------------------------------------------------------------------
# vadvc: per-column tridiagonal system + Thomas sweep (design-note reading D2)
# ----------------------------------------------------------------------------

def vadvc_matrix(w: Grid, lb, ub):
    """Diagonals a, b, c (each [K, nj, ni]) of the per-column system.

    wf(k) = 0.5*(w(i,j,k) + w(i+1,j,k)); a_k = -0.25*wf(k) for k >= 1, a_0 = 0;
    c_k = 0.25*wf(k+1) for k <= K-2, c_{K-1} = 0; b_k = (dtr + |a_k|) + |c_k|
    (b is returned without dtr added: see ``vadvc_solve``).
    """
    box = _box(lb, ub)
    wf = 0.5 * (w.at(box) + w.at(box, 1, 0))
    K = ub[2] - lb[2]
    a = np.zeros_like(wf)
    c = np.zeros_like(wf)
    for k in range(1, K):
        a[k] = -0.25 * wf[k]
    for k in range(0, K - 1):
        c[k] = 0.25 * wf[k + 1]
    return a, c


def vadvc_rhs(phi: np.ndarray, a: np.ndarray, c: np.ndarray, dtr: float) -> np.ndarray:
    """d_k = dtr*phi_k - 0.5*(a_k*(phi_{k-1}-phi_k) + c_k*(phi_{k+1}-phi_k)); a term
    whose coefficient is zero by definition at the column ends is left out."""
    K = phi.shape[0]
    d = np.empty_like(phi)
    for k in range(K):
        lo = k > 0
        hi = k < K - 1
        if lo and hi:
            d[k] = dtr * phi[k] - 0.5 * (a[k] * (phi[k - 1] - phi[k]) + c[k] * (phi[k + 1] - phi[k]))
        elif hi:
            d[k] = dtr * phi[k] - 0.5 * (c[k] * (phi[k + 1] - phi[k]))
        elif lo:
            d[k] = dtr * phi[k] - 0.5 * (a[k] * (phi[k - 1] - phi[k]))
        else:
            d[k] = dtr * phi[k]
    return d


def thomas(a: np.ndarray, b: np.ndarray, c: np.ndarray, d: np.ndarray) -> np.ndarray:
    """Thomas algorithm (forward elimination, back substitution) along axis 0,
    vectorised over the remaining axes, no pivoting:
      c'_0 = c_0/b_0, d'_0 = d_0/b_0
      m = b_k - a_k*c'_{k-1}; c'_k = c_k/m; d'_k = (d_k - a_k*d'_{k-1})/m
      x_{K-1} = d'_{K-1};  x_k = d'_k - c'_k*x_{k+1}
    """
    K = d.shape[0]
    cp = np.empty_like(d)
    dp = np.empty_like(d)
    cp[0] = c[0] / b[0]
    dp[0] = d[0] / b[0]
    for k in range(1, K):
        m = b[k] - a[k] * cp[k - 1]
        cp[k] = c[k] / m
        dp[k] = (d[k] - a[k] * dp[k - 1]) / m
    x = np.empty_like(d)
    x[K - 1] = dp[K - 1]
    for k in range(K - 2, -1, -1):
        x[k] = dp[k] - cp[k] * x[k + 1]
    return x


def vadvc_solve(phi: np.ndarray, w: Grid, lb, ub, dtr: float) -> np.ndarray:
    """Implicit vertical advection of ``phi`` (values over [lb, ub)) by ``w``."""
    a, c = vadvc_matrix(w, lb, ub)
    b = (dtr + np.abs(a)) + np.abs(c)
    d = vadvc_rhs(phi, a, c, dtr)
    return thomas(a, b, c, d)


def hdiff_vadvc(u: Grid, v: Grid, w: Grid, coeff: Grid, lb, ub, dtr: float):
    """u_out = vadvc(hdiff(u)), v_out = vadvc(hdiff(v)); one matrix, two RHS."""
    ud = hdiff(u, coeff, lb, ub)
    vd = hdiff(v, coeff, lb, ub)
    return vadvc_solve(ud, w, lb, ub, dtr), vadvc_solve(vd, w, lb, ub, dtr)


# ----------------------------------------------------------------------------
# fastwaves-like program (Table II "fastwavesuv" shape; reading D3)
# ----------------------------------------------------------------------------

FASTWAVES_INPUTS = ("u_in", "v_in", "utens", "vtens", "pp", "rho", "wgtfac", "hhl", "fx")


def fastwaves_stages(f: dict, lb, ub, dt: float, alpha: float):
    """Six stages, staged over inferred boxes. ``f`` maps input names to Grids.

    S1 ppgk = wgtfac*pp + (1 - wgtfac)*pp(k-1)
    S2 ppgc = ppgk(k+1) - ppgk
    S3 ppgu = (pp(i+1) - pp) + 0.25*(ppgc(i+1) + ppgc)*((hhl(k+1) + hhl)
              - (hhl(i+1,k+1) + hhl(i+1))) / ((hhl(k+1) - hhl) + (hhl(i+1,k+1) - hhl(i+1)))
    S4 ppgv = S3 with i+1 replaced by j+1
    S5 div  = (-u(i+2) + 8*u(i+1) - 8*u(i-1) + u(i-2))/12 + (same for v along j)
    S6 u_out = u_in + dt*((utens - ppgu*2*fx/(rho(i+1) + rho)) + alpha*(div(i+1) - div))
       v_out = v_in + dt*((vtens - ppgv*2*fx/(rho(j+1) + rho)) + alpha*(div(j+1) - div))
    """
    (i0, i1), (j0, j1), (k0, k1) = box = _box(lb, ub)
    pp, hhl = f["pp"], f["hhl"]
    # S2 is read at (i, i+1) and (j, j+1): box grown by one in i and j (bounding box)
    c_box = ((i0, i1 + 1), (j0, j1 + 1), (k0, k1))
    # S1 is read by S2 at k and k+1
    k_box = ((i0, i1 + 1), (j0, j1 + 1), (k0, k1 + 1))
    wg = f["wgtfac"]
    ppgk = Grid(wg.at(k_box) * pp.at(k_box) + (1.0 - wg.at(k_box)) * pp.at(k_box, 0, 0, -1),
                (i0, j0, k0))
    ppgc = Grid(ppgk.at(c_box, 0, 0, 1) - ppgk.at(c_box), (i0, j0, k0))

    def pgrad(di, dj):
        return ((pp.at(box, di, dj) - pp.at(box))
                + 0.25 * (ppgc.at(box, di, dj) + ppgc.at(box))
                * ((hhl.at(box, 0, 0, 1) + hhl.at(box)) - (hhl.at(box, di, dj, 1) + hhl.at(box, di, dj)))
                / ((hhl.at(box, 0, 0, 1) - hhl.at(box)) + (hhl.at(box, di, dj, 1) - hhl.at(box, di, dj))))

    ppgu = Grid(pgrad(1, 0), lb)
    ppgv = Grid(pgrad(0, 1), lb)

    u, v = f["u_in"], f["v_in"]
    div = Grid((-u.at(c_box, 2, 0) + 8.0 * u.at(c_box, 1, 0) - 8.0 * u.at(c_box, -1, 0) + u.at(c_box, -2, 0)) / 12.0
               + (-v.at(c_box, 0, 2) + 8.0 * v.at(c_box, 0, 1) - 8.0 * v.at(c_box, 0, -1) + v.at(c_box, 0, -2)) / 12.0,
               (i0, j0, k0))
    rho, fx = f["rho"], f["fx"]
    u_out = u.at(box) + dt * ((f["utens"].at(box) - ppgu.at(box) * 2.0 * fx.at(box) / (rho.at(box, 1, 0) + rho.at(box)))
                              + alpha * (div.at(box, 1, 0) - div.at(box)))
    v_out = v.at(box) + dt * ((f["vtens"].at(box) - ppgv.at(box) * 2.0 * fx.at(box) / (rho.at(box, 0, 1) + rho.at(box)))
                              + alpha * (div.at(box, 0, 1) - div.at(box)))
    return {"ppgk": ppgk, "ppgc": ppgc, "ppgu": ppgu, "ppgv": ppgv, "div": div,
            "u_out": Grid(u_out, lb), "v_out": Grid(v_out, lb)}


def fastwaves(f: dict, lb, ub, dt: float, alpha: float):
    s = fastwaves_stages(f, lb, ub, dt, alpha)
    return s["u_out"].arr, s["v_out"].arr


def fastwaves_point(f: dict, i, j, k, dt: float, alpha: float):
    """Inlined per-point evaluation of both fastwaves outputs (pure Python)."""
    g = lambda name, a, b, c: f[name].value(a, b, c)

    def ppgk(a, b, c):
        return g("wgtfac", a, b, c) * g("pp", a, b, c) + (1.0 - g("wgtfac", a, b, c)) * g("pp", a, b, c - 1)

    def ppgc(a, b, c):
        return ppgk(a, b, c + 1) - ppgk(a, b, c)

    def pgrad(di, dj):
        h = lambda a, b, c: g("hhl", a, b, c)
        return ((g("pp", i + di, j + dj, k) - g("pp", i, j, k))
                + 0.25 * (ppgc(i + di, j + dj, k) + ppgc(i, j, k))
                * ((h(i, j, k + 1) + h(i, j, k)) - (h(i + di, j + dj, k + 1) + h(i + di, j + dj, k)))
                / ((h(i, j, k + 1) - h(i, j, k)) + (h(i + di, j + dj, k + 1) - h(i + di, j + dj, k))))

    def div(a, b):
        u = lambda x: g("u_in", x, b, k)
        v = lambda y: g("v_in", a, y, k)
        return ((-u(a + 2) + 8.0 * u(a + 1) - 8.0 * u(a - 1) + u(a - 2)) / 12.0
                + (-v(b + 2) + 8.0 * v(b + 1) - 8.0 * v(b - 1) + v(b - 2)) / 12.0)

    uo = g("u_in", i, j, k) + dt * ((g("utens", i, j, k) - pgrad(1, 0) * 2.0 * g("fx", i, j, k)
                                     / (g("rho", i + 1, j, k) + g("rho", i, j, k)))
                                    + alpha * (div(i + 1, j) - div(i, j)))
    vo = g("v_in", i, j, k) + dt * ((g("vtens", i, j, k) - pgrad(0, 1) * 2.0 * g("fx", i, j, k)
                                     / (g("rho", i, j + 1, k) + g("rho", i, j, k)))
                                    + alpha * (div(i, j + 1) - div(i, j)))
    return uo, vo
