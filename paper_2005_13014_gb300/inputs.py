"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module draws random numbers and builds random program structure; it holds
none of the stencil arithmetic. Both the CUDA path and the CPU oracle consume
what it returns, so it imports neither.

Fields are float64 numpy arrays indexed [k, j, i] with ``h`` halo cells on both
sides of every dimension (storage extent n + 2h per dimension). Field number
``f`` of a program is drawn from ``numpy.random.default_rng(seed + f)``.
"""

from __future__ import annotations

import numpy as np

SEED = 2005


def _uniform(shape, lo, hi, seed):
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


def storage_shape(ni, nj, nk, h):
    return (nk + 2 * h, nj + 2 * h, ni + 2 * h)


def hdiff_fields(ni, nj, nk, h, seed=SEED):
    """in ~ U[-1, 1], coeff ~ U[0, 0.1], over the whole storage (halo included)."""
    s = storage_shape(ni, nj, nk, h)
    return {"in": _uniform(s, -1.0, 1.0, seed + 0), "coeff": _uniform(s, 0.0, 0.1, seed + 1)}


def hdiff_vadvc_fields(ni, nj, nk, h, seed=SEED):
    """u, v, w ~ U[-1, 1], coeff ~ U[0, 0.1]."""
    s = storage_shape(ni, nj, nk, h)
    return {"u": _uniform(s, -1.0, 1.0, seed + 0), "v": _uniform(s, -1.0, 1.0, seed + 1),
            "w": _uniform(s, -1.0, 1.0, seed + 2), "coeff": _uniform(s, 0.0, 0.1, seed + 3)}


FASTWAVES_NAMES = ("u_in", "v_in", "utens", "vtens", "pp", "rho", "wgtfac", "hhl", "fx")


def fastwaves_fields(ni, nj, nk, h, seed=SEED):
    """u_in, v_in, utens, vtens, pp ~ U[-1,1]; rho, fx ~ U[0.5,1.5];
    wgtfac ~ U[0.4,0.6]; hhl at storage level k = 100*(nk + 2h - k) + U[0,10]
    (heights fall with k, layer thickness at least 90)."""
    s = storage_shape(ni, nj, nk, h)
    out = {}
    ranges = {"u_in": (-1, 1), "v_in": (-1, 1), "utens": (-1, 1), "vtens": (-1, 1), "pp": (-1, 1),
              "rho": (0.5, 1.5), "wgtfac": (0.4, 0.6), "fx": (0.5, 1.5)}
    for idx, name in enumerate(FASTWAVES_NAMES):
        if name == "hhl":
            levels = 100.0 * (s[0] - np.arange(s[0], dtype=np.float64))
            out[name] = levels[:, None, None] + _uniform(s, 0.0, 10.0, seed + idx)
        else:
            lo, hi = ranges[name]
            out[name] = _uniform(s, float(lo), float(hi), seed + idx)
    return out


def field_uniform(n, h, lo, hi, seed):
    """One field U[lo, hi] over storage with halo h (int or (hi, hj, hk))."""
    hh = (h, h, h) if np.isscalar(h) else tuple(h)
    shape = (n[2] + 2 * hh[2], n[1] + 2 * hh[1], n[0] + 2 * hh[0])
    return _uniform(shape, lo, hi, seed)


def ensemble_members(n=32, seed=SEED):
    """Member interior extents (ni, nj, nk): i and j each from {64,128,256,512},
    k from {60,80,137}."""
    rng = np.random.default_rng(seed)
    ij = np.array([64, 128, 256, 512])
    ks = np.array([60, 80, 137])
    return [(int(rng.choice(ij)), int(rng.choice(ij)), int(rng.choice(ks))) for _ in range(n)]


def dag_shape(seed):
    """Domain of a random program in the varied-shape cost-model experiment:
    i and j each from {64,128,256,512}, k from {60,80,137} (the ensemble
    members' distribution), drawn from the program's seed."""
    rng = np.random.default_rng(seed + 777)
    ij = np.array([64, 128, 256, 512])
    ks = np.array([60, 80, 137])
    return (int(rng.choice(ij)), int(rng.choice(ij)), int(rng.choice(ks)))


def random_dag(seed, max_halo_ij=8, max_halo_k=4):
    """Random stencil program text: 3-12 stages, 1-4 input fields, each stage
    reading 1-3 earlier values at offsets |di|,|dj| <= 2, |dk| <= 1, built from
    convex combinations with dyadic weights, min, max, abs and select, so values
    stay within about [-1, 1]; one or two outputs. Every select whose branches
    differ at the switch point tests an input field, never a computed value. The accumulated offset reach from
    any output down to the inputs stays within (max_halo_ij, max_halo_k)."""
    rng = np.random.default_rng(seed)
    n_in = int(rng.integers(1, 5))
    n_st = max(int(rng.integers(3, 13)), n_in)
    inputs = [f"f{x}" for x in range(n_in)]
    reach = {n: (0, 0, 0) for n in inputs}
    names = list(inputs)
    lines = ["input " + ", ".join(inputs)]

    def offset(src):
        ri, rj, rk = reach[src]
        di = int(rng.integers(-min(2, max_halo_ij - ri), min(2, max_halo_ij - ri) + 1))
        dj = int(rng.integers(-min(2, max_halo_ij - rj), min(2, max_halo_ij - rj) + 1))
        dk = int(rng.integers(-min(1, max_halo_k - rk), min(1, max_halo_k - rk) + 1))
        return di, dj, dk

    def weights(n):
        # dyadic weights (multiples of 1/8, each >= 1/8) summing to one
        cuts = np.sort(rng.choice(np.arange(1, 8), size=n - 1, replace=False)) if n > 1 else np.array([], int)
        parts = np.diff(np.concatenate([[0], cuts, [8]]))
        return [f"{p / 8:.3f}" for p in parts]

    for s in range(n_st):
        name = f"s{s}"
        srcs = [names[-1]]                       # chain: every stage feeds the next
        if s < n_in:
            srcs = [inputs[s]] + ([names[-1]] if s > 0 else [])
        n_reads = int(rng.integers(1, 4))
        while len(srcs) < n_reads:
            srcs.append(names[int(rng.integers(0, len(names)))])
        terms, r = [], [0, 0, 0]
        for src in srcs:
            di, dj, dk = offset(src)
            terms.append(f"{src}[{di},{dj},{dk}]")
            r = [max(r[0], reach[src][0] + abs(di)), max(r[1], reach[src][1] + abs(dj)),
                 max(r[2], reach[src][2] + abs(dk))]
        kind = int(rng.integers(0, 5))
        if len(terms) == 1:
            expr = [f"abs({terms[0]})", f"-{terms[0]}", f"0.5*{terms[0]}"][kind % 3]
        elif kind == 0 or len(terms) == 2 and kind == 3:
            expr = " + ".join(f"{w}*{t}" for w, t in zip(weights(len(terms)), terms))
        elif kind == 1:
            expr = f"min({terms[0]}, {terms[1]})" + (f" * 0.5 + 0.5*{terms[2]}" if len(terms) > 2 else "")
        elif kind == 2:
            expr = f"max({terms[0]}, {terms[1]})" + (f" * 0.5 - 0.5*{terms[2]}" if len(terms) > 2 else "")
        elif kind == 3:
            # the only discontinuous choice tests an input field directly, so both
            # precisions take the same branch (inputs are exact in either)
            cond = inputs[int(rng.integers(0, n_in))]
            ci, cj = int(rng.integers(-1, 2)), int(rng.integers(-1, 2))
            r = [max(r[0], abs(ci)), max(r[1], abs(cj)), r[2]]
            expr = f"select({cond}[{ci},{cj},0] > 0.0, {terms[1]}, {terms[2]})"
        else:
            lets = f"let t = {terms[0]} - {terms[1]}; "
            rest = f" + 0.25*{terms[2]}" if len(terms) > 2 else ""
            expr = "{ " + lets + f"return select(t > 0.0, 0.5*t, -0.25*t){rest} }}"
        lines.append(f"stage {name} = {expr}")
        reach[name] = tuple(r)
        names.append(name)
    outs = [names[-1]]
    if rng.random() < 0.5:
        outs.insert(0, f"s{int(rng.integers(0, n_st - 1))}")
    lines.append("output " + ", ".join(outs))
    return "\n".join(lines) + "\n"


def mlp_init(n_features, hidden=64, seed=SEED):
    """He-uniform weights U[-sqrt(6/fan_in), +sqrt(6/fan_in)], zero biases (float64)."""
    rng = np.random.default_rng(seed)
    def he(o, i):
        lim = np.sqrt(6.0 / i)
        return rng.uniform(-lim, lim, size=(o, i))
    return {"W1": he(hidden, n_features), "b1": np.zeros(hidden),
            "W2": he(hidden, hidden), "b2": np.zeros(hidden),
            "W3": he(1, hidden), "b3": np.zeros(1)}


# input distributions of the Table II stand-ins (programs.TESTSET): uniform
# ranges, or "kup"/"kdown" for fields that increase/decrease with k like
# pressure and geopotential on a k-staggered grid (100 per level + U[0,10])
TESTSET_INPUTS = {
    "uvbke": {"uc": (-1, 1), "vc": (-1, 1), "cosa": (-0.3, 0.3), "rsina": (1.0, 1.1)},
    "p_grad_c": {"uc": (-1, 1), "vc": (-1, 1), "delpc": (1.0, 2.0), "pkc": "kup", "gz": "kdown",
                 "rdxc": (0.5, 1.5), "rdyc": (0.5, 1.5)},
    "hadvuv": {n: (-1, 1) for n in ("uin", "vin", "uatupos", "vatupos", "uatvpos", "vatvpos")},
    "fvtp2d_flux": {n: (-1, 1) for n in ("q", "crx", "cry", "xfx", "yfx", "al", "bl")},
    "hdiffsmag": {"u": (-1, 1), "v": (-1, 1), "hdmask": (0.0, 1.0), "crlavo": (0.9, 1.1), "crlavu": (0.9, 1.1),
                  "crlato": (0.9, 1.1), "crlatu": (0.9, 1.1), "acrlat0": (0.9, 1.1)},
    "hadvuv5th": {n: (-1, 1) for n in ("uin", "vin", "uatupos", "vatupos", "uatvpos", "vatvpos")},
    "nh_p_grad": {"u": (-1, 1), "v": (-1, 1), "rdx": (0.5, 1.5), "rdy": (0.5, 1.5), "gz": "kdown", "pp": (-1, 1),
                  "pk3": "kup", "delp": (1.0, 2.0)},
    "fvtp2d_qi": {"q": (-1, 1), "crx": (-1, 1), "xfx": (-1, 1), "area": (0.5, 1.5), "ra_x": (0.5, 1.5)},
    "fvtp2d_qj": {"q": (-1, 1), "cry": (-1, 1), "yfx": (-1, 1), "area": (0.5, 1.5), "ra_y": (0.5, 1.5),
                  "mfy": (-1, 1)},
}


def testset_fields(name, ni, nj, nk, h, seed=SEED):
    """Storage arrays [k, j, i] (halo h) of one stand-in program's inputs."""
    out = {}
    for x, (fname, dist) in enumerate(TESTSET_INPUTS[name].items()):
        rng = np.random.default_rng(seed + x)
        shape = (nk + 2 * h, nj + 2 * h, ni + 2 * h)
        if isinstance(dist, str):
            k = np.arange(shape[0], dtype=np.float64)[:, None, None]
            ramp = 100.0 * (k if dist == "kup" else (shape[0] - k))
            out[fname] = ramp + rng.uniform(0.0, 10.0, shape)
        else:
            out[fname] = rng.uniform(dist[0], dist[1], shape)
    return out
