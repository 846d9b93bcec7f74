"""Host-side pieces of the cost-model experiment: the feature names match the
library's feature count, and the greedy roofline fusion baseline picks the
fusion with the lowest roofline estimate (constructed cases, no GPU)."""

import numpy as np
import pytest

from paper_2005_13014_gb300 import costmodel as CM


def _cands():
    return [dict(fusion=f, tile_i=ti, tile_j=tj, unroll=u) for f in (0, 1, 2) for (ti, tj) in ((64, 4), (32, 8))
            for u in (1, 2)]


def _features(bytes_pp, ops_pp):
    F = np.zeros((len(bytes_pp), CM.N_FEATURES))
    F[:, CM.F["bytes_per_point"]] = bytes_pp
    F[:, CM.F["ops_per_point"]] = ops_pp
    return F


def test_feature_names_cover_the_library_features(liboec):
    from paper_2005_13014_gb300 import inputs
    from paper_2005_13014_gb300.api import Program
    p = Program(inputs.random_dag(10003), "f32", generic=True)
    c = p.candidates()
    f = p.features((64, 32, 16), 72, 72 * 40, c[0])
    assert f.shape == (CM.N_FEATURES,) == (len(CM.FEATURE_NAMES),)
    inline = [x for x, s in enumerate(c) if s["fusion"] == 0][0]
    none = [x for x, s in enumerate(c) if s["fusion"] == 1][0]
    fi = p.features((64, 32, 16), 72, 72 * 40, c[inline])
    fn = p.features((64, 32, 16), 72, 72 * 40, c[none])
    assert fi[CM.F["fuse_inline"]] == 1 and fn[CM.F["fuse_none"]] == 1
    # stage-by-stage code moves its temporaries: more bytes per point than inlined code
    if p.n_stages > 1:
        assert fn[CM.F["bytes_per_point"]] > fi[CM.F["bytes_per_point"]]


def test_greedy_picks_lowest_roofline_estimate():
    c = _cands()
    n = len(c)
    hbm, ops = 1e12, 1e13
    # memory-bound everywhere: the fusion moving the fewest bytes wins
    b = np.full(n, 40.0)
    o = np.full(n, 10.0)
    for x, s in enumerate(c):
        b[x] = {0: 24.0, 1: 48.0, 2: 30.0}[s["fusion"]]
    g = CM.greedy_fusion(_features(b, o), c, hbm, ops)
    assert c[g]["fusion"] == 0 and c[g]["tile_i"] == 64 and c[g]["unroll"] == 1
    # inlining recomputes so much that it turns compute-bound: partial wins
    for x, s in enumerate(c):
        o[x] = {0: 900.0, 1: 20.0, 2: 60.0}[s["fusion"]]
    g = CM.greedy_fusion(_features(b, o), c, hbm, ops)
    assert c[g]["fusion"] == 2
    est = CM.roofline_seconds_per_point(_features(b, o), hbm, ops)
    pool = [x for x, s in enumerate(c) if s["tile_i"] == 64 and s["unroll"] == 1]
    assert est[g] == min(est[x] for x in pool)
    # a candidate that cannot run is never picked
    usable = np.ones(n, bool)
    usable[g] = False
    g2 = CM.greedy_fusion(_features(b, o), c, hbm, ops, usable=usable)
    assert g2 != g and c[g2]["fusion"] in (0, 1)
    # another tile and unroll
    g3 = CM.greedy_fusion(_features(b, o), c, hbm, ops, tile=(32, 8), unroll=2)
    assert c[g3]["tile_i"] == 32 and c[g3]["unroll"] == 2 and c[g3]["fusion"] == 2
    with pytest.raises(ValueError):
        CM.greedy_fusion(_features(b, o), c, hbm, ops, tile=(128, 1))
