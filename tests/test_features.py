"""Host-side tests of the autotuner's candidate sets and the cost-model
features (no GPU needed)."""

import numpy as np

from paper_2005_13014_gb300 import inputs, programs


def _prog(src, dtype="f32", generic=True):
    from paper_2005_13014_gb300.api import Program
    return Program(src, dtype, generic=generic)


def test_candidate_sets(liboec):
    assert len(_prog(inputs.random_dag(10000)).candidates()) == 108
    assert len(_prog(programs.HDIFF, "f64", generic=False).candidates()) == 233
    assert len(_prog(programs.HDIFF, "f32", generic=False).candidates()) == 95
    assert len(_prog(programs.HDIFF_VADVC, "f64", generic=False).candidates()) == 72
    c = _prog(programs.FASTWAVES, "f64", generic=False).candidates()
    assert len(c) == 152 and {x["arith"] for x in c} == {0, 1}


def test_features_shape_and_schedule_dependence(liboec):
    p = _prog(inputs.random_dag(10007))
    cands = p.candidates()
    F = np.stack([p.features((256, 256, 80), 272, 272 * 272, c) for c in cands])
    assert F.shape == (108, 42) and np.all(np.isfinite(F))
    # program columns identical across schedules, schedule columns not
    assert np.all(F[:, :21] == F[0, :21])
    assert len({tuple(r) for r in F[:, 21:]}) == 108
    onehot = F[:, 21:24]
    assert np.all(onehot.sum(axis=1) == 1)
    # stage-by-stage code stores temporaries, inlined code does not
    none = F[onehot[:, 1] == 1]
    inl = F[onehot[:, 0] == 1]
    if p.n_stages > 1:
        assert np.all(none[:, 32] > 0) and np.all(inl[:, 32] == 0)
    # deterministic
    assert np.array_equal(F[5], p.features((256, 256, 80), 272, 272 * 272, cands[5]))
