"""Autotuning through the tuning database on the GPU: the first call times
every candidate and records the fastest; a second call, and a call after the
database was saved and reopened, take the recorded schedule without timing."""

import numpy as np
import pytest

from paper_2005_13014_gb300 import inputs, programs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_autotune_db_records_then_reuses(tmp_path):
    from paper_2005_13014_gb300.api import Program, TuneDB, device_field
    n, h = (48, 40, 12), 3
    f = inputs.hdiff_vadvc_fields(*n, h, seed=81)
    ins = [device_field(f[k], h, "f64") for k in ("u", "v", "w", "coeff")]
    outs = [device_field(np.zeros_like(f["u"]), h, "f64") for _ in range(2)]
    path = str(tmp_path / "tune.db")
    db = TuneDB(path)
    p = Program(programs.HDIFF_VADVC, "f64")
    assert p.autotune_db(db, ins, outs, (0, 0, 0), n, (h, h, h), [2.0], reps=2) is False
    tuned = p.schedule
    assert len(db) == 1
    rec = db.find(p, ins, outs, (0, 0, 0), n)
    assert rec is not None and rec[0] == tuned and rec[1] > 0
    q = Program(programs.HDIFF_VADVC, "f64")
    assert q.autotune_db(db, ins, outs, (0, 0, 0), n, (h, h, h), [2.0]) is True
    assert q.schedule == tuned
    db.save()
    db.close()
    db2 = TuneDB(path)
    r = Program(programs.HDIFF_VADVC, "f64")
    assert r.autotune_db(db2, ins, outs, (0, 0, 0), n, (h, h, h), [2.0]) is True
    assert r.schedule == tuned
    # the recorded schedule computes the program
    r.apply(ins, outs, (0, 0, 0), n, (h, h, h), [2.0])
    torch.cuda.synchronize()
    assert np.isfinite(outs[0].interior((0, 0, 0), n).cpu().numpy()).all()
