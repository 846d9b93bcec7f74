"""Tuning database (oec_tunedb_*), host side: keys separate what the
schedules depend on (program, dtype, domain extent, strides, alignment),
entries survive a save and a reload, malformed files are refused, and an
invalid schedule is not recorded. Fake device pointers are never read."""

import ctypes as C

import pytest

from paper_2005_13014_gb300 import _lib as L
from paper_2005_13014_gb300 import programs


def _prog(src, dtype="f64"):
    from paper_2005_13014_gb300.api import Program
    return Program(src, dtype=dtype)


def _fake(addr, shape, origin, es=8, dtype=L.F64):
    d = L.FieldDesc()
    d.data = addr
    d.dtype = dtype
    d.ndim = 3
    ni, nj, nk = shape
    d.size = L.I64x3(ni, nj, nk)
    d.stride = L.I64x3(1, ni, ni * nj)
    d.origin = L.I64x3(*origin)
    return d


def _case(p, n, h=3, base=1 << 30, pad=0):
    shp = (n[0] + 2 * h + pad, n[1] + 2 * h, n[2] + 2 * h)
    ins = [_fake(base + x * (1 << 28), shp, (h, h, h)) for x in range(p.n_inputs)]
    outs = [_fake(base + (8 + x) * (1 << 28), shp, (h, h, h)) for x in range(p.n_outputs)]
    return ins, outs


def _arr(descs):
    return (L.FieldDesc * len(descs))(*descs)


def _find(db, p, ins, outs, n):
    s, ms, found = L.Schedule(), C.c_double(), C.c_int()
    L.check(L.lib().oec_tunedb_find(db, p.handle, _arr(ins), len(ins), _arr(outs), len(outs), L.I64x3(0, 0, 0),
                                    L.I64x3(*n), C.byref(s), C.byref(ms), C.byref(found)))
    return (s, ms.value) if found.value else None


def _record(db, p, ins, outs, n, sched, ms):
    s = L.Schedule(*sched)
    return L.lib().oec_tunedb_record(db, p.handle, _arr(ins), len(ins), _arr(outs), len(outs), L.I64x3(0, 0, 0),
                                     L.I64x3(*n), C.byref(s), ms)


def _open(path):
    h = C.c_void_p()
    L.check(L.lib().oec_tunedb_open(path.encode() if path else None, C.byref(h)))
    return h


def test_record_find_save_reload(liboec, tmp_path):
    path = str(tmp_path / "tune.db")
    db = _open(path)                              # no file yet: empty
    assert L.lib().oec_tunedb_count(db) == 0
    hv = _prog(programs.HDIFF_VADVC)
    n = (128, 128, 80)
    ins, outs = _case(hv, n)
    assert _find(db, hv, ins, outs, n) is None
    staged = (1, 0, 32, 8, 1, 4, 2)
    assert _record(db, hv, ins, outs, n, staged, 0.0747) == 0
    s, ms = _find(db, hv, ins, outs, n)
    assert (s.fusion, s.tile_i, s.tile_j, s.k_chunk, s.arith) == (1, 32, 8, 4, 2) and ms == pytest.approx(0.0747)
    # what the key separates: extent, dtype, strides (row padding), program
    n2 = (128, 128, 79)
    assert _find(db, hv, *_case(hv, n2), n2) is None
    hv32 = _prog(programs.HDIFF_VADVC, "f32")
    assert _find(db, hv32, *_case(hv32, n), n) is None
    assert _find(db, hv, *_case(hv, n, pad=1), n) is None
    hd = _prog(programs.HDIFF)
    assert _find(db, hd, *_case(hd, n), n) is None
    assert _record(db, hd, *_case(hd, n), n, (0, 4, 32, 8, 2, 4, 0), 0.017) == 0
    L.check(L.lib().oec_tunedb_save(db, None))
    L.lib().oec_tunedb_close(db)
    text = open(path).read().splitlines()
    assert text[0] == "oec-tunedb 1" and len(text) == 3
    db = _open(path)
    assert L.lib().oec_tunedb_count(db) == 2
    s, ms = _find(db, hv, ins, outs, n)
    assert (s.fusion, s.staging, s.tile_i, s.tile_j, s.unroll, s.k_chunk, s.arith) == staged
    L.lib().oec_tunedb_close(db)


def test_index_bits_survive_a_reload(liboec, tmp_path):
    """The schedule's offset width is stored; entries written without it
    (seven schedule fields) read back as OEC_INDEX_AUTO."""
    path = str(tmp_path / "tune.db")
    db = _open(path)
    hd = _prog(programs.HDIFF, "f32")
    n = (64, 64, 8)
    assert _record(db, hd, *_case(hd, n), n, (0, 0, 64, 4, 2, 0, 0, 64), 0.01) == 0
    L.check(L.lib().oec_tunedb_save(db, None))
    L.lib().oec_tunedb_close(db)
    lines = open(path).read().splitlines()
    assert lines[1].split("\t")[1] == "0 0 64 4 2 0 0 64 0 0"
    db = _open(path)
    s, _ = _find(db, hd, *_case(hd, n), n)
    assert (s.tile_i, s.unroll, s.index_bits) == (64, 2, 64)
    L.lib().oec_tunedb_close(db)
    key = lines[1].split("\t")[0]
    with open(path, "w") as f:
        f.write(f"oec-tunedb 1\n{key}\t0 0 64 4 2 0 0\t0.01\n")
    db = _open(path)
    s, _ = _find(db, hd, *_case(hd, n), n)
    assert (s.tile_i, s.unroll, s.index_bits) == (64, 2, 0)
    L.lib().oec_tunedb_close(db)


def test_sweep_and_slabs_survive_a_reload(liboec, tmp_path):
    """The staged hdiff+vadvc schedule fields sweep and slabs are stored and
    read back; entries written without them read back as 0."""
    path = str(tmp_path / "tune.db")
    db = _open(path)
    hv = _prog(programs.HDIFF_VADVC, "f64")
    n = (64, 32, 16)
    assert _record(db, hv, *_case(hv, n), n, (1, 0, 32, 8, 1, 4, 2, 0, 1, 4), 0.02) == 0
    L.check(L.lib().oec_tunedb_save(db, None))
    L.lib().oec_tunedb_close(db)
    lines = open(path).read().splitlines()
    assert lines[1].split("\t")[1] == "1 0 32 8 1 4 2 0 1 4"
    db = _open(path)
    s, _ = _find(db, hv, *_case(hv, n), n)
    assert (s.tile_j, s.arith, s.sweep, s.slabs) == (8, 2, 1, 4)
    L.lib().oec_tunedb_close(db)
    key = lines[1].split("\t")[0]
    with open(path, "w") as f:
        f.write(f"oec-tunedb 1\n{key}\t1 0 32 8 1 4 2 0\t0.02\n")
    db = _open(path)
    s, _ = _find(db, hv, *_case(hv, n), n)
    assert (s.tile_j, s.sweep, s.slabs) == (8, 0, 0)
    L.lib().oec_tunedb_close(db)


def test_alignment_is_part_of_the_key(liboec):
    db = _open(None)
    hd = _prog(programs.HDIFF, "f32")
    n = (64, 64, 8)
    # rows of 64 + 2*2 + 8 floats from a 16-byte aligned base, corner at column
    # 4: aligned; the same with the base moved by 4 bytes: not
    ins, outs = _case(hd, n, h=2, pad=8)
    for d in ins + outs:
        d.origin = L.I64x3(4, 2, 2)
    assert _record(db, hd, ins, outs, n, (0, 4, 32, 4, 1, 0, 0), 0.01) == 0
    assert _find(db, hd, ins, outs, n) is not None
    for d in ins + outs:
        d.data += 4
    assert _find(db, hd, ins, outs, n) is None
    L.lib().oec_tunedb_close(db)


def test_bad_files_and_schedules_refused(liboec, tmp_path):
    bad = tmp_path / "bad.db"
    bad.write_text("not a database\n")
    h = C.c_void_p()
    assert L.lib().oec_tunedb_open(str(bad).encode(), C.byref(h)) == -1
    bad.write_text("oec-tunedb 1\nkey\t1 2 3\t0.5\n")
    assert L.lib().oec_tunedb_open(str(bad).encode(), C.byref(h)) == -1
    assert ":2:" in L.lib().oec_last_error().decode()
    db = _open(None)
    hd = _prog(programs.HDIFF)
    n = (16, 16, 4)
    assert _record(db, hd, *_case(hd, n), n, (0, 1, 48, 4, 1, 0, 0), 0.1) == -7   # no such SMEM tile
    assert L.lib().oec_tunedb_count(db) == 0
    assert L.lib().oec_tunedb_save(db, None) == -1                                # memory-only, no path
    L.lib().oec_tunedb_close(db)
