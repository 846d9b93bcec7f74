"""Batched ensembles: one persistent launch over members of different sizes
must give, member by member, the same bits as applying the program to each
member alone with the same schedule (both run the same tile sweep), and stay
within the oracle tolerance. Graph replay and direct launch agree."""

import numpy as np
import pytest

from conftest import TOL, rel_err
from oracle import stencils as S
from paper_2005_13014_gb300 import inputs, programs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = [(37, 23, 11), (64, 8, 3), (16, 40, 17), (5, 5, 1), (70, 33, 9), (24, 64, 2)]


def _members(dtype, h=3, shapes=SHAPES, seed=100):
    from paper_2005_13014_gb300.api import device_field
    ms = []
    for x, n in enumerate(shapes):
        f = inputs.hdiff_vadvc_fields(*n, h, seed=seed + 10 * x)
        if dtype == "f32":
            f = {k: v.astype(np.float32).astype(np.float64) for k, v in f.items()}
        d = [device_field(f[k], h, dtype) for k in ("u", "v", "w", "coeff")]
        o = [device_field(np.full_like(f["u"], 3.0), h, dtype) for _ in range(2)]
        ms.append((f, d, o, n))
    return ms


@pytest.mark.parametrize("dtype,arith", [("f64", 0), ("f64", 1), ("f32", 0), ("f32", 1)])
@pytest.mark.parametrize("tile", [(16, 4), (32, 2), (8, 8), (32, 4), (8, 4), (16, 2)])
def test_batch_equals_single_applies_and_oracle(dtype, arith, tile):
    from paper_2005_13014_gb300.api import Batch, Program, device_field
    h = 3
    prog = Program(programs.HDIFF_VADVC, dtype)
    prog.set_schedule(fusion=0, staging=1, tile_i=tile[0], tile_j=tile[1], arith=arith)
    ms = _members(dtype, h)
    batch = Batch(prog, [(d, o, (0, 0, 0), n, (h, h, h)) for (_, d, o, n) in ms], [2.0])
    assert batch.n_items == sum(-(-n[0] // tile[0]) * -(-n[1] // tile[1]) for n in SHAPES)
    for graph in (True, False):
        for (_, _, o, _) in ms:
            for t in o:
                t.tensor.fill_(3.0)
        batch.apply(graph=graph)
        torch.cuda.synchronize()
        for (f, d, o, n) in ms:
            single = [device_field(np.zeros_like(f["u"]), h, dtype) for _ in range(2)]
            prog.apply(d, single, (0, 0, 0), n, (h, h, h), [2.0])
            torch.cuda.synchronize()
            for a, b in zip(o, single):
                assert torch.equal(a.tensor, b.tensor) or torch.equal(
                    a.interior((0, 0, 0), n), b.interior((0, 0, 0), n))
            G = {k: S.Grid.storage(v, h) for k, v in f.items()}
            ru, rv = S.hdiff_vadvc(G["u"], G["v"], G["w"], G["coeff"], (0, 0, 0), n, 2.0)
            gu = o[0].interior((0, 0, 0), n).cpu().numpy().astype(np.float64)
            gv = o[1].interior((0, 0, 0), n).cpu().numpy().astype(np.float64)
            assert max(rel_err(gu, ru), rel_err(gv, rv)) <= TOL[dtype]
            # nothing written outside the member's domain
            full = o[0].tensor.cpu().numpy()
            oi, oj, ok = o[0].origin
            mask = np.ones(full.shape, bool)
            mask[ok:ok + n[2], oj:oj + n[1], oi:oi + n[0]] = False
            assert np.all(full[mask] == 3.0)


@pytest.mark.parametrize("dtype,arith", [("f64", 2), ("f64", 1), ("f32", 1), ("f32", 0)])
def test_staged_batch_equals_single_applies(dtype, arith):
    """Staged batches: every member's chain is a graph branch running the same
    kernels as a single apply, so the bits agree; graph and direct agree."""
    from paper_2005_13014_gb300.api import Batch, Program, device_field
    h = 3
    prog = Program(programs.HDIFF_VADVC, dtype)
    prog.set_schedule(fusion=1, tile_i=32, tile_j=8, k_chunk=4, arith=arith)
    ms = _members(dtype, h)
    batch = Batch(prog, [(d, o, (0, 0, 0), n, (h, h, h)) for (_, d, o, n) in ms], [2.0])
    assert batch.n_items == len(SHAPES)
    for graph in (True, False):
        for (_, _, o, _) in ms:
            for t in o:
                t.tensor.fill_(3.0)
        batch.apply(graph=graph)
        torch.cuda.synchronize()
        for (f, d, o, n) in ms:
            single = [device_field(np.full_like(f["u"], 3.0), h, dtype) for _ in range(2)]
            prog.apply(d, single, (0, 0, 0), n, (h, h, h), [2.0])
            torch.cuda.synchronize()
            for a, b in zip(o, single):
                assert torch.equal(a.tensor, b.tensor)
            G = {k: S.Grid.storage(v, h) for k, v in f.items()}
            ru, rv = S.hdiff_vadvc(G["u"], G["v"], G["w"], G["coeff"], (0, 0, 0), n, 2.0)
            gu = o[0].interior((0, 0, 0), n).cpu().numpy().astype(np.float64)
            gv = o[1].interior((0, 0, 0), n).cpu().numpy().astype(np.float64)
            assert max(rel_err(gu, ru), rel_err(gv, rv)) <= TOL[dtype]


def test_batch_config_ensemble_32_members_f32():
    """The 32-member ensemble of uneven domains (i, j in {64..512}, k in
    {60, 80, 137}), FP32, checked on sampled columns against the oracle."""
    from paper_2005_13014_gb300.api import Batch, Program, device_field
    h = 3
    shapes = inputs.ensemble_members(32)
    prog = Program(programs.HDIFF_VADVC, "f32")
    ms = []
    for x, n in enumerate(shapes):
        f = inputs.hdiff_vadvc_fields(*n, h, seed=inputs.SEED + x)
        d = [device_field(f[k], h, "f32") for k in ("u", "v", "w", "coeff")]
        o = [device_field(np.zeros_like(f["u"]), h, "f32") for _ in range(2)]
        ms.append((f, d, o, n))
    batch = Batch(prog, [(d, o, (0, 0, 0), n, (h, h, h)) for (_, d, o, n) in ms], [2.0])
    batch.apply()
    torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    for (f, d, o, n) in ms[::4]:
        # oracle on a sub-block of columns (the column solve is local to a column)
        i0, j0 = int(rng.integers(0, n[0] - 8)), int(rng.integers(0, n[1] - 8))
        lb, ub = (i0, j0, 0), (i0 + 8, j0 + 8, n[2])
        g = {k: S.Grid.storage(v.astype(np.float32).astype(np.float64), h) for k, v in f.items()}
        ru, rv = S.hdiff_vadvc(g["u"], g["v"], g["w"], g["coeff"], lb, ub, 2.0)
        gu = o[0].interior(lb, ub).cpu().numpy().astype(np.float64)
        gv = o[1].interior(lb, ub).cpu().numpy().astype(np.float64)
        assert max(rel_err(gu, ru), rel_err(gv, rv)) <= TOL["f32"]


@pytest.mark.parametrize("dtype,arith", [("f32", 1), ("f64", 2), ("f32", 0)])
def test_staged_batch_l2_sweep_on_large_members(dtype, arith):
    """Batch members whose column scratch exceeds 48 MB run the column sweep's
    L2 form (recurrence values kept in L2 with evict-last priority and dropped
    once read, four back steps at a time). Column counts that are not multiples
    of 16 and odd level counts (halves of unequal length, partial groups of
    four back steps) give, member by member, the bits of the single applies,
    which use the plain sweep; sampled column blocks match the oracle."""
    from paper_2005_13014_gb300.api import Batch, Program, device_field
    h = 3
    shapes = [(1001, 300, 23), (517, 333, 37), (700, 120, 80), (37, 23, 11)]
    prog = Program(programs.HDIFF_VADVC, dtype)
    prog.set_schedule(fusion=1, tile_i=32, tile_j=8, k_chunk=4, arith=arith)
    ms = _members(dtype, h, shapes=shapes, seed=300)
    batch = Batch(prog, [(d, o, (0, 0, 0), n, (h, h, h)) for (_, d, o, n) in ms], [2.0])
    rng = np.random.default_rng(11)
    for graph in (True, False):
        for (_, _, o, _) in ms:
            for t in o:
                t.tensor.fill_(3.0)
        batch.apply(graph=graph)
        torch.cuda.synchronize()
        for (f, d, o, n) in ms:
            single = [device_field(np.full_like(f["u"], 3.0), h, dtype) for _ in range(2)]
            prog.apply(d, single, (0, 0, 0), n, (h, h, h), [2.0])
            torch.cuda.synchronize()
            for a, b in zip(o, single):
                assert torch.equal(a.tensor, b.tensor)
            del single
    for (f, d, o, n) in ms:
        i0, j0 = int(rng.integers(0, n[0] - 8)), int(rng.integers(0, n[1] - 8))
        lb, ub = (i0, j0, 0), (i0 + 8, j0 + 8, n[2])
        G = {k: S.Grid.storage(v, h) for k, v in f.items()}
        ru, rv = S.hdiff_vadvc(G["u"], G["v"], G["w"], G["coeff"], lb, ub, 2.0)
        gu = o[0].interior(lb, ub).cpu().numpy().astype(np.float64)
        gv = o[1].interior(lb, ub).cpu().numpy().astype(np.float64)
        assert max(rel_err(gu, ru), rel_err(gv, rv)) <= TOL[dtype]


ALIGNED_SHAPES = [(36, 23, 11), (64, 8, 3), (16, 40, 17), (4, 5, 1), (68, 33, 9), (24, 64, 2), (128, 9, 5)]


def _aligned_members(shapes, seed, h=3):
    """FP32 members whose rows are 16-byte aligned at the domain corner (the
    persistent staged batch's warp-row producer needs them)."""
    from paper_2005_13014_gb300.api import device_field
    ms = []
    for x, n in enumerate(shapes):
        f = inputs.hdiff_vadvc_fields(*n, h, seed=seed + 10 * x)
        f = {k: v.astype(np.float32).astype(np.float64) for k, v in f.items()}
        d = [device_field(f[k], h, "f32", align_bytes=16) for k in ("u", "v", "w", "coeff")]
        o = [device_field(np.full_like(f["u"], 3.0), h, "f32", align_bytes=16) for _ in range(2)]
        ms.append((f, d, o, n))
    return ms


def _check_members_against_single(prog, batch, ms, h=3, oracle=True):
    from paper_2005_13014_gb300.api import device_field
    for graph in (True, False):
        for (_, _, o, _) in ms:
            for t in o:
                t.tensor.fill_(3.0)
        batch.apply(graph=graph)
        torch.cuda.synchronize()
        for (f, d, o, n) in ms:
            single = [device_field(np.full_like(f["u"], 3.0), h, "f32", align_bytes=16) for _ in range(2)]
            for t in single:
                t.tensor.fill_(3.0)   # the padding too, as the batch outputs
            prog.apply(d, single, (0, 0, 0), n, (h, h, h), [2.0])
            torch.cuda.synchronize()
            for a, b in zip(o, single):
                assert torch.equal(a.tensor, b.tensor)
            del single
    if oracle:
        rng = np.random.default_rng(5)
        for (f, d, o, n) in ms:
            i0 = int(rng.integers(0, max(1, n[0] - 8)))
            j0 = int(rng.integers(0, max(1, n[1] - 8)))
            lb, ub = (i0, j0, 0), (min(n[0], i0 + 8), min(n[1], j0 + 8), n[2])
            G = {k: S.Grid.storage(v, h) for k, v in f.items()}
            ru, rv = S.hdiff_vadvc(G["u"], G["v"], G["w"], G["coeff"], lb, ub, 2.0)
            gu = o[0].interior(lb, ub).cpu().numpy().astype(np.float64)
            gv = o[1].interior(lb, ub).cpu().numpy().astype(np.float64)
            assert max(rel_err(gu, ru), rel_err(gv, rv)) <= TOL["f32"]


@pytest.mark.parametrize("arith", [1, 0])
@pytest.mark.parametrize("unroll,k_chunk", [(1, 4), (2, 0), (1, 20), (2, 3)])
def test_persistent_staged_batch_equals_single_applies(arith, unroll, k_chunk):
    """FP32 staged batch on the warp-row producer: one persistent launch over
    producer items (row blocks) and column-sweep items (64 columns) of every
    member, the sweeps waiting on row-block counters. Members with partial row
    blocks, partial column groups, one- and two-level columns: member by
    member the bits of the single applies (graph and direct), sampled blocks
    within the oracle tolerance, no bounded wait given up."""
    from paper_2005_13014_gb300 import _lib as L
    from paper_2005_13014_gb300.api import Batch, Program
    h = 3
    prog = Program(programs.HDIFF_VADVC, "f32")
    prog.set_schedule(fusion=1, staging=3, tile_i=32, tile_j=4 * unroll, unroll=unroll, k_chunk=k_chunk, arith=arith)
    ms = _aligned_members(ALIGNED_SHAPES, seed=400)
    batch = Batch(prog, [(d, o, (0, 0, 0), n, (h, h, h)) for (_, d, o, n) in ms], [2.0])
    rows = 4 * unroll
    prod = sum(-(-n[0] // 128) * -(-n[1] // rows) * 2 * -(-n[2] // (k_chunk if 0 < k_chunk <= n[2] else n[2]))
               for n in ALIGNED_SHAPES)
    sweeps = sum(-(-(n[0] * n[1]) // 64) for n in ALIGNED_SHAPES)
    assert batch.n_items == prod + sweeps   # the persistent form
    assert 1 <= batch.n_ctas <= batch.n_items
    _check_members_against_single(prog, batch, ms, h)
    assert L.lib().oec_device_status(None) == 0


def test_persistent_staged_batch_l2_sweep_and_unaligned_fallback():
    """Members with more than 48 MB of column scratch make the persistent
    kernel's sweep take its L2 form (same bits as the single applies' plain
    sweep). Members with rows not 16-byte aligned make the batch fall back to
    the per-member graph branches (one item per member)."""
    from paper_2005_13014_gb300.api import Batch, Program
    h = 3
    prog = Program(programs.HDIFF_VADVC, "f32")
    prog.set_schedule(fusion=1, staging=3, tile_i=32, tile_j=4, unroll=1, k_chunk=20, arith=1)
    shapes = [(1000, 300, 23), (516, 332, 37), (36, 23, 11)]
    ms = _aligned_members(shapes, seed=500)
    batch = Batch(prog, [(d, o, (0, 0, 0), n, (h, h, h)) for (_, d, o, n) in ms], [2.0])
    assert batch.n_items > len(shapes)
    _check_members_against_single(prog, batch, ms, h)
    del batch, ms
    un = _members("f32", h, shapes=[(37, 23, 11), (64, 8, 3)], seed=600)   # ni = 37: rows not aligned
    b2 = Batch(prog, [(d, o, (0, 0, 0), n, (h, h, h)) for (_, d, o, n) in un], [2.0])
    assert b2.n_items == 2
