"""i/j domain decomposition with halo exchange (host logic of a multi-GPU
run), on the CPU: the partition and exchange boxes by construction, and
world_size 2 and 4 gloo process groups that exchange the halos of their
blocks of seeded fields. After one exchange every rank's storage equals the
global field over its block and halo, and the FP64 oracle applied to each
block alone gives, bit for bit, the oracle's result on the whole domain."""

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2005_13014_gb300 import decomp as D  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_split_is_balanced_and_covers():
    for n, p in ((128, 2), (128, 3), (37, 4), (5, 5)):
        s = D.split(n, p)
        assert s[0][0] == 0 and s[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(s, s[1:]))
        sizes = [b - a for a, b in s]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.split(3, 4)


def test_exchange_plan_boxes():
    dec = D.Decomposition((40, 30, 6), 2, 2, (3, 3))
    assert dec.block(3).i == (20, 40) and dec.block(3).j == (15, 30)
    assert dec.neighbour(0, 1, 0) == 1 and dec.neighbour(0, 0, 1) == 2 and dec.neighbour(0, -1, 0) is None
    p1, p2 = dec.exchange_plan(0)          # block 20 x 15 at the lower-left corner
    assert p1 == [(1, ((20, 23), (0, 21)), ((23, 26), (0, 21)))]
    assert p2 == [(2, ((0, 26), (15, 18)), ((0, 26), (18, 21)))]
    p1, p2 = dec.exchange_plan(3)
    assert p1 == [(2, ((3, 6), (0, 21)), ((0, 3), (0, 21)))]
    assert p2 == [(1, ((0, 26), (3, 6)), ((0, 26), (0, 3)))]
    with pytest.raises(ValueError):
        D.Decomposition((8, 8, 2), 4, 1, (3, 3))   # blocks of 2 columns cannot send a halo of 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, px, py, port, out):
    import sys
    sys.path.insert(0, ROOT)
    from oracle import stencils as S
    from paper_2005_13014_gb300 import decomp, inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        n, h = (37, 26, 7), 3
        f = inputs.hdiff_vadvc_fields(*n, h, seed=91)
        dec = decomp.Decomposition(n, px, py, (h, h))
        b = dec.block(rank)
        (i0, i1), (j0, j1) = b.i, b.j
        local = {}
        for k, g in f.items():
            # the block and its halo from the global storage; halo cells that a
            # neighbour owns start as NaN, the domain's own outer halo is the caller's
            t = torch.from_numpy(np.ascontiguousarray(g[:, j0:j1 + 2 * h, i0:i1 + 2 * h])).clone()
            if b.pi > 0:
                t[:, :, :h] = float("nan")
            if b.pi < px - 1:
                t[:, :, -h:] = float("nan")
            if b.pj > 0:
                t[:, :h, :] = float("nan")
            if b.pj < py - 1:
                t[:, -h:, :] = float("nan")
            decomp.exchange(t, dec, rank)
            local[k] = t.numpy()
        same = all(np.array_equal(local[k], f[k][:, j0:j1 + 2 * h, i0:i1 + 2 * h]) for k in f)
        G = {k: S.Grid.storage(v, h) for k, v in local.items()}
        nb = (i1 - i0, j1 - j0, n[2])
        u, v = S.hdiff_vadvc(G["u"], G["v"], G["w"], G["coeff"], (0, 0, 0), nb, 2.0)
        GG = {k: S.Grid.storage(v_, h) for k, v_ in f.items()}
        ru, rv = S.hdiff_vadvc(GG["u"], GG["v"], GG["w"], GG["coeff"], (0, 0, 0), n, 2.0)
        bits = np.array_equal(u, ru[:, j0:j1, i0:i1]) and np.array_equal(v, rv[:, j0:j1, i0:i1])
        out.put((rank, same, bits))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("px,py", [(2, 1), (1, 2), (2, 2)])
def test_blocks_after_halo_exchange_reproduce_the_whole_domain(px, py):
    ws, port = px * py, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, px, py, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(out.get(timeout=5) for _ in range(ws))
    assert [r for r, _, _ in res] == list(range(ws))
    for rank, same, bits in res:
        assert same, f"rank {rank}: halo cells differ from the global field"
        assert bits, f"rank {rank}: block result differs from the whole-domain oracle"
