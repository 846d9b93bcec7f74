"""The ticket order of the persistent staged launches (one FP32 domain, and
an ensemble batch), read on the host through oec_pstaged_ticket_order and
oec_batch_ticket_order (no GPU).

The launch's CTAs take tickets from an atomic counter; a column-sweep item
waits, with a bounded wait, until every producer item of the row blocks its
columns lie in has finished, and producer items never wait. The launch can
only stall if some sweep item's ticket came before a producer item it waits
for: a CTA holding that sweep item could then be waiting on an item that no
running CTA has taken yet. These tests check, over many domain shapes, level
chunks, rows per warp and resident-CTA counts, that the order the kernel
decodes holds every item exactly once and puts each sweep item after all of
its producers. The expected item sets are built here from the launch's
definition (tiles of 128 columns along i, row blocks of 4 x unroll rows, two
fields, level chunks, 64-column groups), not from the library's decoder."""

import ctypes as C

import numpy as np
import pytest

from paper_2005_13014_gb300 import _lib as L


def _order(ni, nj, nk, unroll, k_chunk, grid):
    lib = L.lib()
    n = C.c_int64(0)
    rc = lib.oec_pstaged_ticket_order(ni, nj, nk, unroll, k_chunk, grid, None, 0, C.byref(n))
    assert rc == 0, lib.oec_last_error()
    buf = np.zeros(4 * n.value, np.int32)
    rc = lib.oec_pstaged_ticket_order(ni, nj, nk, unroll, k_chunk, grid,
                                      buf.ctypes.data_as(C.POINTER(C.c_int32)), buf.size, C.byref(n))
    assert rc == 0, lib.oec_last_error()
    return buf.reshape(-1, 4)


def _check(ni, nj, nk, unroll, k_chunk, grid):
    items = _order(ni, nj, nk, unroll, k_chunk, grid)
    rows = 4 * unroll
    tiles_i = -(-ni // 128)
    blocks = -(-nj // rows)
    kc = nk if k_chunk <= 0 or k_chunk > nk else k_chunk
    chunks = -(-nk // kc)
    ncol = ni * nj
    groups = -(-ncol // 64)
    per_block = tiles_i * 2 * chunks
    assert len(items) == blocks * per_block + groups
    x, y, z, w = items.T
    tick = np.arange(len(items))
    prod, grp = x == 0, x == -1
    assert np.all(prod | grp)
    # every producer item (tile along i, row block, chunk and field) once
    key = (z[prod].astype(np.int64) * tiles_i + y[prod]) * (2 * chunks) + w[prod]
    assert np.all((y[prod] >= 0) & (y[prod] < tiles_i) & (z[prod] >= 0) & (z[prod] < blocks))
    assert np.all((w[prod] >= 0) & (w[prod] < 2 * chunks))
    assert np.array_equal(np.sort(key), np.arange(blocks * per_block))
    # every column group once, waiting on the row blocks of its first and last column
    gy = y[grp].astype(np.int64)
    assert np.array_equal(np.sort(gy), np.arange(groups))
    first = 64 * gy
    last = np.minimum(first + 63, ncol - 1)
    assert np.array_equal(z[grp], (first // ni) // rows)
    assert np.array_equal(w[grp], (last // ni) // rows)
    # each group after the last producer item of every row block it waits on
    last_prod = np.full(blocks, -1, np.int64)
    np.maximum.at(last_prod, z[prod], tick[prod])
    gt, gz, gw = tick[grp], z[grp].astype(np.int64), w[grp].astype(np.int64)
    for off in range(int((gw - gz).max()) + 1 if groups else 0):
        b = gz + off
        m = b <= gw
        assert np.all(last_prod[b[m]] < gt[m]), (ni, nj, nk, unroll, k_chunk, grid)
    return items


@pytest.mark.parametrize("n", [(256, 256, 8), (268, 250, 5), (512, 128, 3), (1024, 64, 2), (256, 257, 1),
                               (512, 512, 80), (512, 512, 137)], ids=str)
@pytest.mark.parametrize("unroll,k_chunk", [(1, 4), (2, 0), (1, 20), (2, 3)])
@pytest.mark.parametrize("grid", [1, 456, 608, 100000])
def test_ticket_order_of_the_tested_shapes(n, unroll, k_chunk, grid):
    _check(*n, unroll, k_chunk, grid)


def test_ticket_order_random_shapes():
    rng = np.random.default_rng(20050513)
    for _ in range(300):
        ni = int(rng.integers(1, 1200))
        nj = int(rng.integers(1, 300))
        nk = int(rng.integers(1, 140))
        unroll = int(rng.integers(1, 3))
        k_chunk = int(rng.choice([0, int(rng.integers(1, nk + 4))]))
        grid = int(rng.choice([1, 2, 7, 152, 456, 608, 1 << 20]))
        _check(ni, nj, nk, unroll, k_chunk, grid)


def test_lag_places_groups_behind_their_producers():
    """With many resident CTAs a group's ticket trails its producers by more
    than the CTAs in flight, so its wait usually finds them done; with one
    CTA the order still holds (every wait is for an item already taken)."""
    items = _check(512, 512, 80, 2, 20, 608)
    x, y, z, w = items.T
    tick = np.arange(len(items))
    last_prod = np.full(z.max() + 1, -1)
    np.maximum.at(last_prod, z[x == 0], tick[x == 0])
    g = x == -1
    gap = tick[g] - last_prod[w[g]]
    # all but the groups of the last row blocks trail by at least the grid
    assert np.mean(gap >= 608) > 0.9
    _check(512, 512, 80, 2, 20, 1)


@pytest.mark.parametrize("args", [(0, 8, 8, 1, 0, 10), (8, 0, 8, 1, 0, 10), (8, 8, 0, 1, 0, 10),
                                  (8, 8, 8, 3, 0, 10), (8, 8, 8, 1, 0, 0)], ids=str)
def test_ticket_order_rejects_bad_arguments(args):
    lib = L.lib()
    n = C.c_int64(-5)
    assert lib.oec_pstaged_ticket_order(*args, None, 0, C.byref(n)) == -1
    assert n.value == -5
    assert lib.oec_last_error()


# ---- the persistent staged batch (a table built on the host) ----------------

def _batch_order(sizes, unroll, k_chunk, lag):
    lib = L.lib()
    flat = np.asarray(sizes, np.int32).reshape(-1)
    sp = flat.ctypes.data_as(C.POINTER(C.c_int32))
    n = C.c_int64(0)
    assert lib.oec_batch_ticket_order(len(sizes), sp, unroll, k_chunk, lag, None, 0, C.byref(n)) == 0
    buf = np.zeros(4 * n.value, np.int32)
    rc = lib.oec_batch_ticket_order(len(sizes), sp, unroll, k_chunk, lag,
                                    buf.ctypes.data_as(C.POINTER(C.c_int32)), buf.size, C.byref(n))
    assert rc == 0, lib.oec_last_error()
    return buf.reshape(-1, 4)


def _check_batch(sizes, unroll, k_chunk, lag):
    items = _batch_order(sizes, unroll, k_chunk, lag)
    x, y, z, w = items.T
    tick = np.arange(len(items))
    rows = 4 * unroll
    total = 0
    for m, (ni, nj, nk) in enumerate(sizes):
        tiles_i, blocks = -(-ni // 128), -(-nj // rows)
        kc = nk if k_chunk <= 0 or k_chunk > nk else k_chunk
        chunks = -(-nk // kc)
        ncol = ni * nj
        groups = -(-ncol // 64)
        prod, grp = x == m, x == -1 - m
        key = (z[prod].astype(np.int64) * tiles_i + y[prod]) * (2 * chunks) + w[prod]
        assert np.array_equal(np.sort(key), np.arange(blocks * tiles_i * 2 * chunks)), m
        gy = y[grp].astype(np.int64)
        assert np.array_equal(np.sort(gy), np.arange(groups)), m
        first = 64 * gy
        last = np.minimum(first + 63, ncol - 1)
        assert np.array_equal(z[grp], (first // ni) // rows)
        assert np.array_equal(w[grp], (last // ni) // rows)
        last_prod = np.full(blocks, -1, np.int64)
        np.maximum.at(last_prod, z[prod], tick[prod])
        gt, gz, gw = tick[grp], z[grp].astype(np.int64), w[grp].astype(np.int64)
        for off in range(int((gw - gz).max()) + 1):
            b = gz + off
            k = b <= gw
            assert np.all(last_prod[b[k]] < gt[k]), (m, sizes, unroll, k_chunk, lag)
        # a group trails its last producer by at least the lag, unless it was
        # placed after the table's last producer item
        trail = gt - last_prod[gw]
        assert np.all((trail >= lag) | (gt > tick[x >= 0].max())), m
        total += blocks * tiles_i * 2 * chunks + groups
    assert len(items) == total


def test_batch_ticket_order_of_the_ensemble():
    """The 32-member ensemble's shapes (i, j from 64 to 512, k from 60 to
    137), at the lag the batch uses for 608 resident CTAs and at others."""
    from paper_2005_13014_gb300 import inputs
    shapes = inputs.ensemble_members()
    for unroll, k_chunk in ((2, 20), (1, 8), (2, 0)):
        for lag in (0, 1216, 10 ** 7):
            _check_batch(shapes, unroll, k_chunk, lag)


def test_batch_ticket_order_random_members():
    rng = np.random.default_rng(1305)
    for _ in range(150):
        n = int(rng.integers(1, 6))
        sizes = [(int(rng.integers(1, 700)), int(rng.integers(1, 200)), int(rng.integers(1, 90))) for _ in range(n)]
        _check_batch(sizes, int(rng.integers(1, 3)), int(rng.choice([0, 1, 3, 20, 200])),
                     int(rng.choice([0, 1, 37, 912, 1 << 40])))


@pytest.mark.parametrize("args", [(0, 1, 0, 10), (1, 3, 0, 10), (1, 1, 0, -1)], ids=str)
def test_batch_ticket_order_rejects_bad_arguments(args):
    lib = L.lib()
    n_members, unroll, k_chunk, lag = args
    sizes = np.array([8, 8, 8], np.int32)
    n = C.c_int64(-5)
    rc = lib.oec_batch_ticket_order(n_members, sizes.ctypes.data_as(C.POINTER(C.c_int32)), unroll, k_chunk, lag,
                                    None, 0, C.byref(n))
    assert rc == -1 and n.value == -5
    bad = np.array([8, 0, 8], np.int32)
    assert lib.oec_batch_ticket_order(1, bad.ctypes.data_as(C.POINTER(C.c_int32)), 1, 0, 10, None, 0,
                                      C.byref(n)) == -1
