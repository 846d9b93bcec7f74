"""Domain decomposition of a stencil program over ranks, with halo exchange.

The paper runs one GPU (§VII); a program's domain splits naturally into
i/j blocks, one per rank, because every stage reads its inputs at constant
offsets. Columns are never split along k (the vertical Thomas solve of
hdiff+vadvc runs down whole columns). Before each application a rank needs,
around its block, the halo that shape inference gives for the program's
inputs (paper §V-B): i/j halo 2 for hdiff, and w's extra column at i+1 for
hdiff+vadvc. This module holds the bookkeeping:

  split(n, parts)            balanced 1-D partition of [0, n)
  Decomposition(...)         the px x py grid of blocks, each rank's block and
                             neighbours, and the boxes of one halo exchange
  exchange(storage, ...)     one halo exchange of a rank's field storage over
                             torch.distributed (gloo or NCCL point-to-point):
                             i-direction first, then j-direction with the
                             i-halo columns included, so the corner cells
                             arrive too (kernels that stage a whole window read
                             them)

The domain's own outer halo (beyond the global domain) is the caller's, as
for a single apply. Host logic only: nothing here computes the stencils.
"""

from __future__ import annotations

from dataclasses import dataclass


def split(n: int, parts: int):
    """[start, stop) ranges of a balanced partition of [0, n) into parts
    pieces (the first n % parts pieces one longer)."""
    if parts < 1 or n < parts:
        raise ValueError(f"cannot split {n} points into {parts} non-empty parts")
    q, r = divmod(n, parts)
    out, s = [], 0
    for x in range(parts):
        e = s + q + (1 if x < r else 0)
        out.append((s, e))
        s = e
    return out


@dataclass(frozen=True)
class Block:
    rank: int
    pi: int          # position in the rank grid along i
    pj: int          # and along j
    i: tuple         # [i0, i1) in global logical coordinates
    j: tuple         # [j0, j1)

    @property
    def shape(self):
        return (self.i[1] - self.i[0], self.j[1] - self.j[0])


class Decomposition:
    """A px x py grid of ranks over the global domain (ni, nj, nk); rank r sits
    at (r % px, r // px). halo = (hi, hj): the cells a rank's storage holds
    around its block (at least the program's inferred input halo)."""

    def __init__(self, n, px, py, halo):
        self.n = tuple(n)
        self.px, self.py = px, py
        self.halo = tuple(halo)
        self.si = split(n[0], px)
        self.sj = split(n[1], py)
        hi, hj = self.halo
        if min(b - a for a, b in self.si) < hi or min(b - a for a, b in self.sj) < hj:
            raise ValueError("every block must be at least as wide as the halo it sends")

    @property
    def size(self):
        return self.px * self.py

    def block(self, rank) -> Block:
        pi, pj = rank % self.px, rank // self.px
        return Block(rank, pi, pj, self.si[pi], self.sj[pj])

    def neighbour(self, rank, di, dj):
        """The rank at offset (di, dj) in the grid, or None at the domain edge."""
        b = self.block(rank)
        qi, qj = b.pi + di, b.pj + dj
        if 0 <= qi < self.px and 0 <= qj < self.py:
            return qj * self.px + qi
        return None

    def exchange_plan(self, rank):
        """The two phases of one halo exchange of this rank, as lists of
        (peer, send_box, recv_box) with boxes in the rank's local storage
        coordinates ((i0, i1), (j0, j1)); storage index = logical index of
        the block + halo. Phase 1 moves i-halos over every row of the storage
        (the rows of the domain's own outer j-halo included: a neighbour's
        cells there sit next to this block); phase 2 j-halos over every
        column, the i-halos received in phase 1 included (the corners)."""
        b = self.block(rank)
        hi, hj = self.halo
        ni, nj = b.shape
        plan1, plan2 = [], []
        rows = (0, nj + 2 * hj)
        for di, send_i, recv_i in ((-1, (hi, 2 * hi), (0, hi)), (1, (ni, ni + hi), (ni + hi, ni + 2 * hi))):
            peer = self.neighbour(rank, di, 0)
            if peer is not None:
                plan1.append((peer, (send_i, rows), (recv_i, rows)))
        cols = (0, ni + 2 * hi)
        for dj, send_j, recv_j in ((-1, (hj, 2 * hj), (0, hj)), (1, (nj, nj + hj), (nj + hj, nj + 2 * hj))):
            peer = self.neighbour(rank, 0, dj)
            if peer is not None:
                plan2.append((peer, (cols, send_j), (cols, recv_j)))
        return plan1, plan2


def exchange(storage, dec: Decomposition, rank, group=None):
    """One halo exchange of a rank's field storage (a torch tensor indexed
    [k, j, i] holding the block plus dec.halo cells on each i/j side; k
    unsplit) with its grid neighbours, in place. Every rank of the grid calls
    it; sends and receives are paired by (phase, direction) tags."""
    import torch
    import torch.distributed as dist
    for phase, plan in enumerate(dec.exchange_plan(rank)):
        reqs, recvs = [], []
        for peer, (si, sj), (ri, rj) in plan:
            # the direction of the move, seen from the receiver, makes the tag
            d = (1 if si[0] < ri[0] else -1) if phase == 0 else (1 if sj[0] < rj[0] else -1)
            send = storage[:, sj[0]:sj[1], si[0]:si[1]].contiguous()
            buf = torch.empty_like(storage[:, rj[0]:rj[1], ri[0]:ri[1]].contiguous())
            reqs.append(dist.isend(send, peer, group=group, tag=10 * phase + (1 if d > 0 else 2)))
            reqs.append(dist.irecv(buf, peer, group=group, tag=10 * phase + (2 if d > 0 else 1)))
            recvs.append((buf, ri, rj))
        for r in reqs:
            r.wait()
        for buf, ri, rj in recvs:
            storage[:, rj[0]:rj[1], ri[0]:ri[1]] = buf
