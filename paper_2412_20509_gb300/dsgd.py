"""Sharded sweeps of Algorithm 1 over several ranks (one GPU and one handle each).

Within one sweep the blocks (I_{(sigma_w + k) mod r}, J_k), k < s, touch
disjoint row chunks and disjoint column chunks (Sec. 3.2: the block
estimators of eq. 15 and the local steps of eq. 14 of different blocks of a
sweep read and write disjoint parameters), so they commute and can run on
different ranks. The plan (r >= s; with r < s rows and columns swap roles):

* rank g owns the column chunks k with k mod P == g and runs block k of every
  sweep: a column chunk's factors, smoothed derivatives and visit counts never
  leave their owner during an epoch (the fixed side);
* the row chunk of each block changes from sweep to sweep (the moving side):
  after sweep w every rank sends the row chunks its blocks updated, and every
  rank receives all of them (one all-gather per sweep), so that the next
  sweep's owner of each block holds its row chunk's current state;
* after the last sweep of an epoch the column chunks are all-gathered as well,
  so every rank holds the whole model (deviance, checkpoints, Algorithm 2).

t advances by the whole sweep on every rank and each block keeps its place in
the sweep's step sequence, so every rank ends each epoch with the parameters
of the single-handle fit, bit for bit. A fixed NB shape or Poisson is needed:
the pooled shape update of App. B sums moment statistics over all blocks of a
sweep.

The engine is anything with ``sweep_blocks(sigma, w, blocks)``,
``chunk_floats(side, c)``, ``get_chunk(side, c, out)`` and
``set_chunk(side, c, buf)`` (``paper_2412_20509_gb300.Model``: device buffers,
the collectives on NCCL). Side 0 = row chunks, side 1 = column chunks.
"""
from __future__ import annotations

__all__ = ["blocks_of_rank", "moving_chunk", "sides", "ShardedFit", "run_local_shards"]


def blocks_of_rank(per: int, world: int, rank: int) -> list[int]:
    """The blocks k of every sweep that rank `rank` of `world` runs: k mod world == rank."""
    return [k for k in range(per) if k % world == rank]


def sides(r: int, s: int) -> tuple[int, int]:
    """(fixed side, moving side): (1, 0) when r >= s (column chunks stay, row chunks move), else (0, 1)."""
    return (1, 0) if r >= s else (0, 1)


def moving_chunk(sigma_w: int, k: int, r: int, s: int) -> int:
    """The moving-side chunk of block k in a sweep with offset sigma_w (Algorithm 1's schedule)."""
    return (int(sigma_w) + k) % (r if r >= s else s)


def _chunk_counts(n: int, m: int, nb_row: int, nb_col: int) -> tuple[int, int]:
    return -(-n // nb_row), -(-m // nb_col)


class ShardedFit:
    """One rank's share of a sharded fit, with torch.distributed collectives
    (NCCL for CUDA engines, gloo for CPU engines).

    engine: this rank's handle (it holds the whole count matrix and a replica of
    every parameter; only its own blocks are computed on it). dims: (n, m,
    nb_row, nb_col). device: where the exchange buffers live. group: a
    torch.distributed process group (None = the default group)."""

    def __init__(self, engine, dims, device, dtype=None, group=None):
        import torch
        import torch.distributed as dist
        self.torch, self.dist = torch, dist
        self.engine = engine
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        n, m, nb_row, nb_col = dims
        self.r, self.s = _chunk_counts(n, m, nb_row, nb_col)
        self.per = min(self.r, self.s)
        self.nsw = max(self.r, self.s)
        self.fixed, self.moving = sides(self.r, self.s)
        self.device = device
        self.dtype = dtype or torch.float32
        nmov = self.r if self.moving == 0 else self.s
        nfix = self.s if self.moving == 0 else self.r
        self.mov_floats = max(engine.chunk_floats(self.moving, c) for c in range(nmov))
        self.fix_floats = max(engine.chunk_floats(self.fixed, c) for c in range(nfix))
        self.nfix = nfix
        self.slots = -(-self.per // self.world)   # blocks of the busiest rank per sweep

    def _all_gather(self, send):
        out = self.torch.empty((self.world,) + tuple(send.shape), dtype=send.dtype, device=send.device)
        if hasattr(self.dist, "all_gather_into_tensor") and send.device.type == "cuda":
            self.dist.all_gather_into_tensor(out, send, group=self.group)
        else:
            self.dist.all_gather(list(out.unbind(0)), send, group=self.group)
        return out

    def sweep(self, sigma, w):
        """Run this rank's blocks of sweep w, then exchange the moving chunks they updated."""
        mine = blocks_of_rank(self.per, self.world, self.rank)
        self.engine.sweep_blocks(sigma, w, mine)
        send = self.torch.zeros((self.slots, self.mov_floats), dtype=self.dtype, device=self.device)
        for i, k in enumerate(mine):
            c = moving_chunk(sigma[w], k, self.r, self.s)
            self.engine.get_chunk(self.moving, c, send[i, :self.engine.chunk_floats(self.moving, c)])
        got = self._all_gather(send)
        for g in range(self.world):
            if g == self.rank:
                continue
            for i, k in enumerate(blocks_of_rank(self.per, self.world, g)):
                c = moving_chunk(sigma[w], k, self.r, self.s)
                self.engine.set_chunk(self.moving, c, got[g, i, :self.engine.chunk_floats(self.moving, c)])

    def gather_fixed(self):
        """Every rank receives every fixed-side chunk (end of an epoch)."""
        owned = [c for c in range(self.nfix) if c % self.world == self.rank]
        slots = -(-self.nfix // self.world)
        send = self.torch.zeros((slots, self.fix_floats), dtype=self.dtype, device=self.device)
        for i, c in enumerate(owned):
            self.engine.get_chunk(self.fixed, c, send[i, :self.engine.chunk_floats(self.fixed, c)])
        got = self._all_gather(send)
        for g in range(self.world):
            if g == self.rank:
                continue
            for i, c in enumerate(c2 for c2 in range(self.nfix) if c2 % self.world == g):
                self.engine.set_chunk(self.fixed, c, got[g, i, :self.engine.chunk_floats(self.fixed, c)])

    def epoch(self, sigma):
        """One epoch of Algorithm 1, sharded; afterwards every rank holds the whole model."""
        for w in range(self.nsw):
            self.sweep(sigma, w)
        self.gather_fixed()


def run_local_shards(engines, dims, sigma, make_buffer):
    """The same plan for P engines driven from one process, one after the other
    (P shards on one device, no collective): the exchange is a copy through a
    buffer from make_buffer(floats). After the epoch every engine holds the
    whole model."""
    n, m, nb_row, nb_col = dims
    r, s = _chunk_counts(n, m, nb_row, nb_col)
    per, nsw = min(r, s), max(r, s)
    fixed, moving = sides(r, s)
    P = len(engines)
    nfix = s if moving == 0 else r
    for w in range(nsw):
        for g, e in enumerate(engines):
            e.sweep_blocks(sigma, w, blocks_of_rank(per, P, g))
        for g, e in enumerate(engines):
            for k in blocks_of_rank(per, P, g):
                c = moving_chunk(sigma[w], k, r, s)
                buf = make_buffer(e.chunk_floats(moving, c))
                e.get_chunk(moving, c, buf)
                for h, other in enumerate(engines):
                    if h != g:
                        other.set_chunk(moving, c, buf)
    for c in range(nfix):
        g = c % P
        buf = make_buffer(engines[g].chunk_floats(fixed, c))
        engines[g].get_chunk(fixed, c, buf)
        for h, other in enumerate(engines):
            if h != g:
                other.set_chunk(fixed, c, buf)
