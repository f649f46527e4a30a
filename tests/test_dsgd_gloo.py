"""Sharded sweeps (paper_2412_20509_gb300.dsgd) on CPU ranks: world size 2 over
gloo (127.0.0.1), each rank driving the FP64 oracle on its own blocks of every
sweep and exchanging chunk states with all-gathers. The blocks of a sweep are
disjoint (Sec. 3.2), so after every epoch each rank holds the single-rank fit
bit for bit. Also the host plan itself: every block of a sweep runs on exactly
one rank, and the moving chunks of a sweep are distinct."""
import os
import socket

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2412_20509_gb300 import dsgd  # noqa: E402  (host logic only; no library load)

CASES = {
    # name: (n, m, d, family, nb_row, nb_col) -- r >= s (rows move) and r < s (columns move), ragged chunks
    "rows_move": (300, 200, 3, "negbin", 64, 50),
    "cols_move": (150, 410, 2, "poisson", 64, 50),
    "gamma_rows_move": (300, 200, 3, "gamma", 64, 50),   # a family of Table S1 with float32 responses
}


class OracleEngine:
    """The oracle fit as a shard engine: chunk states packed row by row as
    [free parameters | smoothed gradients | smoothed curvatures | visit count] (FP64)."""

    def __init__(self, fit, nb_row, nb_col):
        self.f, self.nb = fit, (nb_row, nb_col)

    def sweep_blocks(self, sigma, w, blocks):
        self.f.sweep_blocks(sigma, w, blocks)

    def _rows(self, side, c):
        perm = self.f.row_perm if side == 0 else self.f.col_perm
        nb = self.nb[side]
        return perm[c * nb:(c + 1) * nb]

    def _arrays(self, side):
        f = self.f
        return ((f.G, f.U, f.Gb_row, f.Hb_row, f.cnt_row) if side == 0 else (f.B, f.V, f.Gb_col, f.Hb_col, f.cnt_col))

    def chunk_floats(self, side, c):
        a, b, g, _, _ = self._arrays(side)
        return len(self._rows(side, c)) * (a.shape[1] + b.shape[1] + 2 * g.shape[1] + 1)

    def get_chunk(self, side, c, out):
        rows = self._rows(side, c)
        a, b, g, h, cnt = self._arrays(side)
        packed = np.hstack([a[rows], b[rows], g[rows], h[rows], cnt[rows, None].astype(np.float64)])
        out.copy_(torch.from_numpy(packed.ravel()))

    def set_chunk(self, side, c, buf):
        rows = self._rows(side, c)
        a, b, g, h, cnt = self._arrays(side)
        x = buf.numpy().reshape(len(rows), -1)
        o = 0
        for arr in (a, b, g, h):
            arr[rows] = x[:, o:o + arr.shape[1]]
            o += arr.shape[1]
        cnt[rows] = x[:, o].astype(np.int64)


def _setup(case, seed=4):
    import oracle
    n, m, d, fam, nbr, nbc = CASES[case]
    if fam in ("poisson", "negbin"):
        prob = synth.make_problem(n, m, 2, 1, d, fam, seed=seed, zero_frac=0.7 if fam == "negbin" else None,
                                  offset=True)
    else:
        prob = synth.make_family_problem(n, m, 2, 1, d, fam, phi=0.3, seed=seed, offset=True, shift=0.5)
    start = synth.crude_start(prob, d, seed=seed)
    rp, cp = synth.partitions(n, m, seed)
    sig = synth.sweep_orders(n, m, nbr, nbc, 2, seed)
    fit = oracle.OracleFit(prob.Y, prob.X, prob.Z, prob.offset, start, family=fam, nb_row=nbr, nb_col=nbc,
                           row_perm=rp, col_perm=cp, settings=synth.fit_settings())
    return fit, sig, (n, m, nbr, nbc)


def _state(fit):
    return {k: np.array(getattr(fit, k)) for k in ("B", "G", "U", "V", "Gb_row", "Hb_row", "Gb_col", "Hb_col",
                                                   "cnt_row", "cnt_col", "alpha", "t")}


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, case, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        fit, sig, dims = _setup(case)
        shard = dsgd.ShardedFit(OracleEngine(fit, dims[2], dims[3]), dims, device="cpu", dtype=torch.float64)
        for s in sig:
            shard.epoch(s)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), **_state(fit))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("case", list(CASES))
def test_two_gloo_ranks_equal_the_single_rank_fit_bitwise(case, tmp_path, oracle_lib):
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, case, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    ref, sig, _ = _setup(case)
    for s in sig:
        ref.epoch(s)
    want = _state(ref)
    for rank in range(2):
        got = np.load(tmp_path / f"rank{rank}.npz")
        for k, v in want.items():
            np.testing.assert_array_equal(got[k], v, err_msg=f"rank {rank}: {k}")


@pytest.mark.parametrize("per,world", [(5, 2), (4, 4), (3, 5), (98, 3)])
def test_every_block_runs_on_exactly_one_rank(per, world):
    runs = sorted(k for g in range(world) for k in dsgd.blocks_of_rank(per, world, g))
    assert runs == list(range(per))


@pytest.mark.parametrize("r,s", [(98, 5), (5, 98), (7, 7), (3, 1)])
def test_moving_chunks_of_a_sweep_are_distinct(r, s):
    per, nsw = min(r, s), max(r, s)
    sigma = np.random.default_rng(r * s).permutation(nsw)
    fixed, moving = dsgd.sides(r, s)
    assert (fixed, moving) == ((1, 0) if r >= s else (0, 1))
    for w in range(nsw):
        ch = [dsgd.moving_chunk(sigma[w], k, r, s) for k in range(per)]
        assert len(set(ch)) == per and all(0 <= c < nsw for c in ch)


def test_partial_sweeps_equal_the_whole_sweep(oracle_lib):
    """The oracle's block-subset sweep: the blocks of a sweep run in two calls
    (in either order) equal the whole sweep bit for bit, and t advances by one
    sweep per call (Sec. 3.2: a sweep's blocks touch disjoint chunks)."""
    a, sig, dims = _setup("rows_move")
    b, _, _ = _setup("rows_move")
    c, _, _ = _setup("rows_move")
    a.sweeps(sig[0], 0, 3)
    t0 = int(b.t[0])
    for w in range(3):
        b.sweep_blocks(sig[0], w, [0, 2])
        b.t[0] -= 4          # the second call of the same sweep starts from the same t
        b.sweep_blocks(sig[0], w, [1, 3])
        c.sweep_blocks(sig[0], w, [1, 3])
        c.t[0] -= 4
        c.sweep_blocks(sig[0], w, [0, 2])
    assert int(b.t[0]) == t0 + 12
    for other in (b, c):
        for k, v in _state(a).items():
            np.testing.assert_array_equal(_state(other)[k], v, err_msg=k)
