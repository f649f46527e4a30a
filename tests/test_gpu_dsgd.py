"""Sharded sweeps on the GPU through the C ABI (gmf_sgd_sweep_blocks,
gmf_chunk_state): P handles on one device, each running its blocks of every
sweep, with the moving chunks copied between handles after each sweep and the
fixed chunks after each epoch (P shards driven one after the other from one
process; a multi-rank run over NCCL follows the same plan). Every handle ends
each epoch with the single-handle fit bit for bit: the same kernels compute the
same blocks from the same inputs, only fewer of them per launch."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gmf():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_20509_gb300 as g
    return g


CASES = {
    # name: (n, m, p, q, d, family, nb_row, nb_col, y_dtype, precision, flags, shards)
    "fp32_rows_move": (1100, 700, 3, 1, 6, "negbin", 300, 160, "int32", "fp32", 0, 2),
    "fp32_cols_move_3_shards": (300, 1000, 2, 2, 3, "poisson", 100, 96, "int32", "fp32", 0, 3),
    "mixed_cluster": (2000, 1024, 2, 1, 10, "negbin", 500, 256, "uint16", "mixed", 0, 2),
    "mixed_separate_atlas_shape": (4300, 2104, 3, 1, 20, "negbin", 2048, 1024, "uint16", "mixed", 0, 2),
}


def _models(gmf, case, count):
    n, m, p, q, d, fam, nbr, nbc, ydt, prec, flags, _ = CASES[case]
    prob = synth.make_problem(n, m, p, q, d, fam, seed=6, y_dtype=ydt, zero_frac=0.8 if fam == "negbin" else None,
                              offset=True)
    start = synth.crude_start(prob, d, seed=6)
    rp, cp = synth.partitions(n, m, 6)
    Y = torch.from_numpy(prob.Y.view(np.int16) if ydt == "uint16" else prob.Y).cuda()
    kw = dict(family=fam, nb_row=nbr, nb_col=nbc, row_perm=rp, col_perm=cp, settings=synth.fit_settings(),
              precision=prec, flags=flags)
    models = [gmf.Model(Y, prob.X, prob.Z, prob.offset, start, **kw) for _ in range(count)]
    return models, synth.sweep_orders(n, m, nbr, nbc, 2, 6), (n, m, nbr, nbc)


@pytest.mark.parametrize("case", list(CASES))
def test_local_shards_equal_the_single_handle_fit(gmf, case):
    from paper_2412_20509_gb300 import dsgd
    P = CASES[case][-1]
    models, sig, dims = _models(gmf, case, P + 1)
    ref, shards = models[0], models[1:]
    buf = lambda floats: torch.empty(floats, dtype=torch.float32, device="cuda")
    for s in sig:
        ref.epoch(s)
        dsgd.run_local_shards(shards, dims, s, buf)
        want = ref.get_params()
        wema = ref.get_ema()
        for g, mdl in enumerate(shards):
            got, ema = mdl.get_params(), mdl.get_ema()
            for k in ("U", "V", "B", "Gamma"):
                np.testing.assert_array_equal(got[k], want[k], err_msg=f"shard {g} {k}")
            for k in ("Gb_row", "Hb_row", "Gb_col", "Hb_col", "cnt_row", "cnt_col", "t"):
                np.testing.assert_array_equal(ema[k], wema[k], err_msg=f"shard {g} {k}")
    assert shards[0].deviance() == ref.deviance()


def test_sharded_fit_on_a_one_rank_nccl_group(gmf, tmp_path):
    """ShardedFit's collective path with CUDA buffers (all_gather_into_tensor on
    NCCL) on a group of one rank: the plan degenerates to the whole sweep, and
    the fit equals gmf_sgd_epoch's bit for bit."""
    import torch.distributed as dist
    from paper_2412_20509_gb300 import dsgd
    if not dist.is_nccl_available():
        pytest.skip("torch without NCCL")
    dist.init_process_group("nccl", init_method=f"file://{tmp_path}/rdzv", rank=0, world_size=1)
    try:
        models, sig, dims = _models(gmf, "fp32_rows_move", 2)
        shard = dsgd.ShardedFit(models[1], dims, device="cuda")
        for s in sig:
            models[0].epoch(s)
            shard.epoch(s)
        a, b = models[0].get_params(), models[1].get_params()
        for k in ("U", "V", "B", "Gamma"):
            np.testing.assert_array_equal(a[k], b[k])
    finally:
        dist.destroy_process_group()


def test_sweep_blocks_rejects_bad_lists(gmf):
    models, sig, dims = _models(gmf, "fp32_rows_move", 1)
    m = models[0]
    for bad in ([3, 1], [0, 0], [-1], [9]):
        with pytest.raises(gmf.GmfError) as e:
            m.sweep_blocks(sig[0], 0, bad) if bad != [3, 1] else gmf.check(
                gmf.lib().gmf_sgd_sweep_blocks(m._h, np.ascontiguousarray(sig[0], dtype=np.int32).ctypes.data, 0,
                                               np.array(bad, np.int32).ctypes.data, len(bad), None))
        assert e.value.code == gmf.GMF_ERR_ARG
    assert m.chunk_floats(0, 0) == 300 * (m_kp(m) + 2 * (1 + 6) + 1)


def m_kp(model):
    n, m, p, q, d = model.dims
    return (1 + p + q + d + 3) // 4 * 4
