"""Batched rank sweep: every model of a gmf_sweep advances exactly as the same
model fitted alone (same kernels, same arithmetic, deterministic reductions),
so the comparison is bitwise; one model is also checked against the oracle."""
import numpy as np
import pytest

import synth
from tests.test_gpu_parity import rel

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


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_sweep_equals_independent_fits(gmf, precision):
    n, m, nbr, nbc = 900, 640, 300, 256
    d_list = [2, 12, 5, 30]
    prob = synth.make_problem(n, m, 3, 1, 8, "negbin", seed=9, y_dtype="uint16", zero_frac=0.85, offset=True)
    starts = [synth.crude_start(prob, d, seed=9 + d) for d in d_list]
    rp, cp = synth.partitions(n, m, 9)
    st = synth.fit_settings(alpha_mode=1)
    sig = synth.sweep_orders(n, m, nbr, nbc, 3, 9)
    kw = dict(family="negbin", nb_row=nbr, nb_col=nbc, row_perm=rp, col_perm=cp, settings=st, precision=precision)
    sw = gmf.Sweep(prob.Y, prob.X, prob.Z, prob.offset, starts, d_list, **kw)
    solo = [gmf.Model(prob.Y, prob.X, prob.Z, prob.offset, s0, **kw) for s0 in starts]
    for e in range(3):
        sw.epoch(sig[e])
        for mdl in solo:
            mdl.epoch(sig[e])
    for i in range(len(d_list)):
        a, b = sw.models[i].get_params(), solo[i].get_params()
        for k in ("U", "V", "B", "Gamma"):
            np.testing.assert_array_equal(a[k], b[k])
        assert a["alpha"] == b["alpha"]
        assert sw.models[i].deviance() == solo[i].deviance()


def test_sweep_model_matches_oracle(gmf):
    import oracle
    n, m, nbr, nbc = 700, 480, 256, 128
    d_list = [3, 7]
    prob = synth.make_problem(n, m, 2, 1, 5, "poisson", seed=4, offset=True)
    starts = [synth.crude_start(prob, d, seed=4) for d in d_list]
    rp, cp = synth.partitions(n, m, 4)
    st = synth.fit_settings()
    sig = synth.sweep_orders(n, m, nbr, nbc, 4, 4)
    sw = gmf.Sweep(torch.from_numpy(prob.Y).cuda(), prob.X, prob.Z, prob.offset, starts, d_list, family="poisson",
                   nb_row=nbr, nb_col=nbc, row_perm=rp, col_perm=cp, settings=st)
    ref = oracle.OracleFit(prob.Y, prob.X, prob.Z, prob.offset, starts[1], family="poisson", nb_row=nbr, nb_col=nbc,
                           row_perm=rp, col_perm=cp, settings=st)
    for e in range(4):
        sw.epoch(sig[e])
        ref.epoch(sig[e])
    assert sw.models[1].deviance() == pytest.approx(ref.deviance(), rel=1e-4)
    assert rel(sw.models[1].get_params()["U"], ref.U) <= 1e-3


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_sweep_groupings_and_autotune_give_the_same_fits(gmf, precision):
    """Every launch grouping of the models (all in one launch, groups of 2, one
    per launch, a ragged split 3 + 1, and each model's own epoch in turn) gives
    the same fits bit for bit; the
    autotuner times the groupings from saved state, restores it (an autotuned
    sweep then equals one that never ran the trials) and keeps a valid size."""
    n, m, nbr, nbc = 900, 640, 300, 256
    d_list = [2, 12, 5, 30]
    prob = synth.make_problem(n, m, 3, 1, 8, "negbin", seed=11, y_dtype="uint16", zero_frac=0.85, offset=True)
    starts = [synth.crude_start(prob, d, seed=11 + d) for d in d_list]
    rp, cp = synth.partitions(n, m, 11)
    st = synth.fit_settings(alpha_mode=1)
    sig = synth.sweep_orders(n, m, nbr, nbc, 3, 11)
    kw = dict(family="negbin", nb_row=nbr, nb_col=nbc, row_perm=rp, col_perm=cp, settings=st, precision=precision)

    def fit(group=None, tune=False):
        sw = gmf.Sweep(prob.Y, prob.X, prob.Z, prob.offset, starts, d_list, **kw)
        info = None
        if tune:
            info = sw.autotune(sig[0])
        elif group is not None:
            sw.group = group
        for e in range(3):
            sw.epoch(sig[e])
        return sw, info

    ref, _ = fit()
    assert ref.group == len(d_list)
    settings = (2, 1, 3, gmf.GMF_SWEEP_SEQUENTIAL) + ((gmf.GMF_SWEEP_PERSISTENT,) if precision == "mixed" else ())
    for group in settings:
        sw, _ = fit(group)
        assert sw.group == group
        for i in range(len(d_list)):
            a, b = sw.models[i].get_params(), ref.models[i].get_params()
            for k in ("U", "V", "B", "Gamma"):
                np.testing.assert_array_equal(a[k], b[k], err_msg=f"group {group} model {i} {k}")
            assert a["alpha"] == b["alpha"]
    sw, (g, times) = fit(tune=True)
    tried = {4, 2, 1, -1} | ({gmf.GMF_SWEEP_PERSISTENT} if precision == "mixed" else set())
    assert g in tried and sw.group == g and set(times) == tried and all(v > 0 for v in times.values())
    for i in range(len(d_list)):
        a, b = sw.models[i].get_params(), ref.models[i].get_params()
        for k in ("U", "V", "B", "Gamma"):
            np.testing.assert_array_equal(a[k], b[k], err_msg=f"autotuned model {i} {k}")
        ea, eb = sw.models[i].get_ema(), ref.models[i].get_ema()
        for k in ("Gb_row", "Hb_row", "Gb_col", "Hb_col", "cnt_row", "cnt_col", "t"):
            np.testing.assert_array_equal(ea[k], eb[k], err_msg=f"autotuned model {i} {k}")
    with pytest.raises(gmf.GmfError):
        sw.group = 5
    if precision == "fp32":
        with pytest.raises(gmf.GmfError):
            sw.group = gmf.GMF_SWEEP_PERSISTENT


def test_batched_tensor_core_launch_smallest_and_largest_rank_match_oracle(gmf):
    """The batched tensor-core tile launch (one launch for both models, NB,
    uint16) with the smallest and the largest rank of the rank sweep, d = 2
    and d = 50 (K = 7 and 55: one and two 128-byte atoms per split-BF16
    operand half, contraction widths 16 and 64), against the FP64 oracle
    after 3 epochs: deviance within 1e-3 (the mixed-precision bar)."""
    import oracle
    oracle.build()
    n, m, nbr, nbc = 900, 640, 300, 256
    d_list = [2, 50]
    prob = synth.make_problem(n, m, 3, 1, 10, "negbin", seed=13, y_dtype="uint16", zero_frac=0.85, offset=True)
    starts = [synth.crude_start(prob, d, seed=13 + d) for d in d_list]
    rp, cp = synth.partitions(n, m, 13)
    st = synth.fit_settings()
    sig = synth.sweep_orders(n, m, nbr, nbc, 3, 13)
    sw = gmf.Sweep(prob.Y, prob.X, prob.Z, prob.offset, starts, d_list, family="negbin", nb_row=nbr, nb_col=nbc,
                   row_perm=rp, col_perm=cp, settings=st, precision="mixed")
    assert sw.group == len(d_list)
    refs = [oracle.OracleFit(prob.Y, prob.X, prob.Z, prob.offset, s0, family="negbin", nb_row=nbr, nb_col=nbc,
                             row_perm=rp, col_perm=cp, settings=st) for s0 in starts]
    d0 = [r.deviance() for r in refs]
    for e in range(3):
        sw.epoch(sig[e])
        for r in refs:
            r.epoch(sig[e])
    for i, r in enumerate(refs):
        dr, dg = r.deviance(), sw.models[i].deviance()
        assert dr < d0[i]
        assert abs(dg - dr) / dr <= 1e-3, (d_list[i], dg, dr)
        assert rel(sw.models[i].get_params()["U"], r.U) <= 2e-2


@pytest.mark.parametrize("d_list", [[30, 2, 12, 20], [2, 5, 12, 20, 2, 5]])
def test_persistent_launch_with_several_tiles_per_cta(gmf, d_list):
    """The persistent rank-sweep launch with more tiles than resident CTAs, so
    that most CTAs run two or more tiles of different models in turn: one
    TMEM allocation per CTA (512 columns with d = 30 at one CTA per SM; 256
    columns at two CTAs per SM when every d <= 27), mbarrier phases carried
    across tiles. The fits equal those of the grouped launches bit for bit and
    no wait timed out. 3000 x 1024 uint16 counts in 1000 x 512 blocks: 2
    blocks of 8 x 4 tiles per sweep, 64 tiles per model and sweep."""
    n, m, nbr, nbc = 3000, 1024, 1000, 512
    prob = synth.make_problem(n, m, 3, 1, 8, "negbin", seed=21, y_dtype="uint16", zero_frac=0.85, offset=True)
    starts = [synth.crude_start(prob, d, seed=21 + i) for i, d in enumerate(d_list)]
    rp, cp = synth.partitions(n, m, 21)
    st = synth.fit_settings(alpha_mode=1)
    sig = synth.sweep_orders(n, m, nbr, nbc, 2, 21)
    kw = dict(family="negbin", nb_row=nbr, nb_col=nbc, row_perm=rp, col_perm=cp, settings=st, precision="mixed")
    fits = {}
    for group in (len(d_list), gmf.GMF_SWEEP_PERSISTENT):
        sw = gmf.Sweep(prob.Y, prob.X, prob.Z, prob.offset, starts, d_list, **kw)
        sw.group = group
        for e in range(2):
            sw.epoch(sig[e])
        fits[group] = [dict(mdl.get_params(), dev=mdl.deviance()) for mdl in sw.models]  # raises on a flagged wait
    for i in range(len(d_list)):
        a, b = fits[gmf.GMF_SWEEP_PERSISTENT][i], fits[len(d_list)][i]
        for k in ("U", "V", "B", "Gamma"):
            np.testing.assert_array_equal(a[k], b[k], err_msg=f"model {i} {k}")
        assert a["alpha"] == b["alpha"] and a["dev"] == b["dev"]
