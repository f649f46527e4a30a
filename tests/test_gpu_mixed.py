"""Parity of the tensor-core (tcgen05) path with the FP64 oracle.

Tolerances from the arithmetic of the mixed path: eta is a split-BF16 product
(three BF16 products, FP32 accumulate: relative error ~1e-5 of |L||R|); Ddot,
Dddot and the contraction operands are BF16 (unit roundoff 2^-9 ~ 2e-3), so
each block gradient / curvature sum carries up to ~1e-2 relative error against
the scale of its terms. Hence, after one teacher-forced sweep: the parameter
step within 3e-2 (max-norm relative); a sweep moves the parameters by about 1%
of their scale, so the parameters stay within 5e-4; after a
fixed number of epochs: the deviance within 1e-3 of the oracle's (the stated
target for the mixed path).
"""
import numpy as np
import pytest

import synth
from tests.test_gpu_parity import Pair, check_per_entry, rel

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


@pytest.fixture(scope="module")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


MIXED = {
    # K = 1+p+q+d <= 16: one 128-byte atom per eta operand row
    "poisson_cfg1": (1000, 500, 2, 1, 5, "poisson", 100, 100, dict(offset=False)),
    # 2 atoms (K = 25), uint16 counts, ragged 128-tiles, NB shape updates
    "nb_d20_uint16": (900, 640, 3, 1, 20, "negbin", 300, 256,
                      dict(y_dtype="uint16", zero_frac=0.85, alpha_mode=1)),
    # 3 atoms (K = 55), contraction widths 51 / 53 -> 64
    "nb_d50": (640, 384, 3, 1, 50, "negbin", 256, 128, dict(y_dtype="uint16", zero_frac=0.8)),
    # blocks smaller than a tile, r < s role swap, per-visit bias correction, weights
    "nb_swap_small_blocks": (200, 960, 2, 2, 4, "negbin", 100, 96,
                             dict(zero_frac=0.7, bias_corr=1, weights=True)),
}


@pytest.mark.parametrize("case", list(MIXED))
def test_mixed_one_sweep_teacher_forced(gmf, oracle_mod, case):
    n, m, p, q, d, fam, nbr, nbc, extra = MIXED[case]
    P = Pair(gmf, oracle_mod, n, m, p, q, d, fam, nbr, nbc, precision="mixed", **extra)
    for e in range(2):
        P.ref.epoch(P.sigmas[e])
    P.teacher_force()
    before = P.ref_params()
    sig = P.sigmas[5]
    w = int(np.random.default_rng(2).integers(P.nsw))
    P.ref.sweeps(sig, w, w + 1)
    P.gpu.sweeps(sig, w, w + 1)
    got, ref = P.gpu.get_params(), P.ref_params()
    for k in ("U", "V", "B", "Gamma"):
        if ref[k].size == 0:
            continue
        assert rel(got[k], ref[k]) <= 5e-4, (k, rel(got[k], ref[k]))
        check_per_entry(k, got[k], ref[k], before[k], 3e-2, 5e-3)   # and per entry (the atlas shape's bar)
        step_ref = ref[k] - before[k]
        if np.abs(step_ref).max() > 0:
            step_gpu = got[k] - before[k].astype(np.float32).astype(np.float64)
            assert rel(step_gpu, step_ref) <= 3e-2, (k, "step", rel(step_gpu, step_ref))
    ema, rema = P.gpu.get_ema(), P.ref_ema()
    np.testing.assert_array_equal(ema["cnt_row"], rema["cnt_row"])
    np.testing.assert_array_equal(ema["cnt_col"], rema["cnt_col"])
    assert got["alpha"] == pytest.approx(ref["alpha"], rel=1e-3)


@pytest.mark.parametrize("case,epochs", [("poisson_cfg1", 50), ("nb_d20_uint16", 6), ("nb_d50", 4)])
def test_mixed_final_deviance_within_1e3(gmf, oracle_mod, case, epochs):
    n, m, p, q, d, fam, nbr, nbc, extra = MIXED[case]
    P = Pair(gmf, oracle_mod, n, m, p, q, d, fam, nbr, nbc, precision="mixed", **extra)
    d0 = P.ref.deviance()
    for e in range(epochs):
        P.ref.epoch(P.sigmas[e])
        P.gpu.epoch(P.sigmas[e])
    dr, dg = P.ref.deviance(), P.gpu.deviance()
    assert dr < d0
    assert abs(dg - dr) / dr <= 1e-3, (dg, dr)


def test_mixed_full_size_nb_medium(gmf, oracle_mod):
    """The benchmarked workload on the tensor-core path: one epoch, deviance within 1e-3."""
    w = synth.WORKLOADS["nb_medium"]
    P = Pair(gmf, oracle_mod, w.n, w.m, w.p, w.q, w.d, w.family, w.nb_row, w.nb_col, zero_frac=w.zero_frac,
             precision="mixed")
    P.ref.epoch(P.sigmas[0])
    P.gpu.epoch(P.sigmas[0])
    assert P.gpu.deviance() == pytest.approx(P.ref.deviance(), rel=1e-3)
    # Sanity bound only: a full epoch compounds 4 row visits and 40 column visits
    # of steps that each carry the BF16 contraction error (<= 3e-2 of a step).
    got, ref = P.gpu.get_params(), P.ref_params()
    for k in ("U", "V"):
        assert rel(got[k], ref[k]) <= 2e-2


def test_mixed_is_deterministic(gmf, oracle_mod):
    n, m, p, q, d, fam, nbr, nbc, extra = MIXED["nb_d20_uint16"]
    P = Pair(gmf, oracle_mod, n, m, p, q, d, fam, nbr, nbc, precision="mixed", **extra)
    Q = Pair(gmf, oracle_mod, n, m, p, q, d, fam, nbr, nbc, precision="mixed", **extra)
    for e in range(2):
        P.gpu.epoch(P.sigmas[e])
        Q.gpu.epoch(Q.sigmas[e])
    a, b = P.gpu.get_params(), Q.gpu.get_params()
    for k in ("U", "V", "B", "Gamma"):
        np.testing.assert_array_equal(a[k], b[k])


def test_mixed_rejects_unaligned_layouts(gmf, oracle_mod):
    with pytest.raises(gmf.GmfError) as e:
        Pair(gmf, oracle_mod, 100, 50, 2, 1, 3, "poisson", 20, 10, precision="mixed")   # 50 * 4 bytes % 16 != 0
    assert e.value.code == gmf.GMF_ERR_ARG and "16 bytes" in str(e.value)
    with pytest.raises(gmf.GmfError):
        Pair(gmf, oracle_mod, 100, 64, 2, 1, 3, "poisson", 20, 10, precision="mixed")   # nb_col * 4 % 16 != 0


CLUSTER_CASES = {
    # name: (n, m, p, q, d, family, nb_row, nb_col, extra); tiles per block TI x TJ <= 16
    "nb_ragged_12_tiles": (1100, 704, 3, 1, 6, "negbin", 500, 384,
                           dict(zero_frac=0.8, weights=True, alpha_mode=1, bias_corr=1)),
    "poisson_16_tiles_uint16": (2000, 1024, 2, 1, 10, "poisson", 500, 512, dict(y_dtype="uint16")),
    "nb_6_tiles": (300, 256, 2, 2, 3, "negbin", 300, 256, dict(zero_frac=0.6, alpha_mode=1)),
    # fixed NB shape or Poisson: the epoch is one persistent launch
    "nb_ragged_weights_fixed_shape": (1100, 704, 3, 1, 6, "negbin", 500, 384,
                                      dict(zero_frac=0.8, weights=True, bias_corr=1)),
    "poisson_uint16_roles_swapped": (600, 2048, 2, 2, 5, "poisson", 300, 512, dict(y_dtype="uint16")),
    "nb_12_sweeps_16_tiles": (6000, 1024, 2, 1, 10, "negbin", 500, 512, dict(zero_frac=0.5)),
}

MODE_FLAGS = {"persistent": 2, "cluster": 0, "separate": 1}   # gmf.GMF_FLAG_PERSIST, gmf.GMF_FLAG_NO_CLUSTER


def _fit_modes(gmf, case, epochs=3, split=None):
    n, m, p, q, d, fam, nbr, nbc, extra = CLUSTER_CASES[case]
    extra = dict(extra)
    y_dtype = extra.pop("y_dtype", "int32")
    zero_frac = extra.pop("zero_frac", None)
    weights = extra.pop("weights", False)
    prob = synth.make_problem(n, m, p, q, d, fam, seed=3, y_dtype=y_dtype, zero_frac=zero_frac, offset=True)
    start = synth.crude_start(prob, d, seed=3)
    rp, cp = synth.partitions(n, m, 3)
    settings = synth.fit_settings(**extra)
    W = torch.from_numpy(np.random.default_rng(10).uniform(0.5, 1.5, (n, m)).astype(np.float32)).cuda() \
        if weights else None
    sig = synth.sweep_orders(n, m, nbr, nbc, epochs, 3)
    fits = {}
    for mode, flags in MODE_FLAGS.items():
        Yd = torch.from_numpy(prob.Y.view(np.int16) if y_dtype == "uint16" else prob.Y).cuda()
        mdl = gmf.Model(Yd, prob.X, prob.Z, prob.offset, start, family=fam, nb_row=nbr, nb_col=nbc, row_perm=rp,
                        col_perm=cp, settings=settings, W=W, precision="mixed", flags=flags)
        for s_ in sig:
            if split is None:
                mdl.epoch(s_)
            else:   # the epoch as several sweep ranges
                bounds = [0, *split, mdl.num_sweeps]
                for b0, b1 in zip(bounds[:-1], bounds[1:]):
                    mdl.sweeps(s_, b0, b1)
        fits[mode] = mdl
    return fits, settings, fam


def _assert_same_state(a_mdl, b_mdl, label):
    a, b = a_mdl.get_params(), b_mdl.get_params()
    for k in ("B", "Gamma", "U", "V"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=f"{label}: {k}")
    assert a["alpha"] == b["alpha"], label
    ea, eb = a_mdl.get_ema(), b_mdl.get_ema()
    for k in ("Gb_row", "Hb_row", "Gb_col", "Hb_col", "cnt_row", "cnt_col", "t"):
        np.testing.assert_array_equal(ea[k], eb[k], err_msg=f"{label}: {k}")
    assert a_mdl.deviance() == b_mdl.deviance(), label


@pytest.mark.parametrize("case", list(CLUSTER_CASES))
def test_epoch_modes_agree_bitwise(gmf, case):
    """The three ways an epoch can launch -- tiles then a separate strip-update
    launch per sweep; one cluster launch per sweep, the partials exchanged
    through distributed shared memory; one persistent launch per epoch, each
    cluster waiting only for the earlier visits of its moving strip -- run the
    same phases and sum the same partials in the same tile order, so they must
    agree to the bit. Cases with the per-sweep NB shape estimate (alpha_mode 1)
    have no persistent mode and run cluster launches with GMF_FLAG_PERSIST."""
    fits, settings, fam = _fit_modes(gmf, case)
    moment = fam == "negbin" and settings["alpha_mode"] == 1
    assert fits["persistent"].epoch_mode == ("cluster" if moment else "persistent")
    assert fits["cluster"].epoch_mode == "cluster" and fits["separate"].epoch_mode == "separate"
    assert fits["persistent"].launches_per_sweep == (1 if moment else 0)
    assert fits["cluster"].launches_per_sweep == 1 and fits["separate"].launches_per_sweep == 2
    _assert_same_state(fits["persistent"], fits["separate"], "persistent vs separate")
    _assert_same_state(fits["cluster"], fits["separate"], "cluster vs separate")


@pytest.mark.parametrize("case", ["nb_12_sweeps_16_tiles", "poisson_uint16_roles_swapped"])
def test_persistent_sweep_ranges_equal_whole_epochs(gmf, case):
    """gmf_sgd_sweeps over a split of the epoch: each range is one persistent
    launch whose dependency counts start from zero; the result equals the
    per-sweep launches of whole epochs bit for bit."""
    fits, _, _ = _fit_modes(gmf, case, epochs=2, split=[1, 4])
    assert fits["persistent"].epoch_mode == "persistent"
    _assert_same_state(fits["persistent"], fits["separate"], "ranges: persistent vs separate")


def test_persistent_trace_times_one_launch_per_epoch(gmf):
    n, m, p, q, d, fam, nbr, nbc, extra = CLUSTER_CASES["nb_12_sweeps_16_tiles"]
    prob = synth.make_problem(n, m, p, q, d, fam, seed=4, zero_frac=0.5, offset=True)
    start = synth.crude_start(prob, d, seed=4)
    rp, cp = synth.partitions(n, m, 4)
    mdl = gmf.Model(torch.from_numpy(prob.Y).cuda(), prob.X, prob.Z, prob.offset, start, family=fam, nb_row=nbr,
                    nb_col=nbc, row_perm=rp, col_perm=cp, settings=synth.fit_settings(), precision="mixed",
                    flags=gmf.GMF_FLAG_PERSIST)
    assert mdl.epoch_mode == "persistent"
    sig = synth.sweep_orders(n, m, nbr, nbc, 3, 4)
    mdl.trace(True)
    for s_ in sig:
        mdl.epoch(s_)
    ms, launches = mdl.trace_read()
    mdl.trace(False)
    assert launches == 3 and ms > 0.0
    assert np.isfinite(mdl.deviance())


def test_persistent_epoch_equals_cluster_launches_full_size(gmf):
    """The benchmarked workload (20000 x 2000 NB, 4 clusters of 16 CTAs, 40 sweeps
    per epoch, every strip waited on across clusters): two epochs as one
    persistent launch each equal the per-sweep cluster launches bit for bit."""
    w = synth.WORKLOADS["nb_medium"]
    prob = synth.workload_problem(w.name, seed=5)
    start = synth.crude_start(prob, w.d, seed=5)
    rp, cp = synth.partitions(w.n, w.m, 5)
    sig = synth.sweep_orders(w.n, w.m, w.nb_row, w.nb_col, 2, 5)
    Yd = torch.from_numpy(prob.Y).cuda()
    fits = []
    for flags in (gmf.GMF_FLAG_PERSIST, 0):
        mdl = gmf.Model(Yd, prob.X, prob.Z, prob.offset, start, family=w.family, nb_row=w.nb_row, nb_col=w.nb_col,
                        row_perm=rp, col_perm=cp, settings=synth.fit_settings(), precision="mixed", flags=flags)
        for s_ in sig:
            mdl.epoch(s_)
        fits.append(mdl)
    assert fits[0].epoch_mode == "persistent" and fits[1].epoch_mode == "cluster"
    _assert_same_state(fits[0], fits[1], "nb_medium: persistent vs cluster")
