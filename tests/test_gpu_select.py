"""Rank selection (Sec. 4.2) on the GPU: the log-likelihood and Pearson
statistic of gmf_loglik against the FP64 definitions at the same parameters
(FP32 log-gamma terms of one sign, FP64 sums: within 2e-6), and a batched rank
sweep with 30 % of the entries held out, whose per-rank summaries (AIC, BIC,
held-out deviance, eigenvalue-ratio rank of the highest-rank fit) are formed
from the library's numbers by paper_2412_20509_gb300.select."""
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


@pytest.mark.parametrize("family,weights,missing", [("poisson", False, False), ("negbin", True, False),
                                                    ("negbin", False, True)])
def test_loglik_and_pearson_match_definitions(gmf, family, weights, missing):
    from oracle.select import loglik, pearson
    n, m, d = 700, 480, 4
    prob = synth.make_problem(n, m, 2, 1, d, family, seed=12, zero_frac=0.7 if family == "negbin" else None,
                              offset=True)
    obs = synth.holdout_mask(n, m, 0.3, 12) if missing else np.ones((n, m), bool)
    Y = synth.with_missing(prob.Y, obs) if missing else prob.Y
    W = np.random.default_rng(2).uniform(0.5, 1.5, (n, m)).astype(np.float32) if weights else None
    start = synth.crude_start(prob, d, seed=12)
    rp, cp = synth.partitions(n, m, 12)
    model = gmf.Model(torch.from_numpy(Y).cuda(), prob.X, prob.Z, prob.offset, start, family=family, nb_row=128,
                      nb_col=96, row_perm=rp, col_perm=cp, settings=synth.fit_settings(missing=int(missing)),
                      W=None if W is None else torch.from_numpy(W).cuda())
    for s in synth.sweep_orders(n, m, 128, 96, 2, 12):
        model.epoch(s)
    par = model.get_params()
    eta = prob.offset[:, None] + prob.X @ par["B"].T + par["Gamma"] @ prob.Z.T + par["U"] @ par["V"].T
    mu = np.exp(np.clip(eta, -30, 30))
    Wd = None if W is None else W.astype(np.float64)
    got = model.loglik()
    assert got["n_obs"] == int(obs.sum())
    assert got["loglik"] == pytest.approx(loglik(prob.Y, mu, family, par["alpha"], Wd, obs), rel=2e-6)
    assert got["pearson"] == pytest.approx(pearson(prob.Y, mu, family, par["alpha"], Wd, obs), rel=2e-6)


def test_rank_sweep_with_held_out_entries(gmf):
    """Poisson data of rank 4; ranks {1, 2, 4, 6} fitted in one batched sweep
    with 30 % of the entries held out. Each model equals its own single fit bit
    for bit (the imputation runs in the batched tile launch too); the summaries
    follow from the library's numbers; under-fitting ranks predict the held-out
    entries worse than the true rank."""
    from paper_2412_20509_gb300 import select
    n, m, d_true = 1200, 640, 4
    prob = synth.make_problem(n, m, 2, 1, d_true, "poisson", seed=21, offset=True, scale=0.6)
    obs = synth.holdout_mask(n, m, 0.3, 21)
    Ym = synth.with_missing(prob.Y, obs)
    ranks = [1, 2, 4, 6]
    starts = [synth.crude_start(prob, d, seed=21 + d) for d in ranks]
    rp, cp = synth.partitions(n, m, 21)
    kw = dict(family="poisson", nb_row=256, nb_col=128, row_perm=rp, col_perm=cp,
              settings=synth.fit_settings(missing=1, bias_corr=1), precision="mixed")
    Yd = torch.from_numpy(Ym).cuda()
    sw = gmf.Sweep(Yd, prob.X, prob.Z, prob.offset, starts, ranks, **kw)
    solo = gmf.Model(Yd, prob.X, prob.Z, prob.offset, starts[2], **kw)
    for s in synth.sweep_orders(n, m, 256, 128, 20, 21):
        sw.epoch(s)
        solo.epoch(s)
    a, b = sw.models[2].get_params(), solo.get_params()
    for k in ("U", "V", "B", "Gamma"):
        np.testing.assert_array_equal(a[k], b[k])
    Ytrue = torch.from_numpy(prob.Y).cuda()
    sums = [select.fit_summary(mdl, "poisson", Ytrue) for mdl in sw.models]
    for s, d in zip(sums, ranks):
        k = select.free_params(n, m, 2, 1, d, "poisson")
        assert s["d"] == d and s["free_params"] == k
        assert s["aic"] == pytest.approx(-2 * s["loglik"] + 2 * k)
    sw.models[-1].orthogonalize("B1")
    spec = select.singular_values(sw.models[-1])
    assert len(spec) == 6 and np.all(np.diff(spec) <= 0)
    pick = select.select_rank(sums, spec)
    assert set(pick) == {"aic", "bic", "heldout_deviance", "heldout_error", "eigen_ratio"}
    dev = {s["d"]: s["heldout_deviance"] for s in sums}
    assert dev[4] < dev[2] < dev[1] < 1.0
