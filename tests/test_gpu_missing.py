"""Missing entries and held-out evaluation on the GPU (cfg.missing = 1) against
the FP64 oracle: 30 % of the entries, drawn uniformly (the protocol of Sec.
5.2), are marked missing with the count dtype's marker; every block step
imputes them with the current mean (Sec. 3.2). Bars as for complete data:
one teacher-forced sweep within 1e-5 (FP32) / 5e-4 (tensor cores) max-norm
relative, deviance within 1e-4 / 1e-3 after several epochs. The held-out
metrics (gmf_holdout) equal the definitions of Sec. 5.2 evaluated in FP64 at
the same parameters within 1e-5 (FP32 terms, FP64 sums)."""
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


@pytest.fixture(scope="module")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


CASES = {
    # name: (n, m, p, q, d, family, nb_row, nb_col, y_dtype, precision, extra settings)
    "fp32_nb_int32": (1100, 700, 3, 1, 6, "negbin", 300, 160, "int32", "fp32", dict(alpha_mode=1, bias_corr=1)),
    "fp32_poisson_uint16_swap": (300, 1000, 2, 2, 3, "poisson", 200, 100, "uint16", "fp32", {}),
    "mixed_nb_uint16_separate": (4300, 2104, 3, 1, 20, "negbin", 2048, 1024, "uint16", "mixed", {}),
    "mixed_nb_int32_cluster": (1100, 704, 3, 1, 6, "negbin", 500, 384, "int32", "mixed", dict(alpha_mode=1)),
}


class MissingPair:
    def __init__(self, gmf, oracle_mod, case, seed=3, frac=0.3):
        n, m, p, q, d, fam, nbr, nbc, ydt, prec, extra = CASES[case]
        self.prob = synth.make_problem(n, m, p, q, d, fam, seed=seed, y_dtype=ydt,
                                       zero_frac=0.8 if fam == "negbin" else None, offset=True)
        self.obs = synth.holdout_mask(n, m, frac, seed)
        self.Ym = synth.with_missing(self.prob.Y, self.obs)
        self.start = synth.crude_start(self.prob, d, seed=seed)      # an input: drawn from the complete matrix
        self.rp, self.cp = synth.partitions(n, m, seed)
        self.settings = synth.fit_settings(missing=1, **extra)
        self.sigmas = synth.sweep_orders(n, m, nbr, nbc, 8, seed)
        P = self.prob
        self.ref = oracle_mod.OracleFit(self.Ym, P.X, P.Z, P.offset, self.start, family=fam, nb_row=nbr,
                                        nb_col=nbc, row_perm=self.rp, col_perm=self.cp, settings=self.settings)
        dev = lambda a: torch.from_numpy(a.view(np.int16) if a.dtype == np.uint16 else a).cuda()
        self.Ytrue = dev(P.Y)
        self.gpu = gmf.Model(dev(self.Ym), P.X, P.Z, P.offset, self.start, family=fam, nb_row=nbr, nb_col=nbc,
                             row_perm=self.rp, col_perm=self.cp, settings=self.settings, precision=prec)
        self.precision = prec

    def ref_params(self):
        r = self.ref
        return dict(B=r.B.copy(), Gamma=r.G.copy(), U=r.U.copy(), V=r.V.copy(), alpha=float(r.alpha[0]))

    def teacher_force(self):
        r = self.ref
        self.gpu.set_params(self.ref_params())
        self.gpu.set_ema(dict(Gb_row=r.Gb_row, Hb_row=r.Hb_row, Gb_col=r.Gb_col, Hb_col=r.Hb_col,
                              cnt_row=r.cnt_row, cnt_col=r.cnt_col, t=int(r.t[0])))


@pytest.mark.parametrize("case", list(CASES))
def test_missing_one_sweep_teacher_forced(gmf, oracle_mod, case):
    P = MissingPair(gmf, oracle_mod, case)
    for e in range(2):
        P.ref.epoch(P.sigmas[e])
    P.teacher_force()
    w = 1
    P.ref.sweeps(P.sigmas[5], w, w + 1)
    P.gpu.sweeps(P.sigmas[5], w, w + 1)
    got, ref = P.gpu.get_params(), P.ref_params()
    bar = 1e-5 if P.precision == "fp32" else 5e-4
    for k in ("U", "V", "B", "Gamma"):
        assert rel(got[k], ref[k]) <= bar, (k, rel(got[k], ref[k]))
    if "alpha_mode" in CASES[case][-1]:
        assert got["alpha"] == pytest.approx(ref["alpha"], rel=1e-5 if P.precision == "fp32" else 1e-3)


@pytest.mark.parametrize("case", list(CASES))
def test_missing_deviance_and_holdout_metrics(gmf, oracle_mod, case):
    from oracle.holdout import holdout_metrics
    P = MissingPair(gmf, oracle_mod, case)
    d0 = P.ref.deviance()
    for e in range(3):
        P.ref.epoch(P.sigmas[e])
        P.gpu.epoch(P.sigmas[e])
    dr, dg = P.ref.deviance(), P.gpu.deviance()
    assert dr < d0
    assert abs(dg - dr) / dr <= (1e-4 if P.precision == "fp32" else 1e-3), (dg, dr)
    # the metrics at the GPU's own parameters, by the definitions (FP64)
    par = P.gpu.get_params()
    pr = P.prob
    eta = pr.offset[:, None] + pr.X @ par["B"].T + par["Gamma"] @ pr.Z.T + par["U"] @ par["V"].T
    e_ref, d_ref, ybar_ref, nv_ref = holdout_metrics(pr.Y, P.obs, np.exp(np.clip(eta, -30, 30)))
    got = P.gpu.holdout(P.Ytrue)
    assert got["n_heldout"] == nv_ref
    assert got["ybar"] == pytest.approx(ybar_ref, rel=1e-12)
    assert got["error"] == pytest.approx(e_ref, rel=1e-5)
    assert got["deviance"] == pytest.approx(d_ref, rel=1e-5)


def test_holdout_needs_missing_entries(gmf):
    prob = synth.make_problem(200, 96, 2, 1, 2, "poisson", seed=1)
    Y = torch.from_numpy(prob.Y).cuda()
    start = synth.crude_start(prob, 2, seed=1)
    rp, cp = synth.partitions(200, 96, 1)
    kw = dict(family="poisson", nb_row=64, nb_col=32, row_perm=rp, col_perm=cp)
    m0 = gmf.Model(Y, prob.X, prob.Z, prob.offset, start, settings=synth.fit_settings(), **kw)
    with pytest.raises(gmf.GmfError) as e:
        m0.holdout(Y)
    assert e.value.code == gmf.GMF_ERR_STATE
    m1 = gmf.Model(Y, prob.X, prob.Z, prob.offset, start, settings=synth.fit_settings(missing=1), **kw)
    with pytest.raises(gmf.GmfError) as e:
        m1.holdout(Y)                      # nothing marked missing
    assert e.value.code == gmf.GMF_ERR_STATE
