"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 path), from the arithmetic: parameters are stored in FP32
(relative spacing 6e-8), the block sums are FP32 sums of <= nb terms, so one
sweep keeps every parameter matrix within 1e-5 of the oracle in max-norm
relative terms (the stated per-step target) and the step itself
(theta_after - theta_before) within 1e-3 relative; the final deviance of a
fixed number of epochs stays within 1e-4 relative (stated target); the
deviance at identical parameters within 1e-6 (FP32 terms, FP64 total).
"""
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


@pytest.fixture(scope="module")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def rel(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-30))


def check_per_entry(name, got, ref, before, rtol, atol):
    """Each parameter against its own oracle value after a step from `before`:
    |got - ref| <= rtol |step| + atol max|step of its column| + 1e-7 |ref| (the
    last term is the FP32 storage of the parameter)."""
    step = ref - before
    err = np.abs(got - ref)
    colmax = np.abs(step).max(axis=0, keepdims=True)
    bound = rtol * np.abs(step) + atol * colmax + 1e-7 * np.abs(ref)
    bad = err > bound
    assert not bad.any(), (name, int(bad.sum()), float((err - bound).max()), float(colmax.max()))


class Pair:
    """The same fit in the oracle and on the GPU."""

    def __init__(self, gmf, oracle_mod, n, m, p, q, d, family, nb_row, nb_col, *, seed=0, y_dtype="int32",
                 zero_frac=None, offset=True, weights=False, precision="fp32", flags=0, **settings):
        self.prob = synth.make_problem(n, m, p, q, d, family, seed=seed, y_dtype=y_dtype, zero_frac=zero_frac,
                                       offset=offset)
        self.start = synth.crude_start(self.prob, d, seed=seed)
        self.rp, self.cp = synth.partitions(n, m, seed)
        self.settings = synth.fit_settings(**settings)
        self.W = np.random.default_rng(seed + 7).uniform(0.5, 1.5, (n, m)).astype(np.float32) if weights else None
        self.nsw = synth.n_sweeps(n, m, nb_row, nb_col)
        self.sigmas = synth.sweep_orders(n, m, nb_row, nb_col, 64, seed)
        P = self.prob
        self.ref = oracle_mod.OracleFit(P.Y, P.X, P.Z, P.offset, self.start, family=family, nb_row=nb_row,
                                        nb_col=nb_col, row_perm=self.rp, col_perm=self.cp, settings=self.settings,
                                        W=None if self.W is None else self.W.astype(np.float64))
        self.gpu = gmf.Model(torch.from_numpy(P.Y).cuda(), P.X, P.Z, P.offset, self.start, family=family,
                             nb_row=nb_row, nb_col=nb_col, row_perm=self.rp, col_perm=self.cp,
                             settings=self.settings, W=None if self.W is None else torch.from_numpy(self.W).cuda(),
                             precision=precision, flags=flags)

    def ref_params(self):
        r = self.ref
        return dict(B=r.B.copy(), Gamma=r.G.copy(), U=r.U.copy(), V=r.V.copy(), alpha=float(r.alpha[0]))

    def ref_ema(self):
        r = self.ref
        return dict(Gb_row=r.Gb_row.copy(), Hb_row=r.Hb_row.copy(), Gb_col=r.Gb_col.copy(), Hb_col=r.Hb_col.copy(),
                    cnt_row=r.cnt_row.copy(), cnt_col=r.cnt_col.copy(), t=int(r.t[0]))

    def teacher_force(self):
        self.gpu.set_params(self.ref_params())
        self.gpu.set_ema(self.ref_ema())


CASES = {
    # name: (n, m, p, q, d, family, nb_row, nb_col, extra)
    "poisson_cfg1": (1000, 500, 2, 1, 5, "poisson", 100, 100, dict(offset=False)),
    "nb_ragged_weights": (1100, 700, 3, 1, 6, "negbin", 300, 160,
                          dict(zero_frac=0.8, weights=True, alpha_mode=1, bias_corr=1)),
    "nb_swap_r_lt_s": (300, 1000, 2, 2, 3, "negbin", 200, 100, dict(zero_frac=0.7)),
    "tiny_5x4": (5, 4, 2, 1, 2, "poisson", 2, 3, dict()),
    "d0_intercepts": (400, 300, 1, 1, 0, "poisson", 64, 64, dict()),
    "uint16_counts": (900, 650, 3, 1, 10, "negbin", 256, 128, dict(y_dtype="uint16", zero_frac=0.85)),
    "odd_tiles": (130, 67, 2, 1, 9, "negbin", 65, 33, dict(zero_frac=0.5, alpha_mode=1)),
}


@pytest.mark.parametrize("case", list(CASES))
def test_one_sweep_teacher_forced(gmf, oracle_mod, case):
    n, m, p, q, d, fam, nbr, nbc, extra = CASES[case]
    P = Pair(gmf, oracle_mod, n, m, p, q, d, fam, nbr, nbc, **extra)
    # warm up the oracle so the EMA state and counters are non-trivial, then hand its state to the GPU
    for e in range(2):
        P.ref.epoch(P.sigmas[e])
    P.teacher_force()
    before = P.ref_params()
    sig = P.sigmas[5]
    w = int(np.random.default_rng(1).integers(P.nsw))
    # one sweep in both
    P.ref.sweeps(sig, w, w + 1)
    P.gpu.sweeps(sig, w, w + 1)
    got = P.gpu.get_params()
    ref = P.ref_params()
    for k in ("U", "V", "B", "Gamma"):
        if ref[k].size == 0:
            continue
        assert rel(got[k], ref[k]) <= 1e-5, (k, rel(got[k], ref[k]))
        check_per_entry(k, got[k], ref[k], before[k], 1e-3, 1e-5)   # and per entry, as at the atlas shape
        step_ref = ref[k] - before[k]
        if np.abs(step_ref).max() > 0:
            step_gpu = got[k] - before[k].astype(np.float32).astype(np.float64)
            assert rel(step_gpu, step_ref) <= 1e-3, (k, "step", rel(step_gpu, step_ref))
    ema = P.gpu.get_ema()
    rema = P.ref_ema()
    for k in ("Gb_row", "Hb_row", "Gb_col", "Hb_col"):
        if rema[k].size:
            assert rel(ema[k], rema[k]) <= 1e-4, (k, rel(ema[k], rema[k]))
    np.testing.assert_array_equal(ema["cnt_row"], rema["cnt_row"])
    np.testing.assert_array_equal(ema["cnt_col"], rema["cnt_col"])
    assert ema["t"] == rema["t"]
    assert got["alpha"] == pytest.approx(ref["alpha"], rel=1e-6)


@pytest.mark.parametrize("case,epochs", [("poisson_cfg1", 50), ("nb_ragged_weights", 8), ("uint16_counts", 6)])
def test_final_deviance_after_fixed_epochs(gmf, oracle_mod, case, epochs):
    n, m, p, q, d, fam, nbr, nbc, extra = CASES[case]
    P = Pair(gmf, oracle_mod, n, m, p, q, d, fam, nbr, nbc, **extra)
    d0 = P.ref.deviance()
    for e in range(epochs):
        P.ref.epoch(P.sigmas[e])
        P.gpu.epoch(P.sigmas[e])
    dr, dg = P.ref.deviance(), P.gpu.deviance()
    assert dr < d0
    assert abs(dg - dr) / dr <= 1e-4, (dg, dr)
    got = P.gpu.get_params()
    for k in ("U", "V"):
        assert rel(got[k], P.ref_params()[k]) <= 1e-3


def test_deviance_at_identical_parameters(gmf, oracle_mod):
    for fam, extra in (("poisson", dict()), ("negbin", dict(zero_frac=0.85, weights=True))):
        P = Pair(gmf, oracle_mod, 700, 450, 3, 1, 7, fam, 128, 96, seed=4, **extra)
        P.gpu.set_params(P.ref_params())
        assert P.gpu.deviance() == pytest.approx(P.ref.deviance(), rel=1e-6)


def test_full_size_nb_medium_one_epoch(gmf, oracle_mod):
    """The benchmarked workload (20000 x 2000 NB, d = 10, 500 x 500 blocks) in
    the launch configuration the benchmark times: one epoch, whole matrices."""
    w = synth.WORKLOADS["nb_medium"]
    P = Pair(gmf, oracle_mod, w.n, w.m, w.p, w.q, w.d, w.family, w.nb_row, w.nb_col, zero_frac=w.zero_frac,
             offset=True)
    P.ref.epoch(P.sigmas[0])
    P.gpu.epoch(P.sigmas[0])
    got = P.gpu.get_params()
    ref = P.ref_params()
    for k in ("U", "V", "B", "Gamma"):
        assert rel(got[k], ref[k]) <= 1e-4, (k, rel(got[k], ref[k]))
    assert P.gpu.deviance() == pytest.approx(P.ref.deviance(), rel=1e-5)


def test_runs_are_bitwise_deterministic(gmf, oracle_mod):
    n, m, p, q, d, fam, nbr, nbc, extra = CASES["nb_ragged_weights"]
    P = Pair(gmf, oracle_mod, n, m, p, q, d, fam, nbr, nbc, **extra)
    Q = Pair(gmf, oracle_mod, n, m, p, q, d, fam, nbr, nbc, **extra)
    for e in range(3):
        P.gpu.epoch(P.sigmas[e])
        Q.gpu.epoch(Q.sigmas[e])
    a, b = P.gpu.get_params(), Q.gpu.get_params()
    for k in ("U", "V", "B", "Gamma"):
        np.testing.assert_array_equal(a[k], b[k])


def test_checkpoint_resume_is_bitwise(gmf, oracle_mod):
    n, m, p, q, d, fam, nbr, nbc, extra = CASES["nb_ragged_weights"]
    P = Pair(gmf, oracle_mod, n, m, p, q, d, fam, nbr, nbc, **extra)
    Q = Pair(gmf, oracle_mod, n, m, p, q, d, fam, nbr, nbc, **extra)
    for e in range(2):
        P.gpu.epoch(P.sigmas[e])
    ck = P.gpu.state_dict()
    Q.gpu.load_state_dict(ck)
    for e in range(2, 4):
        P.gpu.epoch(P.sigmas[e])
        Q.gpu.epoch(Q.sigmas[e])
    a, b = P.gpu.state_dict(), Q.gpu.state_dict()
    for k in ("U", "V", "B", "Gamma", "Gb_row", "Hb_col"):
        np.testing.assert_array_equal(a[k], b[k])
    assert a["t"] == b["t"] and a["alpha"] == b["alpha"]


def test_update_y_from_host_and_device(gmf, oracle_mod):
    n, m, p, q, d, fam, nbr, nbc, extra = CASES["uint16_counts"]
    P = Pair(gmf, oracle_mod, n, m, p, q, d, fam, nbr, nbc, **extra)
    dev0 = P.gpu.deviance()
    Y2 = np.ascontiguousarray(P.prob.Y[::-1])
    P.gpu.update_y(Y2)
    dev_host = P.gpu.deviance()
    P.gpu.update_y(torch.from_numpy(P.prob.Y).cuda())
    assert P.gpu.deviance() == dev0
    P.gpu.update_y(torch.from_numpy(Y2).cuda())
    assert P.gpu.deviance() == dev_host != dev0


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
@pytest.mark.parametrize("source", ["pinned", "pageable", "unaligned_rows", "pinned_int32", "pinned_staged"])
def test_streamed_counts_equal_synchronous_updates(gmf, oracle_mod, precision, source):
    """gmf_update_y_async with the next matrix's upload issued before the current
    epoch has run gives the same fit, bit for bit, as gmf_update_y between
    epochs: from pinned memory through the direct gather into the second count
    buffer (the handle switches buffers each call); from pageable memory the
    same where the device reads pageable host memory, else through the staging
    copies; rows of 1300 bytes (not a multiple of 16) always through the
    double-buffered staging copies; with GMF_FLAG_STAGED_UPLOAD pinned memory
    through the staging copies as well."""
    # uint16 counts; 656 genes keep the tensor-core layout's 16-byte rows
    n, m, p, q, d, fam, nbr, nbc = 900, 656, 3, 1, 10, "negbin", 256, 128
    if source == "unaligned_rows":
        if precision == "mixed":
            pytest.skip("the tensor-core layout needs 16-byte rows")
        m = 650
    i32 = source == "pinned_int32"
    extra = dict(y_dtype="int32" if i32 else "uint16", zero_frac=0.85)
    P = Pair(gmf, oracle_mod, n, m, p, q, d, fam, nbr, nbc, precision=precision, **extra)
    Q = Pair(gmf, oracle_mod, n, m, p, q, d, fam, nbr, nbc, precision=precision,
             flags=gmf.GMF_FLAG_STAGED_UPLOAD if source == "pinned_staged" else 0, **extra)
    rng = np.random.default_rng(44)
    mats = [np.ascontiguousarray(np.minimum(P.prob.Y.astype(np.int64) + rng.poisson(0.3, P.prob.Y.shape), 65535)
                                 .astype(np.int32 if i32 else np.uint16)) for _ in range(4)]
    srcs = [torch.from_numpy(Y if i32 else Y.view(np.int16)).pin_memory() if source.startswith("pinned") else Y
            for Y in mats]
    for e, Y in enumerate(mats):
        P.gpu.update_y(Y)
        P.gpu.epoch(P.sigmas[e])
    Q.gpu.update_y_async(srcs[0])
    for e in range(len(mats)):
        Q.gpu.epoch(Q.sigmas[e])
        if e + 1 < len(mats):
            Q.gpu.update_y_async(srcs[e + 1])   # its upload overlaps this epoch
    torch.cuda.synchronize()
    assert P.gpu.count_buffers == 1
    assert Q.gpu.count_buffers == {"pinned": 2, "pinned_int32": 2, "unaligned_rows": 1,
                                   "pinned_staged": 1}.get(source, Q.gpu.count_buffers)
    a, b = P.gpu.get_params(), Q.gpu.get_params()
    for k in ("B", "Gamma", "U", "V"):
        np.testing.assert_array_equal(a[k], b[k])
    assert P.gpu.deviance() == Q.gpu.deviance()


def test_bad_sigma_is_rejected(gmf, oracle_mod):
    n, m, p, q, d, fam, nbr, nbc, extra = CASES["tiny_5x4"]
    P = Pair(gmf, oracle_mod, n, m, p, q, d, fam, nbr, nbc, **extra)
    with pytest.raises(gmf.GmfError) as e:
        P.gpu.epoch(np.zeros(P.nsw, dtype=np.int32))
    assert e.value.code == gmf.GMF_ERR_ARG
    with pytest.raises(gmf.GmfError):
        P.gpu.sweeps(P.sigmas[0], 0, P.nsw + 1)
