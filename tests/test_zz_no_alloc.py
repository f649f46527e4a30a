"""gmf_deviance_noalloc: the deviance for callers that cannot allocate device
memory (plug-ins in frameworks that own all device memory through their own
pool). Called through the C ABI twice in a row and checked against the
handle-based gmf_deviance at the deviance tolerance of the other tests (1e-6
relative: FP32 unit deviances, FP64 total). Collected last on purpose."""
import ctypes as C

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


def _factors(prob, params, ld):
    n, m = prob.Y.shape
    p, q, d = prob.X.shape[1], prob.Z.shape[1], params["U"].shape[1]
    L = np.zeros((n, ld), dtype=np.float32)
    R = np.zeros((m, ld), dtype=np.float32)
    L[:, 0] = prob.offset
    L[:, 1:1 + p] = prob.X
    L[:, 1 + p:1 + p + q] = params["Gamma"]
    L[:, 1 + p + q:1 + p + q + d] = params["U"]
    R[:, 0] = 1.0
    R[:, 1:1 + p] = params["B"]
    R[:, 1 + p:1 + p + q] = prob.Z
    R[:, 1 + p + q:1 + p + q + d] = params["V"]
    return L, R, 1 + p + q + d


@pytest.mark.parametrize("family,y_dtype,weights", [("negbin", "int32", True), ("poisson", "uint16", False)])
def test_noalloc_deviance_matches_handle_twice(gmf, family, y_dtype, weights):
    n, m, d = 900, 640, 6
    prob = synth.make_problem(n, m, 3, 1, d, family, seed=21, y_dtype=y_dtype,
                              zero_frac=0.85 if family == "negbin" else None, offset=True)
    start = synth.crude_start(prob, d, seed=21)
    rp, cp = synth.partitions(n, m, 21)
    W = np.random.default_rng(5).uniform(0.5, 1.5, (n, m)).astype(np.float32) if weights else None
    Yd = torch.from_numpy(prob.Y.astype(np.int32) if y_dtype == "int32" else prob.Y.view(np.int16)).cuda()
    Wd = None if W is None else torch.from_numpy(W).cuda()
    model = gmf.Model(torch.from_numpy(prob.Y).cuda() if y_dtype == "int32" else prob.Y, prob.X, prob.Z, prob.offset,
                      start, family=family, nb_row=128, nb_col=128, row_perm=rp, col_perm=cp,
                      settings=synth.fit_settings(), W=Wd if W is not None else None)
    for s in synth.sweep_orders(n, m, 128, 128, 2, 21):
        model.epoch(s)
    ref = model.deviance()
    params = model.get_params()
    L, R, K = _factors(prob, params, 12)
    Ld, Rd = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    ydt = gmf.GMF_Y_INT32 if y_dtype == "int32" else gmf.GMF_Y_UINT16
    fam = gmf.FAMILIES[family]
    for call in range(2):
        rc = gmf.lib().gmf_deviance_noalloc(Yd.data_ptr(), ydt, None if Wd is None else Wd.data_ptr(), n, m,
                                            Ld.data_ptr(), Rd.data_ptr(), K, 12, fam, float(params["alpha"]), 30.0,
                                            out[call:call + 1].data_ptr(), stream)
        assert rc == gmf.GMF_OK, gmf.lib().gmf_last_error()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert got[0] == got[1]
    assert got[0] == pytest.approx(ref, rel=1e-6)


def test_noalloc_rejects_sizes_beyond_scratch(gmf):
    dummy = torch.zeros(4, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = dummy.data_ptr()
    rc = gmf.lib().gmf_deviance_noalloc(p, gmf.GMF_Y_INT32, None, 1 << 20, 1 << 20, p, p, 4, 4, gmf.GMF_POISSON, 1.0,
                                        30.0, out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == gmf.GMF_ERR_ARG
    assert "262144" in gmf.lib().gmf_last_error().decode()


@pytest.mark.parametrize("family,shift,y_mean", [("poisson", 6.0, None), ("negbin", 6.0, None),
                                                 ("poisson", 29.0, 5.0), ("negbin", 29.0, 5.0)])
def test_noalloc_large_counts_and_eta_near_the_clamp(gmf, family, shift, y_mean):
    """Counts far above 256 (beyond the handle kernel's log tables: eta around
    6, counts around 400, where y log(y/mu) - (y - mu) is a small difference of
    large terms) and eta around 29, partly beyond the clamp at 30 (small
    counts, so each term is close to 2 mu): the two deviance kernels and the
    FP64 oracle agree. Bar 1e-5: eta in FP32 carries an error of about
    |eta| * 2^-24, which exp passes on to mu (~2e-6 relative near the clamp)."""
    import oracle
    oracle.build()
    n, m, d = 300, 256, 4
    prob = synth.make_problem(n, m, 2, 1, d, family, seed=8, offset=True)
    params = dict(B=prob.B.copy(), Gamma=prob.Gamma.copy(), U=0.5 * prob.U, V=0.5 * prob.V, alpha=2.0)
    params["B"][:, 0] += shift
    eta = prob.X @ params["B"].T + params["Gamma"] @ prob.Z.T + params["U"] @ params["V"].T + prob.offset[:, None]
    rng = np.random.default_rng(8)
    mean = np.exp(np.clip(eta, -30, 20)) if y_mean is None else np.full(eta.shape, y_mean)
    prob.Y = rng.poisson(mean).astype(np.int32)
    if y_mean is None:
        assert np.median(prob.Y) > 256
    else:
        assert eta.max() > 30 > eta.min() > 20
    rp, cp = synth.partitions(n, m, 8)
    model = gmf.Model(torch.from_numpy(prob.Y).cuda(), prob.X, prob.Z, prob.offset, params, family=family, nb_row=128,
                      nb_col=128, row_perm=rp, col_perm=cp, settings=synth.fit_settings())
    ref = model.deviance()
    stored = model.get_params()   # the handle's FP32 parameters, as doubles
    L, R, K = _factors(prob, stored, 8)
    Yd = torch.from_numpy(prob.Y).cuda()
    Ld, Rd = torch.from_numpy(L).cuda(), torch.from_numpy(R).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = gmf.lib().gmf_deviance_noalloc(Yd.data_ptr(), gmf.GMF_Y_INT32, None, n, m, Ld.data_ptr(), Rd.data_ptr(), K, 8,
                                        gmf.FAMILIES[family], float(stored["alpha"]), 30.0, out.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
    assert rc == gmf.GMF_OK, gmf.lib().gmf_last_error()
    got = float(out.cpu()[0])
    orc = oracle.OracleFit(prob.Y, prob.X, prob.Z, prob.offset, stored, family=family, nb_row=128, nb_col=128,
                           row_perm=rp, col_perm=cp, settings=synth.fit_settings())
    exact = orc.deviance()
    assert got == pytest.approx(ref, rel=1e-5)
    assert got == pytest.approx(exact, rel=1e-5)
    assert ref == pytest.approx(exact, rel=1e-5)


def test_noalloc_takes_no_device_memory(gmf):
    """Free device memory is the same before and after calls (after the first
    call on the device, which only looks up the static array's address)."""
    n, m = 256, 192
    Y = torch.zeros((n, m), dtype=torch.int32, device="cuda")
    L = torch.zeros((n, 4), dtype=torch.float32, device="cuda")
    R = torch.zeros((m, 4), dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    args = (Y.data_ptr(), gmf.GMF_Y_INT32, None, n, m, L.data_ptr(), R.data_ptr(), 1, 4, gmf.GMF_POISSON, 1.0, 30.0,
            out.data_ptr(), st)
    assert gmf.lib().gmf_deviance_noalloc(*args) == gmf.GMF_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        assert gmf.lib().gmf_deviance_noalloc(*args) == gmf.GMF_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert float(out.cpu()[0]) == pytest.approx(2.0 * n * m)   # y = 0, eta = 0: 2 mu per entry
