"""Failure detection in the forms that fault, trap or hang no GPU.

* A non-finite parameter put in from the host (gmf_set_params) makes the next
  epoch's updates non-finite; the kernels flag it in the handle's status word
  and the next synchronous call returns GMF_ERR_NONFINITE.
* The persistent epoch's strip waits are bounded by the global timer. With the
  testing hook gmf_set_wait_limit every dependency count is raised by one, so
  no wait can be satisfied: each gives up after a 2 ms limit, the launch ends
  by itself, the next synchronous call returns GMF_ERR_TIMEOUT, and the CUDA
  context stays usable (a new handle fits and matches a fit that never timed
  out).
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


def _model(gmf, prob, d, nbr, nbc, seed, precision="fp32", flags=0, **settings):
    n, m = prob.Y.shape
    rp, cp = synth.partitions(n, m, seed)
    start = synth.crude_start(prob, d, seed=seed)
    Y = torch.from_numpy(prob.Y.view(np.int16) if prob.Y.dtype == np.uint16 else prob.Y).cuda()
    return gmf.Model(Y, prob.X, prob.Z, prob.offset, start, family=prob.family, nb_row=nbr, nb_col=nbc,
                     row_perm=rp, col_perm=cp, settings=synth.fit_settings(**settings), precision=precision,
                     flags=flags)


@pytest.mark.parametrize("precision", ["fp32", "mixed"])
def test_nonfinite_parameter_is_reported(gmf, precision):
    n, m, d, nbr, nbc = 600, 512, 5, 200, 128
    prob = synth.make_problem(n, m, 3, 1, d, "negbin", seed=31, zero_frac=0.8, offset=True)
    sig = synth.sweep_orders(n, m, nbr, nbc, 2, 31)
    model = _model(gmf, prob, d, nbr, nbc, 31, precision)
    model.epoch(sig[0])
    assert np.isfinite(model.deviance())
    par = model.get_params()
    par["U"][7, 1] = np.nan          # one cell's score, from the host
    model.set_params(par)
    model.epoch(sig[1])
    with pytest.raises(gmf.GmfError) as e:
        model.deviance()
    assert e.value.code == gmf.GMF_ERR_NONFINITE


def test_persistent_strip_wait_times_out_and_the_context_survives(gmf):
    # 6000 x 1024 NB, blocks 500 x 512: 12 row chunks, 2 column chunks, clusters of 4 x 4 tiles; a fixed shape
    # so that the epoch is one persistent launch
    n, m, d, nbr, nbc = 6000, 1024, 10, 500, 512
    prob = synth.make_problem(n, m, 2, 1, d, "negbin", seed=5, zero_frac=0.5, offset=True)
    sig = synth.sweep_orders(n, m, nbr, nbc, 2, 5)
    model = _model(gmf, prob, d, nbr, nbc, 5, "mixed", flags=gmf.GMF_FLAG_PERSIST)
    if model.epoch_mode != "persistent":
        pytest.skip("the persistent epoch is not available for this shape on this device")
    model.set_wait_limit(2_000_000, 1)            # 2 ms per wait; every count one visit short
    torch.cuda.synchronize()
    model.epoch(sig[0])
    torch.cuda.synchronize()                      # the launch ends by itself
    with pytest.raises(gmf.GmfError) as e:
        model.deviance()
    assert e.value.code == gmf.GMF_ERR_TIMEOUT
    del model
    # the context is still usable: a new handle's persistent epoch equals a cluster-launch epoch bit for bit
    fresh = _model(gmf, prob, d, nbr, nbc, 5, "mixed", flags=gmf.GMF_FLAG_PERSIST)
    ref = _model(gmf, prob, d, nbr, nbc, 5, "mixed")
    for s in sig:
        fresh.epoch(s)
        ref.epoch(s)
    a, b = fresh.get_params(), ref.get_params()
    for k in ("U", "V", "B", "Gamma"):
        np.testing.assert_array_equal(a[k], b[k])
    assert fresh.deviance() == ref.deviance()


def test_wait_limit_hook_rejects_bad_values(gmf):
    prob = synth.make_problem(64, 32, 2, 1, 2, "poisson", seed=1)
    model = _model(gmf, prob, 2, 32, 16, 1)
    for bad in ((-1, 0), (0, -1), (10 ** 12, 0)):
        with pytest.raises(gmf.GmfError) as e:
            model.set_wait_limit(*bad)
        assert e.value.code == gmf.GMF_ERR_ARG
    model.set_wait_limit(0, 0)
