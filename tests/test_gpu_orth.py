"""gmf_orthogonalize (Algorithm 2) against the FP64 oracle (oracle/orth.py, the
explicit n x m SVD route) for (B1), (B2), (B3).

Tolerance: the device computes in FP64 but stores the result in FP32
(relative spacing 6e-8) and reads FP32 parameters; the d x d factorizations
amplify that by the condition of U and V (~10 here): 1e-5 max-norm relative per
matrix, and eta unchanged within 1e-5.
"""
import numpy as np
import pytest

import synth
from tests.test_gpu_parity import Pair, rel

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


def eta(X, Z, off, P):
    return X @ P["B"].T + P["Gamma"] @ Z.T + P["U"] @ P["V"].T + off[:, None]


@pytest.mark.parametrize("mode", ["B1", "B2", "B3"])
@pytest.mark.parametrize("q", [1, 2])
def test_orthogonalize_matches_oracle(gmf, oracle_mod, mode, q):
    from oracle.orth import orthogonalize
    P = Pair(gmf, oracle_mod, 900, 640, 3, q, 6, "negbin", 256, 128, zero_frac=0.8)
    for e in range(3):
        P.gpu.epoch(P.sigmas[e])
    before = P.gpu.get_params()
    dev_before = P.gpu.deviance()
    X32 = P.prob.X.astype(np.float32).astype(np.float64)
    Z32 = P.prob.Z.astype(np.float32).astype(np.float64)
    off32 = P.prob.offset.astype(np.float32).astype(np.float64)
    B, G, U, V = orthogonalize(X32, Z32, before["B"], before["Gamma"], before["U"], before["V"], mode)
    P.gpu.orthogonalize(mode)
    after = P.gpu.get_params()
    for k, ref in (("B", B), ("Gamma", G), ("U", U), ("V", V)):
        assert rel(after[k], ref) <= 1e-5, (mode, k, rel(after[k], ref))
    e0, e1 = eta(X32, Z32, off32, before), eta(X32, Z32, off32, after)
    assert rel(e1, e0) <= 1e-5
    assert P.gpu.deviance() == pytest.approx(dev_before, rel=1e-5)
    ema = P.gpu.get_ema()
    assert not ema["Gb_row"].any() and not ema["Hb_col"].any() and not ema["cnt_row"].any()
    # identifiability constraints hold on the result
    assert np.abs(X32.T @ after["Gamma"]).max() <= 1e-4 * np.abs(after["Gamma"]).max() * len(X32) ** 0.5
    assert np.abs(X32.T @ after["U"]).max() <= 1e-4 * np.abs(after["U"]).max() * len(X32) ** 0.5
    if mode == "B1":
        np.testing.assert_allclose(after["V"].T @ after["V"], np.eye(6), atol=1e-5)


def test_fit_continues_after_orthogonalize(gmf, oracle_mod):
    P = Pair(gmf, oracle_mod, 900, 640, 3, 1, 6, "negbin", 256, 128, zero_frac=0.8)
    for e in range(3):
        P.gpu.epoch(P.sigmas[e])
    P.gpu.orthogonalize("B1")
    d0 = P.gpu.deviance()
    for e in range(3, 6):
        P.gpu.epoch(P.sigmas[e])
    assert P.gpu.deviance() < d0
