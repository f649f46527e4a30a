"""Stored oracle values for the 1000 x 500 Poisson workload (50 epochs, blocks
100 x 100): tests/golden/poisson_small_oracle.json, written by
tests/golden/make_golden.py, which calls only oracle/.

CPU: the oracle still produces them (within 1e-10: the host's libm may differ by
an ulp). GPU: the FP32 path follows the oracle's deviance at every one of the 50
epochs within 1e-4 (relative), and the tensor-core path ends within 1e-3."""
import json
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "poisson_small_oracle.json")


def _stored():
    with open(GOLDEN) as fh:
        return json.load(fh)


def test_oracle_reproduces_stored_trajectory(oracle_lib):
    from tests.golden.make_golden import trajectory
    dev, norms = trajectory()
    g = _stored()
    np.testing.assert_allclose(dev, g["deviance_per_epoch"], rtol=1e-10)
    for k, v in g["final_frobenius_norms"].items():
        assert norms[k] == pytest.approx(v, rel=1e-10)


@pytest.mark.gpu
@pytest.mark.parametrize("precision,tol_each,tol_final", [("fp32", 1e-4, 1e-4), ("mixed", None, 1e-3)])
def test_gpu_follows_stored_trajectory(precision, tol_each, tol_final):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2412_20509_gb300 as gmf
    w = synth.WORKLOADS["poisson_small"]
    prob = synth.workload_problem(w.name, seed=0)
    start = synth.crude_start(prob, w.d, seed=0)
    rp, cp = synth.partitions(w.n, w.m, 0)
    sig = synth.sweep_orders(w.n, w.m, w.nb_row, w.nb_col, w.epochs, 0)
    model = gmf.Model(torch.from_numpy(prob.Y).cuda(), prob.X, prob.Z, prob.offset, start, family=w.family,
                      nb_row=w.nb_row, nb_col=w.nb_col, row_perm=rp, col_perm=cp, settings=synth.fit_settings(),
                      precision=precision)
    ref = _stored()["deviance_per_epoch"]
    got = []
    for s in sig:
        model.epoch(s)
        got.append(model.deviance())
    if tol_each is not None:
        np.testing.assert_allclose(got, ref, rtol=tol_each)
    assert got[-1] == pytest.approx(ref[-1], rel=tol_final)
