"""Writes tests/golden/poisson_small_oracle.json: the FP64 oracle's deviance after
each of the 50 epochs of the 1000 x 500 Poisson workload (d = 5, p = 2, q = 1,
blocks 100 x 100, seed 0, default settings) and its final parameters' norms.
Calls only oracle/ (and the seeded input module synth/).

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth  # noqa: E402


def trajectory():
    w = synth.WORKLOADS["poisson_small"]
    prob = synth.workload_problem(w.name, seed=0)
    start = synth.crude_start(prob, w.d, seed=0)
    rp, cp = synth.partitions(w.n, w.m, 0)
    sig = synth.sweep_orders(w.n, w.m, w.nb_row, w.nb_col, w.epochs, 0)
    f = oracle.OracleFit(prob.Y, prob.X, prob.Z, prob.offset, start, family=w.family, nb_row=w.nb_row,
                         nb_col=w.nb_col, row_perm=rp, col_perm=cp, settings=synth.fit_settings())
    dev = []
    for s in sig:
        f.epoch(s)
        dev.append(f.deviance())
    norms = {k: float(np.linalg.norm(getattr(f, k))) for k in ("B", "G", "U", "V")}
    return dev, norms


if __name__ == "__main__":
    oracle.build()
    dev, norms = trajectory()
    out = {"workload": "poisson_small: 1000 x 500 int32 Poisson, d=5, p=2, q=1, blocks 100x100, 50 epochs, seed 0, "
                       "default settings (lambda = (0, 0, 1, 0), a1 = 0.1, a2 = 0.01, k0 = 0.01)",
           "written_by": "tests/golden/make_golden.py (FP64 oracle, oracle/gmf_oracle.c)",
           "deviance_per_epoch": dev, "final_frobenius_norms": norms}
    with open(os.path.join(HERE, "poisson_small_oracle.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", len(dev), "epochs; final deviance", dev[-1])
