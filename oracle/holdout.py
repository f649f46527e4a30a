"""FP64 out-of-sample metrics of Sec. 5.2 (test infrastructure only, like the
rest of ``oracle``): the fit is trained with a set V of held-out entries
treated as missing, and judged on V by

  Error    = sum_V [log{(1 + y) / (1 + mu)}]^2 / sum_V [log{(1 + y) / (1 + ybar_T)}]^2
  Deviance = sum_V D(y, mu) / sum_V D(y, ybar_T)

where ybar_T is the mean of the training (observed) entries and D the Poisson
unit deviance of Table S1 (the paper reports the relative Poisson deviance for
every model). Written directly from those two definitions.
"""
import numpy as np


def poisson_unit_deviance(y, mu):
    """2 [y log(y / mu) - (y - mu)], with 0 log 0 = 0 (Table S1)."""
    y = np.asarray(y, float)
    mu = np.asarray(mu, float)
    pos = y > 0
    ylog = np.zeros(np.broadcast(y, mu).shape)
    yb, mb = np.broadcast_to(y, ylog.shape), np.broadcast_to(mu, ylog.shape)
    ylog[pos] = yb[pos] * np.log(yb[pos] / mb[pos])
    return 2.0 * (ylog - (y - mu))


def holdout_metrics(Y, observed, mu):
    """Y: n x m counts; observed: boolean mask of the training entries (the rest
    is the held-out set V); mu: n x m fitted means. Returns (Error, Deviance,
    ybar_T, |V|)."""
    Y = np.asarray(Y, float)
    obs = np.asarray(observed, bool)
    V = ~obs
    ybar = Y[obs].mean()
    y, m_ = Y[V], np.asarray(mu, float)[V]
    err = np.sum(np.log((1 + y) / (1 + m_)) ** 2) / np.sum(np.log((1 + y) / (1 + ybar)) ** 2)
    dev = np.sum(poisson_unit_deviance(y, m_)) / np.sum(poisson_unit_deviance(y, ybar))
    return float(err), float(dev), float(ybar), int(V.sum())
