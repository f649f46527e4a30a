"""FP64 reference of the rank-selection quantities of Sec. 4.2 (test
infrastructure only, like the rest of ``oracle``):

* the log-likelihood of the observed entries with the full densities of Table
  S1's Poisson and negative binomial laws (log-gamma terms included), from the
  fitted means;
* AIC = -2 l + 2 k and BIC = -2 l + k log N, with k the free parameters
  m p + n q + (n + m) d (+1 for the NB shape) and N the observed entries;
* the Pearson dispersion estimate of App. B, sum w (y - mu)^2 / nu(mu) over
  N_eff = n m - m p - n q - (n + m) d - 1;
* spectral thresholding: with the singular values s_1 >= ... of a high-rank
  fit, the rank with the largest ratio of consecutive eigenvalues s_k^2 /
  s_{k+1}^2 (the paper cites spectral thresholding without fixing a rule;
  this is the eigenvalue-ratio reading).
"""
import math

import numpy as np
from scipy.special import gammaln


def loglik(Y, mu, family, alpha=None, W=None, observed=None):
    Y = np.asarray(Y, float)
    mu = np.asarray(mu, float)
    if family == "poisson":
        lf = Y * np.log(mu) - mu - gammaln(Y + 1)
    else:
        a = np.asarray(alpha, float)      # one shape, or one per gene (broadcast along the columns)
        lf = (gammaln(Y + a) - gammaln(a) - gammaln(Y + 1) + a * np.log(a / (a + mu)) + Y * np.log(mu / (a + mu)))
    if W is not None:
        lf = lf * W
    if observed is not None:
        lf = lf[np.asarray(observed, bool)]
    return float(lf.sum())


def pearson(Y, mu, family, alpha=None, W=None, observed=None):
    Y = np.asarray(Y, float)
    mu = np.asarray(mu, float)
    nu = mu if family == "poisson" else mu * (1 + mu / np.asarray(alpha, float))
    t = (Y - mu) ** 2 / nu
    if W is not None:
        t = t * W
    if observed is not None:
        t = t[np.asarray(observed, bool)]
    return float(t.sum())


def free_params(n, m, p, q, d, family):
    return m * p + n * q + (n + m) * d + (1 if family == "negbin" else 0)


def aic_bic(ll, k, n_obs):
    return -2.0 * ll + 2.0 * k, -2.0 * ll + k * math.log(n_obs)


def pearson_dispersion(stat, n, m, p, q, d):
    return stat / (n * m - m * p - n * q - (n + m) * d - 1)


def eigen_ratio_rank(singular_values):
    s = np.sort(np.asarray(singular_values, float))[::-1]
    lam = s ** 2
    return int(np.argmax(lam[:-1] / lam[1:]) + 1)
