"""Per-gene negative binomial shapes (test infrastructure only, like the rest
of ``oracle``): the moment estimator of App. B, sum w mu^2 / sum w {(y - mu)^2
- mu}, applied to each gene's column instead of the whole matrix. Floored at
eps as in App. B; a gene whose denominator is not positive shows no
overdispersion and gets the cap (a nearly Poisson gene)."""
import numpy as np


def gene_shape_moments(Y, mu, W=None, observed=None, eps=1e-8, cap=1e6):
    Y = np.asarray(Y, float)
    mu = np.asarray(mu, float)
    w = np.ones_like(Y) if W is None else np.asarray(W, float)
    if observed is not None:
        w = w * np.asarray(observed, bool)
    num = (w * mu * mu).sum(axis=0)
    den = (w * ((Y - mu) ** 2 - mu)).sum(axis=0)
    out = np.full(Y.shape[1], float(cap))
    pos = den > 0
    out[pos] = np.minimum(np.maximum(num[pos] / den[pos], eps), cap)
    return out
