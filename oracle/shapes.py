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


def nb_gene_loglik(Y, mu, alpha, W=None, observed=None):
    """Per-gene NB log-likelihood of Table S1's density (App. B), lgamma terms
    included: sum_i w [lgamma(y + a) - lgamma(a) - lgamma(y + 1) + a log(a / (a + mu))
    + y log(mu / (a + mu))] over each column's observed entries; alpha per column."""
    from scipy.special import gammaln
    Y = np.asarray(Y, float)
    mu = np.asarray(mu, float)
    a = np.broadcast_to(np.asarray(alpha, float), (Y.shape[1],))[None, :]
    w = np.ones_like(Y) if W is None else np.asarray(W, float)
    if observed is not None:
        w = w * np.asarray(observed, bool)
    term = (gammaln(Y + a) - gammaln(a) - gammaln(Y + 1.0) + a * np.log(a / (a + mu))
            + np.where(Y > 0, Y * np.log(mu / (a + mu)), 0.0))
    return (w * term).sum(axis=0)


def gene_shape_ml(Y, mu, start, iters=30, tol=1e-6, lo=1e-3, hi=1e4, W=None, observed=None):
    """Maximum-likelihood NB shape per gene with the means held fixed, by
    Newton's method in theta = log alpha, all genes at once. Per gene and
    iteration, from the derivatives of nb_gene_loglik in alpha,
      l'  = sum w [psi(y + a) - psi(a) + log(a / (a + mu)) + (mu - y) / (a + mu)]
      l'' = sum w [psi'(y + a) - psi'(a) + mu / (a (a + mu)) + (y - mu) / (a + mu)^2],
    g = a l' and h = a l' + a^2 l'' are the derivatives in theta; the step is
    -g / h where h < 0, else +-1 towards increasing l; steps are capped at 1,
    theta is kept in [log lo, log hi], and a gene stops once its step is at
    most tol. Returns (alpha, iterations made)."""
    from scipy.special import digamma, polygamma
    Y = np.asarray(Y, float)
    mu = np.asarray(mu, float)
    w = np.ones_like(Y) if W is None else np.asarray(W, float)
    if observed is not None:
        w = w * np.asarray(observed, bool)
    alpha = np.clip(np.broadcast_to(np.asarray(start, float), (Y.shape[1],)).copy(), lo, hi)
    done = np.zeros(Y.shape[1], bool)
    tlo, thi = np.log(lo), np.log(hi)
    it = 0
    while it < iters:
        it += 1
        a = alpha[None, :]
        l1 = (w * (digamma(Y + a) - digamma(a) + np.log(a / (a + mu)) + (mu - Y) / (a + mu))).sum(axis=0)
        l2 = (w * (polygamma(1, Y + a) - polygamma(1, a) + mu / (a * (a + mu)) + (Y - mu) / (a + mu) ** 2)).sum(axis=0)
        g = alpha * l1
        h = alpha * l1 + alpha * alpha * l2
        step = np.where(h < 0, -g / np.where(h < 0, h, -1.0), np.sign(g))
        step = np.clip(step, -1.0, 1.0)
        th = np.log(alpha)
        tn = np.clip(th + step, tlo, thi)
        new = np.where(done, alpha, np.exp(tn))
        done = done | (np.abs(tn - th) <= tol)
        alpha = new
        if done.all():
            break
    return alpha, it
