"""Rank selection over a grid of fits of different latent rank d (Sec. 4.2).

The quantities come from the library (each fit's handle): the log-likelihood
and Pearson statistic of the observed entries (gmf_loglik), the held-out error
and relative Poisson deviance when entries were held out (gmf_holdout), and
the singular values of a high-rank fit after Algorithm 2's (B1)
orthogonalisation (V'V = I and U'U diagonal, so s_k^2 = (U'U)_kk). This module
only combines them:

* information criteria AIC = -2 l + 2 k and BIC = -2 l + k log N, with k =
  m p + n q + (n + m) d free parameters (+1 for the NB shape) and N the
  observed entries;
* out-of-sample error: the rank with the smallest held-out deviance (or error);
* spectral thresholding: the rank with the largest ratio of consecutive
  eigenvalues s_k^2 / s_{k+1}^2 of the high-rank fit (the eigenvalue-ratio
  form of the elbow rule; the paper leaves the rule open);
* the Pearson dispersion estimate of App. B over the effective degrees of
  freedom N_eff = n m - m p - n q - (n + m) d - 1.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["free_params", "information_criteria", "pearson_dispersion", "eigen_ratio_rank", "singular_values",
           "fit_summary", "select_rank"]


def free_params(n, m, p, q, d, family):
    """Free parameters of a fit: B (m x p), Gamma (n x q), U (n x d), V (m x d), and the NB shape."""
    return m * p + n * q + (n + m) * d + (1 if family == "negbin" else 0)


def information_criteria(loglik, k, n_obs):
    """(AIC, BIC) of a log-likelihood with k free parameters and n_obs observations."""
    return -2.0 * loglik + 2.0 * k, -2.0 * loglik + k * math.log(n_obs)


def pearson_dispersion(stat, n, m, p, q, d):
    """Pearson estimate of phi: the statistic over N_eff = n m - m p - n q - (n + m) d - 1."""
    return stat / (n * m - m * p - n * q - (n + m) * d - 1)


def eigen_ratio_rank(sv):
    """The k in [1, len(sv) - 1] with the largest s_k^2 / s_{k+1}^2 (singular values in any order)."""
    s = np.sort(np.asarray(sv, dtype=np.float64))[::-1]
    lam = s * s
    return int(np.argmax(lam[:-1] / lam[1:]) + 1)


def singular_values(model):
    """Singular values of U V' of a (B1-orthogonalised) fit: the column norms of U, largest first."""
    U = model.get_params()["U"]
    return np.sort(np.sqrt((U * U).sum(axis=0)))[::-1]


def fit_summary(model, family, Ytrue=None):
    """The per-fit quantities of the selection from the library: log-likelihood, AIC, BIC, Pearson
    dispersion, deviance and, when entries were held out (Ytrue given), the held-out metrics."""
    n, m, p, q, d = model.dims
    ll = model.loglik()
    k = free_params(n, m, p, q, d, family)
    aic, bic = information_criteria(ll["loglik"], k, ll["n_obs"])
    out = {"d": d, "loglik": ll["loglik"], "free_params": k, "aic": aic, "bic": bic,
           "pearson_phi": pearson_dispersion(ll["pearson"], n, m, p, q, d), "deviance": model.deviance()}
    if Ytrue is not None:
        h = model.holdout(Ytrue)
        out.update(heldout_error=h["error"], heldout_deviance=h["deviance"])
    return out


def select_rank(summaries, spectrum=None):
    """The rank chosen by each criterion from fit_summary() dicts (and, optionally, the singular values of
    the highest-rank fit for spectral thresholding)."""
    pick = lambda key: min(summaries, key=lambda s: s[key])["d"]
    out = {"aic": pick("aic"), "bic": pick("bic")}
    if all("heldout_deviance" in s for s in summaries):
        out["heldout_deviance"] = pick("heldout_deviance")
        out["heldout_error"] = pick("heldout_error")
    if spectrum is not None:
        out["eigen_ratio"] = eigen_ratio_rank(spectrum)
    return out
