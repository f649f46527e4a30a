"""Per-cell projection of new cells by Fisher scoring, FP64 numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Given the column-side parameters (B, V, Z) and the NB shape fixed, each new
cell i is the row problem of Sec. 3 (the equations separate by rows given V):
minimise  -sum_j log f(y_ij; mu_ij) + lam_G/2 |gamma_i|^2 + lam_U/2 |u_i|^2
with eta_ij = o_i + x_i'beta_j + gamma_i'z_j + u_i'v_j, over theta_i =
[gamma_i, u_i]. One Fisher-scoring step (the row step of AIRWLS, Sec. 3.1) is

  theta <- theta + (R' diag(Dddot_i) R + Lambda)^-1 (R' Ddot_i - Lambda theta),
  R = [Z, V]  (m x (q+d)).

The start: u_i from the caller (zeros for a cold start) and, for q = 1 with
Z = 1, gamma_i in closed form as the Poisson intercept given the rest,
gamma_i = log(sum_j y_ij / sum_j exp(eta_ij without gamma)).
"""
from __future__ import annotations

import numpy as np


def _derivs(family, y, eta, alpha, clamp=30.0):
    mu = np.exp(np.clip(eta, -clamp, clamp))
    if family == "poisson":
        nu = mu
    else:
        nu = mu * (1.0 + mu / alpha)
    gdot = 1.0 / mu
    return mu, (y - mu) / (nu * gdot), 1.0 / (nu * gdot * gdot)


def deviance_rows(family, Y, mu, alpha):
    Y = np.asarray(Y, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        ylog = np.where(Y > 0, Y * np.log(np.where(Y > 0, Y, 1.0) / mu), 0.0)
    if family == "poisson":
        D = 2.0 * (ylog - (Y - mu))
    else:
        D = 2.0 * (ylog - (Y + alpha) * np.log((Y + alpha) / (mu + alpha)))
    return D.sum(axis=1)


def project_cells(Y, X, offset, B, Z, V, *, family, alpha, U_start=None, n_steps=3,
                  lam_gamma=0.0, lam_u=1.0, gamma_closed_form=True):
    """Fisher scoring of [gamma_i, u_i] for each row of Y; returns (U, Gamma, dev)."""
    Y = np.asarray(Y, dtype=np.float64)
    n, m = Y.shape
    q = Z.shape[1]
    d = V.shape[1]
    R = np.concatenate([Z, V], axis=1)
    base = X @ B.T + (offset[:, None] if offset is not None else 0.0)
    U = np.zeros((n, d)) if U_start is None else np.array(U_start, dtype=np.float64)
    G = np.zeros((n, q))
    if gamma_closed_form and q >= 1:
        rest = base + U @ V.T
        G[:, 0] = np.log(np.maximum(Y.sum(axis=1), 0.5) / np.exp(np.clip(rest, -30, 30)).sum(axis=1))
    lam = np.array([lam_gamma] * q + [lam_u] * d)
    theta = np.concatenate([G, U], axis=1)
    for _ in range(n_steps):
        eta = base + theta @ R.T
        mu, dd, ddd = _derivs(family, Y, eta, alpha)
        grad = dd @ R - lam * theta                      # R' Ddot_i - Lambda theta
        for i in range(n):
            F = (R * ddd[i][:, None]).T @ R + np.diag(lam)
            theta[i] += np.linalg.solve(F, grad[i])
    eta = base + theta @ R.T
    mu = np.exp(np.clip(eta, -30, 30))
    return theta[:, q:], theta[:, :q], deviance_rows(family, Y, mu, alpha)
