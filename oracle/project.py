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

Step control (a reading: the paper states none for this row problem; its own
AIRWLS runs shorten every step by a fixed 0.2, App. C). Each pass evaluates the
penalised objective f(theta) = 0.5 dev_i(theta) + 0.5 theta' Lambda theta at
the current point. A point with f <= f_best + 1e-5 (1 + |f_best|) is accepted
and the Fisher step is taken from it; otherwise the last step is halved and
tried again from the best point. The slack keeps rounding noise near the
optimum from counting as an increase; far from it, where plain Fisher scoring
overshoots, increases are large. n_steps passes take at most n_steps steps;
the best point and its deviance are returned.
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


SLACK = 1e-5


def project_cells(Y, X, offset, B, Z, V, *, family, alpha, U_start=None, n_steps=3,
                  lam_gamma=0.0, lam_u=1.0, gamma_closed_form=True, halving=True):
    """Fisher scoring of [gamma_i, u_i] for each row of Y; returns (U, Gamma, dev).

    halving=False takes every Fisher step as it comes (plain Fisher scoring)."""
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
    best = theta.copy()
    f_best = np.full(n, np.inf)
    dev_best = np.zeros(n)
    step = np.zeros_like(theta)
    for k in range(n_steps + 1):           # pass k evaluates theta; passes 0..n_steps-1 also step
        eta = base + theta @ R.T
        mu, dd, ddd = _derivs(family, Y, eta, alpha)
        dev = deviance_rows(family, Y, mu, alpha)
        f = 0.5 * dev + 0.5 * (lam * theta ** 2).sum(axis=1)
        grad = dd @ R - lam * theta                      # R' Ddot_i - Lambda theta
        for i in range(n):
            if k == 0 or not halving or f[i] <= f_best[i] + SLACK * (1.0 + abs(f_best[i])):
                best[i], f_best[i], dev_best[i] = theta[i], f[i], dev[i]
                if k < n_steps:
                    F = (R * ddd[i][:, None]).T @ R + np.diag(lam)
                    step[i] = np.linalg.solve(F, grad[i])
                    theta[i] = best[i] + step[i]
            else:
                step[i] *= 0.5
                theta[i] = best[i] + step[i]
    return best[:, q:], best[:, :q], dev_best
