"""FP64 reference of the parameter initialisation of Sec. 4.1 in its
least-squares form (test infrastructure only, like the rest of ``oracle``).

The paper starts Algorithm 1 from column GLMs for B, row GLMs for Gamma given
X B', and the leading singular vectors of a residual matrix for U (then column
GLMs for V); for high-dimensional data it replaces the GLM fits by ordinary
least squares on the link-transformed response, with U and V from the
truncated SVD of the residual. That form, step by step:

  z_ij  = log(y_ij + 1/2)                      (the log link applied to the counts, shifted off zero)
  B     = argmin || z - o 1' - X B' ||_F       (least squares, one column of z per gene)
  Gamma = argmin || E1 - Gamma Z' ||_F,  E1 = z - o 1' - X B'
  E2    = E1 - Gamma Z'
  E2   ~= P diag(s) Q' (the d leading singular triplets),  U = P diag(s)^(1/2),  V = Q diag(s)^(1/2)

(the 1/2 shift and the even split of s between U and V are the readings of
the points the paper leaves open). ``fit_loadings`` is the paper's last step,
the column GLMs for V given U.
"""
import numpy as np


def init_ols(Y, X, Z, offset, d):
    """B (m x p), Gamma (n x q), U (n x d), V (m x d) and the singular values s (length d)."""
    Y = np.asarray(Y, float)
    n, m = Y.shape
    off = np.zeros(n) if offset is None else np.asarray(offset, float)
    zt = np.log(Y + 0.5) - off[:, None]
    B = np.linalg.lstsq(X, zt, rcond=None)[0].T                 # m x p
    E1 = zt - X @ B.T
    Gamma = np.linalg.lstsq(Z, E1.T, rcond=None)[0].T           # n x q
    E2 = E1 - Gamma @ Z.T
    if d == 0:
        return B, Gamma, np.zeros((n, 0)), np.zeros((m, 0)), np.zeros(0)
    P, s, Qt = np.linalg.svd(E2, full_matrices=False)
    r = np.sqrt(s[:d])
    return B, Gamma, P[:, :d] * r, Qt[:d].T * r, s[:d]


# ---------------------------------------------------------------- column GLMs for the loadings (Sec. 4.1)

def _count_derivs(family, y, eta, alpha, clamp=30.0):
    """mu, Ddot / w and Dddot / w of Sec. 3 for the log link (Poisson, NB)."""
    mu = np.exp(np.clip(eta, -clamp, clamp))
    nu = mu if family == "poisson" else mu * (1.0 + mu / alpha)
    return mu, (y - mu) * mu / nu, mu * mu / nu


def _count_deviance(family, y, mu, alpha):
    """Unit deviances of Table S1 (App. B for NB), 0 log 0 = 0."""
    with np.errstate(divide="ignore", invalid="ignore"):
        ylog = np.where(y > 0, y * np.log(np.where(y > 0, y, 1.0) / mu), 0.0)
    if family == "poisson":
        return 2.0 * (ylog - (y - mu))
    return 2.0 * (ylog - (y + alpha) * np.log((y + alpha) / (mu + alpha)))


LOADINGS_SLACK = 1e-5


def fit_loadings(Y, X, Z, offset, B, Gamma, U, V0, *, family, alpha, lam_v=0.0, n_steps=8, W=None,
                 margins=False):
    """The last step of Sec. 4.1: with the scores U and the regression effects
    B, Gamma fixed, one GLM per gene j for its loadings v_j, the scores as the
    design and o_i + x_i'beta_j + gamma_i'z_j as the offset. Each gene
    minimises f_j(v) = 0.5 sum_i w_ij D(y_ij, mu_ij) + 0.5 lam_v |v|^2 (the
    penalised objective of eq. 6 restricted to v_j) by Fisher scoring,
      v <- v + (U' diag(Dddot_.j) U + lam_v I)^-1 (U' Ddot_.j - lam_v v),
    from V0, with the step control of the per-cell projection (the same
    reading: accept a point whose f is within 1e-5 (1 + |f_best|) of the best,
    else halve the last step from the best point). n_steps passes take at most
    n_steps steps. Returns (V, f) with f the genes' objectives at V; with
    margins=True also, per gene, the smallest |(f - f_best)/(1 + |f_best|) -
    1e-5| over its accept / halve tests (how far each decision was from going
    the other way)."""
    Y = np.asarray(Y, float)
    n, m = Y.shape
    d = U.shape[1]
    Wt = np.ones_like(Y) if W is None else np.asarray(W, float)
    base = X @ B.T + Gamma @ Z.T + (0.0 if offset is None else np.asarray(offset, float)[:, None])
    V = np.array(V0, float)
    best = V.copy()
    f_best = np.full(m, np.inf)
    step = np.zeros_like(V)
    margin = np.full(m, np.inf)
    for k in range(n_steps + 1):          # pass k evaluates V; passes 0 .. n_steps-1 also step
        eta = base + U @ V.T
        mu, dd, ddd = _count_derivs(family, Y, eta, alpha)
        f = 0.5 * (Wt * _count_deviance(family, Y, mu, alpha)).sum(axis=0) + 0.5 * lam_v * (V ** 2).sum(axis=1)
        for j in range(m):
            if k > 0:
                margin[j] = min(margin[j], abs((f[j] - f_best[j]) / (1.0 + abs(f_best[j])) - LOADINGS_SLACK))
            if k == 0 or f[j] <= f_best[j] + LOADINGS_SLACK * (1.0 + abs(f_best[j])):
                best[j], f_best[j] = V[j], f[j]
                if k < n_steps:
                    wj = Wt[:, j]
                    F = (U * (wj * ddd[:, j])[:, None]).T @ U + lam_v * np.eye(d)
                    g = U.T @ (wj * dd[:, j]) - lam_v * V[j]
                    step[j] = np.linalg.solve(F, g)
                    V[j] = best[j] + step[j]
            else:
                step[j] *= 0.5
                V[j] = best[j] + step[j]
    if margins:
        return best, f_best, margin
    return best, f_best
