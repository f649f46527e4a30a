"""Independent matrix-form restatement of Algorithm 1 (numpy, FP64).

Used only by the oracle pin tests: it is written separately from the scalar C
oracle (whole-block matrix products instead of per-entry loops, the NB
derivatives in their simplified closed form alpha (y - mu)/(alpha + mu) and
alpha mu/(alpha + mu) instead of the nu / g' form, and likewise for the other
families of Table S1), so that an indexing,
transposition or bookkeeping slip in either one shows up as a mismatch.
"""
import math

import numpy as np


def bias(cfg, t, visits):
    if cfg["bias_corr"] == 0:
        return (1 - cfg["a2"] ** t) / (1 - cfg["a1"] ** t)
    return (1 - (1 - cfg["a2"]) ** visits) / (1 - (1 - cfg["a1"]) ** visits)


class BruteFit:
    def __init__(self, Y, X, Z, offset, start, family, nb_row, nb_col, row_perm, col_perm, cfg, W=None,
                 observed=None, alpha_col=None):
        self.Y = np.asarray(Y, dtype=np.float64)
        self.alpha_col = None if alpha_col is None else np.asarray(alpha_col, float)   # per-gene NB shapes
        # Omega: the observed entries (all by default); the others are imputed by mu each block (Sec. 3.2)
        self.obs = np.ones(self.Y.shape, bool) if observed is None else np.asarray(observed, bool)
        self.W = np.ones_like(self.Y) if W is None else np.asarray(W, dtype=np.float64)
        self.X, self.Z = np.asarray(X, float), np.asarray(Z, float)
        n, m = self.Y.shape
        self.off = np.zeros(n) if offset is None else np.asarray(offset, float)
        self.B = np.array(start["B"], float)
        self.G = np.array(start["Gamma"], float)
        self.U = np.array(start["U"], float)
        self.V = np.array(start["V"], float)
        self.alpha = float(start.get("alpha", 1.0))
        p, q, d = self.X.shape[1], self.Z.shape[1], self.U.shape[1]
        self.GbR = np.zeros((n, q + d)); self.HbR = np.zeros((n, q + d))
        self.GbC = np.zeros((m, p + d)); self.HbC = np.zeros((m, p + d))
        self.cR = np.zeros(n, dtype=np.int64); self.cC = np.zeros(m, dtype=np.int64)
        self.t = 0
        self.family, self.nb_row, self.nb_col = family, nb_row, nb_col
        self.rp, self.cp = np.asarray(row_perm), np.asarray(col_perm)
        self.cfg = cfg

    def epoch(self, sigma):
        cfg = self.cfg
        n, m = self.Y.shape
        p, q, d = self.X.shape[1], self.Z.shape[1], self.U.shape[1]
        r, s = math.ceil(n / self.nb_row), math.ceil(m / self.nb_col)
        swap = r < s
        lam = cfg["lambda_"]
        lam_row = np.array([lam[1]] * q + [lam[2]] * d)
        lam_col = np.array([lam[0]] * p + [lam[3]] * d)
        for w in range(s if swap else r):
            s1 = s2 = 0.0
            t_first = self.t + 1
            for k in range(r if swap else s):
                rc = k if swap else (sigma[w] + k) % r
                cc = (sigma[w] + k) % s if swap else k
                I = self.rp[rc * self.nb_row:(rc + 1) * self.nb_row]
                J = self.cp[cc * self.nb_col:(cc + 1) * self.nb_col]
                Yb, Wb = self.Y[np.ix_(I, J)], self.W[np.ix_(I, J)]
                eta = (self.off[I, None] + self.X[I] @ self.B[J].T + self.G[I] @ self.Z[J].T
                       + self.U[I] @ self.V[J].T)
                e = np.clip(eta, -cfg["eta_clamp"], cfg["eta_clamp"])
                fam = self.family
                mu = e if fam == "gaussian" else (1 / (1 + np.exp(-e)) if fam == "binomial" else np.exp(e))
                ob = self.obs[np.ix_(I, J)]
                Yb = np.where(ob, Yb, mu)
                phi = self.alpha    # the dispersion of the Gaussian, Gamma and inverse Gaussian families
                if fam in ("poisson", "negbin"):
                    if fam == "poisson":
                        f = np.ones_like(mu)
                    else:
                        a = self.alpha if self.alpha_col is None else self.alpha_col[J][None, :]
                        f = a / (a + mu)
                    Dd = Wb * (Yb - mu) * f
                    Ddd = Wb * mu * f
                    s1 += float((Wb * mu * mu).sum())
                    s2 += float((Wb * ((Yb - mu) ** 2 - mu)).sum())
                elif fam == "binomial":           # canonical link: the score is the raw residual
                    Dd = Wb * (Yb - mu)
                    Ddd = Wb * mu * (1 - mu)
                else:
                    # closed forms of the score and Fisher weight under the identity (Gaussian) and log links
                    Dd = {"gaussian": Wb * (Yb - mu), "gamma": Wb * (Yb / mu - 1),
                          "invgauss": Wb * (Yb - mu) / mu ** 2}[fam] / phi
                    Ddd = {"gaussian": Wb, "gamma": Wb, "invgauss": Wb / mu}[fam] / phi
                    pearson = {"gaussian": (Yb - mu) ** 2, "gamma": ((Yb - mu) / mu) ** 2,
                               "invgauss": (Yb - mu) ** 2 / mu ** 3}[fam]
                    s1 += float((Wb * pearson)[ob].sum())
                    s2 += float(ob.sum())
                Rf = np.hstack([self.Z[J], self.V[J]])
                Lf = np.hstack([self.X[I], self.U[I]])
                thR = np.hstack([self.G[I], self.U[I]])
                thC = np.hstack([self.B[J], self.V[J]])
                gR = -(m / len(J)) * (Dd @ Rf) + lam_row * thR
                hR = (m / len(J)) * (Ddd @ (Rf * Rf)) + lam_row + cfg["damping"]
                gC = -(n / len(I)) * (Dd.T @ Lf) + lam_col * thC
                hC = (n / len(I)) * (Ddd.T @ (Lf * Lf)) + lam_col + cfg["damping"]
                self.t += 1
                t = self.t
                rho = cfg["k0"] / (1 + cfg["k0"] * cfg["k1"] * t) ** cfg["tau"]
                self.cR[I] += 1
                self.cC[J] += 1
                cfR = np.array([bias(cfg, t, v) for v in self.cR[I]])[:, None]
                cfC = np.array([bias(cfg, t, v) for v in self.cC[J]])[:, None]
                self.GbR[I] = (1 - cfg["a1"]) * self.GbR[I] + cfg["a1"] * gR
                self.HbR[I] = (1 - cfg["a2"]) * self.HbR[I] + cfg["a2"] * hR
                self.GbC[J] = (1 - cfg["a1"]) * self.GbC[J] + cfg["a1"] * gC
                self.HbC[J] = (1 - cfg["a2"]) * self.HbC[J] + cfg["a2"] * hC
                thR = thR - rho * cfR * self.GbR[I] / self.HbR[I]
                thC = thC - rho * cfC * self.GbC[J] / self.HbC[J]
                self.G[I], self.U[I] = thR[:, :q], thR[:, q:]
                self.B[J], self.V[J] = thC[:, :p], thC[:, p:]
            if self.family == "negbin" and cfg["alpha_mode"] == 1 and s2 > 0:
                ahat = max(cfg["eps"], s1 / s2)
                rho = cfg["k0"] / (1 + cfg["k0"] * cfg["k1"] * t_first) ** cfg["tau"]
                self.alpha = (1 - rho) * self.alpha + rho * ahat
            if self.family in ("gaussian", "gamma", "invgauss") and cfg["alpha_mode"] == 1 and s2 > 0:
                # App. B: the Pearson statistic of the sweep scaled to the whole matrix over the residual dof
                dof = n * m - m * p - n * q - (n + m) * d - 1
                if dof > 0:
                    phat = max(cfg["eps"], (n * m / s2) * s1 / dof)
                    rho = cfg["k0"] / (1 + cfg["k0"] * cfg["k1"] * t_first) ** cfg["tau"]
                    self.alpha = (1 - rho) * self.alpha + rho * phat
