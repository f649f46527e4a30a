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
the points the paper leaves open).
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
