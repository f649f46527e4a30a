"""Algorithm 2 (identifiability projection and orthogonalisation), FP64 numpy.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). Follows the projection
steps of Algorithm 2 in the paper's order, with numpy's SVD and QR as library
steps:

  1. D_G = (X'X)^-1 X' Gamma;  Gamma -= X D_G;  B += Z D_G'
  2. D_U = (X'X)^-1 X' U;      U -= X D_U;      B += V D_U'
  3. D_V = (Z'Z)^-1 Z' V;      V -= Z D_V;      Gamma += U D_V'
  4. (B1) svd(U V') -> U = U~ S~, V = V~; (B2) U = U~, V = V~ S~;
     (B3) whitening by S = cov(U), then qr(V') and a sign fix.

Readings: the sign rule of (B1)/(B2) makes the first entry of magnitude above
1e-12 of each V (B1) or U (B2) column positive. In (B3) the last step uses
D = diag(sign(diag V)), which keeps U V' unchanged (the printed D = diag(V)
would not).
"""
from __future__ import annotations

import numpy as np


def _first_sign(M, tol=1e-12):
    s = np.ones(M.shape[1])
    for c in range(M.shape[1]):
        nz = np.flatnonzero(np.abs(M[:, c]) > tol)
        if len(nz) and M[nz[0], c] < 0:
            s[c] = -1.0
    return s


def project_covariates(X, Z, B, Gamma, U, V):
    """Steps 1-3 of Algorithm 2 (constraint (A)); returns new (B, Gamma, U, V)."""
    B, Gamma, U, V = (np.array(a, dtype=np.float64) for a in (B, Gamma, U, V))
    XtX = X.T @ X
    ZtZ = Z.T @ Z
    DG = np.linalg.solve(XtX, X.T @ Gamma)
    Gamma = Gamma - X @ DG
    B = B + Z @ DG.T
    DU = np.linalg.solve(XtX, X.T @ U)
    U = U - X @ DU
    B = B + V @ DU.T
    DV = np.linalg.solve(ZtZ, Z.T @ V)
    V = V - Z @ DV
    Gamma = Gamma + U @ DV.T
    return B, Gamma, U, V


def orthogonalize(X, Z, B, Gamma, U, V, mode="B1"):
    """Algorithm 2 with the explicit n x m SVD of U V' (small problems)."""
    B, Gamma, U, V = project_covariates(X, Z, B, Gamma, U, V)
    d = U.shape[1]
    n = U.shape[0]
    if mode in ("B1", "B2"):
        Ut, St, Vt = np.linalg.svd(U @ V.T, full_matrices=False)
        Ut, St, Vt = Ut[:, :d], St[:d], Vt[:d].T
        if mode == "B1":
            U, V = Ut * St, Vt
            s = _first_sign(V)
        else:
            U, V = Ut, Vt * St
            s = _first_sign(U)
        U, V = U * s, V * s
    elif mode == "B3":
        one = np.ones((n, 1))
        S = (U.T @ U - (U.T @ one) @ (one.T @ U) / n) / n
        w, Q = np.linalg.eigh(S)
        S_mhalf = (Q / np.sqrt(w)) @ Q.T
        S_half = (Q * np.sqrt(w)) @ Q.T
        U = U @ S_mhalf
        V = V @ S_half
        Qv, Rv = np.linalg.qr(V.T)
        U = U @ Qv
        V = Rv.T
        D = np.sign(np.diag(V))
        D[D == 0] = 1.0
        U, V = U * D, V * D
    else:
        raise ValueError(mode)
    return B, Gamma, U, V
