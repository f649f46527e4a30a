"""Seeded synthetic inputs for GMF fits on count matrices.

This module is shared by the tests, the benchmark and the smoke check. It holds
no part of the estimator: it draws the data (the generative laws of the
workloads below), the random partitions and sweep orders that Algorithm 1
samples (passed to both implementations as inputs), and a crude, deterministic
starting point. Nothing here imports the CUDA package or the oracle.

Workloads (rows = cells, columns = genes; Sec. 2, eq. 3 with an offset):

* ``poisson_small``   1000 x 500 int32, Poisson, d = 5, p = 2, q = 1.
* ``nb_medium``       20000 x 2000 int32, NB, ~85% zeros, d = 10, p = 3, q = 1.
* ``nb_atlas``        200000 x 5000 uint16, NB, ~90% zeros, d = 20.
* ``nb_sweep``        50000 x 3000 uint16, NB (true d = 10) for the rank sweep.
* ``nb_select``       the same law with 30 % of the entries held out, for rank selection.
* ``nb_project``      100000 fit + 100000 held-out cells x 3000 genes, NB, d = 20.

Law (all workloads): eta = o + X B^T + Gamma Z^T + U V^T with
X = [1, N(0,1), ...] (p columns), Z = 1_m (q = 1, so Gamma is a per-cell
intercept), U, V, Gamma and the non-intercept columns of B ~ N(0, 0.5^2). The
NB workloads add a library-size offset o_i = log LogNormal(0, 0.5) and draw a
per-gene NB size alpha_j ~ Gamma(shape 2, scale 0.5). The gene intercept B[:,0]
is N(c, 0.5^2) with c found by bisection so that the expected fraction of zero
counts hits the target.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "WORKLOADS", "Problem", "make_problem", "partitions", "sweep_orders",
    "n_sweeps", "crude_start", "fit_settings", "holdout_mask", "with_missing", "make_family_problem",
]


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n: int
    m: int
    p: int
    q: int
    d: int
    family: str          # "poisson" | "negbin"
    y_dtype: str         # "int32" | "uint16"
    zero_frac: float | None
    offset: bool
    nb_row: int
    nb_col: int
    epochs: int


WORKLOADS = {
    "poisson_small": Workload("poisson_small", 1000, 500, 2, 1, 5, "poisson", "int32", None, False, 100, 100, 50),
    "nb_medium": Workload("nb_medium", 20000, 2000, 3, 1, 10, "negbin", "int32", 0.85, True, 500, 500, 20),
    "nb_atlas": Workload("nb_atlas", 200000, 5000, 3, 1, 20, "negbin", "uint16", 0.90, True, 2048, 1024, 10),
    "nb_sweep": Workload("nb_sweep", 50000, 3000, 3, 1, 10, "negbin", "uint16", 0.90, True, 2048, 1024, 15),
    "nb_select": Workload("nb_select", 50000, 3000, 3, 1, 10, "negbin", "uint16", 0.90, True, 2048, 1024, 15),
    "nb_project": Workload("nb_project", 200000, 3000, 3, 1, 20, "negbin", "uint16", 0.90, True, 2048, 1024, 10),
}


@dataclasses.dataclass
class Problem:
    """One synthetic data set with its true parameters (original row/column order)."""
    Y: np.ndarray            # n x m counts, int32 or uint16, C order
    X: np.ndarray            # n x p float64
    Z: np.ndarray            # m x q float64
    offset: np.ndarray       # n float64 (zeros when the workload has none)
    B: np.ndarray            # m x p true coefficients
    Gamma: np.ndarray        # n x q
    U: np.ndarray            # n x d
    V: np.ndarray            # m x d
    nb_size: np.ndarray | None   # per-gene NB size (None for Poisson)
    family: str
    saturated: int = 0       # counts clipped at 65535 (uint16 workloads)

    @property
    def n(self):
        return self.Y.shape[0]

    @property
    def m(self):
        return self.Y.shape[1]


def _eta(X, B, Gamma, Z, U, V, offset, rows=slice(None)):
    e = X[rows] @ B.T + Gamma[rows] @ Z.T + U[rows] @ V.T
    return e + offset[rows, None]


def _zero_frac(eta, family, size):
    mu = np.exp(np.clip(eta, -30, 30))
    if family == "poisson":
        return float(np.mean(np.exp(-mu)))
    return float(np.mean(np.exp(size[None, :] * (np.log(size[None, :]) - np.log(size[None, :] + mu)))))


def make_problem(n, m, p, q, d, family="poisson", *, seed=0, y_dtype="int32",
                 zero_frac=None, offset=False, scale=0.5):
    """Draw a synthetic count matrix from the GMF law (Sec. 2, eq. 3).

    ``zero_frac`` (NB and Poisson) shifts the gene intercept so that the
    expected fraction of zeros matches it; None leaves the intercept N(0, scale^2).
    """
    rng = np.random.default_rng(seed)
    X = np.empty((n, p))
    X[:, 0] = 1.0
    if p > 1:
        X[:, 1:] = rng.standard_normal((n, p - 1))
    Z = np.ones((m, q)) if q >= 1 else np.zeros((m, 0))
    if q > 1:
        Z[:, 1:] = rng.standard_normal((m, q - 1))
    B = scale * rng.standard_normal((m, p))
    Gamma = scale * rng.standard_normal((n, q))
    U = scale * rng.standard_normal((n, d))
    V = scale * rng.standard_normal((m, d))
    off = rng.normal(0.0, 0.5, size=n) if offset else np.zeros(n)
    size = rng.gamma(2.0, 0.5, size=m) if family == "negbin" else None

    if zero_frac is not None:
        sub = np.sort(rng.choice(n, size=min(n, 2000), replace=False))
        base = _eta(X, B, Gamma, Z, U, V, off, sub)
        lo, hi = -15.0, 15.0
        shift0 = B[:, 0].copy()
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            zf = _zero_frac(base + mid, family, size)
            if zf > zero_frac:
                lo = mid
            else:
                hi = mid
        B[:, 0] = shift0 + 0.5 * (lo + hi)

    # Counts, drawn row-chunk by row-chunk to bound memory.
    saturated = 0
    Y = np.empty((n, m), dtype=np.int32 if y_dtype == "int32" else np.uint16)
    chunk = max(1, int(4_000_000 // max(m, 1)))
    for r0 in range(0, n, chunk):
        rows = slice(r0, min(n, r0 + chunk))
        mu = np.exp(np.clip(_eta(X, B, Gamma, Z, U, V, off, rows), -30, 30))
        if family == "poisson":
            c = rng.poisson(mu)
        else:
            # Gamma-Poisson mixture: lambda ~ Gamma(size, mu/size), y ~ Poisson(lambda)
            c = rng.poisson(rng.gamma(size[None, :], mu / size[None, :]))
        top = 65535 if y_dtype == "uint16" else 2**31 - 1
        saturated += int(np.count_nonzero(c > top))
        Y[rows] = np.minimum(c, top)
    return Problem(Y=np.ascontiguousarray(Y), X=X, Z=Z, offset=off, B=B, Gamma=Gamma,
                   U=U, V=V, nb_size=size, family=family, saturated=saturated)


def make_family_problem(n, m, p, q, d, family, *, phi=0.5, seed=0, offset=False, scale=0.5, shift=0.0):
    """Draw float32 responses from one of the other laws of Table S1 under the
    same linear predictor (eta = o + X B^T + Gamma Z^T + U V^T, gene
    intercepts shifted by `shift`): "gaussian" N(eta, phi) (identity link),
    "binomial" Bernoulli(1 / (1 + e^-eta)) (logit link; 0 / 1 values),
    "gamma" Gamma with mean e^eta and shape 1/phi, "invgauss" inverse Gaussian
    with mean e^eta and shape 1/phi (log links). Returns a Problem whose
    nb_size holds the dispersion phi of every gene."""
    rng = np.random.default_rng([seed, 5])
    X = np.empty((n, p))
    X[:, 0] = 1.0
    if p > 1:
        X[:, 1:] = rng.standard_normal((n, p - 1))
    Z = np.ones((m, q)) if q >= 1 else np.zeros((m, 0))
    if q > 1:
        Z[:, 1:] = rng.standard_normal((m, q - 1))
    B = scale * rng.standard_normal((m, p))
    B[:, 0] += shift
    Gamma = scale * rng.standard_normal((n, q))
    U = scale * rng.standard_normal((n, d))
    V = scale * rng.standard_normal((m, d))
    off = rng.normal(0.0, 0.5, size=n) if offset else np.zeros(n)
    eta = _eta(X, B, Gamma, Z, U, V, off, slice(0, n))
    if family == "gaussian":
        Y = eta + math.sqrt(phi) * rng.standard_normal((n, m))
    elif family == "binomial":
        Y = (rng.random((n, m)) < 1.0 / (1.0 + np.exp(-eta))).astype(np.float64)
    elif family == "gamma":
        mu = np.exp(eta)
        Y = rng.gamma(1.0 / phi, mu * phi)
    elif family == "invgauss":
        mu = np.exp(eta)
        Y = rng.wald(mu, 1.0 / phi)
    else:
        raise ValueError(family)
    return Problem(Y=np.ascontiguousarray(Y, dtype=np.float32), X=X, Z=Z, offset=off, B=B, Gamma=Gamma, U=U, V=V,
                   nb_size=np.full(m, float(phi)), family=family)


def workload_problem(name, seed=0, n=None, m=None):
    """Draw the named workload (optionally at a reduced n x m with the same law)."""
    w = WORKLOADS[name]
    return make_problem(n or w.n, m or w.m, w.p, w.q, w.d, w.family, seed=seed,
                        y_dtype=w.y_dtype, zero_frac=w.zero_frac, offset=w.offset)


def partitions(n, m, seed):
    """Random row and column permutations: chunk c of rows is
    row_perm[c*nb_row:(c+1)*nb_row] (the random partitions of Algorithm 1)."""
    rng = np.random.default_rng([seed, 1])
    return (rng.permutation(n).astype(np.int32), rng.permutation(m).astype(np.int32))


def n_sweeps(n, m, nb_row, nb_col):
    r = -(-n // nb_row)
    s = -(-m // nb_col)
    return max(r, s)


def sweep_orders(n, m, nb_row, nb_col, epochs, seed):
    """One random permutation of the sweep offsets per epoch (the per-block
    sampling of I in Algorithm 1), as int32 arrays."""
    rng = np.random.default_rng([seed, 2])
    w = n_sweeps(n, m, nb_row, nb_col)
    return [rng.permutation(w).astype(np.int32) for _ in range(epochs)]


def crude_start(prob: Problem, d, *, seed=0, scale=0.1):
    """A deterministic starting point shared by both implementations.

    Gene intercepts from column means, per-cell intercepts from row sums, the
    other coefficients zero, and small random latent factors.
    """
    rng = np.random.default_rng([seed, 3])
    n, m = prob.Y.shape
    p = prob.X.shape[1]
    q = prob.Z.shape[1]
    if prob.family in ("gaussian", "binomial"):
        # identity / logit link: column means (clipped into (0, 1) for 0 / 1 data) and row deviations
        Yf = np.nan_to_num(prob.Y.astype(np.float64), nan=float(np.nanmean(prob.Y)))
        link = (lambda v: v) if prob.family == "gaussian" else (lambda v: np.log(v / (1 - v)))
        clip = (lambda v: v) if prob.family == "gaussian" else (lambda v: np.clip(v, 0.02, 0.98))
        B0 = np.zeros((m, p))
        B0[:, 0] = link(clip(Yf.mean(0)))
        G0 = np.zeros((n, q))
        if q >= 1:
            G0[:, 0] = link(clip(Yf.mean(1))) - link(clip(Yf.mean()))
        return dict(B=B0, Gamma=G0, U=scale * rng.standard_normal((n, d)), V=scale * rng.standard_normal((m, d)),
                    alpha=1.0)
    colsum = prob.Y.sum(axis=0, dtype=np.float64)
    rowsum = prob.Y.sum(axis=1, dtype=np.float64)
    B0 = np.zeros((m, p))
    B0[:, 0] = np.log((colsum + 0.5) / n) - prob.offset.mean()
    G0 = np.zeros((n, q))
    if q >= 1:
        expected = np.exp(prob.offset) * np.exp(B0[:, 0]).sum()
        G0[:, 0] = np.log((rowsum + 0.5) / expected)
        G0[:, 0] -= G0[:, 0].mean()
    U0 = scale * rng.standard_normal((n, d))
    V0 = scale * rng.standard_normal((m, d))
    alpha0 = 1.0
    return dict(B=B0, Gamma=G0, U=U0, V=V0, alpha=alpha0)


def fit_settings(**over):
    """Optimiser settings of the paper's sgdGMF runs (Sec. 5.2 / App. C) with the
    unstated constants filled in; keyword arguments override."""
    s = dict(lambda_=(0.0, 0.0, 1.0, 0.0), a1=0.1, a2=0.01, k0=0.01, k1=1e-3, tau=0.75,
             damping=1e-3, eps=1e-8, eta_clamp=30.0, bias_corr=0, alpha_mode=0, missing=0)
    s.update(over)
    return s


def make_problem_device(n, m, p, q, d, family="negbin", *, seed=0, zero_frac=None, offset=True, scale=0.5,
                        device="cuda"):
    """The law of make_problem drawn on a CUDA device with torch's generator
    (for matrices too large to draw with numpy in reasonable time). Returns a
    Problem whose Y is a CUDA uint16-bit tensor (int16 view of the counts,
    saturated at 65535) and whose parameters are numpy arrays. Same law as
    make_problem, different random stream."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    rng = np.random.default_rng([seed, 9])
    X = np.empty((n, p))
    X[:, 0] = 1.0
    if p > 1:
        X[:, 1:] = rng.standard_normal((n, p - 1))
    Z = np.ones((m, q))
    B = scale * rng.standard_normal((m, p))
    Gamma = scale * rng.standard_normal((n, q))
    U = scale * rng.standard_normal((n, d))
    V = scale * rng.standard_normal((m, d))
    off = rng.normal(0.0, 0.5, size=n) if offset else np.zeros(n)
    size = rng.gamma(2.0, 0.5, size=m) if family == "negbin" else None
    if zero_frac is not None:
        sub = np.sort(rng.choice(n, size=min(n, 2000), replace=False))
        base = _eta(X, B, Gamma, Z, U, V, off, sub)
        lo, hi = -15.0, 15.0
        for _ in range(60):
            mid = 0.5 * (lo + hi)
            if _zero_frac(base + mid, family, size) > zero_frac:
                lo = mid
            else:
                hi = mid
        B[:, 0] = B[:, 0] + 0.5 * (lo + hi)
    t = lambda a: torch.as_tensor(a, dtype=torch.float32, device=device)
    Xt, Bt, Gt, Zt, Ut, Vt, ot = map(t, (X, B, Gamma, Z, U, V, off))
    Y = torch.empty((n, m), dtype=torch.int16, device=device)
    st = t(size) if size is not None else None
    chunk = max(1, 20_000_000 // m)
    saturated = 0
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        eta = Xt[r0:r1] @ Bt.T + Gt[r0:r1] @ Zt.T + Ut[r0:r1] @ Vt.T + ot[r0:r1, None]
        mu = torch.exp(eta.clamp(-30, 30))
        if family == "negbin":
            lam = torch._standard_gamma(st.expand_as(mu).contiguous(), generator=g) * (mu / st)
        else:
            lam = mu
        c = torch.poisson(lam, generator=g)
        saturated += int((c > 65535).sum())
        c = c.clamp_(max=65535).to(torch.int32)
        Y[r0:r1] = torch.where(c > 32767, c - 65536, c).to(torch.int16)
    return Problem(Y=Y, X=X, Z=Z, offset=off, B=B, Gamma=Gamma, U=U, V=V, nb_size=size, family=family,
                   saturated=saturated)


MISSING_INT32 = -1        # the count that marks a missing entry in int32 counts
MISSING_UINT16 = 65535    # ... and in uint16 counts


def holdout_mask(n, m, frac, seed):
    """Observed-entry mask with a uniformly drawn held-out fraction `frac` of
    the entries (the evaluation protocol of Sec. 5.2: 30 % in the paper)."""
    rng = np.random.default_rng([seed, 11])
    return rng.random((n, m)) >= frac


def with_missing(Y, observed):
    """A copy of Y with the held-out entries set to the missing marker of its
    dtype (int32: -1, uint16: 65535, float32: NaN)."""
    Y = np.array(Y, copy=True)
    marker = {np.dtype(np.int32): MISSING_INT32, np.dtype(np.uint16): MISSING_UINT16}.get(Y.dtype, np.nan)
    Y[~np.asarray(observed, bool)] = marker
    return Y


def mlp_init(n_in, n_h1, n_h2, n_out, seed):
    """Seeded starting weights of the warm-start encoder: scaled normal weights,
    zero biases (an input shared by the library and the oracle)."""
    rng = np.random.default_rng([seed, 7])
    return dict(W1=rng.standard_normal((n_h1, n_in)) / np.sqrt(n_in), b1=np.zeros(n_h1),
                W2=rng.standard_normal((n_h2, n_h1)) / np.sqrt(n_h1), b2=np.zeros(n_h2),
                W3=rng.standard_normal((n_out, n_h2)) / np.sqrt(n_h2), b3=np.zeros(n_out))
