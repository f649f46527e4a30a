"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test targets a plausible mistake: a dropped term, a wrong sign, a wrong
scale factor, a transposed operand, an off-by-one in t or in the schedule.
"""
import math

import numpy as np
import pytest
from scipy import stats

import synth
from tests.bruteforce import BruteFit

FAM = {"poisson": 0, "negbin": 1}


def loglik(family, y, mu, alpha):
    if family == "poisson":
        return stats.poisson.logpmf(y, mu)
    return stats.nbinom.logpmf(y, alpha, alpha / (alpha + mu))


# ---------------------------------------------------------------- per entry (Sec. 3)

@pytest.mark.parametrize("family", ["poisson", "negbin"])
def test_entry_derivatives_match_finite_differences(oracle_lib, family):
    """Ddot = d log f / d eta (score) and the observed second derivative equals
    Dddot * alpha(mu), alpha(mu) = 1 + (y - mu)(nu'/nu + g''/g') (Sec. 3)."""
    h1, h2 = 1e-5, 2e-3
    for y in (0, 1, 4, 37):
        for eta in (-2.0, 0.3, 2.5):
            for alpha in (0.4, 2.0, 15.0):
                for w in (1.0, 0.6):
                    mu, dd, ddd = oracle_lib.entry(FAM[family], y, eta, w, alpha)
                    assert mu == pytest.approx(math.exp(eta), rel=1e-15)
                    f = lambda e: w * loglik(family, y, math.exp(e), alpha)
                    fd1 = (f(eta + h1) - f(eta - h1)) / (2 * h1)
                    fd2 = -(f(eta + h2) - 2 * f(eta) + f(eta - h2)) / h2 ** 2
                    scale = 1.0 + abs(f(eta))          # finite-difference round-off grows with |f|
                    assert dd == pytest.approx(fd1, rel=1e-7, abs=1e-9 * scale)
                    if family == "poisson":
                        a_mu = 1.0
                    else:
                        nu = mu * (1 + mu / alpha)
                        a_mu = 1 + (y - mu) * ((1 + 2 * mu / alpha) / nu + (-1 / mu ** 2) / (1 / mu))
                    assert ddd * a_mu == pytest.approx(fd2, rel=2e-6, abs=1e-8 * scale)


@pytest.mark.parametrize("family", ["poisson", "negbin"])
def test_fisher_weight_is_expected_observed_information(oracle_lib, family):
    """Dddot is the Fisher weight: E_y[-d^2 log f/d eta^2] under y ~ f(mu)."""
    h = 1e-4
    for eta in (-1.0, 0.5, 1.8):
        for alpha in (0.7, 3.0):
            mu, _, ddd = oracle_lib.entry(FAM[family], 0, eta, 1.0, alpha)
            ys = np.arange(0, 400)
            pmf = np.exp(loglik(family, ys, mu, alpha))
            f = lambda e: loglik(family, ys, math.exp(e), alpha)
            obs = -(f(eta + h) - 2 * f(eta) + f(eta - h)) / h ** 2
            assert float((pmf * obs).sum()) == pytest.approx(ddd, rel=1e-5)


@pytest.mark.parametrize("family", ["poisson", "negbin"])
def test_deviance_matches_likelihood_ratio(oracle_lib, family):
    """D(y, mu) = -2 log{f(y, mu)/f(y, y)} (Sec. 2; Table S1, App. B); zero at
    mu = y, positive elsewhere, linear in w."""
    for y in (0, 1, 3, 20, 250):
        for mu in (0.05, 1.0, 7.5, 300.0):
            for alpha in (0.5, 4.0):
                ref = -2 * (loglik(family, y, mu, alpha) - (loglik(family, y, y, alpha) if y > 0 else 0.0))
                got = oracle_lib.entry_deviance(FAM[family], y, mu, 1.0, alpha)
                assert got == pytest.approx(ref, rel=1e-9, abs=1e-10)
                assert got >= 0
                assert oracle_lib.entry_deviance(FAM[family], y, mu, 0.3, alpha) == pytest.approx(0.3 * got, rel=1e-12)
        if y > 0:
            assert abs(oracle_lib.entry_deviance(FAM[family], y, float(y), 1.0, 2.0)) < 1e-12


# ---------------------------------------------------------------- matrix level (eq. 7-8, 15, App. B)

def tiny_fit(oracle_lib, n, m, p, q, d, family, seed, nb_row=None, nb_col=None, **kw):
    rng = np.random.default_rng(seed)
    X = np.hstack([np.ones((n, 1)), rng.standard_normal((n, p - 1))])
    Z = np.hstack([np.ones((m, 1)), rng.standard_normal((m, q - 1))]) if q else np.zeros((m, 0))
    start = dict(B=0.3 * rng.standard_normal((m, p)), Gamma=0.3 * rng.standard_normal((n, q)),
                 U=0.4 * rng.standard_normal((n, d)), V=0.4 * rng.standard_normal((m, d)), alpha=1.7)
    off = 0.2 * rng.standard_normal(n)
    Y = rng.poisson(2.0, size=(n, m)).astype(np.int32)
    W = kw.pop("W", None)
    settings = synth.fit_settings(**kw)
    rp = kw.get("row_perm", rng.permutation(n).astype(np.int32))
    cp = kw.get("col_perm", rng.permutation(m).astype(np.int32))
    f = oracle_lib.OracleFit(Y, X, Z, off, start, family=family, nb_row=nb_row or n, nb_col=nb_col or m,
                             row_perm=rp, col_perm=cp, settings=settings, W=W)
    return f, dict(Y=Y, X=X, Z=Z, off=off, start=start, rp=rp, cp=cp, settings=settings, W=W)


def nll(family, Y, X, Z, off, B, G, U, V, alpha, W=None):
    eta = off[:, None] + X @ B.T + G @ Z.T + U @ V.T
    ll = loglik(family, Y, np.exp(eta), alpha)
    return -float((ll if W is None else W * ll).sum())


@pytest.mark.parametrize("family", ["poisson", "negbin"])
def test_block_gradient_matches_finite_differences(oracle_lib, family):
    """Full-batch estimators equal d l / d theta of the negative log-likelihood
    for every free block [Gamma, U] and [B, V] (App. B); H matches the second
    derivative for the canonical Poisson link (Z*Z for Gamma, X*X for B)."""
    n, m, p, q, d = 5, 4, 2, 2, 2
    rng = np.random.default_rng(3)
    W = rng.uniform(0.5, 1.5, size=(n, m))
    f, D = tiny_fit(oracle_lib, n, m, p, q, d, family, seed=1, W=W)
    Grow, Hrow, Gcol, Hcol, _ = f.block_grad(np.arange(n), np.arange(m))
    P = {k: np.array(v, dtype=float) for k, v in D["start"].items() if k != "alpha"}
    a = D["start"]["alpha"]
    h, hh = 1e-5, 2e-3

    def L(P):
        return nll(family, D["Y"], D["X"], D["Z"], D["off"], P["B"], P["Gamma"], P["U"], P["V"], a, W)

    def fd(name, i, c):
        Pp = {k: v.copy() for k, v in P.items()}; Pm = {k: v.copy() for k, v in P.items()}
        Pp[name][i, c] += h; Pm[name][i, c] -= h
        g = (L(Pp) - L(Pm)) / (2 * h)
        Pp[name][i, c] += hh - h; Pm[name][i, c] -= hh - h
        h2 = (L(Pp) - 2 * L(P) + L(Pm)) / hh ** 2
        return g, h2

    for i in range(n):
        for c in range(q + d):
            name, cc = ("Gamma", c) if c < q else ("U", c - q)
            g, h2 = fd(name, i, cc)
            assert Grow[i, c] == pytest.approx(g, rel=1e-6, abs=1e-7)
            if family == "poisson":
                assert Hrow[i, c] == pytest.approx(h2, rel=1e-5, abs=1e-6)
    for j in range(m):
        for c in range(p + d):
            name, cc = ("B", c) if c < p else ("V", c - p)
            g, h2 = fd(name, j, cc)
            assert Gcol[j, c] == pytest.approx(g, rel=1e-6, abs=1e-7)
            if family == "poisson":
                assert Hcol[j, c] == pytest.approx(h2, rel=1e-5, abs=1e-6)


def test_block_estimators_are_unbiased_over_a_partition(oracle_lib):
    """sum_J (|J|/m) G_row(I, J) = G_row(I, all) and likewise for the columns
    (eq. 15 and the unbiasedness remark after it), with a ragged last chunk."""
    n, m = 12, 7
    f, D = tiny_fit(oracle_lib, n, m, 2, 1, 3, "negbin", seed=5)
    I = np.arange(n)
    full = f.block_grad(I, np.arange(m))
    acc = [np.zeros_like(full[0]), np.zeros_like(full[1])]
    for J in (np.array([0, 4, 6]), np.array([1, 2, 3]), np.array([5])):
        g = f.block_grad(I, J)
        acc[0] += len(J) / m * g[0]
        acc[1] += len(J) / m * g[1]
    np.testing.assert_allclose(acc[0], full[0], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(acc[1], full[1], rtol=1e-12, atol=1e-12)
    Jall = np.arange(m)
    acc = [np.zeros_like(full[2]), np.zeros_like(full[3])]
    for Ic in (np.arange(0, 5), np.arange(5, 10), np.arange(10, 12)):
        g = f.block_grad(Ic, Jall)
        acc[0] += len(Ic) / n * g[2]
        acc[1] += len(Ic) / n * g[3]
    np.testing.assert_allclose(acc[0], full[2], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(acc[1], full[3], rtol=1e-12, atol=1e-12)


# ---------------------------------------------------------------- Algorithm 1 bookkeeping

@pytest.mark.parametrize("shape,blocks", [((5, 4), (2, 3)), ((12, 7), (5, 3)), ((7, 12), (3, 5))])
@pytest.mark.parametrize("family,bias_corr,alpha_mode", [("poisson", 0, 0), ("negbin", 1, 1), ("negbin", 0, 1)])
def test_epochs_match_independent_matrix_form(oracle_lib, shape, blocks, family, bias_corr, alpha_mode):
    """Three epochs of the C oracle equal an independent numpy restatement of
    Algorithm 1 (brute force on tiny inputs, ragged chunks, both bias readings,
    the NB shape update, and the r < s role swap)."""
    n, m = shape
    f, D = tiny_fit(oracle_lib, n, m, 2, 1, 2, family, seed=7, nb_row=blocks[0], nb_col=blocks[1],
                    bias_corr=bias_corr, alpha_mode=alpha_mode, k0=0.3, k1=0.5, lambda_=(0.1, 0.2, 1.0, 0.3))
    W = np.random.default_rng(9).uniform(0.5, 1.5, size=(n, m))
    f, D = tiny_fit(oracle_lib, n, m, 2, 1, 2, family, seed=7, nb_row=blocks[0], nb_col=blocks[1],
                    bias_corr=bias_corr, alpha_mode=alpha_mode, k0=0.3, k1=0.5, lambda_=(0.1, 0.2, 1.0, 0.3), W=W)
    bf = BruteFit(D["Y"], D["X"], D["Z"], D["off"], D["start"], family, blocks[0], blocks[1], D["rp"], D["cp"],
                  D["settings"], W=W)
    nsw = synth.n_sweeps(n, m, blocks[0], blocks[1])
    rng = np.random.default_rng(11)
    for _ in range(3):
        sigma = rng.permutation(nsw).astype(np.int32)
        f.epoch(sigma)
        bf.epoch(sigma)
    for a, b in ((f.B, bf.B), (f.G, bf.G), (f.U, bf.U), (f.V, bf.V), (f.Gb_row, bf.GbR), (f.Hb_col, bf.HbC)):
        np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-13)
    assert f.alpha[0] == pytest.approx(bf.alpha, rel=1e-12)
    assert int(f.t[0]) == 3 * math.ceil(n / blocks[0]) * math.ceil(m / blocks[1])
    assert (f.cnt_row == 3 * math.ceil(m / blocks[1])).all()
    assert (f.cnt_col == 3 * math.ceil(n / blocks[0])).all()


def test_full_batch_unit_smoothing_is_diagonal_quasi_newton(oracle_lib):
    """With one block (r = s = 1), a1 = a2 = 1 and the per-visit correction,
    one epoch is one step of the diagonal quasi-Newton update (eq. 9-10):
    theta <- theta - rho G/H with the full-data G and H."""
    n, m = 6, 5
    f, D = tiny_fit(oracle_lib, n, m, 2, 1, 2, "negbin", seed=2, a1=1.0, a2=1.0, bias_corr=1,
                    k0=0.7, k1=0.0, damping=0.0, lambda_=(0.0, 0.0, 0.5, 0.5))
    Grow, Hrow, Gcol, Hcol, _ = f.block_grad(np.arange(n), np.arange(m))
    U0, V0, B0, G0 = f.U.copy(), f.V.copy(), f.B.copy(), f.G.copy()
    f.epoch(np.zeros(1, dtype=np.int32))
    lam = 0.5
    np.testing.assert_allclose(f.U, U0 - 0.7 * (Grow[:, 1:] + lam * U0) / (Hrow[:, 1:] + lam), rtol=1e-13)
    np.testing.assert_allclose(f.G, G0 - 0.7 * Grow[:, :1] / Hrow[:, :1], rtol=1e-13)
    np.testing.assert_allclose(f.V, V0 - 0.7 * (Gcol[:, 2:] + lam * V0) / (Hcol[:, 2:] + lam), rtol=1e-13)
    np.testing.assert_allclose(f.B, B0 - 0.7 * Gcol[:, :2] / Hcol[:, :2], rtol=1e-13)


# ---------------------------------------------------------------- convergence to known optima

def _intercepts_fit(oracle_lib, Y, X, settings, nb=None, seed=0):
    n, m = Y.shape
    rng = np.random.default_rng(seed)
    start = dict(B=np.zeros((m, X.shape[1])), Gamma=np.zeros((n, 1)), U=np.zeros((n, 0)),
                 V=np.zeros((m, 0)), alpha=1.0)
    rp, cp = rng.permutation(n).astype(np.int32), rng.permutation(m).astype(np.int32)
    return oracle_lib.OracleFit(Y, X, np.ones((m, 1)), None, start, family="poisson",
                                nb_row=nb[0] if nb else n, nb_col=nb[1] if nb else m,
                                row_perm=rp, col_perm=cp, settings=settings)


def test_d0_poisson_reaches_independence_model(oracle_lib):
    """d = 0 with a gene and a cell intercept is the Poisson independence
    model, whose MLE is mu_ij = y_i. y_.j / y_.. (textbook closed form)."""
    rng = np.random.default_rng(4)
    n, m = 30, 12
    Y = rng.poisson(np.outer(rng.uniform(1, 4, n), rng.uniform(0.5, 3, m))).astype(np.int32)
    st = synth.fit_settings(a1=1.0, a2=1.0, bias_corr=1, k0=0.5, k1=0.0, damping=0.0, lambda_=(0, 0, 0, 0))
    f = _intercepts_fit(oracle_lib, Y, np.ones((n, 1)), st)
    for _ in range(400):
        f.epoch(np.zeros(1, dtype=np.int32))
    mu = np.exp(f.eta())
    ref = np.outer(Y.sum(1), Y.sum(0)) / Y.sum()
    np.testing.assert_allclose(mu, ref, rtol=1e-8)


def _irls_vec(Y, X):
    """Independent Poisson IRLS on the vectorised design of eta_ij = x_i'b_j + g_i."""
    n, m = Y.shape
    p = X.shape[1]
    rows = []
    for i in range(n):
        for j in range(m):
            r = np.zeros(m * p + n)
            r[j * p:(j + 1) * p] = X[i]
            r[m * p + i] = 1.0
            rows.append(r)
    A = np.array(rows)
    y = Y.reshape(-1).astype(float)
    beta = np.zeros(A.shape[1])
    beta[:m * p:p] = np.log(Y.mean(0) + 0.1)
    for _ in range(100):
        eta = A @ beta
        mu = np.exp(eta)
        z = eta + (y - mu) / mu
        sw = np.sqrt(mu)
        beta = np.linalg.lstsq(A * sw[:, None], z * sw, rcond=None)[0]
    return np.exp(A @ beta).reshape(n, m)


def test_d0_poisson_with_covariate_matches_irls(oracle_lib):
    rng = np.random.default_rng(8)
    n, m = 25, 8
    X = np.hstack([np.ones((n, 1)), rng.standard_normal((n, 1))])
    mu0 = np.exp(0.5 + 0.4 * X[:, 1:2] * rng.standard_normal((1, m)) + 0.3 * rng.standard_normal((n, 1)))
    Y = rng.poisson(mu0).astype(np.int32)
    st = synth.fit_settings(a1=1.0, a2=1.0, bias_corr=1, k0=0.4, k1=0.0, damping=0.0, lambda_=(0, 0, 0, 0))
    f = _intercepts_fit(oracle_lib, Y, X, st)
    for _ in range(1500):
        f.epoch(np.zeros(1, dtype=np.int32))
    np.testing.assert_allclose(np.exp(f.eta()), _irls_vec(Y, X), rtol=1e-7)


def test_d0_stochastic_blocks_reach_the_optimum_deviance(oracle_lib):
    """The block-wise stochastic method (r, s > 1, smoothing on) gets within
    1e-3 relative of the MLE deviance of the independence model."""
    rng = np.random.default_rng(6)
    n, m = 60, 24
    Y = rng.poisson(np.outer(rng.uniform(1, 4, n), rng.uniform(0.5, 3, m))).astype(np.int32)
    ref = np.outer(Y.sum(1), Y.sum(0)) / Y.sum()
    d_opt = sum(oracle_lib.entry_deviance(0, y, mu) for y, mu in zip(Y.ravel(), ref.ravel()))
    st = synth.fit_settings(k0=0.5, k1=0.02, tau=0.75, lambda_=(0, 0, 0, 0), bias_corr=1)
    f = _intercepts_fit(oracle_lib, Y, np.ones((n, 1)), st, nb=(20, 8))
    start_dev = f.deviance()
    for e in range(300):
        f.epoch(np.random.default_rng(e).permutation(3).astype(np.int32))
    assert f.deviance() < start_dev
    assert f.deviance() == pytest.approx(d_opt, rel=1e-3)


def test_nb_moment_estimator_recovers_shape(oracle_lib):
    """App. B moment estimator: sum w mu^2 / sum w((y-mu)^2 - mu) recovers a
    known NB shape from data drawn with the true mu plugged in."""
    rng = np.random.default_rng(12)
    n, m, alpha = 400, 500, 2.0
    b = rng.uniform(-0.5, 1.5, m)
    g = rng.uniform(-0.5, 0.5, n)
    mu = np.exp(b[None, :] + g[:, None])
    Y = rng.negative_binomial(alpha, alpha / (alpha + mu)).astype(np.int32)
    start = dict(B=b[:, None].copy(), Gamma=g[:, None].copy(), U=np.zeros((n, 0)), V=np.zeros((m, 0)), alpha=alpha)
    f = oracle_lib.OracleFit(Y, np.ones((n, 1)), np.ones((m, 1)), None, start, family="negbin", nb_row=n,
                             nb_col=m, row_perm=np.arange(n, dtype=np.int32), col_perm=np.arange(m, dtype=np.int32),
                             settings=synth.fit_settings())
    sums = f.block_grad(np.arange(n), np.arange(m))[4]
    assert sums[0] == pytest.approx(float((mu ** 2).sum()), rel=1e-12)
    ahat = sums[0] / sums[1]
    # Var(y) = mu + mu^2/alpha; the ratio's sampling sd here is about 0.02.
    assert abs(ahat - alpha) < 0.1


# ---------------------------------------------------------------- Algorithm 2

@pytest.mark.parametrize("mode", ["B1", "B2", "B3"])
def test_orthogonalize_invariants(mode):
    from oracle.orth import orthogonalize
    rng = np.random.default_rng(13)
    n, m, p, q, d = 40, 15, 2, 2, 3
    X = np.hstack([np.ones((n, 1)), rng.standard_normal((n, p - 1))])
    Z = np.hstack([np.ones((m, 1)), rng.standard_normal((m, q - 1))])
    B, G = rng.standard_normal((m, p)), rng.standard_normal((n, q))
    U, V = rng.standard_normal((n, d)), rng.standard_normal((m, d))
    eta0 = X @ B.T + G @ Z.T + U @ V.T
    B2, G2, U2, V2 = orthogonalize(X, Z, B, G, U, V, mode)
    np.testing.assert_allclose(X @ B2.T + G2 @ Z.T + U2 @ V2.T, eta0, atol=1e-10)
    np.testing.assert_allclose(X.T @ G2, 0, atol=1e-10)
    np.testing.assert_allclose(X.T @ U2, 0, atol=1e-10)
    # every mode: (B3) whitens and triangularises V by multiplying it on the right, which keeps Z'V = 0
    np.testing.assert_allclose(Z.T @ V2, 0, atol=1e-10)
    if mode == "B1":
        np.testing.assert_allclose(V2.T @ V2, np.eye(d), atol=1e-10)
        S = U2.T @ U2
        np.testing.assert_allclose(S - np.diag(np.diag(S)), 0, atol=1e-9)
        assert np.all(np.diff(np.diag(S)) < 0)
        assert np.all(V2[0] > 0)
    if mode == "B2":
        np.testing.assert_allclose(U2.T @ U2, np.eye(d), atol=1e-10)
        assert np.all(U2[0] > 0)
    if mode == "B3":
        Uc = U2 - U2.mean(0)
        np.testing.assert_allclose(Uc.T @ Uc / n, np.eye(d), atol=1e-10)
        np.testing.assert_allclose(np.triu(V2[:d, :d], 1), 0, atol=1e-10)
        assert np.all(np.diag(V2) > 0)


def test_orthogonalize_b1_matches_qr_route():
    """The explicit n x m SVD of Algorithm 2 equals the thin-QR route
    U = Qu Ru, V = Qv Rv, svd(Ru Rv') on a 6 x 5 problem."""
    from oracle.orth import orthogonalize
    rng = np.random.default_rng(14)
    n, m, d = 6, 5, 2
    X, Z = np.ones((n, 1)), np.ones((m, 1))
    B, G = rng.standard_normal((m, 1)), rng.standard_normal((n, 1))
    U, V = rng.standard_normal((n, d)), rng.standard_normal((m, d))
    B2, G2, U2, V2 = orthogonalize(X, Z, B, G, U, V, "B1")
    Uc = U - X @ np.linalg.solve(X.T @ X, X.T @ U)
    Vc = V - Z @ np.linalg.solve(Z.T @ Z, Z.T @ V)
    Qu, Ru = np.linalg.qr(Uc)
    Qv, Rv = np.linalg.qr(Vc)
    P, S, Qt = np.linalg.svd(Ru @ Rv.T)
    Uq, Vq = Qu @ P * S, Qv @ Qt.T
    sgn = np.sign(Vq[0])
    np.testing.assert_allclose(U2, Uq * sgn, atol=1e-10)
    np.testing.assert_allclose(V2, Vq * sgn, atol=1e-10)


# ---------------------------------------------------------------- per-cell Fisher scoring

@pytest.mark.parametrize("family", ["poisson", "negbin"])
def test_projection_converges_to_stationary_point(family):
    from oracle.project import project_cells
    rng = np.random.default_rng(15)
    n, m, p, d = 6, 40, 2, 3
    X = np.hstack([np.ones((n, 1)), rng.standard_normal((n, 1))])
    Z = np.ones((m, 1))
    B, V = 0.3 * rng.standard_normal((m, p)), 0.5 * rng.standard_normal((m, d))
    mu = np.exp(X @ B.T + 0.5 * rng.standard_normal((n, d)) @ V.T)
    Y = rng.poisson(mu)
    U, G, dev = project_cells(Y, X, None, B, Z, V, family=family, alpha=3.0, n_steps=30, lam_u=1.0)
    h = 1e-6
    for i in range(n):
        th = np.concatenate([G[i], U[i]])

        def f(th):
            e = X[i] @ B.T + th[:1] @ Z.T + th[1:] @ V.T
            return -loglik(family, Y[i], np.exp(e), 3.0).sum() + 0.5 * (th[1:] ** 2).sum()

        for c in range(len(th)):
            e = np.zeros_like(th); e[c] = h
            assert abs((f(th + e) - f(th - e)) / (2 * h)) < 1e-6


def test_projection_gamma_closed_form_is_fixed_point():
    """Poisson, u fixed (d = 0): the closed-form gamma is the exact row optimum,
    and Fisher scoring from gamma = 0 converges to it."""
    from oracle.project import project_cells
    rng = np.random.default_rng(16)
    n, m = 5, 30
    X = np.ones((n, 1)); Z = np.ones((m, 1))
    B = rng.standard_normal((m, 1)); V = np.zeros((m, 0))
    Y = rng.poisson(np.exp(B[:, 0])[None, :] * rng.uniform(0.5, 2, (n, 1)))
    _, G_cf, _ = project_cells(Y, X, None, B, Z, V, family="poisson", alpha=1.0, n_steps=0, lam_gamma=0.0)
    _, G_1, _ = project_cells(Y, X, None, B, Z, V, family="poisson", alpha=1.0, n_steps=1, lam_gamma=0.0)
    _, G_cold, _ = project_cells(Y, X, None, B, Z, V, family="poisson", alpha=1.0, n_steps=25, lam_gamma=0.0,
                                 gamma_closed_form=False)
    np.testing.assert_allclose(G_1, G_cf, atol=1e-12)
    np.testing.assert_allclose(G_cold, G_cf, atol=1e-10)



def _far_start_case(seed):
    """A few NB cells and a warm start far from their optimum, where plain
    Fisher scoring overshoots."""
    rng = np.random.default_rng(seed)
    n, m, p, d = 4, 60, 2, 3
    X = np.hstack([np.ones((n, 1)), rng.standard_normal((n, 1))])
    Z = np.ones((m, 1))
    B = 0.3 * rng.standard_normal((m, p))
    V = rng.standard_normal((m, d)) * rng.uniform(0.3, 1.5)
    Ut = rng.standard_normal((n, d)) * rng.uniform(0.5, 2)
    a = rng.uniform(0.5, 5)
    Y = rng.poisson(rng.gamma(a, np.exp(X @ B.T + Ut @ V.T) / a))
    U0 = rng.standard_normal((n, d)) * rng.uniform(1, 3)
    return Y, X, Z, B, V, a, U0


def _row_objective(Y, X, B, Z, V, a, G, U):
    """Penalised per-cell objective from the likelihood itself (lambda_U = 1)."""
    eta = X @ B.T + G @ Z.T + U @ V.T
    return -loglik("negbin", Y, np.exp(eta), a).sum(axis=1) + 0.5 * (U ** 2).sum(axis=1)


def test_projection_step_control_never_raises_the_objective_and_converges():
    """Plain Fisher scoring from a far start overshoots (some cell ends far above
    its best iterate); with step halving the objective of the returned point
    never rises from one pass count to the next, and 40 passes reach the
    stationary point."""
    from oracle.project import project_cells
    overshoot = 0
    for seed in range(8):
        Y, X, Z, B, V, a, U0 = _far_start_case(seed)
        kw = dict(family="negbin", alpha=a, U_start=U0, lam_u=1.0)
        plain = []
        for k in range(12):
            U, G, _ = project_cells(Y, X, None, B, Z, V, n_steps=k, halving=False, **kw)
            plain.append(_row_objective(Y, X, B, Z, V, a, G, U))
        overshoot += int(np.any(plain[-1] > np.min(plain, axis=0) + 1.0))
        prev = None
        for k in range(12):
            U, G, _ = project_cells(Y, X, None, B, Z, V, n_steps=k, **kw)
            f = _row_objective(Y, X, B, Z, V, a, G, U)
            if prev is not None:
                assert np.all(f <= prev + 1e-4 * (1 + np.abs(prev))), (seed, k)
            prev = f
        U, G, _ = project_cells(Y, X, None, B, Z, V, n_steps=40, **kw)
        h = 1e-6
        for i in range(len(Y)):
            th = np.concatenate([G[i], U[i]])

            def fi(t):
                return _row_objective(Y[i:i + 1], X[i:i + 1], B, Z, V, a, t[None, :1], t[None, 1:])[0]

            for c in range(len(th)):
                e = np.zeros_like(th); e[c] = h
                assert abs((fi(th + e) - fi(th - e)) / (2 * h)) < 1e-5 * max(1.0, abs(fi(th))), (seed, i, c)
    assert overshoot >= 2


def test_projection_step_control_is_plain_fisher_when_steps_descend():
    """From the closed-form start on well-scaled cells every Fisher step lowers
    the objective, so step halving changes nothing."""
    from oracle.project import project_cells
    rng = np.random.default_rng(21)
    n, m, p, d = 6, 50, 2, 3
    X = np.hstack([np.ones((n, 1)), rng.standard_normal((n, 1))])
    Z = np.ones((m, 1))
    B, V = 0.3 * rng.standard_normal((m, p)), 0.4 * rng.standard_normal((m, d))
    Y = rng.poisson(np.exp(X @ B.T + 0.5 * rng.standard_normal((n, d)) @ V.T))
    for fam in ("poisson", "negbin"):
        a = project_cells(Y, X, None, B, Z, V, family=fam, alpha=4.0, n_steps=6)
        b = project_cells(Y, X, None, B, Z, V, family=fam, alpha=4.0, n_steps=6, halving=False)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)

# ---------------------------------------------------------------- warm-start encoder (oracle/mlp.py)

def test_mlp_gradients_match_finite_differences():
    from oracle import mlp
    rng = np.random.default_rng(30)
    P = mlp.init_params(7, 5, 4, 3, seed=1)
    for n in ("b1", "b2", "b3"):
        P[n] = 0.3 * rng.standard_normal(P[n].shape)
    Y = rng.poisson(3.0, size=(6, 7))
    T = rng.standard_normal((6, 3))
    _, g = mlp.loss_grad(P, Y, T)
    h = 1e-6
    for n in mlp.NAMES:
        flat = P[n].reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 6)):
            old = flat[idx]
            flat[idx] = old + h
            lp = mlp.loss(P, Y, T)
            flat[idx] = old - h
            lm = mlp.loss(P, Y, T)
            flat[idx] = old
            assert g[n].reshape(-1)[idx] == pytest.approx((lp - lm) / (2 * h), rel=1e-6, abs=1e-9), n


def test_mlp_gelu_is_x_times_normal_cdf():
    from scipy import stats
    from oracle import mlp
    t = np.linspace(-6, 6, 101)
    np.testing.assert_allclose(mlp.gelu(t), t * stats.norm.cdf(t), rtol=1e-12, atol=1e-14)
    h = 1e-6
    np.testing.assert_allclose(mlp.gelu_prime(t), (mlp.gelu(t + h) - mlp.gelu(t - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_mlp_adam_first_step_is_signed_learning_rate():
    """At k = 1 the bias-corrected Adam step is lr * g/(|g| + eps): -lr sign(g)."""
    from oracle import mlp
    P = mlp.init_params(4, 3, 3, 2, seed=2)
    P0 = {k: v.copy() for k, v in P.items()}
    g = {k: np.random.default_rng(3).standard_normal(v.shape) for k, v in P.items()}
    mlp.adam_step(P, g, {}, lr=0.01, eps=0.0)
    for k in P:
        np.testing.assert_allclose(P[k], P0[k] - 0.01 * np.sign(g[k]), rtol=1e-12)


# ---------------------------------------------------------------- missing entries and held-out metrics (Sec. 3.2, 5.2)

@pytest.mark.parametrize("shape,blocks", [((12, 7), (5, 3)), ((7, 12), (3, 5))])
@pytest.mark.parametrize("family,bias_corr,alpha_mode,y_dtype", [("poisson", 0, 0, np.int32), ("negbin", 1, 1, np.int32),
                                                                 ("negbin", 0, 1, np.uint16)])
def test_missing_entries_match_imputation_in_matrix_form(oracle_lib, shape, blocks, family, bias_corr, alpha_mode,
                                                         y_dtype):
    """Entries marked missing (the dtype's sentinel count) are imputed by the
    current mean at every block step, y <- mu on B minus Omega (Sec. 3.2): the
    scalar C oracle equals the matrix-form restatement that replaces the
    unobserved entries of each block by mu (three epochs, ragged chunks, both
    bias readings, the NB shape update from the completed block, r < s)."""
    n, m = shape
    obs = synth.holdout_mask(n, m, 0.3, seed=5)
    assert 0 < (~obs).sum() < n * m
    f0, D = tiny_fit(oracle_lib, n, m, 2, 1, 2, family, seed=7, nb_row=blocks[0], nb_col=blocks[1],
                     bias_corr=bias_corr, alpha_mode=alpha_mode, k0=0.3, k1=0.5, lambda_=(0.1, 0.2, 1.0, 0.3),
                     missing=1)
    Ym = synth.with_missing(D["Y"].astype(y_dtype), obs)
    f = oracle_lib.OracleFit(Ym, D["X"], D["Z"], D["off"], D["start"], family=family, nb_row=blocks[0],
                             nb_col=blocks[1], row_perm=D["rp"], col_perm=D["cp"], settings=D["settings"])
    bf = BruteFit(D["Y"], D["X"], D["Z"], D["off"], D["start"], family, blocks[0], blocks[1], D["rp"], D["cp"],
                  D["settings"], observed=obs)
    nsw = synth.n_sweeps(n, m, blocks[0], blocks[1])
    rng = np.random.default_rng(11)
    for _ in range(3):
        sigma = rng.permutation(nsw).astype(np.int32)
        f.epoch(sigma)
        bf.epoch(sigma)
    # FP64 rounding of three epochs in two summation orders (the unobserved entries make some sums cancel more)
    for a, b in ((f.B, bf.B), (f.G, bf.G), (f.U, bf.U), (f.V, bf.V), (f.Gb_row, bf.GbR), (f.Hb_col, bf.HbC)):
        np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-12)
    assert f.alpha[0] == pytest.approx(bf.alpha, rel=1e-12)


def test_missing_flag_without_missing_entries_changes_nothing(oracle_lib):
    a, D = tiny_fit(oracle_lib, 12, 7, 2, 1, 2, "negbin", seed=3, nb_row=5, nb_col=3, alpha_mode=1)
    b, _ = tiny_fit(oracle_lib, 12, 7, 2, 1, 2, "negbin", seed=3, nb_row=5, nb_col=3, alpha_mode=1, missing=1)
    for s in synth.sweep_orders(12, 7, 5, 3, 2, 3):
        a.epoch(s)
        b.epoch(s)
    for k in ("B", "G", "U", "V", "Gb_row", "Hb_col", "alpha"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))
    assert a.deviance() == b.deviance()


def test_deviance_leaves_out_missing_entries(oracle_lib):
    """With y <- mu a missing entry's unit deviance is D(mu, mu) = 0: the total
    equals the complete matrix's minus the held-out entries' unit deviances."""
    n, m = 9, 8
    obs = synth.holdout_mask(n, m, 0.3, seed=2)
    full, D = tiny_fit(oracle_lib, n, m, 2, 1, 2, "negbin", seed=4)
    f = oracle_lib.OracleFit(synth.with_missing(D["Y"], obs), D["X"], D["Z"], D["off"], D["start"], family="negbin",
                             nb_row=n, nb_col=m, row_perm=D["rp"], col_perm=D["cp"],
                             settings=synth.fit_settings(missing=1))
    mu = np.exp(full.eta())
    held = sum(oracle_lib.entry_deviance(1, D["Y"][i, j], mu[i, j], 1.0, 1.7) for i, j in zip(*np.nonzero(~obs)))
    assert f.deviance() == pytest.approx(full.deviance() - held, rel=1e-12)
    assert held > 0


def test_holdout_metrics_definitions():
    """Sec. 5.2: a perfect prediction scores 0 on both, the training mean
    scores 1 on both, and a 2 x 2 case by hand."""
    from oracle.holdout import holdout_metrics, poisson_unit_deviance
    rng = np.random.default_rng(3)
    Y = rng.poisson(3.0, (20, 15)).astype(float)
    obs = synth.holdout_mask(20, 15, 0.3, seed=1)
    e, d, ybar, nv = holdout_metrics(Y, obs, Y)
    assert e == 0.0 and d == 0.0 and nv == (~obs).sum() and ybar == pytest.approx(Y[obs].mean())
    e, d, _, _ = holdout_metrics(Y, obs, np.full(Y.shape, Y[obs].mean()))
    assert e == pytest.approx(1.0) and d == pytest.approx(1.0)
    # by hand: training entries {2, 4} (mean 3), held-out y = (0, 5) predicted as mu = (1, 4)
    Y2 = np.array([[2.0, 0.0], [5.0, 4.0]])
    obs2 = np.array([[True, False], [False, True]])
    mu2 = np.array([[9.0, 1.0], [4.0, 9.0]])
    e, d, ybar, nv = holdout_metrics(Y2, obs2, mu2)
    num = math.log(1 / 2) ** 2 + math.log(6 / 5) ** 2
    den = math.log(1 / 4) ** 2 + math.log(6 / 4) ** 2
    assert (ybar, nv) == (3.0, 2) and e == pytest.approx(num / den, rel=1e-14)
    dnum = 2 * 1.0 + 2 * (5 * math.log(5 / 4) - 1)
    dden = 2 * 3.0 + 2 * (5 * math.log(5 / 3) - 2)
    assert d == pytest.approx(dnum / dden, rel=1e-14)
    assert poisson_unit_deviance(0.0, 2.5) == pytest.approx(5.0)


# ---------------------------------------------------------------- rank selection quantities (Sec. 4.2, App. B)

@pytest.mark.parametrize("family", ["poisson", "negbin"])
def test_loglik_equals_scipy_log_pmf(family):
    from oracle.select import loglik, pearson
    rng = np.random.default_rng(4)
    mu = rng.gamma(2.0, 1.5, (30, 20))
    Y = rng.poisson(mu).astype(float)
    W = rng.uniform(0.5, 1.5, Y.shape)
    obs = synth.holdout_mask(30, 20, 0.3, seed=4)
    a = 1.7
    ref = loglik_scipy = (W * (stats.poisson.logpmf(Y, mu) if family == "poisson"
                               else stats.nbinom.logpmf(Y, a, a / (a + mu))))[obs].sum()
    assert loglik(Y, mu, family, alpha=a, W=W, observed=obs) == pytest.approx(loglik_scipy, rel=1e-12)
    nu = mu if family == "poisson" else mu + mu ** 2 / a      # Var(y) of the law
    assert pearson(Y, mu, family, alpha=a, W=W, observed=obs) == pytest.approx((W * (Y - mu) ** 2 / nu)[obs].sum(),
                                                                               rel=1e-12)
    assert ref < 0


def test_information_criteria_and_dispersion_by_hand():
    from oracle.select import aic_bic, free_params, pearson_dispersion
    assert free_params(100, 40, 2, 1, 3, "negbin") == 40 * 2 + 100 + 140 * 3 + 1
    aic, bic = aic_bic(-1000.0, 50, 4000)
    assert aic == 2100.0 and bic == pytest.approx(2000.0 + 50 * math.log(4000))
    assert pearson_dispersion(371.0, 20, 10, 2, 1, 1) == pytest.approx(371.0 / (200 - 20 - 20 - 30 - 1))


def test_eigen_ratio_rank_finds_the_gap():
    from oracle.select import eigen_ratio_rank
    assert eigen_ratio_rank([10, 8, 6, 0.6, 0.5, 0.4]) == 3
    assert eigen_ratio_rank([0.4, 9, 0.5, 10]) == 2          # any order
    # the sample singular values of a rank-4 signal plus small noise
    rng = np.random.default_rng(0)
    A = rng.standard_normal((200, 4)) @ np.diag([9, 7, 5, 4]) @ rng.standard_normal((4, 60)) / 8
    s = np.linalg.svd(A + 0.05 * rng.standard_normal(A.shape), compute_uv=False)
    assert eigen_ratio_rank(s[:20]) == 4


# ---------------------------------------------------------------- initialisation (Sec. 4.1, least-squares form)

def test_init_ols_satisfies_its_normal_equations_and_eckart_young():
    """B and Gamma solve their least-squares problems (residuals orthogonal to X and
    to Z), U V' is the best rank-d approximation of the remaining residual (it is
    orthogonal to both factors, and its squared norm is what the trailing singular
    values leave), and U'U = V'V = diag(s)."""
    from oracle.init import init_ols
    prob = synth.make_problem(300, 120, 3, 2, 4, "negbin", seed=6, zero_frac=0.7, offset=True)
    B, G, U, V, s = init_ols(prob.Y, prob.X, prob.Z, prob.offset, 4)
    zt = np.log(prob.Y + 0.5) - prob.offset[:, None]
    E1 = zt - prob.X @ B.T
    np.testing.assert_allclose(prob.X.T @ E1, 0, atol=1e-8)
    E2 = E1 - G @ prob.Z.T
    np.testing.assert_allclose(E2 @ prob.Z, 0, atol=1e-8)
    R = E2 - U @ V.T
    np.testing.assert_allclose(R @ V, 0, atol=1e-8)
    np.testing.assert_allclose(U.T @ R, 0, atol=1e-8)
    np.testing.assert_allclose(U.T @ U, np.diag(s), atol=1e-8)
    np.testing.assert_allclose(V.T @ V, np.diag(s), atol=1e-8)
    sv = np.linalg.svd(E2, compute_uv=False)
    assert np.sum(R ** 2) == pytest.approx(np.sum(sv[4:] ** 2), rel=1e-10)
    assert np.all(np.diff(s) <= 0)


def test_init_ols_starts_closer_than_the_crude_start(oracle_lib):
    """On the synthetic NB law the Sec. 4.1 start has a lower deviance than the crude
    start, and a short fit from it stays lower."""
    from oracle.init import init_ols
    n, m, d = 400, 160, 4
    prob = synth.make_problem(n, m, 2, 1, d, "negbin", seed=8, zero_frac=0.7, offset=True)
    B, G, U, V, _ = init_ols(prob.Y, prob.X, prob.Z, prob.offset, d)
    rp, cp = synth.partitions(n, m, 8)
    kw = dict(family="negbin", nb_row=100, nb_col=80, row_perm=rp, col_perm=cp, settings=synth.fit_settings())
    fi = oracle_lib.OracleFit(prob.Y, prob.X, prob.Z, prob.offset, dict(B=B, Gamma=G, U=U, V=V, alpha=1.0), **kw)
    fc = oracle_lib.OracleFit(prob.Y, prob.X, prob.Z, prob.offset, synth.crude_start(prob, d, seed=8), **kw)
    assert fi.deviance() < fc.deviance()
    for s_ in synth.sweep_orders(n, m, 100, 80, 3, 8):
        fi.epoch(s_)
        fc.epoch(s_)
    assert fi.deviance() < fc.deviance()


@pytest.mark.parametrize("family,lam", [("negbin", 0.0), ("negbin", 0.7), ("poisson", 0.3)])
def test_fit_loadings_reaches_each_columns_glm_optimum(family, lam):
    """Sec. 4.1's column GLMs for V given U: every gene's loadings equal an
    independent minimisation (BFGS) of -sum_i w_ij log f(y_ij; mu_ij) +
    lam/2 |v_j|^2 with scipy's log-pmf, and its score U'Ddot_.j - lam v_j is 0."""
    from scipy import optimize
    from oracle.init import fit_loadings
    rng = np.random.default_rng(3)
    n, m, d, alpha = 80, 6, 3, 1.3
    prob = synth.make_problem(n, m, 2, 1, d, family, seed=5, zero_frac=0.5, offset=True)
    W = rng.uniform(0.5, 1.5, (n, m))
    U = prob.U + 0.2 * rng.standard_normal(prob.U.shape)
    V0 = np.zeros((m, d))
    V, f = fit_loadings(prob.Y, prob.X, prob.Z, prob.offset, prob.B, prob.Gamma, U, V0, family=family, alpha=alpha,
                        lam_v=lam, n_steps=40, W=W)
    base = prob.X @ prob.B.T + prob.Gamma @ prob.Z.T + prob.offset[:, None]
    for j in range(m):
        obj = lambda v: -(W[:, j] * loglik(family, prob.Y[:, j], np.exp(base[:, j] + U @ v), alpha)).sum() \
            + 0.5 * lam * v @ v
        ref = optimize.minimize(obj, np.zeros(d), method="BFGS", options=dict(gtol=1e-10)).x
        np.testing.assert_allclose(V[j], ref, rtol=1e-5, atol=1e-6)
        h = 1e-6
        grad = [(obj(V[j] + h * e) - obj(V[j] - h * e)) / (2 * h) for e in np.eye(d)]
        np.testing.assert_allclose(grad, 0.0, atol=1e-5)


def test_fit_loadings_poisson_intercept_closed_form_and_monotone_objective():
    """With the design a column of ones (d = 1, lam = 0) a Poisson gene's
    loading is log(sum_i y_ij / sum_i exp(offset_ij)); from a far start the
    step control never lets a gene's objective rise with more passes."""
    from oracle.init import fit_loadings
    n, m = 50, 7
    prob = synth.make_problem(n, m, 2, 1, 1, "poisson", seed=9, offset=True)
    U = np.ones((n, 1))
    V, _ = fit_loadings(prob.Y, prob.X, prob.Z, prob.offset, prob.B, prob.Gamma, U, np.zeros((m, 1)),
                        family="poisson", alpha=1.0, n_steps=30)
    base = prob.X @ prob.B.T + prob.Gamma @ prob.Z.T + prob.offset[:, None]
    np.testing.assert_allclose(V[:, 0], np.log(prob.Y.sum(0) / np.exp(base).sum(0)), rtol=1e-10)
    prob = synth.make_problem(60, 5, 2, 1, 2, "negbin", seed=4, zero_frac=0.4, offset=True)
    far = np.full((5, 2), 4.0)
    fs = [fit_loadings(prob.Y, prob.X, prob.Z, prob.offset, prob.B, prob.Gamma, prob.U, far, family="negbin",
                       alpha=1.0, n_steps=k)[1] for k in range(8)]
    for a, b in zip(fs, fs[1:]):
        assert (b <= a + 1e-12 * np.abs(a)).all()
    assert (fs[-1] < 0.5 * fs[0]).all()


# ---------------------------------------------------------------- per-gene NB shapes (App. B per column)

@pytest.mark.parametrize("shape,blocks", [((12, 7), (5, 3)), ((7, 12), (3, 5))])
def test_per_gene_shapes_match_matrix_form(oracle_lib, shape, blocks):
    """alpha_mode 2: every gene uses its own fixed shape in the derivatives; the
    scalar C oracle equals the matrix-form restatement with a column of shapes."""
    n, m = shape
    ac = np.random.default_rng(3).gamma(2.0, 0.5, m) + 0.2
    f0, D = tiny_fit(oracle_lib, n, m, 2, 1, 2, "negbin", seed=7, nb_row=blocks[0], nb_col=blocks[1],
                     bias_corr=1, alpha_mode=2, k0=0.3, k1=0.5, lambda_=(0.1, 0.2, 1.0, 0.3))
    f = oracle_lib.OracleFit(D["Y"], D["X"], D["Z"], D["off"], D["start"], family="negbin", nb_row=blocks[0],
                             nb_col=blocks[1], row_perm=D["rp"], col_perm=D["cp"], settings=D["settings"],
                             alpha_col=ac)
    bf = BruteFit(D["Y"], D["X"], D["Z"], D["off"], D["start"], "negbin", blocks[0], blocks[1], D["rp"], D["cp"],
                  D["settings"], alpha_col=ac)
    rng = np.random.default_rng(11)
    for _ in range(3):
        sigma = rng.permutation(synth.n_sweeps(n, m, blocks[0], blocks[1])).astype(np.int32)
        f.epoch(sigma)
        bf.epoch(sigma)
    for a, b in ((f.B, bf.B), (f.G, bf.G), (f.U, bf.U), (f.V, bf.V), (f.Gb_row, bf.GbR), (f.Hb_col, bf.HbC)):
        np.testing.assert_allclose(a, b, rtol=1e-11, atol=1e-13)
    # the deviance of entry (i, j) uses alpha_j (Table S1 / App. B)
    mu = np.exp(f.eta())
    ref = sum(oracle_lib.entry_deviance(1, D["Y"][i, j], mu[i, j], 1.0, ac[j]) for i in range(n) for j in range(m))
    assert f.deviance() == pytest.approx(ref, rel=1e-12)


def test_gene_shape_moments_recover_known_shapes():
    """Counts drawn from NB(mu, alpha_j) with the true means plugged in: every
    gene's moment estimate is within 25 % of its shape (20000 cells per gene)."""
    from oracle.shapes import gene_shape_moments
    rng = np.random.default_rng(5)
    n, m = 20000, 12
    a = np.linspace(0.5, 4.0, m)
    mu = rng.gamma(4.0, 1.0, (n, 1)) * rng.uniform(0.5, 2.0, (1, m))
    Y = rng.poisson(rng.gamma(a[None, :], mu / a[None, :]))
    est = gene_shape_moments(Y, mu)
    np.testing.assert_allclose(est, a, rtol=0.25)
    # a Poisson gene has no overdispersion: capped
    Yp = rng.poisson(np.full((5000, 3), 3.0))
    assert np.all(gene_shape_moments(Yp, np.full((5000, 3), 3.0), cap=1e6) >= 20)


def test_nb_gene_loglik_equals_scipy_log_pmf():
    """The per-gene NB log-likelihood (Table S1 density, lgamma terms) equals
    scipy's negative binomial log pmf with n = alpha, p = alpha / (alpha + mu)."""
    from scipy.stats import nbinom
    from oracle.shapes import nb_gene_loglik
    rng = np.random.default_rng(11)
    Y = rng.poisson(3.0, (50, 4)).astype(float)
    mu = rng.gamma(2.0, 1.5, (50, 4))
    a = np.array([0.2, 1.0, 7.5, 300.0])
    ref = nbinom.logpmf(Y, a[None, :], a[None, :] / (a[None, :] + mu)).sum(axis=0)
    np.testing.assert_allclose(nb_gene_loglik(Y, mu, a), ref, rtol=1e-12)


def test_gene_shape_ml_is_the_maximiser_and_recovers_known_shapes():
    """Newton's method in log alpha: (1) every interior estimate equals an
    independent bounded scalar maximisation of nb_gene_loglik (Brent's method in
    log alpha) within 1e-5, and the likelihood's derivative there is zero by
    central differences; (2) with counts drawn from NB(mu, alpha_j) and the true
    means, the estimates are within 15 % of the shapes (20000 cells per gene);
    (3) a Poisson gene's estimate is large (its likelihood rises towards the
    Poisson limit; a finite sample may still show slight overdispersion)."""
    from scipy.optimize import minimize_scalar
    from oracle.shapes import gene_shape_ml, nb_gene_loglik
    rng = np.random.default_rng(0)
    n, m = 20000, 6
    mu = np.exp(rng.normal(0, 0.8, (n, m)))
    a_true = np.array([0.3, 1.0, 2.0, 5.0, 20.0, np.inf])
    Y = np.empty((n, m))
    for j in range(m):
        Y[:, j] = rng.poisson(mu[:, j] if np.isinf(a_true[j]) else rng.gamma(a_true[j], mu[:, j] / a_true[j]))
    est, it = gene_shape_ml(Y, mu, np.ones(m), iters=60, tol=1e-8, lo=1e-3, hi=1e4)
    assert it < 60
    np.testing.assert_allclose(est[:5], a_true[:5], rtol=0.15)
    assert est[5] >= 100
    for j in range(6):
        f = lambda t: -nb_gene_loglik(Y[:, j:j + 1], mu[:, j:j + 1], np.exp(t))[0]
        r = minimize_scalar(f, bounds=(np.log(1e-3), np.log(1e4)), method="bounded", options={"xatol": 1e-10})
        if j < 5:  # (the Poisson gene's likelihood is too flat for Brent's method to place to 1e-5)
            assert est[j] == pytest.approx(np.exp(r.x), rel=1e-5)
        assert f(np.log(est[j])) <= f(r.x) + 1e-9 * abs(f(r.x))
        h = 1e-5 * est[j]
        d = (nb_gene_loglik(Y[:, j:j + 1], mu[:, j:j + 1], est[j] + h)[0]
             - nb_gene_loglik(Y[:, j:j + 1], mu[:, j:j + 1], est[j] - h)[0]) / (2 * h)
        assert abs(d) * est[j] <= 1e-5 * n
    # weights and missing entries: an entry with weight 0 (or unobserved) does not count
    W = np.ones((n, m))
    W[: n // 2] = 0.0
    e1, _ = gene_shape_ml(Y, mu, np.ones(m), iters=60, W=W)
    e2, _ = gene_shape_ml(Y[n // 2:], mu[n // 2:], np.ones(m), iters=60)
    obs = W > 0
    e3, _ = gene_shape_ml(Y, mu, np.ones(m), iters=60, observed=obs)
    np.testing.assert_allclose(e1, e2, rtol=1e-12)
    np.testing.assert_allclose(e3, e2, rtol=1e-12)
