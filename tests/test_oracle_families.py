"""Pins of the oracle's other exponential families (Table S1) and of the
smoothed Pearson dispersion (App. B), against what the densities and the
mathematics fix.

Families: Gaussian (identity link), Bernoulli (logit link), Gamma and inverse
Gaussian (log link), with the dispersion phi in the family's scalar slot.
The densities come from scipy.stats, written in the usual mean / shape
parametrisations, so a wrong variance function, link derivative, sign or
power of mu in the oracle shows up as a mismatch.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

import synth
from tests.bruteforce import BruteFit

FAM = {"gaussian": 2, "binomial": 3, "gamma": 4, "invgauss": 5}
CONT = ("gaussian", "gamma", "invgauss")


def mean_of(family, eta):
    if family == "gaussian":
        return eta
    if family == "binomial":
        return 1.0 / (1.0 + math.exp(-eta))
    return math.exp(eta)


def logpdf(family, y, mu, phi):
    """log f(y; mu, phi) in scipy's parametrisations (mean mu, dispersion phi)."""
    if family == "gaussian":
        return stats.norm.logpdf(y, loc=mu, scale=math.sqrt(phi))
    if family == "binomial":
        return stats.bernoulli.logpmf(y, mu)
    if family == "gamma":                      # shape 1/phi, scale mu phi: mean mu, variance phi mu^2
        return stats.gamma.logpdf(y, 1.0 / phi, scale=mu * phi)
    lam = 1.0 / phi                            # inverse Gaussian with mean mu and shape lambda: variance mu^3 / lambda
    return stats.invgauss.logpdf(y, mu / lam, scale=lam)


YS = {"gaussian": (-1.3, 0.0, 0.4, 2.5), "binomial": (0.0, 1.0), "gamma": (0.05, 0.7, 3.0), "invgauss": (0.1, 0.9, 4.0)}
ETAS = {"gaussian": (-1.5, 0.2, 2.0), "binomial": (-2.0, 0.3, 2.5), "gamma": (-1.0, 0.3, 1.2),
        "invgauss": (-0.8, 0.1, 0.9)}


def obs_factor(family, y, mu):
    """alpha(mu) = 1 + (y - mu)(nu'/nu + g''/g') of Sec. 3 for these links."""
    if family in ("gaussian", "binomial"):     # canonical links: observed = expected
        return 1.0
    if family == "gamma":                      # nu = mu^2, g = log: 2/mu - 1/mu
        return 1.0 + (y - mu) / mu
    return 1.0 + 2.0 * (y - mu) / mu           # nu = mu^3: 3/mu - 1/mu


@pytest.mark.parametrize("family", list(FAM))
def test_family_derivatives_match_finite_differences(oracle_lib, family):
    """Ddot = d (w log f)/d eta and the observed second derivative equals
    Dddot * alpha(mu) (Sec. 3), with phi entering as 1/phi."""
    h1, h2 = 1e-5, 2e-3
    for y in YS[family]:
        for eta in ETAS[family]:
            for phi in ((1.0,) if family == "binomial" else (0.3, 1.7)):
                for w in (1.0, 0.6):
                    mu, dd, ddd = oracle_lib.entry(FAM[family], y, eta, w, phi)
                    assert mu == pytest.approx(mean_of(family, eta), rel=1e-15)
                    f = lambda e: w * logpdf(family, y, mean_of(family, e), phi)
                    fd1 = (f(eta + h1) - f(eta - h1)) / (2 * h1)
                    fd2 = -(f(eta + h2) - 2 * f(eta) + f(eta - h2)) / h2 ** 2
                    scale = 1.0 + abs(f(eta))
                    assert dd == pytest.approx(fd1, rel=1e-7, abs=1e-9 * scale)
                    assert ddd * obs_factor(family, y, mu) == pytest.approx(fd2, rel=2e-5, abs=1e-7 * scale)


@pytest.mark.parametrize("family", list(FAM))
def test_family_fisher_weight_is_expected_information(oracle_lib, family):
    """Dddot = E_y[-d^2 log f / d eta^2] under y ~ f(mu, phi) (quadrature over
    the density, a sum for the Bernoulli)."""
    h = 1e-4
    for eta in ETAS[family][:2]:
        phi = 1.0 if family == "binomial" else 0.4
        mu, _, ddd = oracle_lib.entry(FAM[family], 0.0, eta, 1.0, phi)
        obs = lambda y: -(logpdf(family, y, mean_of(family, eta + h), phi) - 2 * logpdf(family, y, mu, phi)
                          + logpdf(family, y, mean_of(family, eta - h), phi)) / h ** 2
        dens = lambda y: math.exp(logpdf(family, y, mu, phi))
        if family == "binomial":
            ex = sum(dens(y) * obs(y) for y in (0.0, 1.0))
        else:
            lo = -np.inf if family == "gaussian" else 0.0
            ex = integrate.quad(lambda y: dens(y) * obs(y), lo, np.inf, limit=200)[0]
        assert ex == pytest.approx(ddd, rel=1e-4)


@pytest.mark.parametrize("family", list(FAM))
def test_family_deviance_is_the_scaled_likelihood_ratio(oracle_lib, family):
    """D(y, mu) = -2 phi w [log f(y; mu) - log f(y; y)], i.e. 2 w times Table
    S1's D / 2a(phi) column with a(phi) = phi / w: zero at mu = y, positive
    elsewhere, linear in w, free of phi."""
    for y in YS[family]:
        for eta in ETAS[family]:
            mu = mean_of(family, eta)
            for phi in ((1.0,) if family == "binomial" else (0.3, 2.0)):
                sat = 0.0 if family == "binomial" else logpdf(family, y, y, phi)
                ref = -2 * phi * (logpdf(family, y, mu, phi) - sat)
                got = oracle_lib.entry_deviance(FAM[family], y, mu, 1.0, phi)
                assert got == pytest.approx(ref, rel=1e-9, abs=1e-11)
                assert got >= 0
                assert oracle_lib.entry_deviance(FAM[family], y, mu, 0.3, phi) == pytest.approx(0.3 * got, rel=1e-12)
        if family != "binomial":
            assert abs(oracle_lib.entry_deviance(FAM[family], y, y, 1.0, 1.0)) < 1e-12


def family_fit(oracle_lib, family, n, m, nb_row, nb_col, *, seed=7, d=2, missing=False, **kw):
    P = synth.make_family_problem(n, m, 2, 1, d, family, phi=0.3, seed=seed, offset=True,
                                  shift=0.5 if family in ("gamma", "invgauss") else 0.0)
    rng = np.random.default_rng(seed)
    start = dict(B=P.B + 0.2 * rng.standard_normal(P.B.shape), Gamma=P.Gamma + 0.2 * rng.standard_normal(P.Gamma.shape),
                 U=P.U + 0.2 * rng.standard_normal(P.U.shape), V=P.V + 0.2 * rng.standard_normal(P.V.shape),
                 alpha=0.8 if family != "binomial" else 1.0)
    rp, cp = rng.permutation(n).astype(np.int32), rng.permutation(m).astype(np.int32)
    obs = synth.holdout_mask(n, m, 0.3, seed=5) if missing else np.ones((n, m), bool)
    Y = synth.with_missing(P.Y, obs) if missing else P.Y
    settings = synth.fit_settings(missing=int(missing), **kw)
    f = oracle_lib.OracleFit(Y, P.X, P.Z, P.offset, start, family=family, nb_row=nb_row, nb_col=nb_col,
                             row_perm=rp, col_perm=cp, settings=settings)
    bf = BruteFit(P.Y, P.X, P.Z, P.offset, start, family, nb_row, nb_col, rp, cp, settings, observed=obs)
    return f, bf, P


@pytest.mark.parametrize("shape,blocks", [((12, 7), (5, 3)), ((7, 12), (3, 5))])
@pytest.mark.parametrize("family,alpha_mode,missing", [("gaussian", 1, False), ("binomial", 0, False),
                                                       ("gamma", 1, False), ("invgauss", 1, True),
                                                       ("gaussian", 0, True)])
def test_family_epochs_match_independent_matrix_form(oracle_lib, shape, blocks, family, alpha_mode, missing):
    """Three epochs of the C oracle equal the matrix-form restatement (closed
    forms of each family's score and Fisher weight, the Pearson dispersion
    pooled per sweep) on ragged chunks and the r < s swap, with and without
    missing entries (NaN marks them in float responses)."""
    n, m = shape
    f, bf, _ = family_fit(oracle_lib, family, n, m, blocks[0], blocks[1], alpha_mode=alpha_mode, missing=missing,
                          k0=0.3, k1=0.5, lambda_=(0.1, 0.2, 1.0, 0.3), bias_corr=1)
    nsw = synth.n_sweeps(n, m, blocks[0], blocks[1])
    rng = np.random.default_rng(11)
    a0 = float(f.alpha[0])
    for _ in range(3):
        sigma = rng.permutation(nsw).astype(np.int32)
        f.epoch(sigma)
        bf.epoch(sigma)
    for a, b in ((f.B, bf.B), (f.G, bf.G), (f.U, bf.U), (f.V, bf.V), (f.Gb_row, bf.GbR), (f.Hb_col, bf.HbC)):
        np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-12)
    assert f.alpha[0] == pytest.approx(bf.alpha, rel=1e-12)
    assert (f.alpha[0] != a0) == (alpha_mode == 1)


@pytest.mark.parametrize("family", CONT)
def test_pearson_dispersion_recovers_phi(oracle_lib, family):
    """App. B: at the generating parameters one full-batch sweep with rho = 1
    sets phi to (1/N) sum w (y - mu)^2 / nu(mu), N = nm - mp - nq - (n+m)d - 1,
    whose expectation there is phi nm / N: within four standard errors, and
    distinguishable from phi itself (N drops (n+m)d + ... = 5 % of nm)."""
    n, m, d, phi = 300, 200, 4, 0.3
    P = synth.make_family_problem(n, m, 2, 1, d, family, phi=phi, seed=3, offset=False,
                                  shift=0.3 if family != "gaussian" else 0.0)
    start = dict(B=P.B, Gamma=P.Gamma, U=P.U, V=P.V, alpha=5.0)
    st = synth.fit_settings(alpha_mode=1, k0=1.0, k1=0.0)
    f = oracle_lib.OracleFit(P.Y, P.X, P.Z, P.offset, start, family=family, nb_row=n, nb_col=m,
                             row_perm=np.arange(n, dtype=np.int32), col_perm=np.arange(m, dtype=np.int32),
                             settings=st)
    f.epoch(np.zeros(1, dtype=np.int32))
    N = n * m - m * 2 - n * 1 - (n + m) * d - 1
    expect = phi * n * m / N
    # standard error of the mean of (y - mu)^2 / nu(mu): its variance over phi^2 is 2 (Gaussian), 2 + 6 phi
    # (Gamma: the fourth cumulant), 2 + 15 phi mu (inverse Gaussian, at the largest mean) -- bounded generously
    mu_max = float(np.exp(P.X @ P.B.T + P.Gamma @ P.Z.T + P.U @ P.V.T).max()) if family != "gaussian" else 1.0
    kurt = {"gaussian": 2.0, "gamma": 2.0 + 6 * phi, "invgauss": 2.0 + 15 * phi * mu_max}[family]
    se = phi * math.sqrt(kurt / (n * m)) * n * m / N
    assert abs(f.alpha[0] - expect) < 4 * se
    if family == "gaussian":
        assert abs(f.alpha[0] - phi) > 4 * se


def test_gaussian_d0_full_batch_reaches_least_squares(oracle_lib):
    """Gaussian with the identity link, d = 0, gene coefficients on [1, x_i] and
    a cell intercept: full-batch smoothing-free steps converge to the
    least-squares fit of the vectorised design (numpy lstsq)."""
    rng = np.random.default_rng(8)
    n, m = 20, 7
    X = np.hstack([np.ones((n, 1)), rng.standard_normal((n, 1))])
    Y = (X @ rng.standard_normal((2, m)) + 0.5 * rng.standard_normal((n, 1))
         + 0.3 * rng.standard_normal((n, m))).astype(np.float32)
    start = dict(B=np.zeros((m, 2)), Gamma=np.zeros((n, 1)), U=np.zeros((n, 0)), V=np.zeros((m, 0)), alpha=1.0)
    st = synth.fit_settings(a1=1.0, a2=1.0, bias_corr=1, k0=0.5, k1=0.0, damping=0.0, lambda_=(0, 0, 0, 0))
    f = oracle_lib.OracleFit(Y, X, np.ones((m, 1)), None, start, family="gaussian", nb_row=n, nb_col=m,
                             row_perm=rng.permutation(n).astype(np.int32), col_perm=rng.permutation(m).astype(np.int32),
                             settings=st)
    for _ in range(3000):
        f.epoch(np.zeros(1, dtype=np.int32))
    rows = []
    for i in range(n):
        for j in range(m):
            r = np.zeros(m * 2 + n)
            r[2 * j:2 * j + 2] = X[i]
            r[2 * m + i] = 1.0
            rows.append(r)
    A = np.array(rows)
    fit = A @ np.linalg.lstsq(A, Y.reshape(-1).astype(np.float64), rcond=None)[0]
    np.testing.assert_allclose(f.eta().reshape(-1), fit, rtol=1e-8, atol=1e-8)


@pytest.mark.parametrize("family", list(FAM))
def test_family_block_gradient_matches_finite_differences(oracle_lib, family):
    """Matrix level (App. B): the full-batch estimators of every free block
    [Gamma, U] and [B, V] equal the derivatives of the weighted negative
    log-likelihood from scipy's densities (phi = 0.7 where the family has one);
    for the canonical links (Gaussian, Bernoulli) the curvature estimates equal
    the exact second derivatives too."""
    n, m, p, q, d, phi = 6, 5, 2, 1, 2, 0.7
    f, _, P = family_fit(oracle_lib, family, n, m, n, m, seed=2, d=d)
    f.alpha[0] = 1.0 if family == "binomial" else phi
    rng = np.random.default_rng(4)
    W = rng.uniform(0.5, 1.5, size=(n, m))
    f.W = np.ascontiguousarray(W)
    f._data.W = f.W.ctypes.data
    Grow, Hrow, Gcol, Hcol, _ = f.block_grad(np.arange(n), np.arange(m))
    Y = P.Y.astype(np.float64)
    th = dict(B=f.B.copy(), Gamma=f.G.copy(), U=f.U.copy(), V=f.V.copy())

    def nll(T):
        eta = P.X @ T["B"].T + T["Gamma"] @ P.Z.T + T["U"] @ T["V"].T + P.offset[:, None]
        mu = np.vectorize(lambda e: mean_of(family, e))(eta)
        return -sum(W[i, j] * logpdf(family, Y[i, j], mu[i, j], f.alpha[0]) for i in range(n) for j in range(m))

    h, hh = 1e-5, 1e-3

    def fd(name, i, c):
        Tp = {k: v.copy() for k, v in th.items()}; Tm = {k: v.copy() for k, v in th.items()}
        Tp[name][i, c] += h; Tm[name][i, c] -= h
        g = (nll(Tp) - nll(Tm)) / (2 * h)
        Tp[name][i, c] += hh - h; Tm[name][i, c] -= hh - h
        return g, (nll(Tp) - 2 * nll(th) + nll(Tm)) / hh ** 2

    canonical = family in ("gaussian", "binomial")
    for i in range(n):
        for c in range(q + d):
            g, h2 = fd(*(("Gamma", i, c) if c < q else ("U", i, c - q)))
            assert Grow[i, c] == pytest.approx(g, rel=1e-6, abs=1e-6)
            if canonical:
                assert Hrow[i, c] == pytest.approx(h2, rel=1e-4, abs=1e-5)
    for j in range(m):
        for c in range(p + d):
            g, h2 = fd(*(("B", j, c) if c < p else ("V", j, c - p)))
            assert Gcol[j, c] == pytest.approx(g, rel=1e-6, abs=1e-6)
            if canonical:
                assert Hcol[j, c] == pytest.approx(h2, rel=1e-4, abs=1e-5)


@pytest.mark.parametrize("family", list(FAM))
def test_family_block_estimators_are_unbiased_over_a_partition(oracle_lib, family):
    """sum_J (|J|/m) G_row(I, J) = G_row(I, all) (eq. 15's unbiasedness) for
    every family, with a ragged last chunk."""
    n, m = 9, 7
    f, _, _ = family_fit(oracle_lib, family, n, m, n, m, seed=6)
    I = np.arange(n)
    full = f.block_grad(I, np.arange(m))
    acc = [np.zeros_like(full[0]), np.zeros_like(full[1])]
    for J in (np.array([0, 4, 6]), np.array([1, 2, 3]), np.array([5])):
        g = f.block_grad(I, J)
        acc[0] += len(J) / m * g[0]
        acc[1] += len(J) / m * g[1]
    np.testing.assert_allclose(acc[0], full[0], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(acc[1], full[1], rtol=1e-12, atol=1e-12)
