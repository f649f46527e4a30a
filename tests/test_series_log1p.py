"""Error bound of the series log1p the tensor-core deviance kernel uses for the
negative binomial term (softplus(eta - log alpha) = max(z, 0) + log1p(e^-|z|)):
log1p(t) = 2 (s + s^3/3 + ... + s^15/15), s = t / (2 + t), t in [0, 1]
(Abramowitz and Stegun 4.1.27). The same operations, in the same order, in
float32 numpy; the kernel's totals are also held to the FP64 oracle and to the
CUDA-core kernel (library log1pf) by the GPU tests."""
import numpy as np

F = np.float32


def log1p_01(t):
    t = F(t)
    s = F(t / F(F(2) + t))
    s2 = F(s * s)
    p = F(1 / 15)
    for c in (13, 11, 9, 7, 5, 3):
        p = F(F(p * s2) + F(1 / c))
    return F(F(2) * F(F(F(s * s2) * p) + s))


def test_series_log1p_is_within_two_float32_ulps_on_its_interval():
    ts = np.concatenate([np.logspace(-12, 0, 4000), np.linspace(0.3, 1.0, 2000)])
    rel = np.array([abs(float(log1p_01(t)) - np.log1p(float(F(t)))) / np.log1p(float(F(t))) for t in ts])
    assert rel.max() < 2.4e-7      # two units of float32 relative spacing (1.19e-7)


def test_softplus_form_equals_log1p_of_the_ratio():
    """alpha softplus(eta - log alpha) = alpha log1p(mu / alpha): the zero-count NB term."""
    for alpha in (0.2, 1.0, 5.0):
        for eta in np.linspace(-12, 6, 200):
            z = eta - np.log(alpha)
            sp = max(z, 0.0) + float(log1p_01(np.exp(-abs(z))))
            ref = np.log1p(np.exp(eta) / alpha)
            assert abs(sp - ref) <= 3e-7 * ref + 1e-7 * max(z, 0.0)
