"""MCMC diagnostics against closed forms: AR(1) autocorrelation rho^tau and
integrated time (1+rho)/(1-rho), i.i.d. ESS = N, R-hat ~ 1 for chains from
one distribution and large for chains with different means."""
import numpy as np
import pytest

from paper_2202_07663_gb300 import diagnostics as dg


def _ar1(rng, rho, chains, n):
    x = np.empty((chains, n))
    x[:, 0] = rng.normal(size=chains) / np.sqrt(1 - rho ** 2)
    e = rng.normal(size=(chains, n))
    for t in range(1, n):
        x[:, t] = rho * x[:, t - 1] + e[:, t]
    return x


def test_autocorr_matches_ar1_and_definition():
    rng = np.random.default_rng(0)
    rho = 0.7
    x = _ar1(rng, rho, 4, 50000)
    r = dg.autocorr(x, 6).mean(axis=0)
    np.testing.assert_allclose(r[:6], rho ** np.arange(6), atol=0.02)
    # direct evaluation of the paper's formula on a short series
    y = rng.normal(size=57)
    mu = y.mean()
    c = [np.sum((y[: 57 - t] - mu) * (y[t:] - mu)) / (57 - t) for t in range(10)]
    np.testing.assert_allclose(dg.autocorr(y, 9), np.array(c) / c[0], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.9])
def test_ess_of_ar1(rho):
    rng = np.random.default_rng(1)
    chains, n = 8, 20000
    x = _ar1(rng, rho, chains, n)
    expect = chains * n * (1 - rho) / (1 + rho)
    assert dg.ess(x) == pytest.approx(expect, rel=0.12)


def test_rhat():
    rng = np.random.default_rng(2)
    same = rng.normal(size=(6, 5000))
    assert dg.rhat(same) < 1.005
    shifted = same + np.arange(6)[:, None] * 0.5
    assert dg.rhat(shifted) > 1.2
    both = np.stack([same, shifted], axis=2)
    r = dg.rhat(both)
    assert r.shape == (2,) and r[0] < 1.005 and r[1] > 1.2


def test_ess_antithetic_chains():
    # AR(1) with rho = -0.5: tau = (1 + rho) / (1 - rho) = 1/3, ESS = 3 N in
    # Geyer's form; the default form cuts the negative lag-1 term and gives N
    rng = np.random.default_rng(3)
    rho, chains, n = -0.5, 8, 20000
    x = _ar1(rng, rho, chains, n)
    assert dg.ess(x, antithetic=True) == pytest.approx(chains * n * (1 - rho) / (1 + rho), rel=0.1)
    assert dg.ess(x) == pytest.approx(chains * n, rel=0.05)
    # positive correlation: both forms agree with the closed form
    y = _ar1(rng, 0.6, chains, n)
    expect = chains * n * 0.4 / 1.6
    assert dg.ess(y, antithetic=True) == pytest.approx(expect, rel=0.12)
