"""Pins of the VI oracle (Sec. 2.4, Table 1) to facts outside it:

- log q against scipy's multivariate normal density;
- d log q / d phi against central differences of scipy's density through
  the Cholesky bijector (layout: u packed row by row, diagonal exponentiated);
- both gradient estimators, averaged over many draws, against the closed-form
  gradient of KL(N(mu, Sigma) || N(m, S)) (a Gaussian target makes the ELBO
  loss the KL itself), and the loss against the closed-form KL;
- the pathwise estimator at fixed draws against central differences of the
  sample-mean loss on a non-Gaussian target;
- Table 1's constants and the quadratic warm-up of the learning rate;
- a VI run on a Gaussian target recovering its mean and covariance.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import vi_oracle as vo


def _rand_phi(rng, d, scale=0.3):
    mu = rng.normal(size=d)
    L = np.tril(rng.normal(size=(d, d)) * scale)
    np.fill_diagonal(L, np.exp(rng.normal(size=d) * 0.3))
    return vo.pack(mu, L)


def _mvn_logpdf_phi(phi, d, z):
    mu, L = vo.unpack(phi, d)
    return stats.multivariate_normal(mean=mu, cov=L @ L.T).logpdf(z)


def test_constants_match_table1(golden_constants):
    g = golden_constants
    assert vo.K_VI == g["vi_iterations"] and vo.N_VI == g["vi_samples"]
    assert vo.LR_PEAK == g["vi_lr_peak"] and vo.LR_WARMUP == g["vi_lr_warmup"]
    assert vo.SIGMA_INIT == g["vi_sigma_init"]
    d = 22
    mu, L = vo.unpack(vo.initial_phi(np.arange(d) * 0.1), d)
    np.testing.assert_allclose(L @ L.T, g["vi_sigma_init"] * np.eye(d), rtol=1e-14, atol=0)
    np.testing.assert_array_equal(mu, np.arange(d) * 0.1)
    assert vo.n_params(d) == d + 253


def test_bijector_layout_and_roundtrip():
    rng = np.random.default_rng(0)
    d = 5
    phi = rng.normal(size=vo.n_params(d))
    mu, L = vo.unpack(phi, d)
    assert np.all(np.triu(L, 1) == 0)
    assert L[0, 0] == pytest.approx(math.exp(phi[d]))
    assert L[1, 0] == phi[d + 1] and L[1, 1] == pytest.approx(math.exp(phi[d + 2]))
    assert L[4, 2] == phi[d + 10 + 2]
    np.testing.assert_allclose(vo.pack(mu, L), phi, rtol=1e-14, atol=1e-15)
    # Sigma = L L^T is positive definite for any phi
    assert np.all(np.linalg.eigvalsh(L @ L.T) > 0)


def test_log_q_matches_scipy():
    rng = np.random.default_rng(1)
    for d in (1, 3, 22):
        phi = _rand_phi(rng, d)
        mu, L = vo.unpack(phi, d)
        z = mu + rng.normal(size=(7, d)) @ L.T * 1.5
        np.testing.assert_allclose(vo.log_q(z, mu, L), np.atleast_1d(_mvn_logpdf_phi(phi, d, z)), rtol=1e-11)


def test_grad_log_q_matches_differences_of_scipy_density():
    rng = np.random.default_rng(2)
    d = 4
    phi = _rand_phi(rng, d)
    mu, L = vo.unpack(phi, d)
    z = mu + rng.normal(size=(3, d)) @ L.T
    g = vo.grad_log_q(z, mu, L)
    h = 1e-5
    for k in range(len(phi)):
        e = np.zeros_like(phi)
        e[k] = h
        fd = (_mvn_logpdf_phi(phi + e, d, z) - _mvn_logpdf_phi(phi - e, d, z)) / (2 * h)
        np.testing.assert_allclose(g[:, k], fd, rtol=1e-6, atol=1e-7)


def _kl_and_grad(phi, d, m, S):
    """Closed-form KL(N(mu, L L^T) || N(m, S)) and its gradient in phi."""
    mu, L = vo.unpack(phi, d)
    Si = np.linalg.inv(S)
    Sig = L @ L.T
    r = m - mu
    kl = 0.5 * (np.trace(Si @ Sig) + r @ Si @ r - d + np.linalg.slogdet(S)[1] - np.linalg.slogdet(Sig)[1])
    gmu = Si @ (mu - m)
    gL = np.tril(Si @ L) - np.diag(1.0 / np.diag(L))
    out = list(gmu)
    for i in range(d):
        for j in range(i + 1):
            out.append(gL[i, j] * L[i, i] if i == j else gL[i, j])
    return kl, np.array(out)


def test_estimators_average_to_the_closed_form_kl_gradient():
    rng = np.random.default_rng(3)
    d = 3
    A = rng.normal(size=(d, d))
    S = A @ A.T + 0.5 * np.eye(d)
    m = rng.normal(size=d)
    target = stats.multivariate_normal(mean=m, cov=S)
    phi = _rand_phi(rng, d, 0.2)
    kl, gk = _kl_and_grad(phi, d, m, S)
    n = 40000
    eps = rng.normal(size=(n, d))
    z = vo.samples(phi, eps)
    logp = target.logpdf(z)
    grad_z = -(z - m) @ np.linalg.inv(S)
    # pathwise: per-draw terms, mean and standard error
    lp, gp = vo.elbo_grad_pathwise(phi, eps, logp, grad_z)
    terms = np.array([vo.elbo_grad_pathwise(phi, eps[i:i + 1], logp[i:i + 1], grad_z[i:i + 1])[1]
                      for i in range(0, 4000)])
    se_p = terms.std(axis=0) / math.sqrt(n) + 1e-12
    assert np.all(np.abs(gp - gk) < 5 * se_p), (gp, gk)
    assert abs(lp - kl) < 0.05
    # score function (Eq. elbo-grad)
    ls, gs = vo.elbo_grad_score(phi, eps, logp)
    mu, L = vo.unpack(phi, d)
    f = vo.log_q(z, mu, L) - logp
    per = f[:, None] * vo.grad_log_q(z, mu, L)
    se_s = per.std(axis=0) / math.sqrt(n)
    assert np.all(np.abs(gs - gk) < 5 * se_s), (gs, gk, se_s)
    assert np.max(se_s) < 0.1 * np.max(np.abs(gk))   # the check has power
    assert ls == lp


def test_pathwise_equals_differences_of_the_sample_loss():
    rng = np.random.default_rng(4)
    d = 4
    a = rng.normal(size=d)

    def logp_fn(z):
        return -0.25 * np.sum(z ** 4, axis=1) - z @ a, -(z ** 3) - a

    phi = _rand_phi(rng, d)
    eps = rng.normal(size=(16, d))

    def loss(ph):
        z = vo.samples(ph, eps)
        return np.mean(_mvn_logpdf_phi(ph, d, z) - logp_fn(z)[0])

    z = vo.samples(phi, eps)
    lp, gz = logp_fn(z)
    l0, g = vo.elbo_grad_pathwise(phi, eps, lp, gz)
    assert l0 == pytest.approx(loss(phi), rel=1e-12)
    h = 1e-6
    for k in range(len(phi)):
        e = np.zeros_like(phi)
        e[k] = h
        assert g[k] == pytest.approx((loss(phi + e) - loss(phi - e)) / (2 * h), rel=1e-5, abs=1e-6)


def test_learning_rate_schedule(golden_constants):
    peak, T = golden_constants["vi_lr_peak"], int(golden_constants["vi_lr_warmup"])
    lr = np.array([vo.learning_rate(t) for t in range(1001)])
    assert lr[0] == 0.0
    assert lr[T] == pytest.approx(peak) and lr[1000] == pytest.approx(peak)
    assert np.all(np.diff(lr) >= 0)
    # quadratic on [0, T]: constant second difference
    d2 = np.diff(lr[:T + 1], 2)
    np.testing.assert_allclose(d2, d2[0], rtol=1e-8)
    assert lr[T // 2] == pytest.approx(0.75 * peak)


def test_vi_recovers_a_gaussian_target():
    rng = np.random.default_rng(5)
    d = 4
    A = rng.normal(size=(d, d))
    S = (A @ A.T + 0.3 * np.eye(d)) * 0.01
    m = rng.normal(size=d)
    Si = np.linalg.inv(S)
    phi = vo.initial_phi(m + 0.05 * rng.normal(size=d))
    mom, vel = np.zeros_like(phi), np.zeros_like(phi)
    for t in range(1, 3001):
        eps = rng.normal(size=(128, d))
        z = vo.samples(phi, eps)
        r = z - m
        logp = -0.5 * np.einsum("ni,ij,nj->n", r, Si, r)
        lr = 2e-2 if t < 2000 else 2e-3
        phi, mom, vel, _, _ = vo.vi_step(phi, mom, vel, t, eps, logp, -r @ Si, estimator="pathwise", lr=lr)
    mu, L = vo.unpack(phi, d)
    sd = np.sqrt(np.diag(S))
    assert np.all(np.abs(mu - m) / sd < 0.1)
    assert np.all(np.abs(L @ L.T - S) < 0.1 * sd[:, None] * sd[None, :])
