"""Pins of the MAP oracle (Sec. 2.2-2.3, Table 1) against facts other than
itself: normalisation of every prior marginal, the change-of-variables
identity behind the log-Jacobian correction, finite differences of the prior
and of the whole objective, Adam's bias-corrected first step, and the
printed schedule constants."""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle
from oracle import map_oracle as mo
from paper_2202_07663_gb300 import inputs


def _support(e):
    if e[0] == "normal":
        return e[1] - 12 * e[2], e[1] + 12 * e[2]
    if e[0] == "lognormal":
        return 1e-9, e[1] * math.exp(12 * e[2])
    if e[0] == "truncnormal":
        return e[3], e[4]
    return e[1], e[2]


@pytest.mark.parametrize("j", range(22))
def test_each_prior_marginal_is_normalised(j):
    """exp(log p_j) integrates to 1 over the support: pins the normalising
    constants (truncation mass, log-normal 1/x term, uniform width)."""
    e = mo.PRIOR[j]
    if e[0] == "lognormal":   # integrate in u = ln x, where the density is smooth and narrow
        c, w = math.log(e[1]), 12 * e[2]
        val, _ = integrate.quad(lambda u: math.exp(mo.log_prior_marginal(j, math.exp(u)) + u), c - w, c + w, limit=400)
    else:
        lo, hi = _support(e)
        val, _ = integrate.quad(lambda x: math.exp(mo.log_prior_marginal(j, x)), lo, hi, limit=400)
    assert val == pytest.approx(1.0, rel=1e-8)


def test_prior_table_matches_the_sampler_and_gradient():
    """The oracle's prior has the distributions the input sampler draws from
    (Eq. sim-dist, prior column); its gradient matches differences; the
    marginals sum to the joint."""
    for e, d in zip(mo.PRIOR, inputs.PAPER_PRIOR_DRAW):
        kind = {"normal": "n", "lognormal": "ln", "truncnormal": "tn", "uniform": "u"}[e[0]]
        assert (kind,) + tuple(e[1:]) == tuple(d)
    th = inputs.draw_table(np.random.default_rng(2), inputs.PAPER_PRIOR_DRAW, 4)
    lp, g = mo.log_prior(th)
    np.testing.assert_allclose(lp, sum(mo.log_prior_marginal(j, th[:, j]) for j in range(22)), rtol=1e-14)
    for j in range(22):
        h = 1e-6 * max(1.0, abs(th[0, j]))
        a, b = th.copy(), th.copy()
        a[:, j] += h
        b[:, j] -= h
        fd = (mo.log_prior(a)[0] - mo.log_prior(b)[0]) / (2 * h)
        np.testing.assert_allclose(g[:, j], fd, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("j", range(22))
def test_change_of_variables(j):
    """Eq. reparam-post: the j-th marginal pulled back to z with its
    log-Jacobian term is a normalised density on R (a wrong Jacobian fails)."""
    z0 = mo.inverse_bijector(inputs.draw_table(np.random.default_rng(3), inputs.PAPER_PRIOR_DRAW, 1))
    np.testing.assert_allclose(mo.inverse_bijector(mo.bijector(z0)[0]), z0, rtol=1e-9, atol=1e-9)

    def dens(x):
        z = z0.copy()
        z[0, j] = x
        th, d, _, _ = mo.bijector(z)
        return math.exp(mo.log_prior_marginal(j, th[0, j])) * d[0, j]

    lo, hi = _support(mo.PRIOR[j])
    b = mo.bijector_kind(mo.PRIOR[j])
    if b[0] == "identity":
        zlo, zhi = lo, hi
    elif b[0] == "exp":
        zlo, zhi = math.log(lo), math.log(hi)
    else:
        zlo, zhi = -60.0, 60.0
    val, _ = integrate.quad(dens, zlo, zhi, limit=400)
    assert val == pytest.approx(1.0, rel=1e-7)


def test_bijector_derivatives_match_differences():
    z = mo.inverse_bijector(inputs.draw_table(np.random.default_rng(4), inputs.PAPER_PRIOR_DRAW, 3))
    th, d, lj, dlj = mo.bijector(z)
    h = 1e-6
    for j in range(22):
        a, b = z.copy(), z.copy()
        a[:, j] += h
        b[:, j] -= h
        np.testing.assert_allclose(d[:, j], (mo.bijector(a)[0][:, j] - mo.bijector(b)[0][:, j]) / (2 * h), rtol=1e-7)
        np.testing.assert_allclose(dlj[:, j], (mo.bijector(a)[2] - mo.bijector(b)[2]) / (2 * h), atol=1e-7)
    np.testing.assert_allclose(lj, np.log(np.abs(d)).sum(axis=1), rtol=1e-12)


def test_objective_gradient_matches_differences():
    spec = inputs.SystemSpec(12, 12, 2, 3, "gaussian", inputs.PIXEL_SCALE, 0.2, 100.0)
    rng = np.random.default_rng(5)
    truth = inputs.draw_table(rng, inputs.PAPER_SIM, 1)[0]
    psf = inputs.make_psf(spec)
    D = inputs.add_noise(rng, oracle.simulate(truth, 12, 12, psf, spec.pixel_scale, 2)[0], 0.2, 100.0)
    z = mo.inverse_bijector(inputs.draw_table(rng, inputs.PAPER_PRIOR_DRAW, 1))

    def f_of(zz):
        th = mo.bijector(zz)[0]
        ll, _, gl = oracle.loglik(th, D, 0.2, psf, spec.pixel_scale, 2, 100.0, grad=True)
        return mo.objective_grad(zz, ll, gl)

    f, g = f_of(z)
    for j in range(22):
        h = 1e-5
        a, b = z.copy(), z.copy()
        a[0, j] += h
        b[0, j] -= h
        fd = (f_of(a)[0][0] - f_of(b)[0][0]) / (2 * h)
        assert g[0, j] == pytest.approx(fd, rel=1e-5, abs=1e-5 * np.abs(g).max())


def test_adam_first_step_and_convergence():
    """Bias-corrected Adam: the first step is -lr * sign(g) in every
    component (to eps); on a quadratic it converges."""
    a = np.array([[3.0, 0.5, 10.0]])
    z = np.array([[1.0, -2.0, 0.3]])
    z1, m, v = mo.adam_step(z, np.zeros_like(z), np.zeros_like(z), 1, a * z, 0.01)
    np.testing.assert_allclose(z1 - z, -0.01 * np.sign(a * z), rtol=1e-7)
    zz, m, v = z.copy(), np.zeros_like(z), np.zeros_like(z)
    for t in range(1, 4001):
        zz, m, v = mo.adam_step(zz, m, v, t, a * zz, 0.01)
    assert np.max(np.abs(zz)) < 5e-3


def test_schedule_matches_table_1(golden_constants):
    assert mo.K_MAP == golden_constants["map_iterations"]
    assert mo.N_MAP == golden_constants["map_starts"]
    assert mo.learning_rate(0) == golden_constants["map_lr_start"]
    assert mo.learning_rate(mo.K_MAP) == pytest.approx(golden_constants["map_lr_end"], rel=1e-12)
    assert mo.learning_rate(150) == pytest.approx(0.5 * (1e-2 + 1e-3), rel=1e-12)


@pytest.mark.parametrize("j", [0, 2, 10, 17])
def test_objective_without_likelihood_is_the_transformed_prior(j):
    """With log L = 0 the objective is -log p~(z), the prior of the
    unconstrained parameters (Eq. reparam-post): exp(-f) is normalised in each
    z_j, and its gradient matches differences. This isolates the log-Jacobian
    terms, which are tiny next to a likelihood gradient."""
    z0 = mo.inverse_bijector(inputs.draw_table(np.random.default_rng(6), inputs.PAPER_PRIOR_DRAW, 1))
    zero = np.zeros(1)
    f0, g0 = mo.objective_grad(z0, zero, np.zeros((1, 22)))
    h = 1e-6
    a, b = z0.copy(), z0.copy()
    a[0, j] += h
    b[0, j] -= h
    fd = (mo.objective_grad(a, zero, np.zeros((1, 22)))[0][0] - mo.objective_grad(b, zero, np.zeros((1, 22)))[0][0])
    assert g0[0, j] == pytest.approx(fd / (2 * h), rel=1e-6, abs=1e-8)
    # normalisation: integral over z_j of exp(-(f(z) - f(z0))) = 1 / p~_j(z0_j), and the
    # same integral with the j-th factor only gives p~_j(z0_j) through the marginal density
    b_kind = mo.bijector_kind(mo.PRIOR[j])

    def ratio(x):
        z = z0.copy()
        z[0, j] = x
        return math.exp(-(mo.objective_grad(z, zero, np.zeros((1, 22)))[0][0] - f0[0]))

    lo, hi = (-60.0, 60.0) if b_kind[0] != "identity" else _support(mo.PRIOR[j])
    if b_kind[0] == "exp":
        c, w = math.log(mo.PRIOR[j][1]), 12 * mo.PRIOR[j][2]
        lo, hi = c - w, c + w
    val, _ = integrate.quad(ratio, lo, hi, limit=400)
    th0, d0, _, _ = mo.bijector(z0)
    p_tilde_j = math.exp(mo.log_prior_marginal(j, th0[0, j])) * d0[0, j]
    assert val * p_tilde_j == pytest.approx(1.0, rel=1e-6)
