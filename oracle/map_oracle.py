"""FP64 oracle of multi-start MAP (arXiv:2202.07663, Sec. 2.2-2.3, Table 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). Plain numpy/scipy
statement of:
  * the prior of Eq. sim-dist (the broader "prior" values), a product of
    independent marginals, evaluated with scipy.stats;
  * the component-wise bijector g of Sec. 2.2 (exp for positive supports,
    Eq. exp; sigmoid for bounded supports, Eq. sigmoid; identity otherwise) and
    the log-Jacobian correction of Eq. reparam-post;
  * the objective of Eq. obj-fun, f(z) = -(log L(g(z)) + log p(g(z)) + log|J|);
  * Adam (Kingma & Ba 2014) with the linear learning-rate schedule of Table 1.
The likelihood and its gradient come from the FP64 model oracle.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import stats

from . import oracle as _model

# (kind, parameters) per parameter, Table 2 order; the prior of Eq. sim-dist.
#   normal(mu, sd) | lognormal(median, sd of log) | truncnormal(mu, sd, lo, hi) | uniform(lo, hi)
PRIOR = [
    ("lognormal", 1.25, 0.4),                   # theta_E
    ("truncnormal", 2.0, 0.5, 1.0, 3.0),        # gamma_epl
    ("normal", 0.0, 0.2), ("normal", 0.0, 0.2),  # e_epl
    ("normal", 0.0, 0.06), ("normal", 0.0, 0.06),  # x_epl, y_epl
    ("normal", 0.0, 0.1), ("normal", 0.0, 0.1),  # gamma_ext
    ("lognormal", 1.6, 0.25),                   # R_l
    ("uniform", 0.5, 8.0),                      # n_l
    ("truncnormal", 0.0, 0.1, -0.15, 0.15), ("truncnormal", 0.0, 0.1, -0.15, 0.15),  # e_l
    ("normal", 0.0, 0.02), ("normal", 0.0, 0.02),  # x_l, y_l
    ("lognormal", 300.0, 0.5),                  # I_l
    ("lognormal", 0.25, 0.25),                  # R_s
    ("uniform", 0.5, 8.0),                      # n_s
    ("truncnormal", 0.0, 0.3, -0.5, 0.5), ("truncnormal", 0.0, 0.3, -0.5, 0.5),  # e_s
    ("normal", 0.0, 0.5), ("normal", 0.0, 0.5),  # x_s, y_s
    ("lognormal", 150.0, 0.9),                  # I_s
]

# Table 1, MAP row
K_MAP = 300
N_MAP = 300
LR_START, LR_END = 1e-2, 1e-3
ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def bijector_kind(entry):
    """Support of the prior decides the bijector: (0, inf) -> exp, (a, b) -> sigmoid, R -> identity."""
    kind = entry[0]
    if kind == "lognormal":
        return ("exp",)
    if kind == "truncnormal":
        return ("sigmoid", entry[3], entry[4])
    if kind == "uniform":
        return ("sigmoid", entry[1], entry[2])
    return ("identity",)


def _dist(entry):
    kind = entry[0]
    if kind == "normal":
        return stats.norm(entry[1], entry[2])
    if kind == "lognormal":
        return stats.lognorm(s=entry[2], scale=entry[1])
    if kind == "truncnormal":
        mu, sd, lo, hi = entry[1:]
        return stats.truncnorm((lo - mu) / sd, (hi - mu) / sd, loc=mu, scale=sd)
    if kind == "uniform":
        return stats.uniform(entry[1], entry[2] - entry[1])
    raise ValueError(kind)


def log_prior_marginal(j: int, x):
    """log density of the j-th prior marginal at x (scipy.stats)."""
    return _dist(PRIOR[j]).logpdf(np.asarray(x, np.float64))


def log_prior(theta):
    """(log p(theta) [B], d log p / d theta [B, 22]) for physical parameters:
    the sum of the independent marginals."""
    theta = np.atleast_2d(np.asarray(theta, np.float64))
    lp = np.zeros(theta.shape[0])
    g = np.zeros_like(theta)
    for j, e in enumerate(PRIOR):
        x = theta[:, j]
        lp += log_prior_marginal(j, x)
        kind = e[0]
        if kind in ("normal", "truncnormal"):
            g[:, j] = -(x - e[1]) / e[2] ** 2
        elif kind == "lognormal":
            g[:, j] = -(np.log(x) - math.log(e[1])) / (e[2] ** 2 * x) - 1.0 / x
    return lp, g


def bijector(z):
    """theta = g(z), d theta / dz, log|J| and d log|J| / dz, component-wise (Sec. 2.2)."""
    z = np.atleast_2d(np.asarray(z, np.float64))
    th, d, lj, dlj = (np.empty_like(z) for _ in range(4))
    for j, e in enumerate(PRIOR):
        b = bijector_kind(e)
        x = z[:, j]
        if b[0] == "exp":
            th[:, j] = np.exp(x)
            d[:, j] = th[:, j]
            lj[:, j] = x
            dlj[:, j] = 1.0
        elif b[0] == "sigmoid":
            a, c = b[1], b[2]
            s = 1.0 / (1.0 + np.exp(-x))
            th[:, j] = a + (c - a) * s
            d[:, j] = (c - a) * s * (1.0 - s)
            lj[:, j] = math.log(c - a) - np.logaddexp(0.0, -x) - np.logaddexp(0.0, x)   # log s + log(1 - s)
            dlj[:, j] = 1.0 - 2.0 * s
        else:
            th[:, j] = x
            d[:, j] = 1.0
            lj[:, j] = 0.0
            dlj[:, j] = 0.0
    return th, d, lj.sum(axis=1), dlj


def inverse_bijector(theta):
    theta = np.atleast_2d(np.asarray(theta, np.float64))
    z = np.empty_like(theta)
    for j, e in enumerate(PRIOR):
        b = bijector_kind(e)
        x = theta[:, j]
        if b[0] == "exp":
            z[:, j] = np.log(x)
        elif b[0] == "sigmoid":
            s = (x - b[1]) / (b[2] - b[1])
            z[:, j] = np.log(s) - np.log1p(-s)
        else:
            z[:, j] = x
    return z


def objective_grad(z, loglik_theta, grad_theta):
    """f(z) = -(log L + log p + log|J|) and df/dz, given log L and its
    gradient at theta = g(z) (Eq. obj-fun, Eq. reparam-post)."""
    th, d, lj, dlj = bijector(z)
    lp, glp = log_prior(th)
    f = -(np.asarray(loglik_theta) + lp + lj)
    g = -((np.asarray(grad_theta) + glp) * d + dlj)
    return f, g


def learning_rate(t: int) -> float:
    """Linear schedule of Table 1: 1e-2 -> 1e-3 over K_MAP iterations (t from 0)."""
    frac = min(t, K_MAP) / K_MAP
    return LR_START + (LR_END - LR_START) * frac


def adam_step(z, m, v, t: int, g, lr: float):
    """One Adam update (t counts from 1): returns (z, m, v)."""
    m = ADAM_B1 * m + (1.0 - ADAM_B1) * g
    v = ADAM_B2 * v + (1.0 - ADAM_B2) * g * g
    mhat = m / (1.0 - ADAM_B1 ** t)
    vhat = v / (1.0 - ADAM_B2 ** t)
    return z - lr * mhat / (np.sqrt(vhat) + ADAM_EPS), m, v


def run_map(z0, image, sigma, psf, pixel_scale, k, gain_exposure, n_steps: int = K_MAP, nthreads: int = 0):
    """Multi-start MAP from z0 [n, 22]; returns (z, f) after n_steps and the
    objective history [n_steps, n] (f at the point each step starts from)."""
    z = np.array(z0, np.float64)
    m = np.zeros_like(z)
    v = np.zeros_like(z)
    hist = []
    for t in range(n_steps):
        th, _, _, _ = bijector(z)
        ll, _, gl = _model.loglik(th.astype(np.float32).astype(np.float64), image, sigma, psf, pixel_scale, k,
                                  gain_exposure, grad=True, nthreads=nthreads)
        f, g = objective_grad(z, ll, gl)
        hist.append(f)
        z, m, v = adam_step(z, m, v, t + 1, g, learning_rate(t))
    th, _, _, _ = bijector(z)
    ll, _, gl = _model.loglik(th.astype(np.float32).astype(np.float64), image, sigma, psf, pixel_scale, k,
                              gain_exposure, grad=True, nthreads=nthreads)
    f, _ = objective_grad(z, ll, gl)
    return z, f, np.array(hist)
