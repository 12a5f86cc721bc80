"""FP64 oracle of full-rank variational inference (arXiv:2202.07663, Sec. 2.4, Table 1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). Plain numpy statement of:
  * the surrogate posterior q = N(mu, Sigma) over the unconstrained parameters,
    Sigma = L L^T, with the Cholesky bijector of Sec. 2.4: an unconstrained
    vector of d(d+1)/2 reals laid into the lower triangle of L, the diagonal
    exponentiated;
  * the ELBO loss of Eq. elbo, E_q[log q - log p~], estimated on n samples;
  * its gradient by the estimator of Eq. elbo-grad (the score-function form,
    E_q[(log q - log p~) grad log q] with the samples held fixed), and by the
    reparameterised (pathwise) form z = mu + L eps, both unbiased for the same
    gradient;
  * the learning-rate schedule of Table 1 (0 -> 1e-3, quadratic over 500
    iterations, read as a degree-2 polynomial schedule that starts at 0) and
    Adam (shared with the MAP oracle);
  * the initialisation of Table 1: mu = the MAP point, Sigma = 1e-6 I.
The variational parameter vector is phi = [mu (d), u (d(d+1)/2)], u packed
row by row: u[i(i+1)/2 + j] = L[i, j] for j < i, log L[i, i] for j = i.
The caller supplies the standard-normal draws eps [n, d] and log p~ (and its
gradient in z, for the pathwise form) at z = mu + L eps.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import solve_triangular

from .map_oracle import adam_step

# Table 1, VI row
K_VI = 1000
N_VI = 500
LR_PEAK = 1e-3
LR_WARMUP = 500
SIGMA_INIT = 1e-6


def n_params(d: int) -> int:
    return d + d * (d + 1) // 2


def unpack(phi, d: int):
    """phi -> (mu [d], L [d, d]) through the Cholesky bijector."""
    phi = np.asarray(phi, np.float64)
    mu = phi[:d].copy()
    L = np.zeros((d, d))
    k = d
    for i in range(d):
        for j in range(i + 1):
            L[i, j] = math.exp(phi[k]) if i == j else phi[k]
            k += 1
    return mu, L


def pack(mu, L):
    """(mu, L) -> phi (inverse of the bijector; L lower triangular, positive diagonal)."""
    d = len(mu)
    out = [float(x) for x in mu]
    for i in range(d):
        for j in range(i + 1):
            out.append(math.log(L[i, i]) if i == j else float(L[i, j]))
    return np.array(out)


def initial_phi(z_map):
    """mu = MAP point, Sigma = SIGMA_INIT * I (Table 1)."""
    d = len(z_map)
    return pack(np.asarray(z_map, np.float64), math.sqrt(SIGMA_INIT) * np.eye(d))


def learning_rate(t: int) -> float:
    """Table 1: 0 -> 1e-3 over 500 iterations, quadratic (t from 0):
    lr = peak - peak (1 - t/500)^2, then constant."""
    frac = min(t, LR_WARMUP) / LR_WARMUP
    return LR_PEAK - LR_PEAK * (1.0 - frac) ** 2


def log_q(z, mu, L):
    """log N(z; mu, L L^T) for z [n, d]: the textbook density written with the
    Cholesky factor, -|L^-1 (z - mu)|^2 / 2 - log det L - d/2 log 2 pi
    (triangular solves; forming Sigma = L L^T would square L's condition number)."""
    z = np.atleast_2d(np.asarray(z, np.float64))
    d = len(mu)
    w = solve_triangular(L, (z - mu).T, lower=True)
    logdet_L = np.sum(np.log(np.diag(L)))
    return -0.5 * np.sum(w * w, axis=0) - logdet_L - 0.5 * d * math.log(2.0 * math.pi)


def _to_u(gmu, gL, L):
    """Gradient in (mu, L) -> gradient in phi (diagonal through exp)."""
    d = len(gmu)
    out = list(gmu)
    for i in range(d):
        for j in range(i + 1):
            out.append(gL[i, j] * L[i, i] if i == j else gL[i, j])
    return np.array(out)


def grad_log_q(z, mu, L):
    """d log q(z; phi) / d phi with z held fixed, per sample: [n, P].
    With w = L^-1 r and a = L^-T w = Sigma^-1 r (r = z - mu):
    d/dmu = a; d/dL = lower part of a w^T (= Sigma^-1 r r^T L^-T) - diag(1/L_ii)."""
    z = np.atleast_2d(np.asarray(z, np.float64))
    out = []
    for zs in z:
        r = zs - mu
        w = solve_triangular(L, r, lower=True)
        a = solve_triangular(L.T, w, lower=False)
        gL = np.tril(np.outer(a, w)) - np.diag(1.0 / np.diag(L))
        out.append(_to_u(a, gL, L))
    return np.array(out)


def elbo_grad_score(phi, eps, logp):
    """Eq. elbo-grad on the samples z_s = mu + L eps_s: the mean over s of
    (log q(z_s) - log p~(z_s)) d log q(z_s)/d phi. Returns (loss, grad [P])."""
    eps = np.atleast_2d(np.asarray(eps, np.float64))
    d = eps.shape[1]
    mu, L = unpack(phi, d)
    z = mu + eps @ L.T
    f = log_q(z, mu, L) - np.asarray(logp, np.float64)
    return f.mean(), (f[:, None] * grad_log_q(z, mu, L)).mean(axis=0)


def elbo_grad_pathwise(phi, eps, logp, grad_z):
    """Reparameterised gradient of the ELBO loss at fixed eps: with
    z = mu + L eps, log q(z) = -|eps|^2/2 - sum log L_ii - d/2 log 2 pi, so
    d loss/d mu = -mean grad_z, d loss/d L_ij = -mean grad_z_i eps_j - delta_ij/L_ii.
    Returns (loss, grad [P])."""
    eps = np.atleast_2d(np.asarray(eps, np.float64))
    d = eps.shape[1]
    mu, L = unpack(phi, d)
    z = mu + eps @ L.T
    gz = np.atleast_2d(np.asarray(grad_z, np.float64))
    f = log_q(z, mu, L) - np.asarray(logp, np.float64)
    gmu = -gz.mean(axis=0)
    gL = np.tril(-(gz.T @ eps) / eps.shape[0]) - np.diag(1.0 / np.diag(L))
    return f.mean(), _to_u(gmu, gL, L)


def samples(phi, eps):
    """z_s = mu + L eps_s."""
    eps = np.atleast_2d(np.asarray(eps, np.float64))
    mu, L = unpack(phi, eps.shape[1])
    return mu + eps @ L.T


def vi_step(phi, m, v, t: int, eps, logp, grad_z=None, estimator: str = "score", lr: float | None = None):
    """One VI iteration (t counts from 1): estimator on the given draws, then
    Adam at the Table 1 rate for iteration t-1. Returns (phi, m, v, loss, grad)."""
    if estimator == "score":
        loss, g = elbo_grad_score(phi, eps, logp)
    else:
        loss, g = elbo_grad_pathwise(phi, eps, logp, grad_z)
    phi, m, v = adam_step(phi, m, v, t, g, learning_rate(t - 1) if lr is None else lr)
    return phi, m, v, loss, g
