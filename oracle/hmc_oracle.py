"""FP64 oracle of the trajectory-length adaptation in HMC (arXiv:2202.07663, Sec. 2.5).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). The paper tunes the
step size and the trajectory length during the first 80% of burn-in with the
methods of Hoffman & Gelman (2014) and Hoffman, Radul & Sountsov (2021). The
second maximises the ChEES criterion (change in the estimator of the
expected square) over the trajectory length T:

  ChEES(T) = 1/4 E[(|q' - E q'|^2 - |q - E q|^2)^2],

q the state a transition starts from and q' its proposal after a trajectory
of length t = u T, u a jitter in (0, 1). Its gradient in log T, per chain,
holding the ensemble means fixed, is

  t (|q' - m'|^2 - |q - m|^2) (q' - m') . v',

v' the velocity M^-1 p' at the end of the trajectory (d q'/dt), m and m' the
chain means of q and q'. Chains are averaged with their acceptance
probabilities as weights; a chain whose proposal is not finite carries no
weight. The jitter u is the base-2 van der Corput (Halton) sequence.
"""
from __future__ import annotations

import numpy as np


def van_der_corput(m: int, base: int = 2) -> float:
    """Radical inverse of m >= 1 in the given base: 1/2, 1/4, 3/4, 1/8, ..."""
    out, f = 0.0, 1.0 / base
    while m > 0:
        m, r = divmod(m, base)
        out += r * f
        f /= base
    return out


def chees_grad_log_t(q_prev, q_prop, v_prop, accept_prob, t: float):
    """Acceptance-weighted mean over chains of t a_c c_c, and of a_c^2 / 4
    (the criterion), with a_c = |q'_c - m'|^2 - |q_c - m|^2 and
    c_c = (q'_c - m') . v'_c; m' averages the finite proposals only.
    Returns (gradient in log T, criterion)."""
    q_prev, q_prop, v_prop = (np.asarray(a, np.float64) for a in (q_prev, q_prop, v_prop))
    w = np.asarray(accept_prob, np.float64).copy()
    ok = np.all(np.isfinite(q_prop), axis=1) & np.all(np.isfinite(v_prop), axis=1) & np.isfinite(w)
    if not ok.any():
        return 0.0, 0.0
    m = q_prev.mean(axis=0)
    mp = q_prop[ok].mean(axis=0)
    grad = crit = sw = 0.0
    for cidx in np.flatnonzero(ok):
        a = np.sum((q_prop[cidx] - mp) ** 2) - np.sum((q_prev[cidx] - m) ** 2)
        c = np.sum((q_prop[cidx] - mp) * v_prop[cidx])
        grad += w[cidx] * t * a * c
        crit += w[cidx] * 0.25 * a * a
        sw += w[cidx]
    if sw <= 0.0:
        return 0.0, 0.0
    return grad / sw, crit / sw
