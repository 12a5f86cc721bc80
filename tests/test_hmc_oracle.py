"""Pins of the trajectory-length oracle (Sec. 2.5; Hoffman, Radul & Sountsov
2021) to facts outside it:

- the base-2 van der Corput sequence's first terms;
- for a standard normal target under exact Hamiltonian flow (q' = q cos t +
  p sin t, v' = -q sin t + p cos t) the criterion is d sin^2(T) and its
  T-derivative d sin(2T) (chain means -> 0): the oracle's estimates over many
  chains match both, and the gradient changes sign at T = pi/2;
- at fixed draws, the per-chain gradient equals central differences of the
  criterion in log T with the chain means held fixed;
- acceptance weights and non-finite proposals.
"""
import math

import numpy as np
import pytest

from oracle import hmc_oracle as ho


def test_van_der_corput():
    assert [ho.van_der_corput(m) for m in range(1, 8)] == [0.5, 0.25, 0.75, 0.125, 0.625, 0.375, 0.875]
    assert ho.van_der_corput(1, 3) == pytest.approx(1 / 3)


def _flow(q, p, t):
    return q * math.cos(t) + p * math.sin(t), -q * math.sin(t) + p * math.cos(t)


@pytest.mark.parametrize("T", [0.4, 0.9, 1.3, 2.0, 2.6])
def test_gaussian_exact_flow_closed_form(T):
    rng = np.random.default_rng(1)
    d, C = 4, 200000
    q = rng.normal(size=(C, d))
    p = rng.normal(size=(C, d))
    qp, vp = _flow(q, p, T)
    g, crit = ho.chees_grad_log_t(q, qp, vp, np.ones(C), T)
    assert crit == pytest.approx(d * math.sin(T) ** 2, rel=0.03, abs=0.02)
    # gradient in log T = T * dChEES/dT = T d sin(2T)
    assert g / T == pytest.approx(d * math.sin(2 * T), rel=0.05, abs=0.05)


def test_gradient_sign_brackets_quarter_period():
    rng = np.random.default_rng(2)
    d, C = 3, 50000
    q, p = rng.normal(size=(C, d)), rng.normal(size=(C, d))
    assert ho.chees_grad_log_t(q, *_flow(q, p, math.pi / 4), np.ones(C), math.pi / 4)[0] > 0
    assert ho.chees_grad_log_t(q, *_flow(q, p, 3 * math.pi / 4), np.ones(C), 3 * math.pi / 4)[0] < 0


def test_gradient_is_derivative_of_criterion_with_means_fixed():
    rng = np.random.default_rng(3)
    d, C = 3, 7
    q, p = rng.normal(size=(C, d)) + 0.3, rng.normal(size=(C, d))
    w = rng.uniform(0.2, 1.0, C)
    T = 1.1
    qp, vp = _flow(q, p, T)
    m, mp = q.mean(0), qp.mean(0)

    def crit(logT):
        x, _ = _flow(q, p, math.exp(logT))
        a = np.sum((x - mp) ** 2, 1) - np.sum((q - m) ** 2, 1)
        return np.sum(w * 0.25 * a * a) / w.sum()

    g, c = ho.chees_grad_log_t(q, qp, vp, w, T)
    assert c == pytest.approx(crit(math.log(T)), rel=1e-12)
    h = 1e-6
    assert g == pytest.approx((crit(math.log(T) + h) - crit(math.log(T) - h)) / (2 * h), rel=1e-6)


def test_weights_and_non_finite_proposals():
    rng = np.random.default_rng(4)
    q, qp, vp = (rng.normal(size=(6, 2)) for _ in range(3))
    w = np.array([1.0, 0.0, 0.5, 1.0, 0.25, 1.0])
    g, c = ho.chees_grad_log_t(q, qp, vp, w, 0.7)
    keep = w > 0
    # zero-weight chains still set the means, but add nothing
    m, mp = q.mean(0), qp.mean(0)
    a = np.sum((qp - mp) ** 2, 1) - np.sum((q - m) ** 2, 1)
    cc = np.sum((qp - mp) * vp, 1)
    assert g == pytest.approx(np.sum((w * 0.7 * a * cc)[keep]) / w.sum(), rel=1e-12)
    # a non-finite proposal leaves the others' means and carries no weight
    qp2 = qp.copy()
    qp2[1, 0] = np.inf
    g2, _ = ho.chees_grad_log_t(q, qp2, vp, w, 0.7)
    mp2 = qp[[0, 2, 3, 4, 5]].mean(0)
    a2 = np.sum((qp - mp2) ** 2, 1) - np.sum((q - m) ** 2, 1)
    c2 = np.sum((qp - mp2) * vp, 1)
    sel = [0, 2, 3, 4, 5]
    assert g2 == pytest.approx(np.sum((w * 0.7 * a2 * c2)[sel]) / w[sel].sum(), rel=1e-12)
    assert ho.chees_grad_log_t(q, qp, vp, np.zeros(6), 0.7) == (0.0, 0.0)
