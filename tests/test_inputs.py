"""The seeded synthetic inputs follow their stated recipes (CPU):

- PSFs: unit sum, the symmetries of a circular profile, and the width read
  back from neighbouring samples (Gaussian FWHM 0.1", Moffat beta 3 with
  FWHM 0.12", at 0.065" pixels);
- draws: truth vectors inside their ranges, multi-start vectors uniform over
  the box with log-uniform amplitudes, perturbed vectors clipped, the
  simulation table's normal, log-normal, uniform and truncated-normal
  marginals;
- noise: Poisson counts at G t_exp plus Gaussian background, so the
  residual variance is M / (G t_exp) + sigma_bkg^2;
- serving stream: Poisson arrivals at the stated rate, shapes and batch
  sizes from the stated sets; seeds are base + system index.
"""
import math

import numpy as np
import pytest

from paper_2202_07663_gb300 import inputs


def _symmetric(a):
    return (np.allclose(a, a.T, rtol=0, atol=1e-15) and np.allclose(a, a[::-1, :], rtol=0, atol=1e-15)
            and np.allclose(a, a[:, ::-1], rtol=0, atol=1e-15))


@pytest.mark.parametrize("K", [5, 11, 21])
def test_gaussian_psf_width(K):
    p = inputs.gaussian_psf(K)
    c = (K - 1) // 2
    assert p.shape == (K, K) and abs(p.sum() - 1.0) < 1e-14 and _symmetric(p)
    assert np.unravel_index(np.argmax(p), p.shape) == (c, c)
    # exp(-1 / (2 s^2)) between the centre and its neighbour gives s in pixels
    s = math.sqrt(-0.5 / math.log(p[c, c + 1] / p[c, c]))
    assert s * inputs.PIXEL_SCALE * 2.0 * math.sqrt(2.0 * math.log(2.0)) == pytest.approx(0.1, rel=1e-12)
    assert s == pytest.approx(0.6533, abs=1e-4)   # 0.04247" at 0.065" pixels
    # separable: every row is a scaled copy of the centre row
    np.testing.assert_allclose(p / p[c][None, :], (p[:, c] / p[c, c])[:, None] * np.ones((1, K)), rtol=1e-12)


@pytest.mark.parametrize("K", [11, 21])
def test_moffat_psf_width(K):
    p = inputs.moffat_psf(K)
    c = (K - 1) // 2
    assert abs(p.sum() - 1.0) < 1e-14 and _symmetric(p)
    beta = 3.0
    # (1 + r^2 / a^2)^-beta between the centre and its neighbours at r = 1 and r = 2
    a1 = 1.0 / math.sqrt((p[c, c + 1] / p[c, c]) ** (-1.0 / beta) - 1.0)
    a2 = 2.0 / math.sqrt((p[c, c + 2] / p[c, c]) ** (-1.0 / beta) - 1.0)
    assert a1 == pytest.approx(a2, rel=1e-12)
    alpha_arcsec = a1 * inputs.PIXEL_SCALE
    assert alpha_arcsec == pytest.approx(0.06 / math.sqrt(2.0 ** (1.0 / 3.0) - 1.0), rel=1e-12)
    assert alpha_arcsec == pytest.approx(0.1177, abs=1e-4)
    # half maximum at half the FWHM
    assert (1.0 + (0.06 / alpha_arcsec) ** 2) ** (-beta) == pytest.approx(0.5, rel=1e-12)


def test_make_psf_kinds():
    assert np.array_equal(inputs.make_psf(inputs.SystemSpec(8, 8, 1, 11, "gaussian")), inputs.gaussian_psf(11))
    assert np.array_equal(inputs.make_psf(inputs.SystemSpec(8, 8, 1, 21, "moffat")), inputs.moffat_psf(21))
    with pytest.raises(ValueError):
        inputs.make_psf(inputs.SystemSpec(8, 8, 1, 5, "airy"))


def test_truth_draws_in_their_ranges():
    rng = np.random.default_rng(0)
    T = np.stack([inputs.draw_truth(rng) for _ in range(4000)])
    for j, (lo, hi) in {0: (1.0, 2.0), 1: (1.8, 2.2), 8: (0.5, 1.5), 9: (2.0, 5.0), 14: (100.0, 1000.0),
                        15: (0.05, 0.3), 16: (0.5, 4.0), 21: (50.0, 500.0)}.items():
        assert T[:, j].min() >= lo and T[:, j].max() <= hi, j
    for j, sd in {2: 0.1, 4: 0.05, 6: 0.05, 10: 0.1, 12: 0.05, 17: 0.15}.items():
        assert T[:, j].std() == pytest.approx(sd, rel=0.06), j
        assert abs(T[:, j].mean()) < 4 * sd / math.sqrt(len(T)), j
    # source offset from the lens centre: N(0, 0.3)
    assert (T[:, 19] - T[:, 4]).std() == pytest.approx(0.3, rel=0.06)
    # log-uniform amplitudes: log I uniform over [log lo, log hi]
    for j, (lo, hi) in {14: (100.0, 1000.0), 21: (50.0, 500.0)}.items():
        u = (np.log(T[:, j]) - math.log(lo)) / (math.log(hi) - math.log(lo))
        assert abs(u.mean() - 0.5) < 0.02 and abs(u.var() - 1.0 / 12.0) < 0.01


def test_box_draws():
    B = 20000
    P = inputs.draw_box(np.random.default_rng(1), B)
    box = inputs.PRIOR_BOX
    assert P.shape == (B, inputs.NPARAM)
    assert np.all(P >= box[:, 0]) and np.all(P <= box[:, 1])
    for j in range(inputs.NPARAM):
        lo, hi = box[j]
        if j in (14, 21):
            u = (np.log(P[:, j]) - math.log(lo)) / (math.log(hi) - math.log(lo))
        else:
            u = (P[:, j] - lo) / (hi - lo)
        assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1.0 / 12.0) < 0.004, j


def test_perturbed_draws():
    rng = np.random.default_rng(2)
    truth = inputs.draw_truth(rng)
    P = inputs.draw_perturbed(rng, truth, 5000, frac=0.01)
    box = inputs.PRIOR_BOX
    lo, hi = np.minimum(box[:, 0], truth), np.maximum(box[:, 1], truth)
    assert np.all(P >= lo) and np.all(P <= hi)
    width = box[:, 1] - box[:, 0]
    inner = (truth - lo > 4 * 0.01 * width) & (hi - truth > 4 * 0.01 * width)   # clipping negligible
    np.testing.assert_allclose(P[:, inner].std(0), 0.01 * width[inner], rtol=0.06)
    assert np.all(np.abs(P[:, inner].mean(0) - truth[inner]) < 5 * 0.01 * width[inner] / math.sqrt(len(P)))
    # a truth outside the box is kept as a bound, not moved inside
    t2 = truth.copy()
    t2[0] = 2.5
    P2 = inputs.draw_perturbed(rng, t2, 1000, frac=0.02)
    assert P2[:, 0].max() <= 2.5 and P2[:, 0].min() >= 1.0


def test_simulation_table_marginals():
    n = 20000
    D = inputs.draw_table(np.random.default_rng(3), inputs.PAPER_SIM, n)
    assert D.shape == (n, len(inputs.PAPER_SIM)) == (n, inputs.NPARAM)
    for j, d in enumerate(inputs.PAPER_SIM):
        x = D[:, j]
        if d[0] == "n":
            assert x.mean() == pytest.approx(d[1], abs=5 * d[2] / math.sqrt(n)) and x.std() == pytest.approx(d[2], rel=0.03)
        elif d[0] == "ln":   # the printed value is the median
            assert np.median(x) == pytest.approx(d[1], rel=0.03) and np.log(x).std() == pytest.approx(d[2], rel=0.03)
        elif d[0] == "u":
            assert x.min() >= d[1] and x.max() <= d[2] and x.mean() == pytest.approx(0.5 * (d[1] + d[2]), rel=0.02)
        else:                # truncated normal: inside the bounds, and the rejection keeps the shape
            assert d[0] == "tn" and x.min() >= d[3] and x.max() <= d[4]
            a, b = (d[3] - d[1]) / d[2], (d[4] - d[1]) / d[2]
            phi = lambda t: math.exp(-0.5 * t * t) / math.sqrt(2 * math.pi)   # noqa: E731
            Phi = lambda t: 0.5 * (1 + math.erf(t / math.sqrt(2)))            # noqa: E731
            Z = Phi(b) - Phi(a)
            mean = d[1] + d[2] * (phi(a) - phi(b)) / Z
            var = d[2] ** 2 * (1 + (a * phi(a) - b * phi(b)) / Z - ((phi(a) - phi(b)) / Z) ** 2)
            assert x.mean() == pytest.approx(mean, abs=5 * math.sqrt(var / n))
            assert x.var() == pytest.approx(var, rel=0.05)
    with pytest.raises(ValueError):
        inputs.draw_table(np.random.default_rng(0), [("gamma", 1.0, 1.0)], 3)


def test_noise_model():
    rng = np.random.default_rng(4)
    M = np.full((200, 200), 3.0)
    M[:100] = 0.5
    for G, sb in ((100.0, 0.2), (1000.0, 0.01)):
        obs = inputs.add_noise(rng, M, sb, G)
        r = obs - M
        for rows, m in ((slice(0, 100), 0.5), (slice(100, 200), 3.0)):
            v = m / G + sb * sb
            assert r[rows].mean() == pytest.approx(0.0, abs=5 * math.sqrt(v / r[rows].size))
            assert r[rows].var() == pytest.approx(v, rel=0.04)
    # no Poisson term without an exposure: background only
    r = inputs.add_noise(rng, M, 0.1, 0.0) - M
    assert r.var() == pytest.approx(0.01, rel=0.03)


def test_serving_stream():
    reqs = inputs.serving_stream(n=4000, rate_hz=20.0, seed=4000)
    t = np.array([r.arrival_s for r in reqs])
    assert np.all(np.diff(t) > 0) and [r.index for r in reqs] == list(range(4000))
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert gaps.mean() == pytest.approx(1 / 20.0, rel=0.05) and gaps.std() == pytest.approx(1 / 20.0, rel=0.06)
    assert {r.spec.H for r in reqs} == {40, 60, 80, 120} and all(r.spec.H == r.spec.W for r in reqs)
    assert {r.spec.k for r in reqs} == {2, 4} and {r.spec.K for r in reqs} == {11, 21}
    assert min(r.B for r in reqs) >= 256 and max(r.B for r in reqs) <= 2048
    assert len({r.seed for r in reqs}) == 4000
    again = inputs.serving_stream(n=4000, rate_hz=20.0, seed=4000)
    assert [(r.arrival_s, r.spec, r.B, r.seed) for r in again] == [(r.arrival_s, r.spec, r.B, r.seed) for r in reqs]


def test_workload_seeds():
    for name, w in inputs.WORKLOADS.items():
        a = inputs.rng_for(name, 3).uniform(size=4)
        b = np.random.default_rng(w["seed"] + 3).uniform(size=4)
        assert np.array_equal(a, b), name
        assert w["spec"].K % 2 == 1 and w["B"] > 0
