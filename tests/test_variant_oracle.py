"""Pins of the variant-likelihood oracle (Sec. 2.1.2, the observed-image
variance) to facts outside it:

- the variance map: sigma_bkg^2 + I_obs / (G t), negative pixels clipped to 0;
- the model is linear in (I_l, I_s): the basis images recombine to the
  model oracle's image at any amplitudes;
- the solved amplitudes are a stationary point of log L: the model
  oracle's forward-mode gradient in I_l and I_s vanishes there, and
  any other amplitudes give a lower log L;
- noiseless data: the solve returns the true amplitudes;
- the profiled gradient equals central differences of the profiled log L
  (amplitudes re-solved at every point);
- degenerate cases: a source whose image misses the detector gets I_s = 0.
"""
import numpy as np
import pytest

import oracle
from oracle import variant_oracle as vo
from paper_2202_07663_gb300 import inputs


@pytest.fixture(scope="module", autouse=True)
def _build():
    oracle.build()


def _system(seed=0, H=24, W=22, k=2, K=5):
    spec = inputs.SystemSpec(H, W, k, K, "gaussian", inputs.PIXEL_SCALE, 0.2, 100.0)
    rng = np.random.default_rng(seed)
    truth = inputs.draw_table(rng, inputs.PAPER_SIM, 1)[0]
    truth[0] = 0.6   # Einstein radius inside the small cut-out
    psf = inputs.make_psf(spec)
    model = oracle.simulate(truth, H, W, psf, spec.pixel_scale, k)[0]
    image = inputs.add_noise(rng, model, spec.sigma_bkg, spec.gain_exposure)
    return spec, truth, psf, model, image


def test_observed_variance_clips_negative_pixels():
    img = np.array([[-1.0, 0.0], [2.0, 10.0]])
    v = vo.observed_variance(img, 0.2, 100.0)
    np.testing.assert_allclose(v, 0.04 + np.array([[0.0, 0.0], [0.02, 0.1]]), rtol=1e-15)
    np.testing.assert_allclose(vo.observed_variance(img, 0.2, 0.0), np.full((2, 2), 0.04), rtol=1e-15)


def test_model_is_linear_in_the_amplitudes():
    spec, truth, psf, model, _ = _system(1)
    A = vo.basis_images(truth, spec.H, spec.W, psf, spec.pixel_scale, spec.k)[0]
    np.testing.assert_allclose(truth[vo.I_L] * A[0] + truth[vo.I_S] * A[1], model, rtol=1e-12,
                               atol=1e-14 * np.abs(model).max())


def test_solved_amplitudes_are_stationary_and_maximal():
    spec, truth, psf, _, image = _system(2)
    rng = np.random.default_rng(3)
    p = inputs.draw_perturbed(rng, truth, 4, frac=0.01)
    ll, _, _, amps = vo.profiled_loglik(p, image, spec.sigma_bkg, psf, spec.pixel_scale, spec.k, spec.gain_exposure)
    var = vo.observed_variance(image, spec.sigma_bkg, spec.gain_exposure)
    q = p.copy()
    q[:, vo.I_L], q[:, vo.I_S] = amps[:, 0], amps[:, 1]
    l2, _, g = oracle.loglik(q, image, np.sqrt(var), psf, spec.pixel_scale, spec.k, 0.0, grad=True)
    np.testing.assert_allclose(l2, ll, rtol=1e-14)
    scale = np.abs(g).max(axis=1)
    assert np.all(np.abs(g[:, vo.I_L]) < 1e-9 * scale) and np.all(np.abs(g[:, vo.I_S]) < 1e-9 * scale)
    for da in ((0.01, 0.0), (0.0, -0.01), (0.003, 0.003)):
        r = q.copy()
        r[:, vo.I_L] *= 1 + da[0]
        r[:, vo.I_S] *= 1 + da[1]
        assert np.all(oracle.loglik(r, image, np.sqrt(var), psf, spec.pixel_scale, spec.k, 0.0)[0] < ll)


def test_noiseless_data_gives_the_true_amplitudes():
    spec, truth, psf, model, _ = _system(4)
    A = vo.basis_images(truth, spec.H, spec.W, psf, spec.pixel_scale, spec.k)
    var = vo.observed_variance(model, spec.sigma_bkg, spec.gain_exposure)
    amps = vo.solve_amplitudes(A, model, var)[0]
    np.testing.assert_allclose(amps, [truth[vo.I_L], truth[vo.I_S]], rtol=1e-9)


def test_profiled_gradient_matches_differences():
    spec, truth, psf, _, image = _system(5)
    p = inputs.draw_perturbed(np.random.default_rng(6), truth, 1, frac=0.01)[0]
    args = (image, spec.sigma_bkg, psf, spec.pixel_scale, spec.k, spec.gain_exposure)
    _, _, g, _ = vo.profiled_loglik(p, *args)
    assert g[0, vo.I_L] == 0.0 and g[0, vo.I_S] == 0.0
    for i in (0, 1, 4, 8, 9, 15, 16, 19):
        h = 1e-5 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (vo.profiled_loglik(pp, *args, grad=False)[0][0] - vo.profiled_loglik(pm, *args, grad=False)[0][0]) / (2 * h)
        assert g[0, i] == pytest.approx(fd, rel=2e-4, abs=1e-4 * np.abs(g).max())


def test_source_off_the_detector_gets_zero_amplitude():
    spec, truth, psf, _, image = _system(7)
    p = truth.copy()
    p[0] = 1e-3          # almost no lensing
    p[19], p[20] = 50.0, 50.0   # source far outside the field
    p[15] = 0.05
    ll, _, _, amps = vo.profiled_loglik(p[None], image, spec.sigma_bkg, psf, spec.pixel_scale, spec.k,
                                        spec.gain_exposure)
    assert amps[0, 1] == 0.0 and amps[0, 0] != 0.0 and np.isfinite(ll[0])
