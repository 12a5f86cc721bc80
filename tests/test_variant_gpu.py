"""The observed-image-variance likelihood on the GPU against its oracle
(Sec. 2.1.2):

- a system built with the observed variance: log L and gradient against the
  model oracle with that variance map and no Poisson term;
- log L profiled over (I_l, I_s): amplitudes, log L and the 20-parameter
  gradient against the variant oracle (FP32 basis images: the amplitudes to
  1e-4 relative, log L and gradient with the FP32 model-error bounds);
- noiseless data gives the true amplitudes; a source off the detector gets
  I_s = 0; a system with the model-dependent variance refuses the call.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import variant_oracle as vo  # noqa: E402
from paper_2202_07663_gb300 import inputs  # noqa: E402
from gpu_common import assert_plain_parity  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def abi():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_07663_gb300 import build, abi as _abi
    build.build()
    oracle.build()
    return _abi


def _system(seed, H=48, W=44, k=2, K=9):
    spec = inputs.SystemSpec(H, W, k, K, "gaussian", inputs.PIXEL_SCALE, 0.2, 100.0)
    rng = np.random.default_rng(seed)
    truth = inputs.draw_table(rng, inputs.PAPER_SIM, 1)[0]
    truth[0] = 0.9
    psf = inputs.make_psf(spec).astype(np.float32)
    model = oracle.simulate(truth, H, W, psf, spec.pixel_scale, k)[0]
    image = inputs.add_noise(rng, model, spec.sigma_bkg, spec.gain_exposure).astype(np.float32)
    return spec, truth, psf, model, image


def test_observed_variance_system_matches_oracle(abi):
    spec, truth, psf, _, image = _system(1)
    params = inputs.draw_perturbed(np.random.default_rng(2), truth, 9, frac=0.02).astype(np.float32)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg,
                     observed_variance=True)
    ll, g = (t.cpu().numpy() for t in s.loglik_grad(torch.from_numpy(params).cuda()))
    s.close()
    sig = np.sqrt(vo.observed_variance(image, np.float32(spec.sigma_bkg), spec.gain_exposure))
    rl, _, rg = oracle.loglik(params.astype(np.float64), image, sig, psf, spec.pixel_scale, spec.k, 0.0, grad=True)
    assert_plain_parity(ll, g, rl, rg, "observed variance")


# K = 9: the 2-D stencil; K = 11 (a Gaussian, rank 1): the separable form,
# in cluster bands below half as many vectors as SMs and whole-image above.
# Named exceptions, measured: vector 78 of the 200-vector draw has a
# source-plane ray 0.28 mas from the source centre (n_s = 2.56), the
# closest of the draw (median 4.5 mas): x_epl 3.35 and x_s 2.47 x the plain
# tolerance, the same with the 2-D stencil (K = 9: 3.37, 2.48).
PROFILED_EXCEPTIONS = {(200, 11): {"x_epl": 4.0, "x_s": 3.0}}


@pytest.mark.parametrize("B,K,H,W", [(1, 9, 48, 44), (13, 9, 48, 44), (64, 9, 48, 44), (5, 11, 48, 44),
                                     (200, 11, 48, 44), (80, 11, 200, 190)])
def test_profiled_loglik_matches_oracle(abi, B, K, H, W):
    """The last case is too large for the whole-image separable buffers: its
    correlation-only pass runs in cluster row bands (4 of 50 rows)."""
    spec, truth, psf, _, image = _system(3, H=H, W=W, K=K)
    params = inputs.draw_perturbed(np.random.default_rng(B), truth, B, frac=0.02).astype(np.float32)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg,
                     observed_variance=True)
    ll, g, amps, c2 = (t.cpu().numpy() for t in s.loglik_grad_profiled(torch.from_numpy(params).cuda(), chi2=True))
    ll_only, g_none, amps2 = s.loglik_grad_profiled(torch.from_numpy(params).cuda(), grad=False)
    s.close()
    assert g_none is None
    np.testing.assert_array_equal(ll_only.cpu().numpy(), ll)
    np.testing.assert_array_equal(amps2.cpu().numpy(), amps)
    rl, rc2, rg, ramps = vo.profiled_loglik(params.astype(np.float64), image, np.float32(spec.sigma_bkg), psf,
                                            spec.pixel_scale, spec.k, spec.gain_exposure)
    np.testing.assert_allclose(amps, ramps, rtol=1e-4)
    assert np.all(g[:, vo.I_L] == 0.0) and np.all(g[:, vo.I_S] == 0.0)
    sig = np.sqrt(vo.observed_variance(image, np.float32(spec.sigma_bkg), spec.gain_exposure))
    at = params.copy()
    at[:, vo.I_L], at[:, vo.I_S] = ramps[:, 0], ramps[:, 1]
    assert_plain_parity(ll, g, rl, rg, "profiled", grad_exceptions=PROFILED_EXCEPTIONS.get((B, K)))
    np.testing.assert_allclose(c2, rc2, rtol=1e-3)


def test_noiseless_data_returns_true_amplitudes_and_degenerate_source(abi):
    spec, truth, psf, model, _ = _system(4)
    s = abi.GLSystem(model.astype(np.float32), psf, spec.pixel_scale, spec.k, spec.gain_exposure,
                     sigma_bkg=spec.sigma_bkg, observed_variance=True)
    p = truth.astype(np.float32)[None].repeat(2, 0)
    p[1, 0] = 1e-3
    p[1, 19], p[1, 20] = 50.0, 50.0
    p[1, 15] = 0.05
    _, _, amps = s.loglik_grad_profiled(torch.from_numpy(p).cuda())
    s.close()
    a = amps.cpu().numpy()
    np.testing.assert_allclose(a[0], [truth[vo.I_L], truth[vo.I_S]], rtol=1e-4)
    assert a[1, 1] == 0.0 and a[1, 0] > 0


def test_model_dependent_variance_refuses_profiling(abi):
    spec, truth, psf, _, image = _system(5)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    with pytest.raises(abi.GLError):
        s.loglik_grad_profiled(torch.from_numpy(truth.astype(np.float32)[None]).cuda())
    s.close()
