"""The MAP -> VI -> HMC pipeline (Sec. 2.6) end to end on a small system,
with shortened stages: every stage runs, the mode is at least as probable as
the truth when the starts are near it, the VI and Laplace preconditioners
both give finite samples near the truth, and the stage timings add up."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2202_07663_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("pre", ["vi", "laplace"])
def test_pipeline_runs_end_to_end(pre):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_07663_gb300 import abi, build, pipeline
    build.build()
    oracle.build()
    spec = inputs.SystemSpec(40, 40, 2, 7, "gaussian", inputs.PIXEL_SCALE, 0.2, 100.0)
    rng = np.random.default_rng(17)
    truth = inputs.draw_table(rng, inputs.PAPER_SIM, 1)[0]
    truth[0] = 0.8
    psf = inputs.make_psf(spec).astype(np.float32)
    model = oracle.simulate(truth, spec.H, spec.W, psf, spec.pixel_scale, spec.k)[0]
    image = inputs.add_noise(rng, model, spec.sigma_bkg, spec.gain_exposure).astype(np.float32)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    starts = torch.from_numpy(inputs.draw_perturbed(np.random.default_rng(3), truth, 8, frac=0.005)
                              .astype(np.float32)).cuda()
    r = pipeline.model_system(s, starts, map_steps=150, vi_steps=200, vi_draws=128, chains=16, n_burn=60,
                              n_samples=60, preconditioner=pre, seed=2)
    ll_t = s.loglik(torch.from_numpy(truth.astype(np.float32)[None]).cuda()).item()
    ll_m = s.loglik(torch.from_numpy(r.theta_map.astype(np.float32)[None]).cuda()).item()
    s.close()
    assert ll_m >= ll_t - 5.0
    th = r.samples.theta.reshape(-1, 22).cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(th))
    z = np.abs(th.mean(0) - truth) / th.std(0)
    assert np.median(z) < 3.0
    assert set(r.seconds) == {"map", "vi", "preconditioner", "hmc", "total"}
    parts = r.seconds["map"] + r.seconds["vi"] + r.seconds["preconditioner"] + r.seconds["hmc"]
    assert abs(parts - r.seconds["total"]) < 1e-3 * max(1.0, r.seconds["total"])
    assert r.grad_evals["map"] == 8 * 151 and r.grad_evals["vi"] == 128 * 200
