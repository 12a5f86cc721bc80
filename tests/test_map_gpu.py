"""Multi-start MAP on the GPU against the MAP oracle (Sec. 2.2-2.3, Table 1):
the fused step kernel and the bijector kernels on identical FP64 inputs, a
short multi-start run against the oracle's run, and the paper's statement
that a few percent of prior-drawn starts reach the global mode."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import map_oracle as mo  # noqa: E402
from paper_2202_07663_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_07663_gb300 import build
    build.build()
    oracle.build()
    from paper_2202_07663_gb300 import abi, map as gmap
    return abi, gmap


def _paper_system(H, seed, K=11):
    spec = inputs.SystemSpec(H, H, 2, K, "gaussian", inputs.PIXEL_SCALE, 0.2, 100.0)
    rng = np.random.default_rng(seed)
    truth = inputs.draw_table(rng, inputs.PAPER_SIM, 1)[0]
    psf = inputs.make_psf(spec).astype(np.float32)
    model = oracle.simulate(truth, spec.H, spec.W, psf, spec.pixel_scale, spec.k)[0]
    image = inputs.add_noise(rng, model, spec.sigma_bkg, spec.gain_exposure).astype(np.float32)
    return spec, truth, psf, image


def test_step_and_bijector_kernels_match_oracle(mods):
    abi, gmap = mods
    lib = abi.lib_handle()
    rng = np.random.default_rng(9)
    n = 257
    theta = inputs.draw_table(rng, inputs.PAPER_PRIOR_DRAW, n).astype(np.float32)
    st = torch.cuda.current_stream().cuda_stream
    pt = gmap.prior_table()
    th_d = torch.from_numpy(theta).cuda()
    z = torch.empty(n, 22, dtype=torch.float64, device="cuda")
    abi._check(lib.gl_map_inverse(n, th_d.data_ptr(), gmap.ctypes.addressof(pt), z.data_ptr(), st), "inverse")
    zo = mo.inverse_bijector(theta.astype(np.float64))
    np.testing.assert_allclose(z.cpu().numpy(), zo, rtol=1e-12, atol=1e-12)
    # one Adam step at t = 3 from nonzero moments
    m = rng.normal(size=(n, 22)) * 10
    v = rng.uniform(1, 100, (n, 22))
    ll = rng.normal(size=n) * 1e3
    gl = rng.normal(size=(n, 22)) * 1e2
    zd, md, vd = (torch.from_numpy(a).cuda().contiguous() for a in (zo, m, v))
    lld, gld = torch.from_numpy(ll).cuda(), torch.from_numpy(gl).cuda().contiguous()
    f = torch.empty(n, dtype=torch.float64, device="cuda")
    th_out = torch.empty(n, 22, dtype=torch.float32, device="cuda")
    lr = 3e-3
    abi._check(lib.gl_map_adam_step(n, zd.data_ptr(), md.data_ptr(), vd.data_ptr(), 3, lr, *gmap.ADAM,
                                    lld.data_ptr(), gld.data_ptr(), gmap.ctypes.addressof(pt), f.data_ptr(),
                                    th_out.data_ptr(), st), "step")
    fo, go = mo.objective_grad(zo, ll, gl)
    zn, mn, vn = mo.adam_step(zo, m, v, 3, go, lr)
    torch.cuda.synchronize()
    np.testing.assert_allclose(f.cpu().numpy(), fo, rtol=1e-12)
    np.testing.assert_allclose(md.cpu().numpy(), mn, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(vd.cpu().numpy(), vn, rtol=1e-12)
    np.testing.assert_allclose(zd.cpu().numpy(), zn, rtol=1e-12, atol=1e-14)
    ref_th = mo.bijector(zn)[0].astype(np.float32)
    np.testing.assert_allclose(th_out.cpu().numpy(), ref_th, rtol=2e-7, atol=1e-30)


def test_multistart_run_in_lockstep_with_oracle(mods):
    """Thirty MAP iterations on the GPU; at every step the oracle applies its
    own prior, bijector, objective and Adam update to the GPU's log-likelihood
    and gradient, and the two states must agree to FP64 rounding. (Whole
    trajectories are not compared: Adam moves a coordinate whose gradient is
    near zero by about +-lr whatever its size, so FP32 noise in such a
    component changes the path.)"""
    abi, gmap = mods
    lib = abi.lib_handle()
    spec, truth, psf, image = _paper_system(20, 101, K=5)
    rng = np.random.default_rng(12)
    n = 16
    theta0 = inputs.draw_table(rng, inputs.PAPER_PRIOR_DRAW, n).astype(np.float32)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    pt = gmap.prior_table()
    st = torch.cuda.current_stream().cuda_stream
    th = torch.from_numpy(theta0).cuda()
    z = torch.empty(n, 22, dtype=torch.float64, device="cuda")
    m = torch.zeros_like(z)
    v = torch.zeros_like(z)
    f = torch.empty(n, dtype=torch.float64, device="cuda")
    abi._check(lib.gl_map_inverse(n, th.data_ptr(), gmap.ctypes.addressof(pt), z.data_ptr(), st), "inverse")
    abi._check(lib.gl_map_transform(n, z.data_ptr(), gmap.ctypes.addressof(pt), th.data_ptr(), st), "transform")
    zo = z.cpu().numpy().copy()
    mo_, vo = np.zeros_like(zo), np.zeros_like(zo)
    for t in range(30):
        ll, g = s.loglik_grad(th)
        lln, gn = ll.cpu().numpy(), g.cpu().numpy()
        lr = gmap.linear_lr(t)
        abi._check(lib.gl_map_adam_step(n, z.data_ptr(), m.data_ptr(), v.data_ptr(), t + 1, lr, *gmap.ADAM,
                                        ll.data_ptr(), g.data_ptr(), gmap.ctypes.addressof(pt), f.data_ptr(),
                                        th.data_ptr(), st), "step")
        fo, go = mo.objective_grad(zo, lln, gn)
        zo, mo_, vo = mo.adam_step(zo, mo_, vo, t + 1, go, lr)
        torch.cuda.synchronize()
        np.testing.assert_allclose(f.cpu().numpy(), fo, rtol=1e-12)
        np.testing.assert_allclose(z.cpu().numpy(), zo, rtol=1e-11, atol=1e-12)
        np.testing.assert_allclose(th.cpu().numpy(), mo.bijector(zo)[0].astype(np.float32), rtol=2.5e-7)
    s.close()


def test_map_from_the_truth_reaches_the_mode(mods):
    """Started at the truth, 300 iterations of the Table 1 schedule end at a
    point at least as probable as the truth (the mode is not the truth: the
    noise moves it) whose reduced chi^2 is within noise of the truth's, and
    at most 1.01 + that noise (Sec. 2.3 marks runs that end at chi2_nu <= 1.01
    as converged to the global mode)."""
    abi, gmap = mods
    spec, truth, psf, image = _paper_system(80, 202)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    tt = torch.from_numpy(truth.astype(np.float32)[None]).cuda()
    res = gmap.MultiStartMAP(s, steps=300).run(tt.repeat(4, 1))
    ll_t, c2_t = (x.cpu().numpy() for x in s.loglik(tt, chi2=True))
    _, c2 = s.loglik(res.theta, chi2=True)
    s.close()
    dof = spec.H * spec.W - 22
    zt = mo.inverse_bijector(truth[None].astype(np.float32).astype(np.float64))
    f_truth = mo.objective_grad(zt, ll_t, np.zeros((1, 22)))[0][0]
    f = res.objective.cpu().numpy()
    assert np.all(f <= f_truth + 1e-3)
    chi2nu, chi2nu_t = c2.cpu().numpy() / dof, c2_t[0] / dof
    noise = np.sqrt(2.0 / dof)
    assert np.all(chi2nu <= chi2nu_t + noise)
    assert np.all(chi2nu <= 1.01 + 2 * noise)


def test_multistart_from_the_prior_descends(mods, golden_constants):
    """n_MAP = 300 prior draws, K_MAP = 300 iterations (Table 1): the starts
    descend (the best by more than two orders of magnitude); the fraction
    reaching the mode depends on the data and is reported by the benchmark,
    not asserted here."""
    abi, gmap = mods
    spec, truth, psf, image = _paper_system(80, 202)
    n = int(golden_constants["map_starts"])
    steps = int(golden_constants["map_iterations"])
    rng = np.random.default_rng(13)
    theta0 = torch.from_numpy(inputs.draw_table(rng, inputs.PAPER_PRIOR_DRAW, n).astype(np.float32)).cuda()
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    res = gmap.MultiStartMAP(s, steps=steps).run(theta0, record=True)
    s.close()
    h = res.history.cpu().numpy()
    f = res.objective.cpu().numpy()
    live = np.isfinite(f)
    assert live.mean() > 0.95
    assert np.mean(f[live] < h[0][live]) > 0.95            # nearly every start descends
    assert np.median(f[live]) < np.median(h[0][live]) / 3.0
    assert np.min(f[live]) < 0.01 * np.median(h[0][live])
    assert res.grad_evals == n * (steps + 1)
