"""Full-rank VI on the GPU against the VI oracle (Sec. 2.4, Table 1):

- gl_vi_sample (z = mu + L eps, theta = g(z)) on identical draws;
- gl_vi_step, both estimators, on identical draws, log densities and
  gradients, for ragged and multi-chunk draw counts: loss, gradient and the
  Adam update to FP64 rounding;
- VI through the GPU path on a 22-dimensional Gaussian target: recovers its
  mean and covariance;
- ten iterations on a lens posterior in lockstep with the oracle (Table 1
  initialisation and schedule): at each step the oracle applies its own
  estimator and Adam update to the GPU's log densities, and the two
  variational states must agree to FP64 rounding. (The oracle rebuilds
  z - mu from z, so an L far from diagonal, which a much larger step would
  make, costs it digits that the GPU, working with the draws, keeps.)
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import map_oracle as mo  # noqa: E402
from oracle import vi_oracle as vo  # noqa: E402
from paper_2202_07663_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_07663_gb300 import build
    build.build()
    oracle.build()
    from paper_2202_07663_gb300 import abi, hmc, map as gmap, vi
    return abi, hmc, gmap, vi


def _rand_phi(rng, d, mu=None, scale=0.3, diag=0.3):
    mu = rng.normal(size=d) if mu is None else mu
    L = np.tril(rng.normal(size=(d, d)) * scale, -1)
    np.fill_diagonal(L, np.exp(rng.normal(size=d) * diag))
    return vo.pack(mu, L)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_sample_kernel_matches_oracle(mods):
    abi, _, gmap, _ = mods
    lib = abi.lib_handle()
    st = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(40)
    # d = 22 with the paper's prior: draws near a prior sample, theta through the bijectors
    z0 = mo.inverse_bijector(inputs.draw_table(rng, inputs.PAPER_PRIOR_DRAW, 1))[0]
    phi = vo.pack(z0, np.tril(rng.normal(size=(22, 22)) * 0.01, -1) + np.diag(np.full(22, 0.02)))
    for n in (1, 77, 1000):
        eps = rng.normal(size=(n, 22))
        z = torch.empty(n, 22, dtype=torch.float64, device="cuda")
        th = torch.empty(n, 22, dtype=torch.float32, device="cuda")
        pt = gmap.prior_table()
        ed, pd = _cuda(eps), _cuda(phi)   # keep the inputs alive until the kernel has run
        abi._check(lib.gl_vi_sample(n, 22, ed.data_ptr(), pd.data_ptr(), gmap.ctypes.addressof(pt), z.data_ptr(),
                                    th.data_ptr(), st), "sample")
        torch.cuda.synchronize()
        zo = vo.samples(phi, eps)
        np.testing.assert_allclose(z.cpu().numpy(), zo, rtol=1e-13, atol=1e-13)
        np.testing.assert_allclose(th.cpu().numpy(), mo.bijector(zo)[0].astype(np.float32), rtol=2e-7, atol=1e-30)
    # generic d without a prior: theta = (float) z
    d, n = 7, 33
    phi = _rand_phi(rng, d)
    eps = rng.normal(size=(n, d))
    z = torch.empty(n, d, dtype=torch.float64, device="cuda")
    th = torch.empty(n, d, dtype=torch.float32, device="cuda")
    ed, pd = _cuda(eps), _cuda(phi)
    abi._check(lib.gl_vi_sample(n, d, ed.data_ptr(), pd.data_ptr(), None, z.data_ptr(), th.data_ptr(), st), "sample")
    torch.cuda.synchronize()
    np.testing.assert_allclose(z.cpu().numpy(), vo.samples(phi, eps), rtol=1e-13, atol=1e-13)
    np.testing.assert_array_equal(th.cpu().numpy(), z.cpu().numpy().astype(np.float32))


@pytest.mark.parametrize("estimator", ["score", "pathwise"])
@pytest.mark.parametrize("d,n", [(22, 500), (22, 77), (7, 1), (7, 6000), (32, 65)])
def test_step_kernel_matches_oracle(mods, estimator, d, n):
    abi, _, _, vi = mods
    lib = abi.lib_handle()
    st = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(41 + d + n)
    phi = _rand_phi(rng, d)
    eps = rng.normal(size=(n, d))
    logp = -1e3 + rng.normal(size=n) * 30
    gz = rng.normal(size=(n, d)) * 50
    P = vo.n_params(d)
    m = rng.normal(size=P) * 0.1
    v = rng.uniform(0.5, 2.0, P)
    t, lr = 3, 7e-4
    phid, md, vd = _cuda(phi), _cuda(m), _cuda(v)
    g = torch.empty(P, dtype=torch.float64, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(lib.gl_vi_workspace_bytes(n, d), dtype=torch.uint8, device="cuda")
    est = vi.SCORE if estimator == "score" else vi.PATHWISE
    ed, lpd, gzd = _cuda(eps), _cuda(logp), _cuda(gz)
    gz_ptr = gzd.data_ptr() if estimator == "pathwise" else None
    abi._check(lib.gl_vi_step(n, d, ed.data_ptr(), lpd.data_ptr(), gz_ptr, est, phid.data_ptr(), md.data_ptr(),
                              vd.data_ptr(), t, lr, *vi.ADAM, g.data_ptr(), loss.data_ptr(), ws.data_ptr(), st), "step")
    torch.cuda.synchronize()
    pn, mn, vn, lo, go = vo.vi_step(phi, m, v, t, eps, logp, gz, estimator=estimator, lr=lr)
    gg = g.cpu().numpy()
    np.testing.assert_allclose(gg, go, rtol=1e-9, atol=1e-9 * np.max(np.abs(go)))
    assert loss.item() == pytest.approx(lo, rel=1e-12)
    np.testing.assert_allclose(md.cpu().numpy(), mn, rtol=1e-9, atol=1e-9 * np.max(np.abs(mn)))
    np.testing.assert_allclose(phid.cpu().numpy(), pn, rtol=1e-12, atol=1e-12)
    # gradient only (no Adam): phi untouched, same gradient
    phid2 = _cuda(phi)
    g2 = torch.empty_like(g)
    abi._check(lib.gl_vi_step(n, d, ed.data_ptr(), lpd.data_ptr(), gz_ptr, est, phid2.data_ptr(), None, None, 0, 0.0,
                              *vi.ADAM, g2.data_ptr(), loss.data_ptr(), ws.data_ptr(), st), "step")
    torch.cuda.synchronize()
    np.testing.assert_array_equal(phid2.cpu().numpy(), phi)
    np.testing.assert_array_equal(g2.cpu().numpy(), gg)


def test_vi_recovers_a_gaussian_target(mods):
    abi, hmc, _, vi = mods
    d = 22
    g = torch.Generator(device="cuda").manual_seed(42)
    A = torch.randn(d, d, dtype=torch.float64, device="cuda", generator=g)
    cov = (A @ A.T / d + 0.2 * torch.eye(d, dtype=torch.float64, device="cuda")) * 1e-4
    mu = torch.randn(d, dtype=torch.float64, device="cuda", generator=g)
    prec = torch.linalg.inv(cov)

    class Gauss:
        needs_q32 = False

        def __call__(self, z, z32, lp, gz):
            r = z - mu
            lp.copy_(-0.5 * (r * (r @ prec)).sum(1))
            if gz is not None:
                gz.copy_(-(r @ prec))

    def lr(t):
        return vi.quadratic_warmup(t, 1e-2, 200) if t < 1200 else (1e-3 if t < 1700 else 1e-4)

    res = vi.FullRankVI(Gauss(), d=d, n=500, steps=2000, estimator="pathwise", seed=1, lr_fn=lr).run(mu + 0.003)
    sd = torch.sqrt(torch.diag(cov))
    assert ((res.mu - mu).abs() / sd).max().item() < 0.1
    C = res.cov
    assert ((torch.diag(C) / torch.diag(cov)) - 1).abs().max().item() < 0.1
    corr = C / torch.sqrt(torch.diag(C)[:, None] * torch.diag(C)[None, :])
    corr0 = cov / (sd[:, None] * sd[None, :])
    assert (corr - corr0).abs().max().item() < 0.05
    assert torch.isfinite(res.loss).all()
    assert res.loss[-100:].mean().item() < res.loss[:10].mean().item()


def _paper_system(H, seed, K=11):
    spec = inputs.SystemSpec(H, H, 2, K, "gaussian", inputs.PIXEL_SCALE, 0.2, 100.0)
    rng = np.random.default_rng(seed)
    truth = inputs.draw_table(rng, inputs.PAPER_SIM, 1)[0]
    psf = inputs.make_psf(spec).astype(np.float32)
    model = oracle.simulate(truth, spec.H, spec.W, psf, spec.pixel_scale, spec.k)[0]
    image = inputs.add_noise(rng, model, spec.sigma_bkg, spec.gain_exposure).astype(np.float32)
    return spec, truth, psf, image


@pytest.mark.parametrize("estimator", ["pathwise", "score"])
def test_vi_lockstep_with_oracle_on_a_lens_posterior(mods, estimator):
    abi, hmc, gmap, vi = mods
    lib = abi.lib_handle()
    st = torch.cuda.current_stream().cuda_stream
    spec, truth, psf, image = _paper_system(30, 103, K=5)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    post = hmc.PosteriorTarget(s)
    d, n = 22, 96
    phi = vo.initial_phi(mo.inverse_bijector(truth)[0])
    P = vo.n_params(d)
    m, v = np.zeros(P), np.zeros(P)
    phid, md, vd = _cuda(phi), torch.zeros(P, dtype=torch.float64, device="cuda"), \
        torch.zeros(P, dtype=torch.float64, device="cuda")
    g = torch.empty(P, dtype=torch.float64, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    ws = torch.empty(lib.gl_vi_workspace_bytes(n, d), dtype=torch.uint8, device="cuda")
    z = torch.empty(n, d, dtype=torch.float64, device="cuda")
    lp = torch.empty(n, dtype=torch.float64, device="cuda")
    gz = torch.empty(n, d, dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(7)
    est = vi.SCORE if estimator == "score" else vi.PATHWISE
    for t in range(1, 11):
        eps = rng.normal(size=(n, d))
        ed = _cuda(eps)
        abi._check(lib.gl_vi_sample(n, d, ed.data_ptr(), phid.data_ptr(), None, z.data_ptr(), None, st), "sample")
        post(z, None, lp, gz if estimator == "pathwise" else None)
        lr = vo.learning_rate(t - 1)   # Table 1 schedule: L stays well conditioned
        abi._check(lib.gl_vi_step(n, d, ed.data_ptr(), lp.data_ptr(), gz.data_ptr() if est == vi.PATHWISE else None,
                                  est, phid.data_ptr(), md.data_ptr(), vd.data_ptr(), t, lr, *vi.ADAM, g.data_ptr(),
                                  loss.data_ptr(), ws.data_ptr(), st), "step")
        torch.cuda.synchronize()
        np.testing.assert_allclose(z.cpu().numpy(), vo.samples(phi, eps), rtol=1e-12, atol=1e-13)
        phi, m, v, lo, go = vo.vi_step(phi, m, v, t, eps, lp.cpu().numpy(), gz.cpu().numpy(), estimator=estimator,
                                       lr=lr)
        assert loss.item() == pytest.approx(lo, rel=1e-11)
        np.testing.assert_allclose(phid.cpu().numpy(), phi, rtol=1e-10, atol=1e-12)
    s.close()


@pytest.mark.parametrize("estimator", ["score", "pathwise"])
def test_moments_then_apply(mods, estimator):
    """The step split in two: one part gives gl_vi_step's bits; draws spread
    over uneven parts (as over processes) give the oracle's step on all draws."""
    abi, _, _, vi = mods
    lib = abi.lib_handle()
    st = torch.cuda.current_stream().cuda_stream
    d, n = 22, 500
    rng = np.random.default_rng(97)
    phi = _rand_phi(rng, d)
    eps = rng.normal(size=(n, d))
    logp = -1e3 + rng.normal(size=n) * 30
    gz = rng.normal(size=(n, d)) * 50
    P = vo.n_params(d)
    Q = 1 + P
    m = rng.normal(size=P) * 0.1
    v = rng.uniform(0.5, 2.0, P)
    t, lr = 5, 4e-4
    est = vi.SCORE if estimator == "score" else vi.PATHWISE
    ed, lpd, gzd = _cuda(eps), _cuda(logp), _cuda(gz)
    ws = torch.empty(lib.gl_vi_workspace_bytes(n, d), dtype=torch.uint8, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")

    def gz_ptr(lo):
        return gzd[lo:].data_ptr() if estimator == "pathwise" else None

    def apply(nparts, sums):
        phid, md, vd = _cuda(phi), _cuda(m), _cuda(v)
        g = torch.empty(P, dtype=torch.float64, device="cuda")
        abi._check(lib.gl_vi_apply(n, d, nparts, sums.data_ptr(), est, phid.data_ptr(), md.data_ptr(), vd.data_ptr(),
                                   t, lr, *vi.ADAM, g.data_ptr(), loss.data_ptr(), st), "apply")
        torch.cuda.synchronize()
        return phid.cpu().numpy(), md.cpu().numpy(), g.cpu().numpy(), loss.item()

    # one part: bitwise gl_vi_step
    phid, md, vd = _cuda(phi), _cuda(m), _cuda(v)
    g = torch.empty(P, dtype=torch.float64, device="cuda")
    abi._check(lib.gl_vi_step(n, d, ed.data_ptr(), lpd.data_ptr(), gz_ptr(0), est, phid.data_ptr(), md.data_ptr(),
                              vd.data_ptr(), t, lr, *vi.ADAM, g.data_ptr(), loss.data_ptr(), ws.data_ptr(), st), "step")
    torch.cuda.synchronize()
    ref = (phid.cpu().numpy(), md.cpu().numpy(), g.cpu().numpy(), loss.item())
    sums = torch.empty(1, Q, dtype=torch.float64, device="cuda")
    abi._check(lib.gl_vi_moments(n, d, ed.data_ptr(), lpd.data_ptr(), gz_ptr(0), est, _cuda(phi).data_ptr(),
                                 ws.data_ptr(), sums.data_ptr(), st), "moments")
    one = apply(1, sums)
    for a, b in zip(one[:3], ref[:3]):
        np.testing.assert_array_equal(a, b)
    assert one[3] == ref[3]
    # three uneven parts against the oracle on all draws
    cuts = [0, 1, 320, n]
    sums = torch.empty(3, Q, dtype=torch.float64, device="cuda")
    pd = _cuda(phi)
    for k in range(3):
        lo, hi = cuts[k], cuts[k + 1]
        abi._check(lib.gl_vi_moments(hi - lo, d, ed[lo:].data_ptr(), lpd[lo:].data_ptr(), gz_ptr(lo), est,
                                     pd.data_ptr(), ws.data_ptr(), sums[k].data_ptr(), st), "moments")
    pn, mn, gn, ln = apply(3, sums)
    po, mo_, vo_, lo_, go = vo.vi_step(phi, m, v, t, eps, logp, gz, estimator=estimator, lr=lr)
    np.testing.assert_allclose(gn, go, rtol=1e-9, atol=1e-9 * np.max(np.abs(go)))
    assert ln == pytest.approx(lo_, rel=1e-12)
    np.testing.assert_allclose(mn, mo_, rtol=1e-9, atol=1e-9 * np.max(np.abs(mo_)))
    np.testing.assert_allclose(pn, po, rtol=1e-12, atol=1e-12)
    # invalid arguments are refused before any launch
    assert lib.gl_vi_apply(n, d, 0, sums.data_ptr(), est, pd.data_ptr(), None, None, 0, 0.0, *vi.ADAM,
                           g.data_ptr(), loss.data_ptr(), st) != 0
    assert lib.gl_vi_moments(0, d, ed.data_ptr(), lpd.data_ptr(), gz_ptr(0), est, pd.data_ptr(), ws.data_ptr(),
                             sums.data_ptr(), st) != 0
