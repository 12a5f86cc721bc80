"""The HMC path (100x100, k=4, 21x21 Moffat PSF): the adjoint behind torch.autograd.Function, and HMC kernels.

- autograd gradient of LogLik vs the FP64 oracle and vs central finite
  differences (h = 1e-4) of the oracle's log L, on the 100x100, k=4, 21x21
  Moffat system;
- FP64 Hamiltonian/accept kernel vs a numpy statement of the same rule;
- leapfrog kernels: exact time reversibility and correct moments on a
  Gaussian target whose gradient is computed by torch in FP64;
- a short lens HMC run: chains move, acceptance is sane, log L finite.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_2202_07663_gb300 import inputs  # noqa: E402
from gpu_common import assert_plain_parity, make_system, oracle_eval  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_07663_gb300 import build
    build.build()
    oracle.build()
    from paper_2202_07663_gb300 import abi, hmc
    return abi, hmc


def test_autograd_gradient_vs_oracle_and_central_differences(mods):
    abi, hmc = mods
    spec = inputs.WORKLOADS[inputs.HMC]["spec"]
    truth, image, psf = make_system(spec, 3000)
    params = inputs.draw_perturbed(np.random.default_rng(31), truth, 3).astype(np.float32)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    p = torch.from_numpy(params).double().cuda().requires_grad_(True)
    ll = hmc.loglik(p, s)
    (g,) = torch.autograd.grad(ll.sum(), p)
    ll_nograd = hmc.loglik(p.detach(), s)
    s.close()
    ll, g = ll.detach().cpu().numpy(), g.cpu().numpy()
    np.testing.assert_array_equal(ll, ll_nograd.cpu().numpy())
    rl, _, rg = oracle_eval(spec, image, psf, params)
    assert_plain_parity(ll, g, rl, rg, "autograd vs oracle")
    # central differences of the FP64 oracle, h = 1e-4 (relative for |p| > 1)
    fd = np.empty_like(rg)
    base = params.astype(np.float64)
    for i in range(22):
        h = 1e-4 * np.maximum(1.0, np.abs(base[:, i]))
        pp, pm = base.copy(), base.copy()
        pp[:, i] += h
        pm[:, i] -= h
        lp = oracle.loglik(pp, image, np.float32(spec.sigma_bkg), psf, spec.pixel_scale, spec.k, spec.gain_exposure)[0]
        lm = oracle.loglik(pm, image, np.float32(spec.sigma_bkg), psf, spec.pixel_scale, spec.k, spec.gain_exposure)[0]
        fd[:, i] = (lp - lm) / (2 * h)
    # FD truncation error is O(h^2); same tolerance rule as the oracle comparison
    assert_plain_parity(ll, g, rl, fd, "autograd vs central differences")


def _numpy_finish(p0, logp0, p, grad_new, logp_new, q_new, inv_mass, log_u, eps, q, logp, grad):
    p = p + 0.5 * eps * grad_new
    h0 = -logp0 + 0.5 * np.sum(p0 * p0 * inv_mass, axis=1)
    h1 = -logp_new + 0.5 * np.sum(p * p * inv_mass, axis=1)
    fin = np.isfinite(h0) & np.isfinite(h1)
    acc = fin & (log_u < h0 - h1)
    aprob = np.where(fin, np.minimum(1.0, np.exp(np.where(fin, h0 - h1, 0.0))), 0.0)
    q = np.where(acc[:, None], q_new, q)
    grad = np.where(acc[:, None], grad_new, grad)
    logp = np.where(acc, logp_new, logp)
    return p, q, logp, grad, acc.astype(np.int32), aprob


def test_finish_kernel_matches_numpy(mods):
    abi, _ = mods
    rng = np.random.default_rng(5)
    B, d = 300, 22
    arrs = {k: rng.normal(size=(B, d)) for k in ("p0", "p", "grad_new", "q_new", "q", "grad")}
    inv_mass = rng.uniform(0.5, 2.0, d)
    logp0 = rng.normal(size=B) * 3
    logp_new = logp0 + rng.normal(size=B) * 2
    logp_new[:5] = np.nan
    log_u = np.log(rng.uniform(size=B))
    logp = logp0.copy()
    eps = 0.17
    ref = _numpy_finish(arrs["p0"], logp0, arrs["p"], arrs["grad_new"], logp_new, arrs["q_new"], inv_mass, log_u,
                        eps, arrs["q"], logp, arrs["grad"])
    t = {k: torch.from_numpy(v).cuda().contiguous() for k, v in arrs.items()}
    tl0, tln, tim, tlu, tlp = (torch.from_numpy(x).cuda().contiguous() for x in (logp0, logp_new, inv_mass, log_u,
                                                                                   logp))
    acc = torch.empty(B, dtype=torch.int32, device="cuda")
    aprob = torch.empty(B, dtype=torch.float64, device="cuda")
    abi.gl_hmc_finish(B, d, t["p0"].data_ptr(), tl0.data_ptr(), t["p"].data_ptr(), t["grad_new"].data_ptr(),
                      tln.data_ptr(), t["q_new"].data_ptr(), tim.data_ptr(), tlu.data_ptr(), eps, t["q"].data_ptr(),
                      tlp.data_ptr(), t["grad"].data_ptr(), acc.data_ptr(), torch.cuda.current_stream().cuda_stream,
                      accept_prob=aprob.data_ptr())
    torch.cuda.synchronize()
    np.testing.assert_allclose(t["p"].cpu().numpy(), ref[0], rtol=1e-15, atol=1e-15)
    np.testing.assert_array_equal(acc.cpu().numpy(), ref[4])
    np.testing.assert_array_equal(t["q"].cpu().numpy(), ref[1])
    np.testing.assert_array_equal(tlp.cpu().numpy(), ref[2])
    np.testing.assert_array_equal(t["grad"].cpu().numpy(), ref[3])
    np.testing.assert_allclose(aprob.cpu().numpy(), ref[5], rtol=1e-14, atol=0)
    assert 0 < ref[4].sum() < B and ref[4][:5].sum() == 0


def _gauss(mu, prec):
    def lg(q32):
        q = q32.double()
        r = q - mu
        return -0.5 * (r * (r @ prec)).sum(1), -(r @ prec)
    return lg


def test_leapfrog_is_reversible_and_hmc_samples_a_gaussian(mods):
    abi, hmc = mods
    d, B = 22, 2048
    g = torch.Generator(device="cuda").manual_seed(3)
    mu = torch.randn(d, dtype=torch.float64, device="cuda", generator=g)
    sd = torch.exp(torch.randn(d, dtype=torch.float64, device="cuda", generator=g) * 0.5)
    prec = torch.diag(1.0 / sd ** 2)
    lg = _gauss(mu, prec)
    # reversibility: L steps forward, flip momentum, L steps back (FP64 state; the
    # likelihood sees FP32 positions, so compare with FP32-level tolerance)
    q0 = (mu + sd * torch.randn(B, d, dtype=torch.float64, device="cuda", generator=g)).contiguous()
    p = torch.randn(B, d, dtype=torch.float64, device="cuda", generator=g).contiguous()
    inv_mass = (sd ** 2).contiguous()
    q = q0.clone()
    q32 = torch.empty(B, d, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    _, gr = lg(q.float())
    gr = gr.contiguous()
    eps, L = 0.3, 6
    for sign in (1.0, -1.0):
        if sign < 0:
            p.neg_()
        for l in range(L):
            abi.gl_hmc_leapfrog(B, d, q.data_ptr(), p.data_ptr(), gr.data_ptr(), inv_mass.data_ptr(), eps,
                                0.5 if l == 0 else 1.0, q32.data_ptr(), st)
            _, gr = lg(q32)
            gr = gr.contiguous()
        p.add_(0.5 * eps * gr)
    torch.cuda.synchronize()
    assert torch.max(torch.abs(q - q0) / sd).item() < 1e-5
    # sampling: chain means and variances match the target
    sampler = hmc.HMC(q0, inv_mass, 0.5, 8, logp_grad=lg, seed=11)
    sampler.run(30)
    qs = []
    for _ in range(40):
        sampler.run(1)
        qs.append(sampler.q.clone())
    Q = torch.stack(qs).reshape(-1, d)
    z_mean = ((Q.mean(0) - mu) / (sd / math.sqrt(Q.shape[0] / 8))).abs().max().item()
    ratio = (Q.var(0) / sd ** 2)
    assert z_mean < 6.0
    assert torch.all((ratio > 0.85) & (ratio < 1.15)), ratio
    assert sampler.n_accepted / sampler.n_proposed > 0.5


def test_lens_hmc_runs(mods):
    abi, hmc = mods
    spec = inputs.SystemSpec(40, 40, 2, 11, "moffat")
    truth, image, psf = make_system(spec, 3100)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    q0 = torch.from_numpy(inputs.draw_perturbed(np.random.default_rng(4), truth, 64, frac=0.002)).cuda()
    inv_mass = hmc.laplace_inv_mass(s, torch.from_numpy(truth).cuda())
    sampler = hmc.HMC(q0, inv_mass, 0.05, 8, system=s, seed=2)
    lp0 = sampler.logp.clone()
    sampler.tune_step_size(rounds=4, iters=2)
    stats = sampler.run(10)
    assert torch.isfinite(sampler.logp).all()
    assert 0.2 < stats.acceptance <= 1.0
    assert (sampler.q - q0.double()).abs().max().item() > 0
    assert sampler.logp.mean().item() > lp0.mean().item() - 50.0
    s.close()
