"""Inference spread over two processes (gloo, host-side exchanges; both on
the one GPU, whose kernels never wait on each other) against one process:

* both processes end with the same MAP point, variational posterior and
  samples, bit for bit;
* MAP and HMC give one process's results (per-start and per-chain work is
  independent of the batch it runs in; the global quantities are reduced
  from the same gathered values);
* VI differs only by the order in which the draws' moment sums are added.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SETTINGS = dict(map_steps=60, vi_steps=40, vi_draws=48, chains=10, n_burn=30, n_samples=12, seed=4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(group):
    import sys
    sys.path.insert(0, ROOT)
    import oracle
    from paper_2202_07663_gb300 import abi, hmc, inputs, map as gmap, pipeline
    spec = inputs.SystemSpec(32, 32, 2, 7, "gaussian", inputs.PIXEL_SCALE, 0.2, 100.0)
    rng = np.random.default_rng(23)
    truth = inputs.draw_table(rng, inputs.PAPER_SIM, 1)[0]
    truth[0] = 0.8
    psf = inputs.make_psf(spec).astype(np.float32)
    model = oracle.simulate(truth, spec.H, spec.W, psf, spec.pixel_scale, spec.k)[0]
    image = inputs.add_noise(rng, model, spec.sigma_bkg, spec.gain_exposure).astype(np.float32)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    starts = torch.from_numpy(inputs.draw_perturbed(np.random.default_rng(6), truth, 9, frac=0.01)
                              .astype(np.float32)).cuda()
    r = pipeline.model_system(s, starts, group=group, **SETTINGS)
    # HMC on its own around the MAP point (no VI rounding upstream)
    th = torch.from_numpy(r.theta_map.astype(np.float32))[None].cuda()
    z0 = gmap.MultiStartMAP(s, steps=0).run(th).z[0].clone()
    cov = torch.diag(torch.full((22,), 1e-6, dtype=torch.float64, device="cuda"))
    ps = hmc.sample_posterior(s, z0, cov, chains=10, n_burn=30, n_samples=12, seed=9, group=group)
    torch.cuda.synchronize()
    s.close()
    return dict(theta_map=r.theta_map, map_objective=r.map_objective, vi_mu=r.vi_mu.cpu().numpy(),
                vi_cov=r.vi_cov.cpu().numpy(), z=r.samples.z.cpu().numpy(), evals=dict(r.grad_evals),
                hmc_z=ps.z.cpu().numpy(), hmc_eps=ps.run.step_size, hmc_T=ps.run.trajectory_length)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        out[rank] = _run(dist.group.WORLD)
    finally:
        dist.destroy_process_group()


def _single(_, out):
    torch.cuda.set_device(0)
    out["single"] = _run(None)


def test_two_processes_match_one():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle
    from paper_2202_07663_gb300 import build
    build.build()
    oracle.build()
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:   # no fork of this (threaded, CUDA) process
        out = m.dict()
        mp.spawn(_single, args=(out,), nprocs=1, join=True)
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    a, b, one = res[0], res[1], res["single"]
    for k in ("theta_map", "vi_mu", "vi_cov", "z", "hmc_z"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    assert a["map_objective"] == b["map_objective"] and a["hmc_eps"] == b["hmc_eps"] and a["hmc_T"] == b["hmc_T"]
    # shards: 9 starts -> 5 + 4, 48 draws -> 24 + 24, 10 chains -> 5 + 5
    assert a["evals"]["map"] == 5 * 61 and b["evals"]["map"] == 4 * 61
    assert a["evals"]["vi"] == b["evals"]["vi"] == 24 * 40
    assert one["evals"]["map"] == 9 * 61 and one["evals"]["vi"] == 48 * 40
    np.testing.assert_array_equal(a["theta_map"], one["theta_map"])
    assert a["map_objective"] == one["map_objective"]
    np.testing.assert_allclose(a["vi_mu"], one["vi_mu"], rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(a["vi_cov"], one["vi_cov"], rtol=1e-7, atol=1e-14)
    np.testing.assert_allclose(a["hmc_z"], one["hmc_z"], rtol=1e-10, atol=1e-12)
    assert a["hmc_eps"] == pytest.approx(one["hmc_eps"], rel=1e-12)
    assert a["hmc_T"] == pytest.approx(one["hmc_T"], rel=1e-12)
