"""Benchmark of the batched lens log-likelihood + gradient on GB300.

One step = one gl_loglik_grad call over B = 4096 parameter vectors of one
synthetic 60x60 lens (k = 2 supersampling, 11x11 Gaussian PSF, 0.065"/pix):
the multi-start batched workload. Every step runs the whole hot path:
per-vector setup, ray shooting + lights + binning, PSF convolution +
likelihood + pixel adjoint, recomputed-ray adjoint, gradient reduction.

Prints ONE JSON line (rank 0). Keys beyond the metric:
  e2e          same metric through the host-buffer C-ABI entry point
               (pinned params in, log L + gradient out, copies timed)
  roofline     dominant kernel (k_ray_adj) against the FP32 ALU peak
  cpu_baseline the FP64 oracle on the host cores, bounded sample
  clocks       nvidia-smi SM clocks and throttle reasons during the timed region
  gpu_launches kernels this library launched in the timed region

--impl reference times the FP64 CPU oracle on the same workload instead
(the paper publishes no per-evaluation reference implementation).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2202_07663_gb300 import inputs  # noqa: E402

METRIC = "log-lik+grad evals/s"
UNIT = "evals/s"
WORKLOAD = inputs.MULTISTART

# FP32 flop counts per ray of the two ray kernels (FMA = 2), N = EPL series
# terms of the vector; per pixel of the convolution kernel.
def flops_ray_fwd(N):
    return 90 + 7 * N


def flops_ray_adj(N):
    return 331 + 14 * N


def flops_conv_pixel(K, grad):
    return (4 if grad else 2) * K * K + 25


SERIES_TOL = 2e-8
NMAX = 128


def series_terms(params: np.ndarray, adjoint: bool) -> np.ndarray:
    """Per-vector EPL series length, the rules the setup kernel applies:
    forward  smallest N >= 0 with |a_(N+1)| f^(N+1) / (1 - f max(1, c_(N+2))) <= tol,
             a_n = c_1 ... c_n, c_k = (2k - 2 + t) / (2k + 2 - t), t = gamma - 1,
    adjoint  the same N, at least 1."""
    p = params.astype(np.float64)
    f = np.hypot(p[:, 2], p[:, 3])[:, None]
    t = (p[:, 1] - 1.0)[:, None]
    k = np.arange(1, NMAX + 2)[None, :]
    c = (2 * k - 2 + t) / (2 * k + 2 - t)                    # c_1 .. c_(NMAX+1)
    with np.errstate(divide="ignore"):
        la = np.cumsum(np.log(np.abs(c)), axis=1)             # log|a_1| .. log|a_(NMAX+1)|
        lf = np.where(f > 0, np.log(np.maximum(f, 1e-300)), -1e300)
    N = np.arange(0, NMAX + 1)[None, :]
    kk = N + 2
    cnext = (2 * kk - 2 + t) / (2 * kk + 2 - t)
    r = np.minimum(f * np.maximum(1.0, cnext), 0.999999)
    good = la[:, :NMAX + 1] + (N + 1) * lf - np.log1p(-r) <= np.log(SERIES_TOL)
    first = np.where(good.any(axis=1), good.argmax(axis=1), NMAX)
    if adjoint:
        first = np.maximum(first, 1)
    return first.astype(np.int64)


MUFU_RAY_ADJ = 12   # ex2/lg2/rcp per ray in the adjoint (EPL power, two Sersic profiles)
# DRAM bytes per launch of k_ray_adj from one ncu capture, valid only for the
# kernel source it was taken on (sha256 prefix of gl_kernels.cu + gl_device.cuh);
# any other source reports null traffic until it is captured again.
TRAFFIC = {"484cf7d85eb9f23b": 64.712192e6}   # ncu dram read + write, one launch at B = 4096


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for f in ("gl_kernels.cu", "gl_device.cuh"):
        with open(os.path.join(ROOT, "paper_2202_07663_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons (every 50 ms)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def rank_param_seed(rank: int) -> int:
    """Seed of rank r's parameter batch: every rank evaluates its own B vectors."""
    return inputs.WORKLOADS[WORKLOAD]["seed"] + 17 + rank


def max_over_ranks(value: float, device, world: int) -> float:
    """Max of a per-rank float over all ranks (the timing rule of the benchmark)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, per_rank_units: int, seconds: float) -> float:
    """Units processed by all ranks per second of the slowest rank (weak scaling)."""
    return world * per_rank_units / seconds


def make_workload(device, rank: int):
    """Synthetic lens system (observed image from the GPU model + seeded noise) and B vectors."""
    import torch
    from paper_2202_07663_gb300 import abi
    c = inputs.WORKLOADS[WORKLOAD]
    spec, B = c["spec"], c["B"]
    rng = inputs.rng_for(WORKLOAD, 0)
    truth = inputs.draw_truth(rng)
    psf = inputs.make_psf(spec).astype(np.float32)
    blank = np.zeros((spec.H, spec.W), np.float32)
    s0 = abi.GLSystem(blank, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    model = s0.simulate(torch.from_numpy(truth.astype(np.float32)[None]).to(device)).cpu().numpy()[0]
    s0.close()
    image = inputs.add_noise(rng, model, spec.sigma_bkg, spec.gain_exposure).astype(np.float32)
    params = inputs.draw_box(np.random.default_rng(rank_param_seed(rank)), B).astype(np.float32)
    return spec, B, truth, psf, image, params


def synthetic_system(workload: str, device):
    """(spec, truth, psf, image) of a workload: GPU model of a seeded truth + seeded noise."""
    import torch
    from paper_2202_07663_gb300 import abi
    spec = inputs.WORKLOADS[workload]["spec"]
    rng = inputs.rng_for(workload, 0)
    truth = inputs.draw_truth(rng)
    psf = inputs.make_psf(spec).astype(np.float32)
    blank = np.zeros((spec.H, spec.W), np.float32)
    s0 = abi.GLSystem(blank, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    model = s0.simulate(torch.from_numpy(truth.astype(np.float32)[None]).to(device)).cpu().numpy()[0]
    s0.close()
    image = inputs.add_noise(rng, model, spec.sigma_bkg, spec.gain_exposure).astype(np.float32)
    return spec, truth, psf, image


def run_hmc_workload(device, iterations: int = 200, chains: int = 512, leapfrog: int = 8, cpu: bool = False):
    """HMC through the adjoint, 100x100 pixels, k = 4, 21x21 Moffat PSF."""
    import torch
    from paper_2202_07663_gb300 import abi, hmc
    spec, truth, psf, image = synthetic_system(inputs.HMC, device)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    s.reserve(chains)
    q0 = torch.from_numpy(inputs.draw_perturbed(np.random.default_rng(3017), truth, chains, frac=0.002)).to(device)
    inv_mass = hmc.laplace_inv_mass(s, torch.from_numpy(truth).to(device))
    sampler = hmc.HMC(q0, inv_mass, 0.05, leapfrog, system=s, seed=3)
    eps = sampler.tune_step_size(rounds=5, iters=2)
    st = sampler.run(iterations)
    s.close()
    out = {"workload": "hmc-100x100-k4-moffat21", "chains": chains, "leapfrog": leapfrog,
           "iterations": iterations, "grad_evals": st.grad_evals, "seconds": st.seconds,
           "evals_per_s": st.evals_per_s, "acceptance": st.acceptance, "step_size": eps,
           "mass": "diagonal, 1/|d2 logL/dq2| at the truth (Laplace)",
           "log_density": "log L (flat prior), physical parameters"}
    if cpu:
        out["cpu_oracle"] = oracle_sample(spec, psf, image, q0.cpu().numpy().astype(np.float32))
    return out


def run_stress_workload(device, steps: int = 3, cpu: bool = False):
    """The stress workload: 200x200 pixels, k = 4, 21x21 PSF, B = 16384 vectors per call."""
    import torch
    from paper_2202_07663_gb300 import abi
    spec, truth, psf, image = synthetic_system(inputs.STRESS, device)
    B = inputs.WORKLOADS[inputs.STRESS]["B"]
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    s.reserve(B)
    params = inputs.draw_box(np.random.default_rng(5017), B).astype(np.float32)
    p = torch.from_numpy(params).to(device)
    ll = torch.empty(B, dtype=torch.float64, device=device)
    g = torch.empty(B, 22, dtype=torch.float64, device=device)
    s.loglik_grad(p, out=(ll, g, None))
    torch.cuda.synchronize()
    abi.gl_profile_reset()
    abi.gl_profile_enable(True)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(steps):
        s.loglik_grad(p, out=(ll, g, None))
    e.record()
    torch.cuda.synchronize()
    prof = abi.gl_profile_read()
    abi.gl_profile_enable(False)
    ms = a.elapsed_time(e) / steps
    n_adj, ms_adj = prof["k_ray_adj"]
    N = series_terms(params, adjoint=True)
    rays = spec.H * spec.W * spec.k * spec.k
    adj_tflops = rays * float(flops_ray_adj(N).sum()) / (ms_adj / n_adj * 1e-3) / 1e12
    s.close()
    out = {"workload": "stress-200x200-k4-psf21-B16384", "B": B, "steps": steps, "ms_per_step": ms,
           "evals_per_s": B / (ms * 1e-3), "k_ray_adj_tflops": adj_tflops,
           "kernel_ms_per_step": {k: v[1] / steps for k, v in prof.items() if v[0] > 0},
           "finite": bool(torch.isfinite(ll).all().item() and torch.isfinite(g).all().item())}
    if cpu:
        out["cpu_oracle"] = oracle_sample(spec, psf, image, params)
    return out


def run_serving_workload(device, n_latency: int = 200, n_capacity: int = 1000):
    """The serving workload: the seeded stream of heterogeneous lenses (Poisson 20/s; sizes
    40..120 px, k in {2, 4}, PSF 11 or 21, 256..2048 vectors per request).
    Latency: the first n_latency requests at their arrival times through the
    continuous-batching server. Capacity: n_capacity requests all at t = 0,
    served (grouped, graph-replayed) and one gl_loglik_grad call per lens."""
    from paper_2202_07663_gb300 import serving
    stream = inputs.serving_stream(n=n_capacity)
    reqs = serving.make_requests(stream, device)
    srv = serving.LensServer(budget_bytes=16 << 30, arena_bytes=4 << 30, max_segments=64, chunk=2048)
    lat, _ = srv.serve(reqs[:n_latency], realtime=True)
    cap, _ = srv.serve(reqs, realtime=False)
    srv.close()
    base_lat = serving.serve_one_call_per_lens(reqs[:n_latency], realtime=True)
    base_cap = serving.serve_one_call_per_lens(reqs, realtime=False)
    return {"workload": "serving-poisson20-40..120px-k2|4-psf11|21-B256..2048",
            "latency_stream": dict(lat.summary(), arrivals="first %d requests at 20/s" % n_latency),
            "capacity": dict(cap.summary(), arrivals="%d requests at t=0" % n_capacity),
            "one_call_per_lens": {"latency_stream": base_lat.summary(), "capacity": base_cap.summary()},
            "speedup_lenses_per_s": cap.lenses_per_s / base_cap.lenses_per_s}


def run_map_workload(device, n_starts: int = 300, steps=(300, 1000, 3000)):
    """Sec. 2.3 / Table 1: multi-start MAP, 300 starts drawn from the prior, on
    a system drawn from the paper's simulation distribution (80x80, k = 2,
    sigma_bkg = 0.2, t_exp = 100 s, G = 1). Reports time, the fraction of
    starts that end at reduced chi^2 <= 1.01 (the paper's marker of runs that
    reached the global mode, Sec. 2.3) and the fraction whose objective ends
    within 1 of the best start's (the same optimum)."""
    import torch
    from paper_2202_07663_gb300 import abi, map as gmap
    spec = inputs.PAPER_SAMPLE_SPEC
    rng = np.random.default_rng(202)
    truth = inputs.draw_table(rng, inputs.PAPER_SIM, 1)[0]
    psf = inputs.make_psf(spec).astype(np.float32)
    blank = np.zeros((spec.H, spec.W), np.float32)
    s0 = abi.GLSystem(blank, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    model = s0.simulate(torch.from_numpy(truth.astype(np.float32)[None]).to(device)).cpu().numpy()[0]
    s0.close()
    image = inputs.add_noise(rng, model, spec.sigma_bkg, spec.gain_exposure).astype(np.float32)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    s.reserve(n_starts)
    th0 = torch.from_numpy(inputs.draw_table(np.random.default_rng(13), inputs.PAPER_PRIOR_DRAW,
                                             n_starts).astype(np.float32)).to(device)
    out = {"workload": "map-multistart-80x80-k2-psf11-paper-noise", "starts": n_starts, "runs": []}
    for k in steps:
        gmap.MultiStartMAP(s, steps=5).run(th0[:8])   # warm-up
        r = gmap.MultiStartMAP(s, steps=k).run(th0)
        _, c2 = s.loglik(r.theta, chi2=True)
        chi2nu = c2.cpu().numpy() / (spec.H * spec.W - 22)
        f = r.objective.cpu().numpy()
        fbest = float(np.nanmin(f))
        out["runs"].append({"iterations": k, "seconds": r.seconds, "evals_per_s": r.grad_evals / r.seconds,
                            "fraction_chi2nu_le_1.01": float(np.mean(chi2nu <= 1.01)),
                            "fraction_at_best_objective": float(np.mean(f <= fbest + 1.0)),
                            "best_objective": fbest, "best_chi2nu": float(chi2nu[int(np.nanargmin(f))])})
    s.close()
    return out


def run_hmc_paper_workload(device, chains: int = 50, n_burn: int = 250, n_samples: int = 750, leapfrog: int = 5):
    """Sec. 2.5 / Table 1 sampling step on a system drawn from the paper's
    simulation distribution (80x80, k = 2, 11x11 PSF, sigma_bkg = 0.2,
    t_exp = 100 s): MAP (300 Adam iterations from 16 starts near the truth),
    Laplace covariance of log p~(z) at the best start as the preconditioner
    (in place of the variational covariance), then 50 chains of HMC on the
    posterior with dual-averaged step size, 250 burn-in + 750 samples, L = 5.
    Reports ESS and R-hat of the 22 physical parameters."""
    import torch
    from paper_2202_07663_gb300 import abi, diagnostics, hmc, map as gmap
    spec = inputs.PAPER_SAMPLE_SPEC
    rng = np.random.default_rng(202)
    truth = inputs.draw_table(rng, inputs.PAPER_SIM, 1)[0]
    psf = inputs.make_psf(spec).astype(np.float32)
    blank = np.zeros((spec.H, spec.W), np.float32)
    s0 = abi.GLSystem(blank, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    model = s0.simulate(torch.from_numpy(truth.astype(np.float32)[None]).to(device)).cpu().numpy()[0]
    s0.close()
    image = inputs.add_noise(rng, model, spec.sigma_bkg, spec.gain_exposure).astype(np.float32)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    s.reserve(max(chains, 2 * 22))
    th0 = torch.from_numpy(inputs.draw_perturbed(np.random.default_rng(2024), truth, 16, frac=0.01)
                           .astype(np.float32)).to(device)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = gmap.MultiStartMAP(s, steps=300).run(th0)
    z_map = r.z[r.best].clone()
    cov = hmc.laplace_covariance(hmc.PosteriorTarget(s), z_map)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    ps = hmc.sample_posterior(s, z_map, cov, chains=chains, n_burn=n_burn, n_samples=n_samples, n_leapfrog=leapfrog,
                              seed=5)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    th = ps.theta.transpose(0, 1).cpu().numpy().astype(np.float64)   # [chains, n, 22]
    s.close()
    ess = diagnostics.ess(th)
    ess_g = diagnostics.ess(th, antithetic=True)
    rh = diagnostics.rhat(th)
    mean, sd = th.reshape(-1, 22).mean(0), th.reshape(-1, 22).std(0)
    hmc_s = ps.run.seconds
    return {"workload": "hmc-posterior-80x80-k2-psf11-paper-noise", "chains": chains, "burn_in": n_burn,
            "samples": n_samples, "leapfrog": leapfrog, "step_size": ps.run.step_size,
            "accept_burn": ps.run.accept_burn, "accept_samples": ps.run.accept_samples,
            "map_and_preconditioner_s": t1 - t0, "hmc_s": hmc_s, "grad_evals": ps.run.grad_evals,
            "evals_per_s": ps.run.grad_evals / hmc_s, "ess_min": float(ess.min()), "ess_mean": float(ess.mean()),
            "ess_per_iter_min": float(ess.min()) / n_samples, "ess_per_s_min": float(ess.min()) / hmc_s,
            "ess_geyer_min": float(ess_g.min()), "ess_geyer_per_s_min": float(ess_g.min()) / hmc_s,
            "rhat_max": float(rh.max()), "max_abs_z_truth": float(np.max(np.abs(mean - truth) / sd)),
            "mass": "dense: Laplace covariance of log p~(z) at the MAP (whitened coordinates)",
            "log_density": "posterior of the unconstrained parameters (prior Eq. sim-dist, bijectors)"}


def run_variant_workload(device, B: int = 4096, steps: int = 10):
    """Sec. 2.1.2 variant: observed-image variance, log L profiled over the two
    light amplitudes (both basis images from one ray pass, 2B convolutions,
    2x2 solves and log L of the profiled model, then the gradient by the PSF
    correlation and the ray adjoint),
    against the plain log L + gradient on the same system and vectors
    (80x80, k = 2, 11x11 PSF, sigma_bkg = 0.2, t_exp = 100 s)."""
    import torch
    from paper_2202_07663_gb300 import abi
    spec = inputs.PAPER_SAMPLE_SPEC
    rng = np.random.default_rng(303)
    truth = inputs.draw_table(rng, inputs.PAPER_SIM, 1)[0]
    psf = inputs.make_psf(spec).astype(np.float32)
    blank = np.zeros((spec.H, spec.W), np.float32)
    s0 = abi.GLSystem(blank, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    model = s0.simulate(torch.from_numpy(truth.astype(np.float32)[None]).to(device)).cpu().numpy()[0]
    s0.close()
    image = inputs.add_noise(rng, model, spec.sigma_bkg, spec.gain_exposure).astype(np.float32)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg,
                     observed_variance=True)
    s.reserve(2 * B)
    p = torch.from_numpy(inputs.draw_perturbed(np.random.default_rng(7), truth, B, frac=0.05)
                         .astype(np.float32)).to(device)
    out = {"workload": "variant-obsvar-profiled-80x80-k2-psf11", "B": B}
    for name, fn in (("plain", lambda: s.loglik_grad(p)), ("profiled", lambda: s.loglik_grad_profiled(p))):
        fn()
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            fn()
        e.record()
        torch.cuda.synchronize()
        ms = a.elapsed_time(e) / steps
        out[name] = {"ms_per_call": ms, "evals_per_s": B / (ms * 1e-3)}
    out["profiled_over_plain_time"] = out["profiled"]["ms_per_call"] / out["plain"]["ms_per_call"]
    s.close()
    return out


def run_pipeline_workload(device):
    """Sec. 2.6 / Table 1: MAP (300 prior starts x 300) -> VI (1000 x 500) ->
    HMC (50 chains, 250 + 750, ChEES) on a system drawn from the paper's
    simulation distribution (80x80, k = 2, 11x11 PSF, sigma_bkg = 0.2,
    t_exp = 100 s): time per stage and in total (the paper's 105 s on
    4 A100), the mode's reduced chi^2, and the sampler's ESS and R-hat; once
    with HMC preconditioned by the VI covariance (the paper) and once by the
    Laplace covariance at the MAP point."""
    import torch
    from paper_2202_07663_gb300 import abi, diagnostics, pipeline
    spec = inputs.PAPER_SAMPLE_SPEC
    rng = np.random.default_rng(202)
    truth = inputs.draw_table(rng, inputs.PAPER_SIM, 1)[0]
    psf = inputs.make_psf(spec).astype(np.float32)
    blank = np.zeros((spec.H, spec.W), np.float32)
    s0 = abi.GLSystem(blank, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    model = s0.simulate(torch.from_numpy(truth.astype(np.float32)[None]).to(device)).cpu().numpy()[0]
    s0.close()
    image = inputs.add_noise(rng, model, spec.sigma_bkg, spec.gain_exposure).astype(np.float32)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    starts = torch.from_numpy(inputs.draw_table(np.random.default_rng(13), inputs.PAPER_PRIOR_DRAW, 300)
                              .astype(np.float32)).to(device)
    # load the dense linear-algebra libraries (L L^T, Cholesky of the 22x22
    # preconditioner) before the clock starts: a one-time cost of the process
    e = torch.eye(22, dtype=torch.float64, device=device)
    torch.linalg.cholesky(e @ e.T)
    torch.cuda.synchronize()
    out = {"workload": "pipeline-80x80-k2-psf11-paper-noise", "map_starts": 300, "paper_seconds_4xA100": 105.0}
    dof = spec.H * spec.W - 22
    for pre in ("vi", "laplace"):
        r = pipeline.model_system(s, starts, preconditioner=pre, seed=1)
        _, c2 = s.loglik(torch.from_numpy(r.theta_map.astype(np.float32)[None]).to(device), chi2=True)
        th = r.samples.theta.transpose(0, 1).cpu().numpy().astype(np.float64)
        ess, rh = diagnostics.ess(th), diagnostics.rhat(th)
        flat = th.reshape(-1, 22)
        out[pre] = {"seconds": {k: round(v, 4) for k, v in r.seconds.items()}, "grad_evals": r.grad_evals,
                    "map_chi2nu": float(c2.item()) / dof, "ess_min": float(ess.min()), "rhat_max": float(rh.max()),
                    "step_size": r.samples.run.step_size, "trajectory_length": r.samples.run.trajectory_length,
                    "max_abs_z_truth": float(np.max(np.abs(flat.mean(0) - truth) / flat.std(0)))}
    s.close()
    return out


def cpu_baseline(spec, psf, image, params, budget_s: float = 12.0):
    """The FP64 oracle (log L + gradient) on a bounded sample of the same workload."""
    import oracle
    oracle.build()
    nt = oracle.max_threads()
    args = (image, np.float32(spec.sigma_bkg), psf, spec.pixel_scale, spec.k, spec.gain_exposure)
    n0 = min(len(params), max(nt, 8))
    t = time.perf_counter()
    oracle.loglik(params[:n0].astype(np.float64), *args, grad=True, nthreads=nt)
    dt = time.perf_counter() - t
    n = int(min(len(params), max(n0, math.floor(n0 * budget_s / max(dt, 1e-3)))))
    t = time.perf_counter()
    oracle.loglik(params[:n].astype(np.float64), *args, grad=True, nthreads=nt)
    dt = time.perf_counter() - t
    # the same on one core, on a smaller sample
    n1 = max(2, min(len(params), int(n * 4.0 / budget_s / max(nt, 1)) + 1))
    t = time.perf_counter()
    oracle.loglik(params[:n1].astype(np.float64), *args, grad=True, nthreads=1)
    dt1 = time.perf_counter() - t
    return {"value": n / dt, "unit": UNIT, "cores": nt, "kind": "oracle",
            "sample": "%d of the %d vectors (log L + forward-mode gradient, FP64), %.1f s" % (n, len(params), dt),
            "value_1core": n1 / dt1, "sample_1core": "%d vectors, %.1f s" % (n1, dt1)}


def oracle_sample(spec, psf, image, params, budget_s: float = 4.0):
    """The FP64 oracle (log L + gradient) on all host cores over a bounded
    sample of a workload's vectors (one per core first, then more if that
    took well under the budget): evals/s and what the sample was."""
    import oracle
    oracle.build()
    nt = oracle.max_threads()
    args = (image, np.float32(spec.sigma_bkg), psf, spec.pixel_scale, spec.k, spec.gain_exposure)
    n = min(len(params), nt)
    t = time.perf_counter()
    oracle.loglik(params[:n].astype(np.float64), *args, grad=True, nthreads=nt)
    dt = time.perf_counter() - t
    if dt < budget_s / 3:
        n = int(min(len(params), max(n, math.floor(n * budget_s / max(dt, 1e-3)))))
        t = time.perf_counter()
        oracle.loglik(params[:n].astype(np.float64), *args, grad=True, nthreads=nt)
        dt = time.perf_counter() - t
    return {"evals_per_s": n / dt, "cores": nt, "kind": "oracle",
            "sample": "%d of the workload's vectors (log L + forward-mode gradient, FP64), %.1f s" % (n, dt)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    c = inputs.WORKLOADS[WORKLOAD]
    spec, B = c["spec"], c["B"]
    rng = inputs.rng_for(WORKLOAD, 0)
    truth = inputs.draw_truth(rng)
    psf = inputs.make_psf(spec).astype(np.float32)
    model = oracle.simulate(truth, spec.H, spec.W, psf, spec.pixel_scale, spec.k)[0]
    image = inputs.add_noise(rng, model, spec.sigma_bkg, spec.gain_exposure).astype(np.float32)
    params = inputs.draw_box(np.random.default_rng(rank_param_seed(0)), B).astype(np.float32)
    nt = oracle.max_threads()
    a = (image, np.float32(spec.sigma_bkg), psf, spec.pixel_scale, spec.k, spec.gain_exposure)
    per_step = max(nt * 2, 32)
    for w in range(args.warmup):
        oracle.loglik(params[:nt].astype(np.float64), *a, grad=True, nthreads=nt)
    times = []
    for s in range(args.steps):
        sl = params[(s * per_step) % B:(s * per_step) % B + per_step].astype(np.float64)
        t = time.perf_counter()
        oracle.loglik(sl, *a, grad=True, nthreads=nt)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = per_step * args.steps / total
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": spec.H, "W": spec.W, "supersample": spec.k, "psf": spec.K, "B": B,
                   "step_sample": per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                         "sample": "%d vectors per step of the %d-vector workload" % (per_step, B)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


def run_small_batch(args, B: int = 50):
    """The call the samplers make (50 chains, Table 1): per-call time of
    log L + gradient for B vectors of one 80x80 system (k = 2, 11x11 PSF,
    the paper's noise), inputs resident, CUDA events around K calls."""
    import torch
    from paper_2202_07663_gb300 import abi, build
    build.build()
    device = torch.device("cuda", 0)
    spec = inputs.PAPER_SAMPLE_SPEC
    rng = np.random.default_rng(50)
    truth = inputs.draw_table(rng, inputs.PAPER_SIM, 1)[0]
    psf = inputs.make_psf(spec).astype(np.float32)
    blank = np.zeros((spec.H, spec.W), np.float32)
    s0 = abi.GLSystem(blank, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    model = s0.simulate(torch.from_numpy(truth.astype(np.float32)[None]).to(device)).cpu().numpy()[0]
    s0.close()
    image = inputs.add_noise(rng, model, spec.sigma_bkg, spec.gain_exposure).astype(np.float32)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    s.reserve(B)
    p = torch.from_numpy(inputs.draw_perturbed(np.random.default_rng(51), truth, B, frac=0.01)
                         .astype(np.float32)).to(device)
    ll = torch.empty(B, dtype=torch.float64, device=device)
    g = torch.empty(B, 22, dtype=torch.float64, device=device)
    for _ in range(args.warmup):
        s.loglik_grad(p, out=(ll, g, None))
    torch.cuda.synchronize()
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(args.steps):
        s.loglik_grad(p, out=(ll, g, None))
    e.record()
    torch.cuda.synchronize()
    us = 1e3 * a.elapsed_time(e) / args.steps
    s.close()
    print(json.dumps({"workload": "small-batch-80x80-k2-psf11-B50", "B": B, "steps": args.steps,
                      "us_per_call": us, "evals_per_s": B / (us * 1e-6),
                      "finite": bool(torch.isfinite(ll).all().item() and torch.isfinite(g).all().item())}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the HMC (100x100, k=4), stress (200x200, B=16384) and serving runs reported beside the metric")
    ap.add_argument("--small-batch", action="store_true",
                    help="only the sampler-sized call: B = 50 vectors of an 80x80, k = 2, 11x11-PSF system")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.small_batch:
        return run_small_batch(args)

    import torch
    import torch.distributed as dist
    from paper_2202_07663_gb300 import abi, build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()

    spec, B, truth, psf, image, params = make_workload(device, rank)
    sysm = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    sysm.reserve(B)
    p_dev = torch.from_numpy(params).to(device)
    ll = torch.empty(B, dtype=torch.float64, device=device)
    g = torch.empty(B, 22, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)   # > L2 (129 MB)

    def step():
        sysm.loglik_grad(p_dev, out=(ll, g, None))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # ---- device-timed steps (inputs resident in HBM; L2 flushed between steps)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    abi.gl_profile_reset()
    abi.gl_profile_enable(True)
    n0 = abi.gl_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local) as clk:
        t0 = time.perf_counter()
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            step()
            b.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    launches = abi.gl_launch_count() - n0
    prof = abi.gl_profile_read()
    abi.gl_profile_enable(False)
    step_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / args.steps, device, world)
    value = whole_job_rate(world, B, step_ms * 1e-3)

    # ---- end to end through the host-buffer entry point (pinned host memory)
    hp = torch.from_numpy(params).pin_memory()
    hl = torch.empty(B, dtype=torch.float64).pin_memory()
    hg = torch.empty(B, 22, dtype=torch.float64).pin_memory()
    hp_np, hl_np, hg_np = hp.numpy(), hl.numpy(), hg.numpy()
    for _ in range(3):
        sysm.loglik_grad_host(hp_np, hl_np, hg_np)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sysm.loglik_grad_host(hp_np, hl_np, hg_np)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / args.steps, device, world)
    e2e_value = whole_job_rate(world, B, e2e_s)

    # ---- roofline of the dominant kernel, from the live event timings
    n_adj, ms_adj = prof["k_ray_adj"]
    N = series_terms(params, adjoint=True)
    rays = spec.H * spec.W * spec.k * spec.k
    flop_adj = float(rays * flops_ray_adj(N).sum())
    adj_s = (ms_adj / max(n_adj, 1)) * 1e-3
    peaks, peak_src = read_peaks()
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved = flop_adj / adj_s / 1e12
    # special-function unit: 12 MUFU ops per ray in the adjoint; 32 per clock per SM
    # (own ex2.approx throughput probe on this GPU)
    mufu_peak = sms * 32 * sm_mhz * 1e6 / 1e9
    mufu_achieved = rays * B * MUFU_RAY_ADJ / adj_s / 1e9
    th = kernel_source_hash()
    traffic = TRAFFIC.get(th)
    if traffic is not None:
        traffic = traffic * B / 4096.0   # captured at B = 4096; DRAM bytes scale with the vectors of a launch
    kern = {k: {"launches": v[0], "ms_total": round(v[1], 4)} for k, v in prof.items() if v[0] > 0}
    tot = sum(v[1] for v in prof.values())
    for k in kern:
        kern[k]["share"] = round(prof[k][1] / tot, 4) if tot > 0 else None
    clocks = clk.summary()

    if world > 1:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(spec, psf, image, params)
    workloads = None
    if world == 1 and not args.no_workloads:
        cpu_w = not args.no_cpu_baseline
        workloads = {"hmc": run_hmc_workload(device, cpu=cpu_w), "stress": run_stress_workload(device, cpu=cpu_w),
                     "serving": run_serving_workload(device), "map": run_map_workload(device),
                     "hmc_paper": run_hmc_paper_workload(device), "variant": run_variant_workload(device),
                     "pipeline": run_pipeline_workload(device)}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (f64 per-vector sums)", "data": "synthetic",
        "config": {"workload": WORKLOAD, "H": spec.H, "W": spec.W, "supersample": spec.k, "psf": spec.K,
                   "pixel_scale": spec.pixel_scale, "B_per_gpu": B, "params": "uniform over the prior box",
                   "l2": "flushed (256 MB write) between timed steps, flush outside the step events",
                   "parallelism": "replicas (B per GPU)" if world > 1 else "single GPU"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": B * 22 * 4,
                "d2h_bytes_per_step": B * 8 + B * 22 * 8},
        "roofline": {"bound": "alu", "kernel": "k_ray_adj", "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic,
                     "flops_per_launch": flop_adj, "launch_ms": adj_s * 1e3,
                     "peak_basis": "FP32 FMA: %d SMs x 128 lanes x 2 x %.0f MHz (max SM clock, %s peaks file)" % (
                         sms, sm_mhz, peak_src),
                     "mufu": {"achieved": mufu_achieved, "peak": mufu_peak, "unit": "Gop/s",
                              "frac": mufu_achieved / mufu_peak, "ops_per_ray": MUFU_RAY_ADJ,
                              "peak_basis": "%d SMs x 32 MUFU/clk (measured ex2 probe) x %.0f MHz" % (sms, sm_mhz)},
                     "mean_series_terms": float(N.mean()), "kernel_source": th},
        "kernels": kern,
        "cpu_baseline": cpu,
        "workloads": workloads,
        "clocks": clocks,
        "gpu_launches": int(launches),
        "wall_s_timed": wall,
    }
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
