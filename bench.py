"""Benchmark of the batched lens log-likelihood + gradient on GB300.

One step = one gl_loglik_grad call over B = 4096 parameter vectors of one
synthetic 60x60 lens (k = 2 supersampling, 11x11 Gaussian PSF, 0.065"/pix):
the multi-start batched workload. Every step runs the whole hot path:
per-vector setup, ray shooting + lights + binning, PSF convolution +
likelihood + pixel adjoint, recomputed-ray adjoint, gradient reduction.

Prints ONE JSON line (rank 0). Keys beyond the metric:
  e2e          same metric through the host-buffer C-ABI entry point
               (pinned params in, log L + gradient out, copies timed)
  roofline     dominant kernel (k_ray_adj) against the measured FP32 peak
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


def flops_conv_pixel(K, grad, R=0):
    """K x K stencil: 2 K^2 flops per pass; R separable terms: a K-tap
    horizontal and a K-tap vertical pass per term, 4 K R flops per pass.
    Two passes (model, adjoint correlation) with the gradient; ~25 for the
    likelihood terms."""
    per_pass = 4 * K * R if R > 0 else 2 * K * K
    return (2 if grad else 1) * per_pass + 25


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


MUFU_RAY_ADJ = 13   # ex2/lg2/rcp per ray in the adjoint: EPL 5 (lg2, ex2, three rcp), each Sersic profile 4
# DRAM bytes per launch of k_ray_adj from one ncu capture, keyed by workload
# and the kernel source it was taken on (sha256 prefix of gl_kernels.cu +
# gl_device.cuh); any other source reports null traffic until it is captured again.
TRAFFIC = {("multistart-60x60-k2-psf11-B4096", "7e5e9fc077046014"): 64.524e6}


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


def rank_param_seed(workload: str, rank: int) -> int:
    """Seed of rank r's parameter batch: every rank evaluates its own B vectors."""
    return inputs.WORKLOADS[workload]["seed"] + 17 + rank


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


BENCH_INPUTS = os.path.join(ROOT, "tests", "golden", "bench_inputs")


def load_observed(workload: str):
    """(spec, truth, psf, image) of a benchmark workload. The observed image
    was written by the FP64 oracle (model of the seeded truth + seeded noise,
    tests/golden/bench_inputs/make_bench_images.py), so both arms of the
    benchmark and its error report use the same data, none of it from the
    CUDA path."""
    spec = inputs.WORKLOADS[workload]["spec"]
    image = np.load(os.path.join(BENCH_INPUTS, workload + ".image.npy"))
    truth = np.load(os.path.join(BENCH_INPUTS, workload + ".truth.npy"))
    if not np.array_equal(inputs.draw_truth(inputs.rng_for(workload, 0)), truth):
        raise RuntimeError("stored benchmark input of %s does not match its seed" % workload)
    psf = inputs.make_psf(spec).astype(np.float32)
    return spec, truth, psf, image.astype(np.float32)


def workload_params(workload: str, rank: int, truth: np.ndarray) -> np.ndarray:
    c = inputs.WORKLOADS[workload]
    rng = np.random.default_rng(rank_param_seed(workload, rank))
    if c["draw"] == "box":
        return inputs.draw_box(rng, c["B"]).astype(np.float32)
    return inputs.draw_perturbed(rng, truth, c["B"]).astype(np.float32)


def workload_config(workload: str) -> dict:
    """The config object of a workload, the same in both arms of the benchmark."""
    c = inputs.WORKLOADS[workload]
    spec = c["spec"]
    return {"workload": workload, "H": spec.H, "W": spec.W, "supersample": spec.k, "psf": spec.K,
            "psf_kind": spec.psf, "pixel_scale": spec.pixel_scale, "sigma_bkg": spec.sigma_bkg,
            "gain_exposure": spec.gain_exposure, "B_per_gpu": c["B"],
            "params": "uniform over the prior box" if c["draw"] == "box" else "truth + N(0, 0.02 box width)",
            "image": "oracle model of the seeded truth + seeded noise (stored input)",
            "l2": "GPU arm: flushed by a 256 MB write between timed steps, outside the step events"}


TOL_UNITS = ("multiples of the tolerance: log L |dl| / (1e-4 max(|l|, 1)); gradient "
             "|dg_i| / (1e-3 (|g_i| + 1e-2 max_j |g_j|)), per component")


def error_stats(ll, g, rl, rg) -> dict:
    """Error of the GPU results against the FP64 oracle, per vector (log L)
    and per component (gradient), in multiples of the stated tolerance."""
    el = np.abs(ll - rl) / (1e-4 * np.maximum(np.abs(rl), 1.0))
    eg = np.abs(g - rg) / (1e-3 * (np.abs(rg) + 1e-2 * np.max(np.abs(rg), axis=1, keepdims=True)))
    per = eg.max(axis=0)
    j = int(np.argmax(per))
    return {"vectors": int(len(ll)), "unit": TOL_UNITS,
            "loglik": {"max": float(el.max()), "p99": float(np.percentile(el, 99)),
                       "frac_over_1": float(np.mean(el > 1))},
            "grad": {"max": float(eg.max()), "p99": float(np.percentile(eg, 99)),
                     "frac_over_1": float(np.mean(eg > 1)), "worst_param": inputs.PARAM_NAMES[j]}}


def oracle_sample(spec, psf, image, params, budget_s: float, min_n: int = 8):
    """The FP64 oracle (log L + gradient) on all host cores over a bounded,
    evenly spread sample of a workload's vectors (first and last included):
    (timing dict, sample indices, oracle log L, oracle gradient)."""
    import oracle
    oracle.build()
    nt = oracle.max_threads()
    args = (image, np.float32(spec.sigma_bkg), psf, spec.pixel_scale, spec.k, spec.gain_exposure)
    B = len(params)

    def pick(n):
        return np.unique(np.linspace(0, B - 1, min(n, B)).round().astype(np.int64))

    idx = pick(max(nt, min_n))
    t = time.perf_counter()
    oracle.loglik(params[idx].astype(np.float64), *args, grad=True, nthreads=nt)
    dt = time.perf_counter() - t
    if dt < budget_s / 3:
        idx = pick(int(max(len(idx), math.floor(len(idx) * budget_s / max(dt, 1e-3)))))
        t = time.perf_counter()
    rl, _, rg = oracle.loglik(params[idx].astype(np.float64), *args, grad=True, nthreads=nt)
    dt = time.perf_counter() - t
    timing = {"value": len(idx) / dt, "unit": UNIT, "cores": nt, "kind": "oracle",
              "sample": "%d of the %d vectors, evenly spread, first and last included (log L + forward-mode "
                        "gradient, FP64), %.1f s" % (len(idx), B, dt)}
    return timing, idx, rl, rg


def cpu_baseline(spec, psf, image, params, ll_gpu, g_gpu, budget_s: float = 12.0):
    """The CPU-baseline leg: the FP64 oracle timed on a bounded sample of the
    workload (all host cores, and one core on a smaller sample), and the error
    of the GPU results on that sample against it."""
    import oracle
    timing, idx, rl, rg = oracle_sample(spec, psf, image, params, budget_s)
    args = (image, np.float32(spec.sigma_bkg), psf, spec.pixel_scale, spec.k, spec.gain_exposure)
    n1 = max(2, min(len(idx), int(len(idx) * 3.0 / budget_s / max(timing["cores"], 1)) + 1))
    t = time.perf_counter()
    oracle.loglik(params[idx[:n1]].astype(np.float64), *args, grad=True, nthreads=1)
    dt1 = time.perf_counter() - t
    timing.update(value_1core=n1 / dt1, sample_1core="%d vectors, %.1f s" % (n1, dt1))
    err = error_stats(ll_gpu[idx], g_gpu[idx], rl, rg)
    err["sample"] = "the CPU-baseline sample (%d vectors)" % len(idx)
    return timing, err


def measured_peaks():
    """FP32 FMA and ex2 rates of this GPU from the library's probe kernels."""
    from paper_2202_07663_gb300 import abi
    return {"fp32_tflops": abi.gl_profile_peak(abi.GL_PEAK_FP32_FMA) / 1e12,
            "mufu_ex2_gops": abi.gl_profile_peak(abi.GL_PEAK_MUFU_EX2) / 1e9}


def measure(workload: str, device, rank: int, world: int, steps: int, warmup: int, cpu: bool, peaks: dict,
            cpu_budget_s: float = 12.0) -> dict:
    """One benchmark line for a workload: device-timed steps (inputs resident,
    L2 flushed between steps, clocks sampled), the end-to-end rate through the
    host-buffer entry point, the roofline of the dominant kernel against the
    measured FP32 peak, kernel shares, and (rank 0, one GPU) the oracle
    baseline with the per-result error."""
    import torch
    import torch.distributed as dist
    from paper_2202_07663_gb300 import abi
    spec, truth, psf, image = load_observed(workload)
    B = inputs.WORKLOADS[workload]["B"]
    params = workload_params(workload, rank, truth)
    sysm = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    psf_rank = sysm.psf_rank()   # separable PSF terms the convolution runs with (0: K x K stencil)
    sysm.reserve(B)
    p_dev = torch.from_numpy(params).to(device)
    ll = torch.empty(B, dtype=torch.float64, device=device)
    g = torch.empty(B, 22, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(device)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=device)   # > L2 (129 MB)

    def step():
        sysm.loglik_grad(p_dev, out=(ll, g, None))

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()

    # ---- device-timed steps (inputs resident in HBM; L2 flushed between steps).
    # Only the dominant kernel is bracketed by the library's events here: an
    # event between two kernels of a call ends their programmatic overlap, and
    # bracketing all five lengthened the 60x60 step by ~30 us (two boundaries:
    # ~8 us). The other kernels' times come from a profiled pass below.
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    abi.gl_profile_reset()
    abi.gl_profile_select([abi.GL_K_RAY_ADJ])
    abi.gl_profile_enable(True)
    n0 = abi.gl_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    local = int(os.environ.get("LOCAL_RANK", "0"))
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
    prof_timed = abi.gl_profile_read()
    abi.gl_profile_enable(False)
    step_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev) / steps, device, world)
    value = whole_job_rate(world, B, step_ms * 1e-3)
    ll_host, g_host = ll.cpu().numpy(), g.cpu().numpy()

    # ---- profiled pass: every kernel bracketed (shares; slower steps, not the metric)
    psteps = min(steps, 100)
    pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(psteps)]
    abi.gl_profile_reset()
    abi.gl_profile_select(range(abi.GL_KERNEL_KINDS))
    abi.gl_profile_enable(True)
    for a, b in pev:
        flush.zero_()
        a.record(stream)
        step()
        b.record(stream)
    torch.cuda.synchronize()
    prof = abi.gl_profile_read()
    abi.gl_profile_enable(False)
    profiled_ms = sum(a.elapsed_time(b) for a, b in pev) / psteps
    del flush

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
    for _ in range(steps):
        sysm.loglik_grad_host(hp_np, hl_np, hg_np)
    e2e_s = max_over_ranks((time.perf_counter() - t0) / steps, device, world)
    e2e_value = whole_job_rate(world, B, e2e_s)
    sysm.close()

    # ---- roofline of the dominant kernel (and the rates of the others), from the live event timings
    rays = spec.H * spec.W * spec.k * spec.k
    N_adj = series_terms(params, adjoint=True)
    N_fwd = series_terms(params, adjoint=False)
    work = {"k_ray_adj": float(rays * flops_ray_adj(N_adj).sum()),
            "k_ray_fwd": float(rays * flops_ray_fwd(N_fwd).sum()),
            "k_conv": float(B * spec.H * spec.W * flops_conv_pixel(spec.K, True, psf_rank))}
    n_adj, ms_adj = prof_timed["k_ray_adj"]   # the timed steps' own adjoint launches
    adj_s = (ms_adj / max(n_adj, 1)) * 1e-3
    fp32_peak = peaks["fp32_tflops"]
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    nominal = read_peaks()[0]
    fp32_nominal = sms * 128 * 2 * float(nominal.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    achieved = work["k_ray_adj"] / adj_s / 1e12
    mufu_peak = peaks["mufu_ex2_gops"]
    mufu_achieved = rays * B * MUFU_RAY_ADJ / adj_s / 1e9
    th = kernel_source_hash()
    traffic = TRAFFIC.get((workload, th))
    tot = sum(v[1] for v in prof.values())
    kern = {}
    for k, (n, ms) in prof.items():
        if n == 0:
            continue
        kern[k] = {"launches": n, "ms_total": round(ms, 4), "share": round(ms / tot, 4) if tot > 0 else None}
        if k in work:
            kern[k]["tflops"] = work[k] / (ms / n * 1e-3) / 1e12
            kern[k]["frac_fp32_peak"] = kern[k]["tflops"] / fp32_peak
    if "k_conv" in kern:
        kern["k_conv"]["psf_terms"] = psf_rank   # 0: K x K stencil; R: R pairs of 1-D passes
    clocks = clk.summary()
    cpu_base, err = None, None
    if cpu and rank == 0 and world == 1:
        cpu_base, err = cpu_baseline(spec, psf, image, params, ll_host, g_host, budget_s=cpu_budget_s)
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (f64 per-vector sums)", "data": "synthetic",
        "config": dict(workload_config(workload),
                       parallelism="replicas (B per GPU)" if world > 1 else "single GPU"),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": B * 22 * 4,
                "d2h_bytes_per_step": B * 8 + B * 22 * 8},
        "roofline": {"bound": "alu", "kernel": "k_ray_adj", "achieved": achieved, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic,
                     "flops_per_launch": work["k_ray_adj"], "launch_ms": adj_s * 1e3,
                     "launch_basis": "CUDA events around every k_ray_adj launch of the timed steps, on the "
                                     "launching stream (the only kernel bracketed in them)",
                     "peak_basis": "measured: packed-FMA probe kernel of this library (gl_profile_peak) on this "
                                   "GPU before the timed steps, best of five launches",
                     "peak_nominal": fp32_nominal, "frac_of_nominal": achieved / fp32_nominal,
                     "nominal_basis": "%d SMs x 128 FP32 lanes x 2 x %.0f MHz (max SM clock)" % (
                         sms, float(nominal.get("sm_max_mhz", 2070.0))),
                     "mufu": {"achieved": mufu_achieved, "peak": mufu_peak, "unit": "Gop/s",
                              "frac": mufu_achieved / mufu_peak, "ops_per_ray": MUFU_RAY_ADJ,
                              "peak_basis": "measured: ex2 probe kernel (gl_profile_peak)"},
                     "mean_series_terms": float(N_adj.mean()), "kernel_source": th},
        "kernels": kern,
        "kernels_basis": "a profiled pass of %d more steps with every kernel bracketed by CUDA events on the "
                         "launching stream (the events end the programmatic overlap between kernels, so those "
                         "steps took %.4f ms against the metric's %.4f)" % (psteps, profiled_ms, step_ms),
        "cpu_baseline": cpu_base,
        "error": err,
        "clocks": clocks,
        "gpu_launches": int(launches),
        "wall_s_timed": wall,
    }


def run_hmc_workload(device, iterations: int = 200, chains: int = 512, leapfrog: int = 8, cpu: bool = False):
    """HMC through the adjoint (100x100 pixels, k = 4, 21x21 Moffat PSF): 512
    chains x 8 leapfrog steps x 200 iterations, the log density and its
    gradient through the torch.autograd.Function (LogLik + autograd.grad);
    the same run through the library's direct call beside it, so that the
    Function's overhead is measured. With cpu, the error of the gradient
    evaluations against the FP64 oracle on a sample of the chains' start
    points."""
    import torch
    from paper_2202_07663_gb300 import abi, hmc
    spec, truth, psf, image = load_observed(inputs.HMC)
    s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
    s.reserve(chains)
    q0 = torch.from_numpy(inputs.draw_perturbed(np.random.default_rng(3017), truth, chains, frac=0.002)).to(device)
    inv_mass = hmc.laplace_inv_mass(s, torch.from_numpy(truth).to(device))
    out = {"workload": "hmc-100x100-k4-moffat21", "chains": chains, "leapfrog": leapfrog, "iterations": iterations,
           "mass": "diagonal, 1/|d2 logL/dq2| at the truth (Laplace)",
           "log_density": "log L (flat prior), physical parameters"}
    eps = None
    for name, target in (("autograd", hmc.AutogradTarget(s)), ("direct", hmc.LensTarget(s))):
        sampler = hmc.HMC(q0, inv_mass, 0.05, leapfrog, target=target, seed=3)
        if eps is None:
            eps = sampler.tune_step_size(rounds=5, iters=2)
        else:
            sampler.eps = eps
        st = sampler.run(iterations)
        out[name] = {"grad_evals": st.grad_evals, "seconds": st.seconds, "evals_per_s": st.evals_per_s,
                     "acceptance": st.acceptance}
    out.update(step_size=eps, grad_evals=out["autograd"]["grad_evals"], seconds=out["autograd"]["seconds"],
               evals_per_s=out["autograd"]["evals_per_s"], acceptance=out["autograd"]["acceptance"],
               autograd_over_direct_time=out["autograd"]["seconds"] / out["direct"]["seconds"])
    if cpu:
        q = q0.to(torch.float32).contiguous()
        ll, g = s.loglik_grad(q)
        timing, idx, rl, rg = oracle_sample(spec, psf, image, q.cpu().numpy(), budget_s=4.0, min_n=16)
        out["cpu_oracle"] = timing
        out["error"] = dict(error_stats(ll.cpu().numpy()[idx], g.cpu().numpy()[idx], rl, rg),
                            sample="%d of the chains' start points" % len(idx))
    s.close()
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
    # warm-up of both forms (first launches of each kernel variant load its code)
    srv.serve(reqs[:40], realtime=False)
    serving.serve_one_call_per_lens(reqs[:40], realtime=False)
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


def run_map_workload(device, n_starts: int = 300, steps=(300, 1000, 3000), seeds=(202, 303, 404, 505, 606, 707)):
    """Sec. 2.3 / Table 1: multi-start MAP, 300 starts drawn from the prior,
    on six systems drawn from the paper's simulation distribution (80x80,
    k = 2, sigma_bkg = 0.2, t_exp = 100 s, G = 1), for 300, 1000 and 3000
    Adam iterations (10^-2 -> 10^-3 linearly over the run). Per system and
    iteration count: time, the best start's distance to the global optimum in
    objective (df = f - f_opt, f the negative log posterior; f_opt the lowest
    value over every run, including 16 starts near the truth run for 3000
    iterations), the fractions of starts with df <= 1 and <= 5, and with
    reduced chi^2 <= 1.01 (the paper's marker, Sec. 2.3)."""
    import torch
    from paper_2202_07663_gb300 import abi, map as gmap
    spec = inputs.PAPER_SAMPLE_SPEC
    psf = inputs.make_psf(spec).astype(np.float32)
    dof = spec.H * spec.W - 22
    th0 = torch.from_numpy(inputs.draw_table(np.random.default_rng(13), inputs.PAPER_PRIOR_DRAW,
                                             n_starts).astype(np.float32)).to(device)
    out = {"workload": "map-multistart-80x80-k2-psf11-paper-noise", "starts": n_starts, "systems": []}
    for seed in seeds:
        rng = np.random.default_rng(seed)
        truth = inputs.draw_table(rng, inputs.PAPER_SIM, 1)[0]
        blank = np.zeros((spec.H, spec.W), np.float32)
        s0 = abi.GLSystem(blank, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
        model = s0.simulate(torch.from_numpy(truth.astype(np.float32)[None]).to(device)).cpu().numpy()[0]
        s0.close()
        image = inputs.add_noise(rng, model, spec.sigma_bkg, spec.gain_exposure).astype(np.float32)
        s = abi.GLSystem(image, psf, spec.pixel_scale, spec.k, spec.gain_exposure, sigma_bkg=spec.sigma_bkg)
        s.reserve(n_starts)
        near = torch.from_numpy(inputs.draw_perturbed(np.random.default_rng(seed + 1), truth, 16, frac=0.005)
                                .astype(np.float32)).to(device)
        gmap.MultiStartMAP(s, steps=5).run(th0[:8])   # warm-up
        f_near = gmap.MultiStartMAP(s, steps=max(steps)).run(near).objective.cpu().numpy()
        runs = []
        for k in steps:
            r = gmap.MultiStartMAP(s, steps=k).run(th0)
            _, c2 = s.loglik(r.theta, chi2=True)
            runs.append((k, r, r.objective.cpu().numpy(), c2.cpu().numpy() / dof))
        f_opt = float(min(np.nanmin(f_near), *(np.nanmin(f) for _, _, f, _ in runs)))
        rec = {"seed": seed, "f_opt": f_opt, "runs": []}
        for k, r, f, chi2nu in runs:
            df = f - f_opt
            b = int(np.nanargmin(f))
            rec["runs"].append({"iterations": k, "seconds": r.seconds, "evals_per_s": r.grad_evals / r.seconds,
                                "best_df": float(df[b]), "best_chi2nu": float(chi2nu[b]),
                                "fraction_df_le_1": float(np.mean(df <= 1)), "fraction_df_le_5": float(np.mean(df <= 5)),
                                "fraction_chi2nu_le_1.01": float(np.mean(chi2nu <= 1.01))})
        out["systems"].append(rec)
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
    out["what_it_buys"] = ("the two light amplitudes solved in closed form per call (Sec. 2.1.2): a sampler or "
                           "optimiser works in 20 parameters instead of 22, and the variance uses the observed "
                           "image, not the model; the call costs the 2 basis images, 2B convolutions and a 2x2 "
                           "solve per vector more than the plain one")
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


def run_reference(args):
    """The reference arm: the FP64 oracle timed on the host cores on the same
    workload (same stored observed image, same parameter vectors, same config
    object), each step a bounded sample of the vectors."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    workload = args.workload
    spec, truth, psf, image = load_observed(workload)
    params = workload_params(workload, 0, truth)
    B = len(params)
    nt = oracle.max_threads()
    a = (image, np.float32(spec.sigma_bkg), psf, spec.pixel_scale, spec.k, spec.gain_exposure)
    per_step = max(nt * 2, 32) if spec.H * spec.W * spec.k ** 2 <= 40000 else nt
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
        "config": dict(workload_config(workload), parallelism="single GPU" if args.gpus <= 1 else
                       "replicas (B per GPU)"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nt, "kind": "oracle",
                         "sample": "%d vectors per step of the %d-vector workload (log L + forward-mode gradient, "
                                   "FP64)" % (per_step, B)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


def small_batch_workload(device, steps: int = 200, warmup: int = 5, B: int = 50, graph: bool = True) -> dict:
    """The call the samplers make (50 chains, Table 1): per-call time of
    log L + gradient for B vectors of one 80x80 system (k = 2, 11x11 PSF,
    the paper's noise), inputs resident, CUDA events around the calls on one
    stream, issued one by one and (graph) replayed from a CUDA graph of 10
    calls."""
    import torch
    from paper_2202_07663_gb300 import abi
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
    st = torch.cuda.Stream(device)
    a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(st):
        for _ in range(warmup):
            s.loglik_grad(p, out=(ll, g, None))
        st.synchronize()
        a.record(st)
        for _ in range(steps):
            s.loglik_grad(p, out=(ll, g, None))
        e.record(st)
        st.synchronize()
        eager_us = 1e3 * a.elapsed_time(e) / steps
        graph_us = None
        if graph:
            gr = torch.cuda.CUDAGraph()
            with torch.cuda.graph(gr, stream=st):
                for _ in range(10):
                    s.loglik_grad(p, out=(ll, g, None))
            for _ in range(3):
                gr.replay()
            st.synchronize()
            reps = max(1, steps // 10)
            a.record(st)
            for _ in range(reps):
                gr.replay()
            e.record(st)
            st.synchronize()
            graph_us = 1e3 * a.elapsed_time(e) / (10 * reps)
    finite = bool(torch.isfinite(ll).all().item() and torch.isfinite(g).all().item())
    s.close()
    out = {"workload": "small-batch-80x80-k2-psf11-B50", "B": B, "steps": steps,
           "us_per_call": eager_us, "evals_per_s": B / (eager_us * 1e-6), "finite": finite}
    if graph_us is not None:
        out.update(graph_us_per_call=graph_us, graph_evals_per_s=B / (graph_us * 1e-6))
    return out


def run_small_batch(args, B: int = 50):
    """--small-batch: the samplers' call alone (one JSON line)."""
    import torch
    from paper_2202_07663_gb300 import build
    build.build()
    print(json.dumps(small_batch_workload(torch.device("cuda", 0), args.steps, args.warmup, B, graph=False)))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 400 for the 60x60 workload, 20 for the 200x200 stress workload)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=[inputs.MULTISTART, inputs.STRESS],
                    help="the metric's workload (default) or the 200x200, k = 4, B = 16384 stress workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the workloads reported beside the metric (stress, HMC, serving, MAP, ...)")
    ap.add_argument("--small-batch", action="store_true",
                    help="only the sampler-sized call: B = 50 vectors of an 80x80, k = 2, 11x11-PSF system")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.steps is None:
        args.steps = 20 if args.workload == inputs.STRESS else 400
    if args.impl == "reference":
        return run_reference(args)
    if args.small_batch:
        return run_small_batch(args)

    import torch
    import torch.distributed as dist
    from paper_2202_07663_gb300 import build

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
    peaks = measured_peaks()
    cpu = not args.no_cpu_baseline
    out = measure(args.workload, device, rank, world, args.steps, args.warmup, cpu, peaks)
    if world > 1:
        dist.barrier()
    if rank != 0:
        dist.destroy_process_group()
        return 0
    if world == 1 and not args.no_workloads and args.workload == WORKLOAD:
        out["workloads"] = {
            "stress": measure(inputs.STRESS, device, 0, 1, 20, 3, cpu, peaks),
            "hmc": run_hmc_workload(device, cpu=cpu), "serving": run_serving_workload(device),
            "map": run_map_workload(device), "hmc_paper": run_hmc_paper_workload(device),
            "variant": run_variant_workload(device), "pipeline": run_pipeline_workload(device),
            "small_batch": small_batch_workload(device)}
    out["peaks"] = peaks
    print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
