"""The modelling pipeline of arXiv:2202.07663 (Sec. 2.6, Table 1) for one lens system:

1. multi-start MAP: n_MAP = 300 starts drawn from the prior, K_MAP = 300 Adam
   iterations (10^-2 -> 10^-3 linear); the best start's point is the mode;
2. full-rank VI: mu = the MAP point, Sigma = 10^-6 I, K_VI = 1000 iterations of
   n_VI = 500 draws (0 -> 10^-3 quadratic over 500);
3. HMC: n_HMC = 50 chains drawn from the VI posterior, mass Sigma_VI^-1,
   eps0 = 0.3, L0 = 5, step size and trajectory length adapted over the
   first 80% of n_burn = 250, then n_sample = 750.

``preconditioner="laplace"`` replaces the VI covariance (for HMC's mass and
the chains' start) by the Laplace covariance of log p~(z) at the VI mean
(see ``hmc.laplace_covariance``). It is taken at the VI mean, not at the MAP
point: when the best start ends at a local mode (the paper's 300 iterations
do not always reach the global one), the Hessian there describes the wrong
basin and the chains stay in it, while VI has already moved its mean toward
the posterior mass.
Every stage runs in the library's kernels; this module only sequences them.

With a process group (one GPU per process, ``distributed``) the starts, the
VI draws and the chains are split over the processes; every process ends
with the same MAP point, variational posterior and all chains' samples.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import abi, distributed, hmc, map as gmap, vi

NPARAM = abi.NPARAM


@dataclasses.dataclass
class PipelineResult:
    theta_map: np.ndarray            # [22] best MAP point (physical)
    map_objective: float
    vi_mu: torch.Tensor              # [22] unconstrained
    vi_cov: torch.Tensor             # [22, 22]
    samples: hmc.PosteriorSamples
    seconds: dict                    # per stage and total
    grad_evals: dict


def model_system(system: abi.GLSystem, theta_starts: torch.Tensor, prior=None, map_steps: int = 300,
                 vi_steps: int = 1000, vi_draws: int = 500, chains: int = 50, n_burn: int = 250,
                 n_samples: int = 750, preconditioner: str = "vi", seed: int = 0,
                 vi_estimator: str = "pathwise", group=None) -> PipelineResult:
    """Run MAP -> VI -> HMC on ``system`` from the given multi-start points
    (physical, [n_MAP, 22]; the paper draws them from the prior; with a
    process group every process passes all of them)."""
    if preconditioner not in ("vi", "laplace"):
        raise ValueError("preconditioner must be 'vi' or 'laplace'")
    dev = theta_starts.device
    prior = gmap.PAPER_PRIOR if prior is None else prior
    rank, size = distributed.world(group)
    n_map = theta_starts.shape[0]
    if min(n_map, vi_draws, chains) < size:
        raise ValueError("fewer starts, draws or chains than processes")
    lo, hi = distributed.shard(n_map, rank, size)
    local = [hi - lo] + [b - a for a, b in (distributed.shard(n, rank, size) for n in (vi_draws, chains))]
    system.reserve(max(local + [2 * NPARAM]))
    sec, evals = {}, {}
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()

    m = gmap.MultiStartMAP(system, prior=prior, steps=map_steps).run(theta_starts[lo:hi])
    _, map_objective, (theta_map, z_map) = distributed.best_row(m.objective, [m.theta, m.z], group)
    torch.cuda.synchronize(dev)
    t1 = time.perf_counter()
    sec["map"], evals["map"] = t1 - t0, m.grad_evals

    post = hmc.PosteriorTarget(system, prior)
    r = vi.FullRankVI(post, n=vi_draws, steps=vi_steps, estimator=vi_estimator, seed=seed, group=group).run(z_map)
    torch.cuda.synchronize(dev)
    t2 = time.perf_counter()
    sec["vi"], evals["vi"] = t2 - t1, r.evals

    if preconditioner == "vi":
        mu, cov = r.mu, r.cov
    else:
        mu, cov = r.mu, hmc.laplace_covariance(post, r.mu)
        evals["laplace"] = 2 * NPARAM
    torch.cuda.synchronize(dev)
    t3 = time.perf_counter()
    sec["preconditioner"] = t3 - t2
    ps = hmc.sample_posterior(system, mu, cov, chains=chains, n_burn=n_burn, n_samples=n_samples, seed=seed + 7,
                              prior=prior, group=group)
    torch.cuda.synchronize(dev)
    t4 = time.perf_counter()
    sec["hmc"], evals["hmc"] = t4 - t3, ps.run.grad_evals
    sec["total"] = t4 - t0
    return PipelineResult(theta_map.cpu().numpy().astype(np.float64), map_objective, r.mu, r.cov, ps, sec, evals)
