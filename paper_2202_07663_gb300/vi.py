"""Full-rank variational inference on the GPU (arXiv:2202.07663, Sec. 2.4, Table 1).

q = N(mu, L L^T) over the unconstrained parameters, L through the Cholesky
bijector (``gl_vi_*``). Each iteration draws eps ~ N(0, I) [n, d] from a seeded
torch generator, maps the draws (``gl_vi_sample``), evaluates the target's log
density (and its gradient for the pathwise estimator), and takes one Adam step
on the estimated ELBO gradient (``gl_vi_step``). Table 1: n = 500 draws,
1000 iterations, learning rate 0 -> 1e-3 quadratic over 500 iterations,
mu = the MAP point, Sigma = 1e-6 I at the start.

Targets are the ones ``hmc`` defines (``PosteriorTarget`` for a lens system,
``FunctionTarget`` for tests): ``target(z64, z32, logp_out, grad_out_or_None)``.

With a process group the n draws of each iteration are split over the
processes (``distributed``): each evaluates its rows, reduces them to moment
sums (``gl_vi_moments``), and every process applies the same step from all
processes' sums (``gl_vi_apply``); ``VIResult.evals`` counts this process's
evaluations.
"""
from __future__ import annotations

import dataclasses
import math
import time
from typing import Optional

import torch

from . import abi, distributed

SCORE, PATHWISE = 0, 1
ADAM = (0.9, 0.999, 1e-8)


def quadratic_warmup(t: int, peak: float = 1e-3, steps: int = 500) -> float:
    """0 -> peak over `steps` iterations as a degree-2 polynomial (t from 0)."""
    frac = min(t, steps) / steps
    return peak - peak * (1.0 - frac) ** 2


def n_params(d: int) -> int:
    return d + d * (d + 1) // 2


def pack(mu: torch.Tensor, L: torch.Tensor) -> torch.Tensor:
    """(mu, lower-triangular L with positive diagonal) -> phi (float64)."""
    d = mu.shape[0]
    rows = []
    for i in range(d):
        r = L[i, : i + 1].clone()
        r[i] = torch.log(r[i])
        rows.append(r)
    return torch.cat([mu.to(torch.float64)] + [r.to(torch.float64) for r in rows]).contiguous()


def unpack(phi: torch.Tensor, d: int):
    """phi -> (mu [d], L [d, d])."""
    mu = phi[:d].clone()
    L = torch.zeros(d, d, dtype=torch.float64, device=phi.device)
    k = d
    for i in range(d):
        L[i, : i + 1] = phi[k:k + i + 1]
        L[i, i] = torch.exp(phi[k + i])
        k += i + 1
    return mu, L


@dataclasses.dataclass
class VIResult:
    phi: torch.Tensor            # [P] float64
    mu: torch.Tensor             # [d]
    L: torch.Tensor              # [d, d] lower triangular
    loss: torch.Tensor           # [steps] ELBO-loss estimates, float64
    seconds: float
    evals: int

    @property
    def cov(self) -> torch.Tensor:
        return self.L @ self.L.T


class FullRankVI:
    """Stochastic VI with Adam; ``estimator`` 'pathwise' (reparameterised) or 'score' (Eq. elbo-grad)."""

    def __init__(self, target, d: int = abi.NPARAM, n: int = 500, steps: int = 1000, lr_peak: float = 1e-3,
                 warmup: int = 500, estimator: str = "pathwise", seed: int = 0, lr_fn=None, group=None):
        if estimator not in ("pathwise", "score"):
            raise ValueError("estimator must be 'pathwise' or 'score'")
        self.target = target
        self.d, self.n, self.steps = int(d), int(n), int(steps)
        self.lr_fn = lr_fn if lr_fn is not None else (lambda t: quadratic_warmup(t, lr_peak, warmup))
        self.est = PATHWISE if estimator == "pathwise" else SCORE
        self.seed = seed
        self.group = group

    def run(self, mu0: torch.Tensor, sigma0: float = 1e-6, phi0: Optional[torch.Tensor] = None) -> VIResult:
        dev = mu0.device
        d, n = self.d, self.n
        P = n_params(d)
        rank, size = distributed.world(self.group)
        lo, hi = distributed.shard(n, rank, size)
        nl = hi - lo                                  # this process's draws
        lib = abi.lib_handle()
        st = torch.cuda.current_stream(dev).cuda_stream
        f64 = dict(dtype=torch.float64, device=dev)
        if phi0 is None:
            phi = pack(mu0.to(**f64), math.sqrt(sigma0) * torch.eye(d, **f64))
        else:
            phi = phi0.to(**f64).clone().contiguous()
        m = torch.zeros(P, **f64)
        v = torch.zeros(P, **f64)
        g = torch.empty(P, **f64)
        loss = torch.empty(self.steps, **f64)
        eps_all = torch.empty(n, d, **f64)
        eps = eps_all[lo:hi]
        z = torch.empty(nl, d, **f64)
        z32 = torch.empty(nl, d, dtype=torch.float32, device=dev)
        logp = torch.empty(nl, **f64)
        gz = torch.empty(nl, d, **f64) if self.est == PATHWISE else None
        ws = torch.empty(max(1, lib.gl_vi_workspace_bytes(max(1, nl), d)), dtype=torch.uint8, device=dev)
        sums = torch.zeros(1 + P, **f64)
        gen = torch.Generator(device=dev)
        gen.manual_seed(self.seed)
        need32 = getattr(self.target, "needs_q32", True)
        b1, b2, ae = ADAM
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for t in range(self.steps):
            torch.randn(n, d, generator=gen, out=eps_all)   # every process draws all n, keeps its rows
            gzp = gz.data_ptr() if gz is not None else None
            if nl:
                abi._check(lib.gl_vi_sample(nl, d, eps.data_ptr(), phi.data_ptr(), None, z.data_ptr(),
                                            z32.data_ptr() if need32 else None, st), "gl_vi_sample")
                self.target(z, z32, logp, gz)
            if size == 1:
                abi._check(lib.gl_vi_step(n, d, eps.data_ptr(), logp.data_ptr(), gzp, self.est, phi.data_ptr(),
                                          m.data_ptr(), v.data_ptr(), t + 1, self.lr_fn(t), b1, b2, ae, g.data_ptr(),
                                          loss[t:].data_ptr(), ws.data_ptr(), st), "gl_vi_step")
                continue
            if nl:
                abi._check(lib.gl_vi_moments(nl, d, eps.data_ptr(), logp.data_ptr(), gzp, self.est, phi.data_ptr(),
                                             ws.data_ptr(), sums.data_ptr(), st), "gl_vi_moments")
            parts = distributed.gather_parts(sums, self.group)
            abi._check(lib.gl_vi_apply(n, d, size, parts.data_ptr(), self.est, phi.data_ptr(), m.data_ptr(),
                                       v.data_ptr(), t + 1, self.lr_fn(t), b1, b2, ae, g.data_ptr(),
                                       loss[t:].data_ptr(), st), "gl_vi_apply")
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        mu, L = unpack(phi, d)
        return VIResult(phi, mu, L, loss, dt, nl * self.steps)
