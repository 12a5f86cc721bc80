"""Autograd wrapper of the lens log-likelihood and an HMC driver on top of it.

``LogLik`` is a ``torch.autograd.Function``: its forward runs the CUDA
log-likelihood (with the hand-written adjoint when the input requires a
gradient; the adjoint recomputes every ray, none is stored) and its backward
scales the stashed gradient by the incoming one.

``HMC`` runs many chains of Hamiltonian Monte Carlo (arXiv:2202.07663,
Sec. 2.5) on the log-likelihood as log density: leapfrog updates and the FP64
Hamiltonian/accept step are the library's CUDA kernels (``gl_hmc_*``); the
random numbers (momenta, accept uniforms) come from a seeded torch generator
and are passed in. The mass matrix is diagonal.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Optional, Tuple

import torch

from . import abi

NPARAM = abi.NPARAM


class LogLik(torch.autograd.Function):
    """log L(params) for a resident ``abi.GLSystem``; params [B, 22] (float32 or float64)."""

    @staticmethod
    def forward(ctx, params, system):
        p32 = params.detach().to(torch.float32).contiguous()
        if params.requires_grad:
            ll, g = system.loglik_grad(p32)
            ctx.save_for_backward(g)
        else:
            ll = system.loglik(p32)
        ctx.in_dtype = params.dtype
        return ll.to(params.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return (grad_out.to(g.dtype)[:, None] * g).to(ctx.in_dtype), None


def loglik(params, system):
    return LogLik.apply(params, system)


def laplace_inv_mass(system, q: torch.Tensor, rel_step: float = 1e-3, floor: float = 1e-12) -> torch.Tensor:
    """Diagonal inverse mass from the Hessian diagonal of log L at q [22]:
    central differences of the gradient, 44 vectors in one call; 1/|H_ii|."""
    q = q.to(torch.float64)
    h = rel_step * torch.clamp(q.abs(), min=1e-2)
    eye = torch.eye(NPARAM, dtype=torch.float64, device=q.device)
    pts = torch.cat([q[None] + eye * h[:, None], q[None] - eye * h[:, None]], 0).to(torch.float32).contiguous()
    _, g = system.loglik_grad(pts)
    hdiag = (g[:NPARAM].diagonal() - g[NPARAM:].diagonal()) / (2 * h)
    return 1.0 / torch.clamp(hdiag.abs(), min=floor)


@dataclasses.dataclass
class HMCStats:
    iterations: int
    leapfrog_steps: int
    grad_evals: int
    acceptance: float
    seconds: float

    @property
    def evals_per_s(self) -> float:
        return self.grad_evals / self.seconds


class HMC:
    """B chains of HMC with diagonal mass. ``logp_grad(q32) -> (logp f64 [B], grad f64 [B, d])``
    defaults to the lens log-likelihood of ``system``; the leapfrog and accept
    steps run in the library's kernels."""

    def __init__(self, q0: torch.Tensor, inv_mass: torch.Tensor, step_size: float, n_leapfrog: int,
                 system=None, logp_grad: Optional[Callable] = None, seed: int = 0):
        self.q = q0.to(torch.float64).contiguous().clone()
        self.B, self.d = self.q.shape
        self.dev = self.q.device
        self.inv_mass = inv_mass.to(torch.float64).to(self.dev).contiguous()
        self.eps = float(step_size)
        self.L = int(n_leapfrog)
        self.system = system
        self.logp_grad = logp_grad or self._lens_logp_grad
        self.gen = torch.Generator(device=self.dev)
        self.gen.manual_seed(seed)
        B, d = self.B, self.d
        f64 = dict(dtype=torch.float64, device=self.dev)
        self.p = torch.empty(B, d, **f64)
        self.p0 = torch.empty(B, d, **f64)
        self.qp = torch.empty(B, d, **f64)
        self.gp = torch.empty(B, d, **f64)
        self.lp_new = torch.empty(B, **f64)
        self.q32 = torch.empty(B, d, dtype=torch.float32, device=self.dev)
        self.accepted = torch.zeros(B, dtype=torch.int32, device=self.dev)
        self.logp, self.grad = self.logp_grad(self.q.to(torch.float32).contiguous())
        self.logp = self.logp.clone()
        self.grad = self.grad.clone()
        self.n_accepted = 0
        self.n_proposed = 0
        self.grad_evals = 0

    def _lens_logp_grad(self, q32):
        return self.system.loglik_grad(q32)

    def _lens_into(self, q32):
        self.system.loglik_grad(q32, out=(self.lp_new, self.gp, None))

    def step(self) -> None:
        """One HMC iteration (L leapfrog steps + FP64 accept) for all chains."""
        stream = torch.cuda.current_stream(self.dev).cuda_stream
        B, d = self.B, self.d
        torch.randn(B, d, generator=self.gen, dtype=torch.float64, device=self.dev, out=self.p0)
        self.p0.mul_(torch.rsqrt(self.inv_mass))
        self.p.copy_(self.p0)
        self.qp.copy_(self.q)
        self.gp.copy_(self.grad)
        for l in range(self.L):
            abi.gl_hmc_leapfrog(B, d, self.qp.data_ptr(), self.p.data_ptr(), self.gp.data_ptr(),
                                self.inv_mass.data_ptr(), self.eps, 0.5 if l == 0 else 1.0, self.q32.data_ptr(),
                                stream)
            if self.system is not None and self.logp_grad == self._lens_logp_grad:
                self._lens_into(self.q32)
            else:
                lp, g = self.logp_grad(self.q32)
                self.lp_new.copy_(lp)
                self.gp.copy_(g)
        log_u = torch.rand(B, generator=self.gen, dtype=torch.float64, device=self.dev).log_()
        abi.gl_hmc_finish(B, d, self.p0.data_ptr(), self.logp.data_ptr(), self.p.data_ptr(), self.gp.data_ptr(),
                          self.lp_new.data_ptr(), self.qp.data_ptr(), self.inv_mass.data_ptr(), log_u.data_ptr(),
                          self.eps, self.q.data_ptr(), self.logp.data_ptr(), self.grad.data_ptr(),
                          self.accepted.data_ptr(), stream)
        self.grad_evals += B * self.L
        self.n_proposed += B

    def run(self, n_iter: int) -> HMCStats:
        import time
        torch.cuda.synchronize(self.dev)
        acc = torch.zeros((), dtype=torch.int64, device=self.dev)
        e0 = self.grad_evals
        t0 = time.perf_counter()
        for _ in range(n_iter):
            self.step()
            acc += self.accepted.sum()
        torch.cuda.synchronize(self.dev)
        dt = time.perf_counter() - t0
        a = int(acc.item())
        self.n_accepted += a
        return HMCStats(n_iter, n_iter * self.L, self.grad_evals - e0, a / max(1, n_iter * self.B), dt)

    def tune_step_size(self, target: float = 0.65, rounds: int = 6, iters: int = 3) -> float:
        """Crude step-size search toward a target acceptance (geometric updates)."""
        for _ in range(rounds):
            st = self.run(iters)
            self.eps *= math.exp(1.5 * (st.acceptance - target))
        return self.eps
