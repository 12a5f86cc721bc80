"""Autograd wrapper of the lens log-likelihood and an HMC driver on top of it.

``LogLik`` is a ``torch.autograd.Function``: its forward runs the CUDA
log-likelihood (with the hand-written adjoint when the input requires a
gradient; the adjoint recomputes every ray, none is stored) and its backward
scales the stashed gradient by the incoming one.

``HMC`` runs many chains of Hamiltonian Monte Carlo (arXiv:2202.07663,
Sec. 2.5): leapfrog updates and the FP64 Hamiltonian/accept step are the
library's CUDA kernels (``gl_hmc_*``); the random numbers (momenta, accept
uniforms) come from a seeded torch generator and are passed in. The mass
matrix is diagonal. Targets:

- ``LensTarget``: log L in the physical parameters (the HMC throughput workload);
- ``AutogradTarget``: the same log L through ``LogLik`` and ``torch.autograd``;
- ``PosteriorTarget``: the posterior of the unconstrained parameters,
  log p~(z) = log L(g(z)) + log p(g(z)) + log|J| (Eq. reparam-post), through
  ``gl_map_transform`` and ``gl_posterior_grad`` — the paper's sampler;
- ``FunctionTarget``: any ``logp_grad(q32) -> (logp, grad)`` (tests).

``run_adaptive`` adapts, during the first 80% of burn-in (Sec. 2.5), the
step size by dual averaging (Hoffman & Gelman 2014) toward a target
acceptance probability (0.75) and, optionally, the trajectory length by the
ChEES criterion (Hoffman, Radul & Sountsov 2021; ``gl_hmc_chees``), with
jittered leapfrog counts; then fixes both.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import time
from typing import Callable, Optional

import numpy as np
import torch

from . import abi, distributed

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


# ------------------------------------------------------------- targets ----

class LensTarget:
    """log L in the physical parameters; consumes the leapfrog's FP32 positions."""
    needs_q32 = True

    def __init__(self, system):
        self.system = system

    def __call__(self, q64, q32, lp_out, g_out):
        self.system.loglik_grad(q32, out=(lp_out, g_out, None))


class AutogradTarget:
    """log L in the physical parameters through ``LogLik`` and
    ``torch.autograd.grad``: the chain's FP64 positions are the leaf, the
    Function's forward runs the likelihood and the adjoint, its backward
    scales the stashed gradient. The same numbers as ``LensTarget`` (which
    calls the library directly), plus autograd's bookkeeping."""
    needs_q32 = False

    def __init__(self, system):
        self.system = system

    def __call__(self, q64, q32, lp_out, g_out):
        q = q64.detach().requires_grad_(g_out is not None)
        with torch.enable_grad():
            ll = LogLik.apply(q, self.system)
            if g_out is not None:
                (g,) = torch.autograd.grad(ll.sum(), q)
                g_out.copy_(g)
        lp_out.copy_(ll.detach())


class PosteriorTarget:
    """log p~(z) of the unconstrained parameters (Sec. 2.2) for one system."""
    needs_q32 = False

    def __init__(self, system, prior=None):
        from . import map as gmap
        self.system = system
        self.prior = gmap.prior_table(prior if prior is not None else gmap.PAPER_PRIOR)
        self._buf = {}   # per batch size, kept: captured graphs hold their pointers

    def __call__(self, q64, q32, lp_out, g_out):
        B = q64.shape[0]
        if B not in self._buf:
            dev = q64.device
            self._buf[B] = (torch.empty(B, NPARAM, dtype=torch.float32, device=dev),
                            torch.empty(B, dtype=torch.float64, device=dev),
                            torch.empty(B, NPARAM, dtype=torch.float64, device=dev))
        th, ll, gt = self._buf[B]
        lib = abi.lib_handle()
        st = torch.cuda.current_stream(q64.device).cuda_stream
        pp = ctypes.addressof(self.prior)
        abi._check(lib.gl_map_transform(B, q64.data_ptr(), pp, th.data_ptr(), st), "gl_map_transform")
        if g_out is None:   # log density only (no adjoint pass)
            self.system.loglik(th, out=ll)
            abi._check(lib.gl_posterior_grad(B, q64.data_ptr(), ll.data_ptr(), None, pp, lp_out.data_ptr(), None, st),
                       "gl_posterior_grad")
            return
        self.system.loglik_grad(th, out=(ll, gt, None))
        abi._check(lib.gl_posterior_grad(B, q64.data_ptr(), ll.data_ptr(), gt.data_ptr(), pp, lp_out.data_ptr(),
                                         g_out.data_ptr(), st), "gl_posterior_grad")


class FunctionTarget:
    """Wraps ``logp_grad(q32) -> (logp float64 [B], grad float64 [B, d])``."""
    needs_q32 = True

    def __init__(self, fn: Callable):
        self.fn = fn

    def __call__(self, q64, q32, lp_out, g_out):
        lp, g = self.fn(q32)
        lp_out.copy_(lp)
        if g_out is not None:
            g_out.copy_(g)


class WhitenedTarget:
    """A target seen through z = mu + L x (Sigma = L L^T): HMC with identity
    mass on x is HMC with mass Sigma^-1 on z, the paper's preconditioning
    (Sec. 2.5). log p is unchanged (constant Jacobian); grad_x = L^T grad_z."""
    needs_q32 = False

    def __init__(self, inner, mu: torch.Tensor, L: torch.Tensor):
        self.inner = inner
        self.mu = mu.to(torch.float64).contiguous()
        self.L = torch.tril(L.to(torch.float64)).contiguous()
        self.d = self.mu.shape[0]
        self._buf = {}   # per batch size, kept: captured graphs and the chained steps hold their pointers

    def to_z(self, x: torch.Tensor) -> torch.Tensor:
        xc = x.to(torch.float64).contiguous()
        z = torch.empty_like(xc)
        abi.gl_hmc_affine(xc.shape[0], self.d, xc.data_ptr(), self.mu.data_ptr(), self.L.data_ptr(), z.data_ptr(),
                          None, torch.cuda.current_stream(x.device).cuda_stream)
        return z

    def _buffers(self, B, dev):
        if B not in self._buf:
            d = self.d
            self._buf[B] = (torch.empty(B, d, dtype=torch.float64, device=dev),
                            torch.empty(B, d, dtype=torch.float32, device=dev),
                            torch.empty(B, d, dtype=torch.float64, device=dev),
                            torch.empty(B, dtype=torch.float64, device=dev))
        return self._buf[B]

    @property
    def lens_posterior(self) -> bool:
        """Whether this is the whitened lens posterior (the fused launches apply)."""
        return isinstance(self.inner, PosteriorTarget) and self.d == NPARAM

    def leapfrog_first(self, x, p, grad, inv_mass, eps, eps_dev, kick):
        """The first leapfrog step of a trajectory (lens posterior only):
        gl_hmc_leapfrog_whitened on (x, p) with the gradient ``grad`` (the
        update, whitening and bijectors in one launch), then log L and its
        gradient at the new point, kept in this target's buffers."""
        B = x.shape[0]
        z, z32, gz, ll = self._buffers(B, x.device)
        st = torch.cuda.current_stream(x.device).cuda_stream
        lib = abi.lib_handle()
        abi._check(lib.gl_hmc_leapfrog_whitened(B, x.data_ptr(), p.data_ptr(), grad.data_ptr(), inv_mass.data_ptr(),
                                                float(eps), eps_dev.data_ptr() if eps_dev is not None else None,
                                                float(kick), self.mu.data_ptr(), self.L.data_ptr(),
                                                ctypes.addressof(self.inner.prior), z.data_ptr(), z32.data_ptr(), st),
                   "gl_hmc_leapfrog_whitened")
        self.inner.system.loglik_grad(z32, out=(ll, gz, None))

    def leapfrog_next(self, x, p, inv_mass, eps, eps_dev, kick):
        """A later leapfrog step: the posterior gradient at the point of the
        last evaluation, the update and the transform in one launch
        (gl_hmc_leapfrog_whitened_chain), then log L and its gradient at
        the new point, in this target's buffers."""
        B = x.shape[0]
        z, z32, gz, ll = self._buffers(B, x.device)
        st = torch.cuda.current_stream(x.device).cuda_stream
        lib = abi.lib_handle()
        abi._check(lib.gl_hmc_leapfrog_whitened_chain(B, x.data_ptr(), p.data_ptr(), z.data_ptr(), gz.data_ptr(),
                                                      inv_mass.data_ptr(), float(eps),
                                                      eps_dev.data_ptr() if eps_dev is not None else None,
                                                      float(kick), self.mu.data_ptr(), self.L.data_ptr(),
                                                      ctypes.addressof(self.inner.prior), z32.data_ptr(), st),
                   "gl_hmc_leapfrog_whitened_chain")
        self.inner.system.loglik_grad(z32, out=(ll, gz, None))

    def posterior_at_last(self, B, dev, lp_out, g_out):
        """log p~ and its gradient in x at the point of the last evaluation."""
        z, _, gz, ll = self._buffers(B, dev)
        abi._check(abi.lib_handle().gl_posterior_whitened_grad(
            B, z.data_ptr(), ll.data_ptr(), gz.data_ptr(), self.L.data_ptr(), ctypes.addressof(self.inner.prior),
            lp_out.data_ptr(), g_out.data_ptr(), torch.cuda.current_stream(dev).cuda_stream),
            "gl_posterior_whitened_grad")

    def __call__(self, q64, q32, lp_out, g_out):
        B, d = q64.shape
        z, z32, gz, ll = self._buffers(B, q64.device)
        st = torch.cuda.current_stream(q64.device).cuda_stream
        if self.lens_posterior:
            # the lens posterior: whitening and bijectors in one launch, the
            # posterior gradient and its pull-back in another (same sums)
            lib = abi.lib_handle()
            pp = ctypes.addressof(self.inner.prior)
            abi._check(lib.gl_posterior_whitened_transform(B, q64.data_ptr(), self.mu.data_ptr(), self.L.data_ptr(),
                                                           pp, z.data_ptr(), z32.data_ptr(), st),
                       "gl_posterior_whitened_transform")
            if g_out is None:
                self.inner.system.loglik(z32, out=ll)
            else:
                self.inner.system.loglik_grad(z32, out=(ll, gz, None))
            abi._check(lib.gl_posterior_whitened_grad(B, z.data_ptr(), ll.data_ptr(),
                                                      gz.data_ptr() if g_out is not None else None,
                                                      self.L.data_ptr(), pp, lp_out.data_ptr(),
                                                      g_out.data_ptr() if g_out is not None else None, st),
                       "gl_posterior_whitened_grad")
            return
        abi.gl_hmc_affine(B, d, q64.data_ptr(), self.mu.data_ptr(), self.L.data_ptr(), z.data_ptr(),
                          z32.data_ptr() if self.inner.needs_q32 else None, st)
        self.inner(z, z32, lp_out, gz if g_out is not None else None)
        if g_out is not None:
            abi.gl_hmc_affine_pullback(B, d, gz.data_ptr(), self.L.data_ptr(), g_out.data_ptr(), st)


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


def laplace_inv_mass_target(target, q: torch.Tensor, step: float = 1e-4, floor: float = 1e-12) -> torch.Tensor:
    """Diagonal inverse mass 1/|d2 logp/dq2| of any target at q [d] (central
    differences of its gradient, 2d points in one evaluation)."""
    q = q.to(torch.float64)
    d = q.shape[0]
    eye = torch.eye(d, dtype=torch.float64, device=q.device) * step
    pts = torch.cat([q[None] + eye, q[None] - eye], 0).contiguous()
    lp = torch.empty(2 * d, dtype=torch.float64, device=q.device)
    g = torch.empty(2 * d, d, dtype=torch.float64, device=q.device)
    target(pts, pts.to(torch.float32).contiguous(), lp, g)
    hdiag = (g[:d].diagonal() - g[d:].diagonal()) / (2 * step)
    return 1.0 / torch.clamp(hdiag.abs(), min=floor)


def laplace_covariance(target, q: torch.Tensor, step: float = 1e-4) -> torch.Tensor:
    """Covariance (-H)^-1 of a target at q [d] (a mode): the Hessian by central
    differences of the gradient (2d points, one evaluation), symmetrised; a
    non-positive-definite Hessian falls back to its diagonal. Setup of the
    preconditioner when no variational covariance is at hand; float64 [d, d]."""
    q = q.to(torch.float64)
    d = q.shape[0]
    eye = torch.eye(d, dtype=torch.float64, device=q.device) * step
    pts = torch.cat([q[None] + eye, q[None] - eye], 0).contiguous()
    lp = torch.empty(2 * d, dtype=torch.float64, device=q.device)
    g = torch.empty(2 * d, d, dtype=torch.float64, device=q.device)
    target(pts, pts.to(torch.float32).contiguous(), lp, g)
    Hm = ((g[:d] - g[d:]) / (2 * step)).cpu().numpy()
    Hm = -0.5 * (Hm + Hm.T)
    try:
        np.linalg.cholesky(Hm)
        C = np.linalg.inv(Hm)
    except np.linalg.LinAlgError:
        C = np.diag(1.0 / np.maximum(np.abs(np.diag(Hm)), 1e-12))
    return torch.from_numpy(0.5 * (C + C.T)).to(q.device)


# ------------------------------------------------------------ sampler -----

class DualAveraging:
    """Step-size adaptation of Hoffman & Gelman (2014), Sec. 3.2.1."""

    def __init__(self, eps0: float, target: float = 0.75, gamma: float = 0.05, t0: float = 10.0, kappa: float = 0.75):
        self.mu = math.log(10.0 * eps0)
        self.target, self.gamma, self.t0, self.kappa = target, gamma, t0, kappa
        self.hbar = 0.0
        self.log_eps_bar = 0.0
        self.m = 0

    def update(self, accept_prob: float) -> float:
        self.m += 1
        w = 1.0 / (self.m + self.t0)
        self.hbar = (1.0 - w) * self.hbar + w * (self.target - accept_prob)
        log_eps = self.mu - math.sqrt(self.m) / self.gamma * self.hbar
        eta = self.m ** (-self.kappa)
        self.log_eps_bar = eta * log_eps + (1.0 - eta) * self.log_eps_bar
        return math.exp(log_eps)

    def final(self) -> float:
        return math.exp(self.log_eps_bar)


def van_der_corput(m: int, base: int = 2) -> float:
    """Radical inverse of m >= 1: the jitter sequence 1/2, 1/4, 3/4, 1/8, ..."""
    out, f = 0.0, 1.0 / base
    while m > 0:
        m, r = divmod(m, base)
        out += r * f
        f /= base
    return out


class TrajectoryAdam:
    """Trajectory-length adaptation of Hoffman, Radul & Sountsov (2021):
    Adam ascent on log T along the ChEES gradient, beta1 = 0, beta2 = 0.95,
    rate 0.025; T capped at t_max."""

    def __init__(self, T0: float, lr: float = 0.025, beta2: float = 0.95, eps: float = 1e-8,
                 t_max: float = float("inf")):
        self.log_t = math.log(T0)
        self.lr, self.b2, self.eps, self.log_t_max = lr, beta2, eps, math.log(t_max)
        self.v = 0.0
        self.n = 0

    def update(self, grad: float) -> float:
        if math.isfinite(grad):
            self.n += 1
            self.v = self.b2 * self.v + (1.0 - self.b2) * grad * grad
            vhat = self.v / (1.0 - self.b2 ** self.n)
            self.log_t = min(self.log_t + self.lr * grad / (math.sqrt(vhat) + self.eps), self.log_t_max)
        return math.exp(self.log_t)


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


@dataclasses.dataclass
class AdaptiveRun:
    samples: torch.Tensor        # [n_samples, chains, d] float64 (positions of the target)
    step_size: float
    accept_burn: float
    accept_samples: float
    seconds: float
    grad_evals: int
    trajectory_length: float = float("nan")   # adapted T (jittered runs), else eps * L
    mean_leapfrog: float = float("nan")       # leapfrog steps per iteration while sampling


class HMC:
    """B chains of HMC with diagonal mass on a target (default: the lens log L of ``system``)."""

    def __init__(self, q0: torch.Tensor, inv_mass: torch.Tensor, step_size: float, n_leapfrog: int,
                 system=None, logp_grad: Optional[Callable] = None, target=None, seed: int = 0,
                 graphs: bool = False, group=None, fuse: bool = True, graph_chunk: int = 8):
        # with a process group, q0 holds every chain and this process runs its
        # shard of them; random draws are made for all chains and sliced
        self.group = group
        rank, size = distributed.world(group)
        self.B_total = q0.shape[0]
        if self.B_total < size:
            raise ValueError("fewer chains than processes")
        self.rows = distributed.shard(self.B_total, rank, size)
        self.row_counts = distributed.counts(self.B_total, size)
        self.size = size
        self.q = q0[self.rows[0]:self.rows[1]].to(torch.float64).contiguous().clone()
        self.B, self.d = self.q.shape
        self.dev = self.q.device
        self.inv_mass = inv_mass.to(torch.float64).to(self.dev).contiguous()
        self.eps = float(step_size)
        self.L = int(n_leapfrog)
        if target is None:
            target = FunctionTarget(logp_grad) if logp_grad is not None else LensTarget(system)
        self.target = target
        # the whitened lens posterior takes the leapfrog update in its first launch
        self.fused = bool(fuse) and isinstance(target, WhitenedTarget) and target.lens_posterior
        self.gen = torch.Generator(device=self.dev)
        self.gen.manual_seed(seed)
        B, d = self.B, self.d
        f64 = dict(dtype=torch.float64, device=self.dev)
        self.p = torch.empty(B, d, **f64)
        self.p0_all = torch.empty(self.B_total, d, **f64)
        self.p0 = self.p0_all[self.rows[0]:self.rows[1]]
        self.u_all = torch.empty(self.B_total, **f64)
        self.qp = torch.empty(B, d, **f64)
        self.gp = torch.empty(B, d, **f64)
        self.lp_new = torch.empty(B, **f64)
        self.q32 = torch.empty(B, d, dtype=torch.float32, device=self.dev)
        self.accepted = torch.zeros(B, dtype=torch.int32, device=self.dev)
        self.accept_prob = torch.zeros(B, **f64)
        self.logp = torch.empty(B, **f64)
        self.grad = torch.empty(B, d, **f64)
        self.q_prev = torch.empty(B, d, **f64)
        self.chees = torch.zeros(3, **f64)
        # one leapfrog update + one target evaluation, captured once per kick
        # (0.5 opens a trajectory, 1 continues it) and replayed; eps is read
        # from eps_dev when the graph runs. Continuing steps are also captured
        # graph_chunk at a time, so that most of a trajectory's steps share a
        # graph launch.
        self.graphs = bool(graphs)
        if int(graph_chunk) < 1:
            raise ValueError("graph_chunk must be at least 1")
        self.graph_chunk = int(graph_chunk)
        self.eps_dev = torch.full((1,), self.eps, **f64)
        self._eps_dev_val = self.eps
        self._graph = {}
        self.q32.copy_(self.q)
        self.target(self.q, self.q32, self.logp, self.grad)
        self.n_accepted = 0
        self.n_proposed = 0
        self.grad_evals = 0

    def step(self, n_leapfrog: Optional[int] = None) -> None:
        """One HMC iteration (L leapfrog steps + FP64 accept) for all chains."""
        stream = torch.cuda.current_stream(self.dev).cuda_stream
        B, d = self.B, self.d
        L = self.L if n_leapfrog is None else int(n_leapfrog)
        if L < 1:
            raise ValueError("an HMC iteration needs at least one leapfrog step")
        self.q_prev.copy_(self.q)
        torch.randn(self.B_total, d, generator=self.gen, dtype=torch.float64, device=self.dev, out=self.p0_all)
        self.p0.mul_(torch.rsqrt(self.inv_mass))
        self.p.copy_(self.p0)
        self.qp.copy_(self.q)
        self.gp.copy_(self.grad)
        q32 = self.q32.data_ptr() if self.target.needs_q32 else None
        if self.graphs:
            if self._eps_dev_val != self.eps:
                self.eps_dev.fill_(self.eps)
                self._eps_dev_val = self.eps
            # the first step, then the others in graphs of graph_chunk steps and single-step graphs
            self._leapfrog_graph(0.5).replay()
            rest = L - 1
            if 1 < self.graph_chunk <= rest:   # captured the first time a trajectory is long enough
                chunk = self._leapfrog_graph(1.0, self.graph_chunk)
                while rest >= self.graph_chunk:
                    chunk.replay()
                    rest -= self.graph_chunk
            for _ in range(rest):
                self._leapfrog_graph(1.0).replay()
        elif self.fused:
            for l in range(L):
                if l == 0:
                    self.target.leapfrog_first(self.qp, self.p, self.gp, self.inv_mass, self.eps, None, 0.5)
                else:
                    self.target.leapfrog_next(self.qp, self.p, self.inv_mass, self.eps, None, 1.0)
        else:
            for l in range(L):
                abi.gl_hmc_leapfrog(B, d, self.qp.data_ptr(), self.p.data_ptr(), self.gp.data_ptr(),
                                    self.inv_mass.data_ptr(), self.eps, 0.5 if l == 0 else 1.0, q32, stream)
                self.target(self.qp, self.q32, self.lp_new, self.gp)
        if self.fused:   # the fused steps leave log p~ and its gradient at the last point to here
            self.target.posterior_at_last(B, self.dev, self.lp_new, self.gp)
        torch.rand(self.B_total, generator=self.gen, dtype=torch.float64, device=self.dev, out=self.u_all)
        log_u = self.u_all[self.rows[0]:self.rows[1]].log_()
        abi.gl_hmc_finish(B, d, self.p0.data_ptr(), self.logp.data_ptr(), self.p.data_ptr(), self.gp.data_ptr(),
                          self.lp_new.data_ptr(), self.qp.data_ptr(), self.inv_mass.data_ptr(), log_u.data_ptr(),
                          self.eps, self.q.data_ptr(), self.logp.data_ptr(), self.grad.data_ptr(),
                          self.accepted.data_ptr(), stream, self.accept_prob.data_ptr())
        self.grad_evals += B * L
        self.n_proposed += B

    def _leapfrog_graph(self, kick: float, steps: int = 1):
        g = self._graph.get((kick, steps))
        if g is None:
            g = torch.cuda.CUDAGraph()
            q32 = self.q32.data_ptr() if self.target.needs_q32 else None
            if self.fused:   # buffers allocated before the capture
                self.target._buffers(self.B, self.dev)
            with torch.cuda.graph(g, capture_error_mode="thread_local"):
                st = torch.cuda.current_stream(self.dev).cuda_stream
                for _ in range(steps):
                    if self.fused and kick == 0.5:
                        self.target.leapfrog_first(self.qp, self.p, self.gp, self.inv_mass, 0.0, self.eps_dev, kick)
                    elif self.fused:
                        self.target.leapfrog_next(self.qp, self.p, self.inv_mass, 0.0, self.eps_dev, kick)
                    else:
                        abi.gl_hmc_leapfrog_dev(self.B, self.d, self.qp.data_ptr(), self.p.data_ptr(),
                                                self.gp.data_ptr(), self.inv_mass.data_ptr(),
                                                self.eps_dev.data_ptr(), kick, q32, st)
                        self.target(self.qp, self.q32, self.lp_new, self.gp)
            self._graph[(kick, steps)] = g
        return g

    def chees_gradient(self, t: float):
        """(gradient in log T, criterion, weight sum) of the last iteration
        over all chains (device); with a process group the chains' rows are
        gathered first and every process evaluates the same criterion."""
        rows = (self.q_prev, self.qp, self.p, self.accept_prob)
        if self.size > 1:
            rows = tuple(distributed.gather_rows(x, self.group, self.row_counts).contiguous() for x in rows)
        abi.gl_hmc_chees(self.B_total, self.d, rows[0].data_ptr(), rows[1].data_ptr(), rows[2].data_ptr(),
                         self.inv_mass.data_ptr(), rows[3].data_ptr(), t, self.chees.data_ptr(),
                         torch.cuda.current_stream(self.dev).cuda_stream)
        return self.chees

    def mean_accept_prob(self) -> torch.Tensor:
        """The last iteration's acceptance probability averaged over all chains (device scalar)."""
        return distributed.mean(self.accept_prob, self.group, self.row_counts)

    def run(self, n_iter: int) -> HMCStats:
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

    def run_adaptive(self, n_burn: int, n_samples: int, adapt_frac: float = 0.8, target_accept: float = 0.75,
                     adapt_trajectory: bool = False, max_leapfrog: int = 256) -> AdaptiveRun:
        """Burn-in with adaptation over its first adapt_frac, then n_samples
        recorded iterations. The step size (shared by all chains) follows dual
        averaging on the chains' mean acceptance probability. With
        adapt_trajectory, each iteration runs ceil(u_m T / eps) leapfrog steps
        (u_m the van der Corput jitter, also while sampling) and T follows the
        ChEES gradient (Adam on log T), starting from eps * L; both are frozen
        when adaptation ends (eps at its dual-averaged value)."""
        torch.cuda.synchronize(self.dev)
        t0 = time.perf_counter()
        e0 = self.grad_evals
        n_adapt = int(adapt_frac * n_burn)
        da = DualAveraging(self.eps, target=target_accept)
        T = self.eps * self.L
        ta = TrajectoryAdam(T, t_max=max_leapfrog * self.eps) if adapt_trajectory else None
        it = 0

        def n_steps():
            nonlocal it
            it += 1
            if not adapt_trajectory:
                return self.L, self.eps * self.L
            t = van_der_corput(it) * T
            return min(max_leapfrog, max(1, math.ceil(t / self.eps))), t

        ab = torch.zeros((), dtype=torch.float64, device=self.dev)
        for i in range(n_burn):
            L, t = n_steps()
            self.step(L)
            if i < n_adapt:
                if adapt_trajectory:
                    self.chees_gradient(t)
                    g = float(self.chees[0].item())
                    T = ta.update(g)
                self.eps = da.update(float(self.mean_accept_prob().item()))
                if i == n_adapt - 1:
                    self.eps = da.final()
            ab += self.mean_accept_prob()
        out = torch.empty(n_samples, self.B, self.d, dtype=torch.float64, device=self.dev)
        asum = torch.zeros((), dtype=torch.float64, device=self.dev)
        nl = 0
        for i in range(n_samples):
            L, _ = n_steps()
            nl += L
            self.step(L)
            out[i].copy_(self.q)
            asum += self.mean_accept_prob()
        torch.cuda.synchronize(self.dev)
        return AdaptiveRun(out, self.eps, float(ab.item()) / max(1, n_burn), float(asum.item()) / max(1, n_samples),
                           time.perf_counter() - t0, self.grad_evals - e0, T, nl / max(1, n_samples))


@dataclasses.dataclass
class PosteriorSamples:
    theta: torch.Tensor          # [n_samples, chains, 22] float32, physical parameters
    z: torch.Tensor              # [n_samples, chains, 22] float64, unconstrained
    run: AdaptiveRun


def sample_posterior(system, z_center: torch.Tensor, cov: torch.Tensor, chains: int = 50, n_burn: int = 250,
                     n_samples: int = 750, n_leapfrog: int = 5, seed: int = 0, prior=None,
                     step_size: float = 0.3, adapt_trajectory: bool = True,
                     max_leapfrog: int = 256, graphs: bool = True, group=None) -> PosteriorSamples:
    """The sampling step of the pipeline (Sec. 2.5, Table 1): chains drawn from
    N(z_center, cov) (the variational posterior in the paper), HMC on log p~(z)
    with mass cov^-1 (whitened coordinates); over the first 80% of burn-in the
    step size follows dual averaging toward acceptance 0.75 and, with
    adapt_trajectory, the trajectory length (from step_size * n_leapfrog,
    Table 1's 0.3 x 5) follows the ChEES gradient; otherwise n_leapfrog is
    fixed. With graphs, each leapfrog step is a replayed CUDA graph.
    The system's scratch is reserved for the chains first (no allocation
    may happen inside a captured graph). With a process group the chains are
    split over the processes and every process returns all chains' samples
    (``run.grad_evals`` counts this process's evaluations)."""
    dev = z_center.device
    rank, size = distributed.world(group)
    lo, hi = distributed.shard(chains, rank, size)
    system.reserve(max(1, hi - lo))
    L = torch.linalg.cholesky(cov.to(torch.float64).to(dev))
    post = PosteriorTarget(system, prior)
    target = WhitenedTarget(post, z_center.to(dev), L)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    x0 = torch.randn(chains, NPARAM, dtype=torch.float64, device=dev, generator=g)
    sampler = HMC(x0, torch.ones(NPARAM, dtype=torch.float64, device=dev), step_size, n_leapfrog, target=target,
                  seed=seed + 1, graphs=graphs, group=group)
    run = sampler.run_adaptive(n_burn, n_samples, adapt_trajectory=adapt_trajectory, max_leapfrog=max_leapfrog)
    if size > 1:
        chains_first = run.samples.transpose(0, 1).contiguous()
        run.samples = distributed.gather_rows(chains_first, group, sampler.row_counts).transpose(0, 1).contiguous()
    n = n_samples * chains
    z = target.to_z(run.samples.reshape(n, NPARAM))
    th = torch.empty(n, NPARAM, dtype=torch.float32, device=dev)
    pt = post.prior
    abi._check(abi.lib_handle().gl_map_transform(n, z.data_ptr(), ctypes.addressof(pt), th.data_ptr(),
                                                 torch.cuda.current_stream(dev).cuda_stream), "gl_map_transform")
    return PosteriorSamples(th.reshape(n_samples, chains, NPARAM), z.reshape(n_samples, chains, NPARAM), run)
