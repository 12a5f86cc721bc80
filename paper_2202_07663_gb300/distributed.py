"""Inference for one lens system spread over processes (one GPU each).

The steps of Sec. 2.3-2.5 are data-parallel in one unit each: MAP in its
start points, VI in the Monte-Carlo draws of each ELBO-gradient estimate,
HMC in its chains. Every process runs the library's kernels on its share of
that unit; the exchanges are small all-gathers through ``torch.distributed``
(NCCL on GPUs, gloo on CPU):

* MAP: the best start over all processes (``best_row``);
* VI: each process's moment sums (``gl_vi_moments``), added in rank order
  inside ``gl_vi_apply``;
* HMC: the chains' acceptance probabilities (the dual-averaging mean) and,
  while the trajectory length adapts, the rows ``gl_hmc_chees`` reads.

Gathered values are combined in rank order on every process, so all of them
hold bit-identical global state (step size, trajectory length, variational
parameters, best start) without a broadcast. Random numbers for a unit are
drawn for all units from one shared seed and sliced to the process's rows, so
a run on several processes makes the draws a single process would make.

With ``group=None`` and no initialised process group everything is local
(one process, no communication).
"""
from __future__ import annotations

from typing import List, Optional, Sequence, Tuple

import torch
import torch.distributed as dist


def world(group=None) -> Tuple[int, int]:
    """(rank, world size) in ``group``; (0, 1) without a process group."""
    if not (dist.is_available() and dist.is_initialized()):
        return 0, 1
    return dist.get_rank(group), dist.get_world_size(group)


def shard(n: int, rank: int, size: int) -> Tuple[int, int]:
    """Rows [lo, hi) of n units for ``rank`` of ``size``: contiguous, in rank
    order, the first n % size ranks one row longer."""
    if size < 1 or not 0 <= rank < size or n < 0:
        raise ValueError("bad shard request")
    q, r = divmod(n, size)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def counts(n: int, size: int) -> List[int]:
    return [b - a for a, b in (shard(n, r, size) for r in range(size))]


def gather_parts(x: torch.Tensor, group=None) -> torch.Tensor:
    """[size, *x.shape]: every process's ``x`` (equal shapes) in rank order."""
    _, size = world(group)
    if size == 1:
        return x.unsqueeze(0)
    dev = x.device
    if dev.type != "cpu" and dist.get_backend(group) == "gloo":
        x = x.cpu()            # gloo exchanges host memory
    parts = [torch.empty_like(x) for _ in range(size)]
    dist.all_gather(parts, x.contiguous(), group=group)
    return torch.stack(parts).to(dev)


def gather_rows(x: torch.Tensor, group=None, row_counts: Optional[Sequence[int]] = None) -> torch.Tensor:
    """Concatenate every process's rows of ``x`` (first dimensions may differ)
    in rank order. ``row_counts`` (per rank) saves one exchange when known."""
    _, size = world(group)
    if size == 1:
        return x
    if row_counts is None:
        n = torch.tensor([x.shape[0]], dtype=torch.int64, device=x.device)
        row_counts = [int(c) for c in gather_parts(n, group).reshape(-1).tolist()]
    if len(row_counts) != size or row_counts[dist.get_rank(group)] != x.shape[0]:
        raise ValueError("row_counts does not match the process group")
    m = max(row_counts)
    pad = x.new_zeros((m,) + tuple(x.shape[1:]))
    pad[: x.shape[0]] = x
    parts = gather_parts(pad, group)
    return torch.cat([parts[r, :c] for r, c in enumerate(row_counts)])


def mean(x: torch.Tensor, group=None, row_counts: Optional[Sequence[int]] = None) -> torch.Tensor:
    """Mean of a 1-D tensor over all processes' entries (the same bits on
    every process: the gathered vector is reduced identically everywhere)."""
    return gather_rows(x, group, row_counts).mean()


def best_row(objective: torch.Tensor, rows: Sequence[torch.Tensor], group=None):
    """Global argmin of ``objective`` over all processes' entries, non-finite
    values left out, ties to the lowest global index (rank order, then local
    order). Returns (global index, value, [row of each tensor in ``rows``]) on
    every process; index -1, value inf and NaN rows if no entry is finite."""
    rank, size = world(group)
    dev = objective.device
    f = torch.nan_to_num(objective.to(torch.float64), nan=float("inf"), posinf=float("inf"), neginf=float("inf"))
    n = f.shape[0]
    widths = [max(1, int(torch.Size(r.shape[1:]).numel())) for r in rows]
    cand = torch.full((3 + sum(widths),), float("nan"), dtype=torch.float64, device=dev)
    cand[0] = float("inf")
    cand[1] = -1.0
    cand[2] = float(n)
    if n:
        i = int(torch.argmin(f).item())       # first minimum: lowest local index
        if torch.isfinite(f[i]):
            cand[0] = f[i]
            cand[1] = i
            k = 3
            for r, w in zip(rows, widths):
                cand[k:k + w] = r[i].reshape(-1).to(torch.float64)
                k += w
    allc = gather_parts(cand, group).cpu()
    best, gidx, off = None, -1, 0
    for r in range(size):
        v, li, nr = float(allc[r, 0]), int(allc[r, 1]), int(allc[r, 2])
        if li >= 0 and (best is None or v < float(allc[best, 0])):
            best, gidx = r, off + li
        off += nr
    if best is None:
        out = [torch.full(t.shape[1:], float("nan"), dtype=t.dtype, device=dev) for t in rows]
        return -1, float("inf"), out
    out, k = [], 3
    row = allc[best].to(dev)
    for t, w in zip(rows, widths):
        out.append(row[k:k + w].reshape(t.shape[1:]).to(t.dtype))
        k += w
    return gidx, float(allc[best, 0]), out
