"""Continuous-batching lens server on top of the graph-replayed batcher.

Requests (one lens system + a batch of parameter vectors) arrive over time.
The scheduler admits them first-come first-served while the device-memory
budget allows (resident image, variance and PSF, plus the request's
parameters and results), uploads each admitted system on a side stream, and
forms batches of (request, vector range) segments round-robin over the
admitted requests, limited by the batcher's scratch arena and segment count.
Batches run as replays of one captured CUDA graph; up to ``max_inflight``
batches are queued on the GPU while the host forms the next, so requests
admitted while others run join the following batch. A request completes when
its last range has run and its results are copied back to pinned host
memory; its latency is completion minus arrival.
"""
from __future__ import annotations

import collections
import dataclasses
import time
from typing import Callable, Deque, Dict, List, Optional, Sequence, Tuple

import numpy as np

from . import inputs

NPARAM = 22
IO_BYTES_PER_VECTOR = NPARAM * 4 + 8 + NPARAM * 8     # params f32, log L f64, grad f64


@dataclasses.dataclass
class Job:
    """Host-side state of one request."""
    index: int
    arrival_s: float
    B: int
    resident_bytes: int
    next_vec: int = 0          # first vector not yet scheduled
    admitted_s: Optional[float] = None
    done_s: Optional[float] = None

    @property
    def bytes(self) -> int:
        return self.resident_bytes + self.B * IO_BYTES_PER_VECTOR

    @property
    def remaining(self) -> int:
        return self.B - self.next_vec


class Scheduler:
    """Admission by memory budget (FIFO) and round-robin batch formation."""

    def __init__(self, budget_bytes: int, arena_bytes: int, max_segments: int, chunk: int,
                 segment_bytes: Callable[[Job, int], int]):
        self.budget = int(budget_bytes)
        self.arena = int(arena_bytes)
        self.max_segments = int(max_segments)
        self.chunk = int(chunk)
        self.segment_bytes = segment_bytes
        self.used = 0
        self.waiting: Deque[Job] = collections.deque()
        self.active: List[Job] = []
        self.finished: List[Job] = []
        self._rr = 0

    def arrive(self, job: Job) -> None:
        if job.bytes > self.budget:
            raise ValueError("request %d needs %d bytes, more than the whole budget" % (job.index, job.bytes))
        self.waiting.append(job)

    def admit(self, now: float, max_ready: Optional[int] = None) -> List[Job]:
        """Admit waiting jobs FIFO while the budget allows and, with max_ready,
        while fewer than max_ready admitted jobs still have vectors to schedule
        (uploading a system blocks the host, so it is done as the batches need
        it, while the GPU works on the batches already queued)."""
        out = []
        ready = sum(1 for j in self.active if j.remaining > 0)
        while self.waiting and self.used + self.waiting[0].bytes <= self.budget and (
                max_ready is None or ready < max_ready):
            ready += 1
            j = self.waiting.popleft()
            j.admitted_s = now
            self.used += j.bytes
            self.active.append(j)
            out.append(j)
        return out

    def next_batch(self) -> List[Tuple[Job, int, int]]:
        """Segments (job, first vector, count): at most one per job, round-robin
        from where the previous batch stopped, within the arena and segment limits."""
        cands = [j for j in self.active if j.remaining > 0]
        if not cands:
            return []
        n = len(cands)
        start = self._rr % n
        order = cands[start:] + cands[:start]
        segs, used = [], 0
        for j in order:
            if len(segs) == self.max_segments:
                break
            c = min(self.chunk, j.remaining)
            need = self.segment_bytes(j, c)
            while c > 1 and used + need > self.arena:
                c //= 2
                need = self.segment_bytes(j, c)
            if used + need > self.arena:
                break
            segs.append((j, j.next_vec, c))
            j.next_vec += c
            used += need
        self._rr = start + len(segs)
        return segs

    def complete(self, job: Job, now: float) -> None:
        job.done_s = now
        self.used -= job.bytes
        self.active.remove(job)
        self.finished.append(job)

    def idle(self) -> bool:
        return not self.waiting and not self.active


# ------------------------------------------------------------------ GPU ----

@dataclasses.dataclass
class LensInput:
    """A request's host data: observed image, PSF and parameter vectors."""
    index: int
    arrival_s: float
    spec: inputs.SystemSpec
    image: np.ndarray
    psf: np.ndarray
    params: np.ndarray          # float32 [B, 22] (pinned copy made by the server)


def make_requests(stream: Sequence[inputs.LensRequest], device) -> List[LensInput]:
    """Observed images for a request stream: GPU model of a seeded truth + seeded noise.
    (Input preparation; not part of serving.)"""
    import torch
    from . import abi
    out = []
    cache: Dict[Tuple, object] = {}
    for r in stream:
        rng = np.random.default_rng(r.seed)
        truth = inputs.draw_truth(rng)
        psf = inputs.make_psf(r.spec).astype(np.float32)
        key = (r.spec.H, r.spec.W, r.spec.k, r.spec.K)
        if key not in cache:
            cache[key] = abi.GLSystem(np.zeros((r.spec.H, r.spec.W), np.float32), psf, r.spec.pixel_scale, r.spec.k,
                                      r.spec.gain_exposure, sigma_bkg=r.spec.sigma_bkg)
        model = cache[key].simulate(torch.from_numpy(truth.astype(np.float32)[None]).to(device)).cpu().numpy()[0]
        image = inputs.add_noise(rng, model, r.spec.sigma_bkg, r.spec.gain_exposure).astype(np.float32)
        params = inputs.draw_perturbed(rng, truth, r.B).astype(np.float32)
        out.append(LensInput(r.index, r.arrival_s, r.spec, image, psf, params))
    for s in cache.values():
        s.close()
    return out


@dataclasses.dataclass
class ServeStats:
    n: int
    seconds: float
    latencies_s: np.ndarray
    batches: int
    vectors: int

    @property
    def lenses_per_s(self) -> float:
        return self.n / self.seconds

    def summary(self) -> dict:
        lat = self.latencies_s * 1e3
        return {"lenses": self.n, "seconds": self.seconds, "lenses_per_s": self.lenses_per_s,
                "evals_per_s": self.vectors / self.seconds, "batches": self.batches,
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                               "mean": float(lat.mean()), "max": float(lat.max())}}


class LensServer:
    """Serves LensInput streams through a Batcher (continuous batching)."""

    def __init__(self, budget_bytes: int = 8 << 30, arena_bytes: int = 2 << 30, max_segments: int = 64,
                 chunk: int = 2048, max_inflight: int = 2, max_H: int = 128, max_W: int = 128, max_K: int = 21):
        import torch
        from . import abi
        self.abi = abi
        self.batcher = abi.Batcher(max_segments, arena_bytes, max_H, max_W, max_K)
        self.budget, self.arena, self.max_segments = budget_bytes, arena_bytes, max_segments
        self.chunk, self.max_inflight = chunk, max_inflight
        self.compute = torch.cuda.Stream()
        self.upload = torch.cuda.Stream()

    def close(self) -> None:
        self.batcher.close()

    def serve(self, reqs: Sequence[LensInput], realtime: bool = True, keep_results: bool = False):
        """Runs the stream; arrival times are honoured when realtime, else all
        requests arrive at t = 0 (capacity). Returns (ServeStats, results)."""
        import torch
        abi = self.abi
        dev = torch.device("cuda", torch.cuda.current_device())
        # host-side pinned buffers (input preparation)
        host = {}
        for r in reqs:
            host[r.index] = (torch.from_numpy(r.params).pin_memory(),
                             torch.empty(r.params.shape[0], dtype=torch.float64).pin_memory(),
                             torch.empty(r.params.shape[0], NPARAM, dtype=torch.float64).pin_memory())
        state: Dict[int, dict] = {}

        def seg_bytes(job: Job, n: int) -> int:
            return abi.Batcher.segment_bytes(state[job.index]["sys"], n)

        sched = Scheduler(self.budget, self.arena, self.max_segments, self.chunk, seg_bytes)
        pending = collections.deque(sorted(reqs, key=lambda r: r.arrival_s))
        by_index = {r.index: r for r in reqs}
        inflight: Deque[Tuple[object, List]] = collections.deque()
        finishing: List[Tuple[Job, object]] = []
        batches = vectors = 0
        t0 = time.perf_counter()
        while pending or not sched.idle() or inflight or finishing:
            now = time.perf_counter() - t0
            while pending and (not realtime or pending[0].arrival_s <= now):
                r = pending.popleft()
                resident = 4 * (2 * r.spec.H * r.spec.W + r.spec.K * r.spec.K)
                sched.arrive(Job(r.index, r.arrival_s if realtime else 0.0, r.params.shape[0], resident))
            for j in sched.admit(now, max_ready=2 * self.max_segments):
                r = by_index[j.index]
                with torch.cuda.stream(self.upload):
                    sysm = abi.GLSystem(r.image, r.psf, r.spec.pixel_scale, r.spec.k, r.spec.gain_exposure,
                                        sigma_bkg=r.spec.sigma_bkg)
                    hp, hl, hg = host[r.index]
                    p = hp.to(dev, non_blocking=True)
                    ll = torch.empty(j.B, dtype=torch.float64, device=dev)
                    g = torch.empty(j.B, NPARAM, dtype=torch.float64, device=dev)
                    ev = torch.cuda.Event()
                    ev.record(self.upload)
                state[j.index] = {"sys": sysm, "p": p, "ll": ll, "g": g, "ready": ev, "waited": False}
            # retire finished batches and requests
            while inflight and inflight[0][0].query():
                inflight.popleft()
            still = []
            for j, ev in finishing:
                if ev.query():
                    sched.complete(j, time.perf_counter() - t0)
                else:
                    still.append((j, ev))
            finishing = still
            if len(inflight) < self.max_inflight:
                segs = sched.next_batch()
                if segs:
                    systems, pp, bb, lp, gp = [], [], [], [], []
                    for j, a, c in segs:
                        st = state[j.index]
                        if not st["waited"]:
                            self.compute.wait_event(st["ready"])
                            st["waited"] = True
                        systems.append(st["sys"])
                        pp.append(st["p"].data_ptr() + a * NPARAM * 4)
                        bb.append(c)
                        lp.append(st["ll"].data_ptr() + a * 8)
                        gp.append(st["g"].data_ptr() + a * NPARAM * 8)
                    self.batcher.run(systems, pp, bb, lp, gp, stream=self.compute.cuda_stream)
                    done_ev = torch.cuda.Event()
                    done_ev.record(self.compute)
                    inflight.append((done_ev, segs))
                    batches += 1
                    vectors += sum(c for _, _, c in segs)
                    for j, a, c in segs:
                        if j.remaining == 0:       # last range scheduled: copy results back
                            st = state[j.index]
                            _, hl, hg = host[j.index]
                            with torch.cuda.stream(self.compute):
                                hl.copy_(st["ll"], non_blocking=True)
                                hg.copy_(st["g"], non_blocking=True)
                                ev = torch.cuda.Event()
                                ev.record(self.compute)
                            finishing.append((j, ev))
                    continue
            if not (inflight or finishing) and sched.idle() and pending and realtime:
                time.sleep(max(0.0, min(1e-3, pending[0].arrival_s - (time.perf_counter() - t0))))
            elif inflight or finishing:
                time.sleep(0)   # yield; completion is polled
        torch.cuda.synchronize()
        total = time.perf_counter() - t0
        jobs = sorted(sched.finished, key=lambda j: j.index)
        results = {}
        if keep_results:
            for r in reqs:
                _, hl, hg = host[r.index]
                results[r.index] = (hl.numpy().copy(), hg.numpy().copy())
        for st in state.values():
            st["sys"].close()
        lat = np.array([j.done_s - j.arrival_s for j in jobs])
        return ServeStats(len(jobs), total, lat, batches, vectors), results


def serve_one_call_per_lens(reqs: Sequence[LensInput], realtime: bool = True):
    """Baseline: each lens in its own gl_loglik_grad call (system created on
    arrival, results copied back), in arrival order, no batching across lenses."""
    import torch
    from . import abi
    dev = torch.device("cuda", torch.cuda.current_device())
    lat = []
    t0 = time.perf_counter()
    vectors = 0
    for r in sorted(reqs, key=lambda r: r.arrival_s):
        if realtime:
            while time.perf_counter() - t0 < r.arrival_s:
                time.sleep(max(0.0, min(1e-3, r.arrival_s - (time.perf_counter() - t0))))
        sysm = abi.GLSystem(r.image, r.psf, r.spec.pixel_scale, r.spec.k, r.spec.gain_exposure,
                            sigma_bkg=r.spec.sigma_bkg)
        hp = torch.from_numpy(r.params).pin_memory()
        p = hp.to(dev, non_blocking=True)
        ll, g = sysm.loglik_grad(p)
        hl, hg = ll.cpu(), g.cpu()
        done = time.perf_counter() - t0
        lat.append(done - (r.arrival_s if realtime else 0.0))
        vectors += r.params.shape[0]
        sysm.close()
    torch.cuda.synchronize()
    total = time.perf_counter() - t0
    return ServeStats(len(reqs), total, np.array(lat), len(reqs), vectors)
