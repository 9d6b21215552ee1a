"""Continuous-batching server for probed-gradient requests on one GPU.

Requests (one shot gradient each: a grid, nt, r, and device-resident model,
wavelet and observed data) arrive over time.  The scheduler admits them, in
arrival order, as soon as a slot and enough of the device-memory budget are
free -- the footprint is the probed workspace that ``tp_workspace_bytes``
reports plus the gradient -- so requests that arrive while others run join
them on the GPU.  Every admitted request runs on a stream of its own; its
whole gradient is captured once into a CUDA graph and launched as one graph,
and kernels of different requests overlap on the device.  When a request
completes its memory returns to the budget and the next waiting request is
admitted.  With a graph cache, requests of one shape (grid, time axis,
geometry counts, probes) replay a gradient captured once for that shape: the
first such request pays the capture, later ones copy their inputs into the
cached graph's buffers and replay it.  Latency = completion - arrival (host
clock).

The scheduling policy (``Scheduler``) is host logic only and is tested on the
CPU with a simulated executor; ``GpuExecutor`` runs requests through the C ABI.
"""
from __future__ import annotations

import dataclasses
import time
from collections import deque
from typing import Callable, List, Optional

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the run
    footprint: int                 # device bytes while admitted
    work: float = 0.0              # grid-point updates (2 N nt)
    payload: object = None         # executor-specific
    admitted: Optional[float] = None
    done: Optional[float] = None

    @property
    def latency(self) -> Optional[float]:
        return None if self.done is None else self.done - self.arrival


class Scheduler:
    """FIFO admission by device-memory footprint and slot count."""

    def __init__(self, budget_bytes: int, max_slots: int):
        if budget_bytes <= 0 or max_slots <= 0:
            raise ValueError("budget and slots must be positive")
        self.budget = int(budget_bytes)
        self.max_slots = int(max_slots)
        self.used = 0
        self.queue: deque = deque()
        self.active: dict = {}
        self.peak_used = 0
        self.peak_active = 0

    def arrive(self, req: Request):
        if req.footprint > self.budget:
            raise ValueError(f"request {req.rid} needs {req.footprint} bytes, more than the budget {self.budget}")
        self.queue.append(req)

    def admissible(self) -> List[Request]:
        """Pops and returns the requests that fit now (head-of-line order:
        a request that does not fit blocks the ones behind it, so no request
        waits forever)."""
        out = []
        while self.queue and len(self.active) < self.max_slots and self.used + self.queue[0].footprint <= self.budget:
            r = self.queue.popleft()
            self.used += r.footprint
            self.active[r.rid] = r
            out.append(r)
        self.peak_used = max(self.peak_used, self.used)
        self.peak_active = max(self.peak_active, len(self.active))
        return out

    def complete(self, rid: int):
        r = self.active.pop(rid)
        self.used -= r.footprint
        return r

    def idle(self) -> bool:
        return not self.queue and not self.active


def run(requests: List[Request], sched: Scheduler, start: Callable[[Request], None],
        poll: Callable[[], List[int]], clock: Callable[[], float] = time.perf_counter,
        sleep: Callable[[float], None] = lambda s: time.sleep(s)) -> List[Request]:
    """Drives arrivals, admission and completion until every request is done.
    `start(req)` launches a request asynchronously; `poll()` returns the ids
    of requests that finished since the last call."""
    pending = deque(sorted(requests, key=lambda r: r.arrival))
    t0 = clock()
    while pending or not sched.idle():
        now = clock() - t0
        while pending and pending[0].arrival <= now:
            sched.arrive(pending.popleft())
        for r in sched.admissible():
            r.admitted = clock() - t0
            start(r)
        for rid in poll():
            r = sched.complete(rid)
            r.done = clock() - t0
        if sched.idle() and pending:
            sleep(max(0.0, min(pending[0].arrival - (clock() - t0), 0.01)))
        else:
            sleep(0.0002)
    return requests


def summarize(requests: List[Request], makespan: float, captured=None) -> dict:
    """Latency percentiles of all requests; with `captured` (ids of requests
    that had their graph captured), also of the others (served by a replay)."""
    lat = np.array([r.latency for r in requests], dtype=np.float64) * 1e3
    work = float(sum(r.work for r in requests))
    out = {"requests": len(requests), "p50_ms": float(np.percentile(lat, 50)),
           "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
           "gpts_per_s": work / makespan / 1e9 if makespan > 0 else None, "makespan_s": makespan}
    if captured is not None:
        rep = np.array([r.latency for r in requests if r.rid not in captured], dtype=np.float64) * 1e3
        out["replayed_requests"] = int(rep.size)
        if rep.size:
            out["replayed_p50_ms"] = float(np.percentile(rep, 50))
            out["replayed_p99_ms"] = float(np.percentile(rep, 99))
    return out


# ---------------------------------------------------------------- GPU side
class GraphSlot:
    """A captured gradient for one request shape, replayable for any request
    of that shape: its own copies of the geometry, inputs and outputs (the
    graph holds their device addresses) and its own workspace."""

    def __init__(self, job, stream):
        import torch
        from . import api, native
        p0 = job.problem
        g = p0.grid
        self.problem = api.Problem(g.ndim, g.nx, g.ny, g.nz, g.h, g.dt, g.nt, g.order, p0.src.clone(), p0.rec.clone(),
                                   vmax=g.vmax, device=p0.device, form=p0.form, sponge=g.sponge,
                                   sponge_eta=g.sponge_eta)
        self.probe = job.probe
        self.vel, self.wavelet, self.d_obs = job.vel.clone(), job.wavelet.clone(), job.d_obs.clone()
        self.grad = torch.empty(self.problem.shape, dtype=torch.float32, device=p0.device)
        self.scalars = torch.empty(2, dtype=torch.float64, device=p0.device)
        self.bytes = job.footprint() + sum(t.numel() * t.element_size() for t in (self.vel, self.wavelet, self.d_obs))
        with torch.cuda.stream(stream):
            self.problem.workspace(native.OP_GRADIENT_PROBED, self.probe)  # allocated outside the capture
            t0 = time.perf_counter()
            self.graph = torch.cuda.CUDAGraph()
            self.graph.capture_begin(capture_error_mode="thread_local")
            try:
                self.problem.gradient_probed(self.vel, self.wavelet, self.d_obs, self.probe, grad=self.grad,
                                             scalars=self.scalars)
            finally:
                self.graph.capture_end()
            self.capture_s = time.perf_counter() - t0

    def run(self, job):
        """On the current stream: the job's geometry and inputs in, one replay,
        its gradient and (misfit, |g|) out."""
        self.problem.src.copy_(job.problem.src, non_blocking=True)
        self.problem.rec.copy_(job.problem.rec, non_blocking=True)
        self.vel.copy_(job.vel, non_blocking=True)
        self.wavelet.copy_(job.wavelet, non_blocking=True)
        self.d_obs.copy_(job.d_obs, non_blocking=True)
        self.graph.replay()
        job.grad.copy_(self.grad, non_blocking=True)
        job.scalars.copy_(self.scalars, non_blocking=True)


class GraphCache:
    """Captured gradients kept per request shape.  A request takes an idle
    slot of its shape (a replay) or has one captured; finished requests return
    their slot.  Idle slots are freed least recently used first while the
    cached bytes exceed max_bytes (slots in use are never freed)."""

    def __init__(self, max_bytes: int):
        from collections import OrderedDict
        self.max_bytes = int(max_bytes)
        self.idle = OrderedDict()  # key -> [slots]
        self.bytes = 0
        self.captures = 0
        self.capture_s = 0.0
        self.reuses = 0
        self.evictions = 0

    def acquire(self, key, job, stream):
        slots = self.idle.get(key)
        if slots:
            self.idle.move_to_end(key)
            self.reuses += 1
            return slots.pop(), False
        slot = GraphSlot(job, stream)
        self.bytes += slot.bytes
        self.captures += 1
        self.capture_s += slot.capture_s
        self._evict()
        return slot, True

    def release(self, key, slot):
        self.idle.setdefault(key, []).append(slot)
        self.idle.move_to_end(key)
        self._evict()

    def _evict(self):
        while self.bytes > self.max_bytes:
            key = next((k for k, v in self.idle.items() if v), None)
            if key is None:
                return
            slot = self.idle[key].pop(0)
            if not self.idle[key]:
                del self.idle[key]
            self.bytes -= slot.bytes
            self.evictions += 1
            del slot


class GpuExecutor:
    """Runs each request's probed gradient on its own stream: replayed from a
    per-shape graph cache (cache_bytes > 0), as one CUDA graph captured for
    the request (use_graphs), or as direct launches."""

    def __init__(self, use_graphs: bool = True, cache_bytes: int = 0):
        import torch
        self.torch = torch
        self.use_graphs = use_graphs
        self.cache = GraphCache(cache_bytes) if cache_bytes > 0 else None
        self.finished: List[int] = []
        self.events = {}
        self.live = {}
        self.captured = set()  # ids of requests that had their graph captured

    def start(self, req: Request):
        torch = self.torch
        job = req.payload
        stream = torch.cuda.Stream()
        slot = None
        with torch.cuda.stream(stream):
            if self.cache is not None:
                job.allocate(workspace=False)
                slot, new = self.cache.acquire(job.key(), job, stream)
                if new:
                    self.captured.add(req.rid)
                slot.run(job)
            else:
                job.allocate()
                if self.use_graphs:
                    # capture on this request's stream only: no device-wide
                    # synchronisation, so the other requests keep running
                    g = torch.cuda.CUDAGraph()
                    g.capture_begin(capture_error_mode="thread_local")
                    try:
                        job.launch()
                    finally:
                        g.capture_end()
                    g.replay()
                    job.graph = g
                    self.captured.add(req.rid)
                else:
                    job.launch()
            ev = torch.cuda.Event()
            ev.record(stream)
        self.events[req.rid] = ev
        self.live[req.rid] = (stream, job, slot)

    def poll(self) -> List[int]:
        done = [rid for rid, ev in self.events.items() if ev.query()]
        for rid in done:
            self.events.pop(rid)
            _, job, slot = self.live.pop(rid)
            if slot is not None:
                self.cache.release(job.key(), slot)
            job.finish()
        return done

    def stats(self) -> dict:
        c = self.cache
        if c is None:
            return {"graph_cache": False, "captures": len(self.captured)}
        return {"graph_cache": True, "captures": c.captures, "graph_reuse": c.reuses,
                "capture_ms_total": 1e3 * c.capture_s, "capture_ms_mean": 1e3 * c.capture_s / max(c.captures, 1),
                "evictions": c.evictions, "cache_bytes": c.bytes}


class GradientJob:
    """One shot-gradient request: device inputs, workspace, outputs."""

    def __init__(self, problem, vel, wavelet, d_obs, probe):
        self.problem, self.vel, self.wavelet, self.d_obs, self.probe = problem, vel, wavelet, d_obs, probe
        self.grad = None
        self.scalars = None
        self.graph = None
        self.result = None

    def key(self):
        """Requests with equal keys replay the same captured gradient: the grid
        and time axis (vmax included: the stability check runs at capture), the
        form, the counts of the geometry and the probe specification."""
        g, geo, pr = self.problem.grid, self.problem.geom, self.probe
        return ((g.ndim, g.nx, g.ny, g.nz, g.h, g.dt, g.nt, g.order, g.vmax, g.form, g.sponge, g.sponge_eta),
                (geo.nshots, geo.nsrc, geo.nrec), (pr.kind, pr.r, pr.T, pr.seed, pr.scale, pr.acc))

    def footprint(self) -> int:
        from . import native
        return self.problem.workspace_bytes(native.OP_GRADIENT_PROBED, self.probe) + 4 * self.problem.N + 512

    def allocate(self, workspace: bool = True):
        import torch
        from . import native
        self.grad = torch.empty(self.problem.shape, dtype=torch.float32, device=self.problem.device)
        self.scalars = torch.empty(2, dtype=torch.float64, device=self.problem.device)
        if workspace:
            self.problem.workspace(native.OP_GRADIENT_PROBED, self.probe)

    def launch(self):
        self.problem.gradient_probed(self.vel, self.wavelet, self.d_obs, self.probe, grad=self.grad,
                                     scalars=self.scalars)

    def finish(self):
        self.result = (self.grad, self.scalars)
        self.graph = None
        self.problem.release()  # workspace memory back to the pool
