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
admitted.  Latency = completion - arrival (host clock).

The scheduling policy (``Scheduler``) is host logic only and is tested on the
CPU with a simulated executor; ``GpuExecutor`` runs requests through the C ABI.
"""
from __future__ import annotations

import dataclasses
import threading
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


def summarize(requests: List[Request], makespan: float) -> dict:
    lat = np.array([r.latency for r in requests], dtype=np.float64) * 1e3
    work = float(sum(r.work for r in requests))
    return {"requests": len(requests), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
            "gpts_per_s": work / makespan / 1e9 if makespan > 0 else None, "makespan_s": makespan}


# ---------------------------------------------------------------- GPU side
class GpuExecutor:
    """Runs each request's probed gradient on its own stream, as one CUDA
    graph captured from the C-ABI call (or as direct launches)."""

    def __init__(self, use_graphs: bool = True):
        import torch
        self.torch = torch
        self.use_graphs = use_graphs
        self.lock = threading.Lock()
        self.finished: List[int] = []
        self.events = {}
        self.live = {}

    def start(self, req: Request):
        torch = self.torch
        job = req.payload
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
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
            else:
                job.launch()
            ev = torch.cuda.Event()
            ev.record(stream)
        self.events[req.rid] = ev
        self.live[req.rid] = (stream, job)

    def poll(self) -> List[int]:
        done = [rid for rid, ev in self.events.items() if ev.query()]
        for rid in done:
            self.events.pop(rid)
            _, job = self.live.pop(rid)
            job.finish()
        return done


class GradientJob:
    """One shot-gradient request: device inputs, workspace, outputs."""

    def __init__(self, problem, vel, wavelet, d_obs, probe):
        self.problem, self.vel, self.wavelet, self.d_obs, self.probe = problem, vel, wavelet, d_obs, probe
        self.grad = None
        self.scalars = None
        self.graph = None
        self.result = None

    def footprint(self) -> int:
        from . import native
        return self.problem.workspace_bytes(native.OP_GRADIENT_PROBED, self.probe) + 4 * self.problem.N + 512

    def allocate(self):
        import torch
        from . import native
        self.grad = torch.empty(self.problem.shape, dtype=torch.float32, device=self.problem.device)
        self.scalars = torch.empty(2, dtype=torch.float64, device=self.problem.device)
        self.problem.workspace(native.OP_GRADIENT_PROBED, self.probe)

    def launch(self):
        self.problem.gradient_probed(self.vel, self.wavelet, self.d_obs, self.probe, grad=self.grad,
                                     scalars=self.scalars)

    def finish(self):
        self.result = (self.grad, self.scalars)
        self.graph = None
        self.problem.release()  # workspace memory back to the pool
