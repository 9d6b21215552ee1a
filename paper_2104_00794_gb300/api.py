"""Torch-facing helpers over the C ABI (device memory and streams only).

``Problem`` holds one batch of shots on the device (grid, geometry) and
allocates the caller-owned workspace with torch; every computation is a call
into libtprobe through ``native``.  Tensors passed in must be contiguous
float32 CUDA tensors of the documented shapes.
"""
from __future__ import annotations

import dataclasses
import functools
from typing import Optional

import torch

from . import native


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _on_device(fn):
    """Runs a method with its object's device current, so that the current
    stream and every launch inside the library belong to that device."""
    @functools.wraps(fn)
    def run(self, *args, **kw):
        with torch.cuda.device(self.device):
            return fn(self, *args, **kw)
    return run


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _f32(t, device) -> torch.Tensor:
    t = torch.as_tensor(t, device=device)
    if t.dtype != torch.float32:
        t = t.to(torch.float32)
    return t.contiguous()


@dataclasses.dataclass
class ProbeSpec:
    kind: str = "rademacher"
    r: int = 4
    T: int = 32
    seed: int = 2104
    scale: float = 0.0
    Z_user: Optional[torch.Tensor] = None
    acc: str = "f32"  # accumulator storage: "f32", "bf16", "bf16_kahan", "f32_fold" (one set, r <= 32)

    def to_c(self) -> native.tp_probe:
        return native.tp_probe(native.PROBE_KINDS[self.kind], int(self.r), int(self.T), int(self.seed) & (2**64 - 1),
                               _ptr(self.Z_user) if self.Z_user is not None else None, float(self.scale),
                               native.ACC_TYPES[self.acc])


class Problem:
    """A batch of shots on one model grid, with device-resident geometry."""

    def __init__(self, ndim, nx, ny, nz, h, dt, nt, order, src, rec, vmax: float = 0.0, device="cuda",
                 form: str = "auto", sponge: int = 0, sponge_eta: float = 0.0):
        """form: the fp32 time stepping (tp_grid.form).  "auto" takes the
        compensated forward where the library supports it (2-D grids without an
        absorbing layer whose shot fits one thread-block cluster) and the
        levels form elsewhere."""
        self.device = torch.device(device)
        self.src = torch.as_tensor(src, dtype=torch.int64, device=self.device).contiguous()
        self.rec = torch.as_tensor(rec, dtype=torch.int64, device=self.device).contiguous()
        if self.src.dim() == 1:
            self.src = self.src[None]
        if self.rec.dim() == 1:
            self.rec = self.rec[None]
        self.nshots = int(self.src.shape[0])
        if self.rec.shape[0] != self.nshots:
            raise ValueError("src and rec need the same number of shots")
        auto = form == "auto"
        self.grid = native.tp_grid(int(ndim), int(nx), int(ny), int(nz), float(h), float(dt), int(nt), int(order),
                                   float(vmax), native.TIME_FORMS["compensated" if auto else form], int(sponge),
                                   float(sponge_eta))
        self.geom = native.tp_geom(self.nshots, int(self.src.shape[1]), self.src.data_ptr(),
                                   int(self.rec.shape[1]), self.rec.data_ptr())
        if auto and not native.tp_form_supported(self.grid, self.geom):
            self.grid.form = native.TIME_FORMS["levels"]
        self.form = {v: k for k, v in native.TIME_FORMS.items()}[self.grid.form]
        self._ws = {}

    @classmethod
    def from_workload(cls, w, nt=None, vmax=None, device="cuda", form="auto"):
        vm = float(max(w.vel_true.max(), w.vel0.max())) if vmax is None else vmax
        return cls(w.ndim, w.nx, w.ny, w.nz, w.h, w.dt, w.nt if nt is None else nt, w.order, w.src, w.rec,
                   vmax=vm, device=device, form=form, sponge=getattr(w, "sponge", 0),
                   sponge_eta=getattr(w, "sponge_eta", 0.0))

    # ---------------------------------------------------------------- sizes
    @property
    def nt(self):
        return self.grid.nt

    @property
    def N(self):
        return self.grid.nx * self.grid.ny * self.grid.nz

    @property
    def shape(self):
        g = self.grid
        return (g.nz, g.ny, g.nx) if g.ndim == 3 else (g.nz, g.nx)

    def workspace_bytes(self, op: int, probe: Optional[ProbeSpec] = None) -> int:
        return native.tp_workspace_bytes(op, self.grid, self.geom, probe.to_c() if probe is not None else None)

    def workspace(self, op: int, probe: Optional[ProbeSpec] = None) -> tuple[int, int]:
        """(pointer, bytes) of a cached, 256-byte aligned workspace for `op`."""
        n = self.workspace_bytes(op, probe)
        buf = self._ws.get(op)
        if buf is None or buf.numel() < n + 256:
            self._ws.pop(op, None)
            buf = torch.empty(n + 256, dtype=torch.uint8, device=self.device)
            self._ws[op] = buf
        p = buf.data_ptr()
        p += (-p) % 256
        return p, n

    def release(self):
        self._ws.clear()

    # ---------------------------------------------------------------- operators
    @_on_device
    def forward(self, vel, wavelet, d_out=None):
        vel, wavelet = _f32(vel, self.device), _f32(wavelet, self.device)
        if d_out is None:
            d_out = torch.empty((self.nshots, self.nt, self.geom.nrec), dtype=torch.float32, device=self.device)
        ws, n = self.workspace(native.OP_FORWARD)
        native.tp_forward(self.grid, self.geom, _ptr(vel), _ptr(wavelet), _ptr(d_out), ws, n, _stream())
        return d_out

    @_on_device
    def adjoint(self, vel, d_in, q_out=None):
        vel, d_in = _f32(vel, self.device), _f32(d_in, self.device)
        if q_out is None:
            q_out = torch.empty((self.nshots, self.nt, self.geom.nsrc), dtype=torch.float32, device=self.device)
        ws, n = self.workspace(native.OP_ADJOINT)
        native.tp_adjoint(self.grid, self.geom, _ptr(vel), _ptr(d_in), _ptr(q_out), ws, n, _stream())
        return q_out

    @_on_device
    def gradient_probed(self, vel, wavelet, d_obs, probe: ProbeSpec, grad=None, scalars=None):
        """(grad [dJ/dm], scalars[2] = (misfit, ||grad||)) as device tensors."""
        vel, wavelet, d_obs = _f32(vel, self.device), _f32(wavelet, self.device), _f32(d_obs, self.device)
        if grad is None:
            grad = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        if scalars is None:
            scalars = torch.empty(2, dtype=torch.float64, device=self.device)
        ws, n = self.workspace(native.OP_GRADIENT_PROBED, probe)
        native.tp_gradient_probed(self.grid, self.geom, probe.to_c(), _ptr(vel), _ptr(wavelet), _ptr(d_obs),
                                  _ptr(grad), scalars.data_ptr(), scalars.data_ptr() + 8, ws, n, _stream())
        return grad, scalars

    @_on_device
    def gradient_full(self, vel, wavelet, d_obs, grad=None, scalars=None):
        vel, wavelet, d_obs = _f32(vel, self.device), _f32(wavelet, self.device), _f32(d_obs, self.device)
        if grad is None:
            grad = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        if scalars is None:
            scalars = torch.empty(2, dtype=torch.float64, device=self.device)
        ws, n = self.workspace(native.OP_GRADIENT_FULL)
        native.tp_gradient_full(self.grid, self.geom, _ptr(vel), _ptr(wavelet), _ptr(d_obs), _ptr(grad),
                                scalars.data_ptr(), scalars.data_ptr() + 8, ws, n, _stream())
        return grad, scalars

    # ------------------------------------------------------------ split Algorithm 1
    def state_bytes(self, probe: ProbeSpec) -> int:
        return native.tp_probed_state_bytes(self.grid, self.geom, probe.to_c())

    def new_state(self, probe: ProbeSpec) -> torch.Tensor:
        """Caller-owned, 256-byte aligned buffer for the probes and forward accumulators."""
        n = self.state_bytes(probe)
        buf = torch.empty(n + 256, dtype=torch.uint8, device=self.device)
        off = (-buf.data_ptr()) % 256
        return buf[off:off + n]

    @_on_device
    def probed_forward(self, vel, wavelet, probe: ProbeSpec, state: torch.Tensor, d_out=None):
        """d = F(m; q) and the forward probe accumulators into `state` (Algorithm 1 lines 0-3)."""
        vel, wavelet = _f32(vel, self.device), _f32(wavelet, self.device)
        if d_out is None:
            d_out = torch.empty((self.nshots, self.nt, self.geom.nrec), dtype=torch.float32, device=self.device)
        ws, n = self.workspace(native.OP_PROBED_FORWARD, probe)
        native.tp_probed_forward(self.grid, self.geom, probe.to_c(), _ptr(vel), _ptr(wavelet), _ptr(d_out),
                                 state.data_ptr(), state.numel(), ws, n, _stream())
        return d_out

    @_on_device
    def probed_backward(self, vel, wavelet, adj_src, probe: ProbeSpec, state: torch.Tensor, wrt_velocity=False,
                        grad=None, gnorm=None):
        """Gradient (dJ/dm, or dJ/dv) from the adjoint source and `state` (Algorithm 1 lines 4-8)."""
        vel, wavelet, adj_src = _f32(vel, self.device), _f32(wavelet, self.device), _f32(adj_src, self.device)
        if grad is None:
            grad = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        if gnorm is None:
            gnorm = torch.empty(1, dtype=torch.float64, device=self.device)
        ws, n = self.workspace(native.OP_PROBED_BACKWARD, probe)
        native.tp_probed_backward(self.grid, self.geom, probe.to_c(), _ptr(vel), _ptr(wavelet), _ptr(adj_src),
                                  1 if wrt_velocity else 0, _ptr(grad), gnorm.data_ptr(), state.data_ptr(),
                                  state.numel(), ws, n, _stream())
        return grad, gnorm

    @_on_device
    def probed_image(self, vel, adj_src, probe: ProbeSpec, state: torch.Tensor, cond: str = "gradient",
                     image=None):
        """Imaging condition on the probed fields (Eq. 5): scale * sum_i <D P_i, D V_i>
        with P_i from `state` (probed_forward) and V_i from an adjoint run driven by
        adj_src; cond "correlation" (D = identity) or "gradient" (D = spatial gradient)."""
        vel, adj_src = _f32(vel, self.device), _f32(adj_src, self.device)
        if image is None:
            image = torch.empty(self.shape, dtype=torch.float32, device=self.device)
        ws, n = self.workspace(native.OP_PROBED_BACKWARD, probe)
        native.tp_probed_image(self.grid, self.geom, probe.to_c(), _ptr(vel), _ptr(adj_src),
                               native.IMAGE_CONDS[cond], _ptr(image), state.data_ptr(), state.numel(), ws, n,
                               _stream())
        return image

    @_on_device
    def qr_probes(self, d_obs, r: int, seed: int = 2104, kind: str = "rademacher") -> torch.Tensor:
        """Range-finding probes of Eq. 6, [nshots, nt, r], from the observed
        records; use them as ProbeSpec(kind="user", Z_user=Q, r=r)."""
        d_obs = _f32(d_obs, self.device)
        nt, nrec = self.nt, self.geom.nrec
        spec = ProbeSpec(kind=kind, r=r, seed=seed)
        n = native.tp_qr_workspace_bytes(nt, nrec, self.nshots, r)
        buf = torch.empty(n + 256, dtype=torch.uint8, device=self.device)
        ws = buf.data_ptr() + (-buf.data_ptr()) % 256
        Q = torch.empty((self.nshots, nt, r), dtype=torch.float32, device=self.device)
        native.tp_qr_probes(spec.to_c(), nt, nrec, self.nshots, _ptr(d_obs), _ptr(Q), ws, n, _stream())
        native.tp_workspace_status(ws, n, _stream())
        return Q

    @_on_device
    def probes(self, probe: ProbeSpec, shot: int = 0, nt: Optional[int] = None):
        nt = self.nt if nt is None else nt
        Z = torch.empty((nt, probe.r), dtype=torch.float32, device=self.device)
        native.tp_probes(probe.to_c(), nt, shot, _ptr(Z), _stream())
        return Z

    @_on_device
    def status(self, op: int):
        """Raises the device-side errors of the last `op` call (and clears them): a bounded wait
        that timed out (TP_ERR_TIMEOUT), a source or receiver index outside the grid when the
        call ran without a host check (vmax given; TP_ERR_ARG), rank-deficient QR probes."""
        buf = self._ws.get(op)
        if buf is None:
            return
        p = buf.data_ptr()
        p += (-p) % 256
        native.tp_workspace_status(p, buf.numel() - 256, _stream())


class GraphedGradient:
    """One Problem's gradient captured once as CUDA graphs and replayed per call.

    Every kernel of the gradient is enqueued by the library without host
    synchronisation (given the grid's vmax), so the whole call -- a few
    thousand kernels for nt = 2000 -- is captured once and launched as
    graphs.  Inputs (host tensors, preferably pinned, or device tensors) are
    copied into static device buffers, the graphs are replayed on the current
    stream, and the gradient and (misfit, |g|) are copied into the caller's
    outputs when given (else the static device tensors are returned,
    overwritten by the next call).  The probed gradient runs as its two
    halves (tp_probed_forward; tp_residual and tp_probed_backward), which give
    tp_gradient_probed's result bit for bit; d_obs is first read by the
    residual, so its upload runs on a second stream beside the forward half.
    The probes are fixed at capture (the spec's seed); use a new
    GraphedGradient for new probes."""

    def __init__(self, problem: Problem, probe: Optional[ProbeSpec] = None, full: bool = False):
        self.device = problem.device
        with torch.cuda.device(self.device):
            self._capture(problem, probe, full)

    def _capture(self, problem: Problem, probe: Optional[ProbeSpec], full: bool):
        if not problem.grid.vmax > 0.0:
            raise ValueError("a graphed gradient needs the grid's vmax (no host synchronisation inside the call)")
        if not full and probe is None:
            raise ValueError("probe spec required for the probed gradient")
        self.problem, self.probe, self.full = problem, probe, full
        g, dev = problem.grid, problem.device
        shape = problem.shape
        self.vel = torch.ones(shape, dtype=torch.float32, device=dev)
        self.vel.mul_(float(g.vmax))
        self.wavelet = torch.zeros((problem.nshots, problem.nt, problem.geom.nsrc), dtype=torch.float32, device=dev)
        self.d_obs = torch.zeros((problem.nshots, problem.nt, problem.geom.nrec), dtype=torch.float32, device=dev)
        self.grad = torch.empty(shape, dtype=torch.float32, device=dev)
        self.scalars = torch.empty(2, dtype=torch.float64, device=dev)
        if full:
            parts = [self._full]
        else:
            self.state = problem.new_state(probe)
            self.d_syn = torch.empty_like(self.d_obs)
            n = native.tp_residual_workspace_bytes()
            self._rbuf = torch.empty(n + 256, dtype=torch.uint8, device=dev)
            self._rws = (self._rbuf.data_ptr() + (-self._rbuf.data_ptr()) % 256, n)
            parts = [self._forward_half, self._backward_half]
        for run in parts:  # allocates the workspaces outside the capture
            run()
        # the graphs keep raw pointers into the workspaces: hold them, so that
        # problem.release() cannot free them under the graphs
        ops = [native.OP_GRADIENT_FULL] if full else [native.OP_PROBED_FORWARD, native.OP_PROBED_BACKWARD]
        self._ws = [problem._ws[op] for op in ops]
        torch.cuda.synchronize(dev)
        side = torch.cuda.Stream(device=dev)
        self.graphs = []
        with torch.cuda.stream(side):
            for run in parts:
                gr = torch.cuda.CUDAGraph()
                gr.capture_begin()
                run()
                gr.capture_end()
                self.graphs.append(gr)
        torch.cuda.synchronize(dev)
        self._upload = torch.cuda.Stream(device=dev)

    def _full(self):
        self.problem.gradient_full(self.vel, self.wavelet, self.d_obs, grad=self.grad, scalars=self.scalars)

    def _forward_half(self):
        self.problem.probed_forward(self.vel, self.wavelet, self.probe, self.state, d_out=self.d_syn)

    def _backward_half(self):
        native.tp_residual(self.d_syn.data_ptr(), self.d_obs.data_ptr(), self.d_syn.numel(),
                           self.scalars.data_ptr(), self._rws[0], self._rws[1], _stream())
        self.problem.probed_backward(self.vel, self.wavelet, self.d_syn, self.probe, self.state, grad=self.grad,
                                     gnorm=self.scalars[1:])

    @_on_device
    def __call__(self, vel, wavelet, d_obs, grad_out: Optional[torch.Tensor] = None,
                 scalars_out: Optional[torch.Tensor] = None):
        main = torch.cuda.current_stream()
        self.vel.copy_(vel, non_blocking=True)
        self.wavelet.copy_(wavelet, non_blocking=True)
        if self.full:
            self.d_obs.copy_(d_obs, non_blocking=True)
            self.graphs[0].replay()
        else:
            self._upload.wait_stream(main)  # the previous call's backward half has read d_obs
            self.graphs[0].replay()
            with torch.cuda.stream(self._upload):  # beside the forward half
                self.d_obs.copy_(d_obs, non_blocking=True)
                if d_obs.is_cuda:
                    d_obs.record_stream(self._upload)
            main.wait_stream(self._upload)
            self.graphs[1].replay()
        if grad_out is not None:
            grad_out.copy_(self.grad, non_blocking=True)
        if scalars_out is not None:
            scalars_out.copy_(self.scalars, non_blocking=True)
        return (self.grad if grad_out is None else grad_out), (self.scalars if scalars_out is None else scalars_out)


def memory_model(problem: Problem, probe: ProbeSpec) -> dict:
    """Gradient memory: the paper's counts (N nt values for the history,
    2 N r for the probed accumulators) and this library's workspace bytes."""
    N, nt, r, S = problem.N, problem.nt, probe.r, problem.nshots
    return {
        "full_history_values": N * nt * S,
        "probed_accumulator_values": 2 * N * r * S,
        "paper_reduction_factor": nt / (2.0 * r),
        "workspace_full_bytes": problem.workspace_bytes(native.OP_GRADIENT_FULL),
        "workspace_probed_bytes": problem.workspace_bytes(native.OP_GRADIENT_PROBED, probe),
    }
