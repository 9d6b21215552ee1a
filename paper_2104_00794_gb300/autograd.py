"""Differentiable forward modelling with a probed backward pass.

``ProbedModeling`` wraps F(m; q) (Eq. 2) as a ``torch.autograd.Function`` of
the velocity.  Its forward runs the library's forward sweep and keeps only
the probes and the forward probe accumulators (Algorithm 1 lines 0-3, 2 N r
values with the adjoint ones instead of the N nt history); its backward runs
the adjoint sweep driven by dL/dd, the adjoint accumulation and the combine
(Algorithm 1 lines 4-8) and returns dL/dv through the chain rule
dm/dv = -2 / v^3, all inside the CUDA kernels.  With identity probes
(r = nt) the backward is the exact adjoint-state gradient; with r random
probes it is the unbiased estimate of Eq. 4.
"""
from __future__ import annotations

import torch

from .api import Problem, ProbeSpec


class ProbedModeling(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vel: torch.Tensor, problem: Problem, wavelet: torch.Tensor, probe: ProbeSpec):
        state = problem.new_state(probe)
        d = problem.probed_forward(vel.detach(), wavelet, probe, state)
        ctx.problem, ctx.probe, ctx.state = problem, probe, state
        ctx.save_for_backward(vel, wavelet)
        return d

    @staticmethod
    def backward(ctx, grad_d: torch.Tensor):
        vel, wavelet = ctx.saved_tensors
        grad_v, _ = ctx.problem.probed_backward(vel.detach(), wavelet, grad_d.contiguous(), ctx.probe, ctx.state,
                                                wrt_velocity=True)
        ctx.state = None
        return grad_v, None, None, None


def modeling(vel: torch.Tensor, problem: Problem, wavelet: torch.Tensor, probe: ProbeSpec) -> torch.Tensor:
    """Synthetic data [nshots, nt, nrec] = F(vel), differentiable in vel."""
    return ProbedModeling.apply(vel, problem, wavelet, probe)
