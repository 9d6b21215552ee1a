"""Full-waveform inversion with probed gradients (§Example).

The paper inverts with a spectral projected gradient method (SPG) under box
constraints on the squared slowness m, using randomized-trace gradients with
new probes at every iteration.  This module holds that loop:

  * ``spg``: SPG with a nonmonotone line search (Birgin, Martinez & Raydan,
    2000): step d = P(x - alpha g) - x, Barzilai-Borwein alpha = s.s / s.y
    (safeguarded), backtracking until f(x + lam d) <= max of the last M
    values + gamma lam g.d.  It is written against plain callables and
    operators, so it runs on numpy arrays (tested on the CPU) and on device
    tensors alike.
  * ``invert``: the FWI driver on the GPU.  The objective is the data misfit
    1/2 |F(m) - d_obs|^2 of all shots (one forward per evaluation); the
    gradient is the probed gradient of the library (new probes each call,
    seed + call index) or the full-storage gradient.  m is bounded by
    [1/vmax^2, 1/vmin^2].

The optimiser's vector updates (axpy, clamp, dot products) are a few O(N)
operations per iteration next to the 2 N nt stencil updates of a gradient;
they run as torch operations on the device.
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional


@dataclasses.dataclass
class SpgResult:
    x: object
    f: List[float]            # objective after each iteration (f[0]: start)
    evals: int                # objective evaluations (line-search trials included)
    grads: int                # gradient evaluations


def spg(x0, fg: Callable, f: Callable, proj: Callable, dot: Callable, maxabs: Callable, iters: int,
        memory: int = 5, gamma: float = 1e-4, alpha_min: float = 1e-10, alpha_max: float = 1e10,
        alpha0: Optional[float] = None, step0: Optional[float] = None,
        max_backtracks: int = 10) -> SpgResult:
    """Spectral projected gradient.  fg(x) -> (f, g); f(x) -> f; proj(x) -> the
    projection onto the feasible set; dot(a, b) -> float; maxabs(a) -> float.
    First step length: alpha0 if given; else, with step0, the alpha whose
    gradient step changes the largest entry of x by the fraction step0; else
    1 / max|P(x - g) - x| (the published default)."""
    x = proj(x0)
    fx, g = fg(x)
    hist = [float(fx)]
    evals, grads = 1, 1
    if alpha0 is not None:
        alpha = alpha0
    elif step0 is not None:
        alpha = step0 * maxabs(x) / max(maxabs(g), 1e-300)
    else:
        alpha = 1.0 / max(maxabs(proj(x - g) - x), 1e-300)
    for _ in range(iters):
        d = proj(x - alpha * g) - x
        gd = dot(g, d)
        if gd >= 0.0:  # projected gradient vanished: stationary
            break
        fmax = max(hist[-memory:])
        lam = 1.0
        x_new, f_new = None, None
        for _ in range(max_backtracks + 1):
            x_try = x + lam * d
            f_try = float(f(x_try))
            evals += 1
            if f_try <= fmax + gamma * lam * gd:
                x_new, f_new = x_try, f_try
                break
            lam *= 0.5
        if x_new is None:  # no acceptable step along d
            break
        fx_new, g_new = fg(x_new)
        grads += 1
        s = x_new - x
        y = g_new - g
        sy = dot(s, y)
        alpha = alpha_max if sy <= 0.0 else min(alpha_max, max(alpha_min, dot(s, s) / sy))
        x, g = x_new, g_new
        hist.append(float(fx_new))
    return SpgResult(x, hist, evals, grads)


def update_mask(shape, top: int, side: int, bottom: int):
    """1 where the model is updated, 0 in the `top` rows (next to the sources
    and receivers, where the gradient is dominated by their near field) and
    within `side` / `bottom` cells of the absorbing faces."""
    import numpy as np
    m = np.zeros(shape, dtype=np.float32)
    sl = [slice(top, shape[0] - bottom)] + [slice(side, n - side) for n in shape[1:]]
    m[tuple(sl)] = 1.0
    return m


def invert(problem, vel0, wavelet, d_obs, vmin: float, vmax: float, iters: int, probe=None,
           full: bool = False, memory: int = 5, seed: int = 2104, mask=None, step0: float = 0.02) -> SpgResult:
    """FWI of `problem`'s shots by SPG on the squared slowness.  `probe`
    (api.ProbeSpec) selects probed gradients, its seed advanced per call;
    `full=True` uses the full-storage gradient instead.  `mask` (the model's
    shape, 0/1) restricts the update; `step0` sets the first step (the largest
    entry of m moves by that fraction).  Returns the velocity model in ``x``
    (device tensor, the shape of vel0).

    The line search's misfits go through tp_misfit_noalloc, whose scratch is
    one array per device shared by every call in the process: two inversions
    run at the same time in one process (threads on different streams) must
    be serialised, or their misfits race on that array."""
    import torch

    dev = problem.device
    vel0 = torch.as_tensor(vel0, device=dev, dtype=torch.float32)
    wavelet = torch.as_tensor(wavelet, device=dev, dtype=torch.float32).contiguous()
    d_obs = torch.as_tensor(d_obs, device=dev, dtype=torch.float32).contiguous()
    mlo, mhi = 1.0 / vmax ** 2, 1.0 / vmin ** 2
    calls = [0]
    mk = None if mask is None else torch.as_tensor(mask, device=dev, dtype=torch.float32)

    def vel_of(m):
        return torch.rsqrt(m).contiguous()

    from . import native
    J = torch.empty(1, dtype=torch.float64, device=dev)

    def misfit(m):
        d = problem.forward(vel_of(m), wavelet)
        # J = 1/2 |d - d_obs|^2 in fp64 by the library's reduction kernels
        with torch.cuda.device(dev):
            native.tp_misfit_noalloc(d.data_ptr(), d_obs.data_ptr(), d.numel(), J.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
        return float(J.item())

    def fg(m):
        v = vel_of(m)
        if full:
            g, sc = problem.gradient_full(v, wavelet, d_obs)
        else:
            spec = dataclasses.replace(probe, seed=seed + calls[0])
            g, sc = problem.gradient_probed(v, wavelet, d_obs, spec)
        calls[0] += 1
        return float(sc[0]), (g * mk if mk is not None else g.clone())

    res = spg((1.0 / vel0.double() ** 2).float(), fg, misfit,
              proj=lambda m: torch.clamp(m, mlo, mhi),
              dot=lambda a, b: float(torch.sum(a.double() * b.double())),
              maxabs=lambda a: float(torch.max(torch.abs(a))), iters=iters, memory=memory, step0=step0)
    res.x = vel_of(res.x)
    return res
