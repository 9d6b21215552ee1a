"""Seeded synthetic inputs for the probed-gradient workloads.

This module only *generates inputs*: velocity models, acquisition geometry
and the source wavelet.  It holds none of the method's arithmetic (no
stencil, no probes, no gradient), so both the CUDA path and the FP64 checker
can take their inputs from here without sharing any of the computation.

The paper's only experiment (Section "Example") uses the 2-D overthrust
model, 8 Hz Ricker wavelet, 3 s of recording and r = 16 probes.  That model
is not available here; the seeded models below stand in for it with the
same kind of structure (smooth background, random perturbations, a
high-velocity body, layered 3-D media).

Conventions shared by every consumer:
  * grids are stored z-major, x fastest: ``vel[z, y, x]`` (3-D) or
    ``vel[z, x]`` (2-D, ``ny == 1``);
  * a grid point's flat index is ``(z * ny + y) * nx + x``;
  * the wavelet of shot ``s`` is ``wavelet[s, t, k]`` for source ``k``;
  * every array handed out is float32 (the precision the GPU path reads);
    the checker converts these exact float32 values to float64.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

DEFAULT_SEED = 2104

# Courant numbers v*dt/h at which the leapfrog scheme with a centred
# 2k-order Laplacian stops being stable (max |symbol| of the Laplacian):
# listed here only so that generated models can be clipped safely.
CFL_LIMIT = {(2, 4): 0.6124, (3, 4): 0.5000, (2, 8): 0.5546, (3, 8): 0.4529}


@dataclasses.dataclass
class Workload:
    """One seeded problem: grid, geometry, models, wavelet, probe spec."""

    name: str
    ndim: int
    nx: int
    ny: int
    nz: int
    h: float
    dt: float
    nt: int
    order: int
    f0: float
    nshots: int
    src: np.ndarray          # int64 [nshots, nsrc] flat indices
    rec: np.ndarray          # int64 [nshots, nrec] flat indices
    vel_true: np.ndarray     # float32 [nz, (ny,) nx]  m/s
    vel0: np.ndarray         # float32, the model the gradient is taken at
    wavelet: np.ndarray      # float32 [nshots, nt, nsrc]
    r: int = 4
    probe_kind: str = "rademacher"
    seed: int = DEFAULT_SEED
    T: int = 32
    sponge: int = 0           # absorbing layer width in cells on every face but the top (0: none)
    sponge_eta: float = 0.0   # its peak damping [1/s]

    @property
    def N(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def nsrc(self) -> int:
        return int(self.src.shape[1])

    @property
    def nrec(self) -> int:
        return int(self.rec.shape[1])

    def describe(self) -> dict:
        return {
            "workload": self.name, "ndim": self.ndim,
            "grid": [self.nz, self.ny, self.nx] if self.ndim == 3 else [self.nz, self.nx],
            "h_m": self.h, "dt_s": self.dt, "nt": self.nt, "order": self.order,
            "f0_hz": self.f0, "shots": self.nshots, "nrec": self.nrec,
            "r": self.r, "probes": self.probe_kind, "T": self.T, "seed": self.seed,
        }


# ----------------------------------------------------------------- wavelet
def ricker(nt: int, dt: float, f0: float, t0: Optional[float] = None) -> np.ndarray:
    """Ricker wavelet w(t) = (1 - 2 pi^2 f0^2 tau^2) exp(-pi^2 f0^2 tau^2),
    tau = t*dt - t0, sampled at t = 0..nt-1 (float64, peak amplitude 1).
    The delay defaults to t0 = 1/f0."""
    if t0 is None:
        t0 = 1.0 / f0
    tau = np.arange(nt, dtype=np.float64) * dt - t0
    a = (math.pi * f0 * tau) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def _wavelets(nshots: int, nsrc: int, nt: int, dt: float, f0: float) -> np.ndarray:
    w = ricker(nt, dt, f0).astype(np.float32)
    return np.ascontiguousarray(np.broadcast_to(w[None, :, None], (nshots, nt, nsrc)))


# ----------------------------------------------------------------- indexing
def flat_index(nx: int, ny: int, z, y, x) -> np.ndarray:
    return (np.asarray(z, np.int64) * ny + np.asarray(y, np.int64)) * nx + np.asarray(x, np.int64)


def surface_receivers_2d(nx: int, row: int = 0, stride: int = 1) -> np.ndarray:
    xs = np.arange(0, nx, stride)
    return flat_index(nx, 1, row, 0, xs)


def surface_receivers_3d(nx: int, ny: int, row: int = 0, stride: int = 1) -> np.ndarray:
    ys, xs = np.meshgrid(np.arange(0, ny, stride), np.arange(0, nx, stride), indexing="ij")
    return flat_index(nx, ny, row, ys.ravel(), xs.ravel())


# ----------------------------------------------------------------- models
def two_layer_2d(nz: int, nx: int, v_top: float, v_bot: float, iface_row: int) -> np.ndarray:
    v = np.full((nz, nx), v_top, dtype=np.float64)
    v[iface_row:, :] = v_bot
    return v.astype(np.float32)


def _smooth_random_field(shape, sigma: float, seed: int) -> np.ndarray:
    """i.i.d. normal field from numpy's PCG64 stream, Gaussian-filtered and
    scaled to unit max |value|."""
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    f = gaussian_filter(rng.standard_normal(shape), sigma=sigma, mode="reflect")
    return f / np.max(np.abs(f))


def gradient_lens_2d(nz: int, nx: int, seed: int, vmin=1500.0, vmax=4500.0,
                     perturb=0.05, sigma=4.0, lens_dv=800.0, lens_centre=(0.45, 0.60),
                     lens_axes=(15.0, 60.0), vclip: Optional[float] = None,
                     background_only: bool = False) -> np.ndarray:
    """Smooth linear-in-depth background vmin..vmax, times (1 + perturb*field)
    with a Gaussian-filtered random field, plus an elliptic high-velocity
    lens (centre as fractions of (z, x); semi-axes in cells)."""
    z = np.arange(nz, dtype=np.float64)[:, None] / max(nz - 1, 1)
    v = np.broadcast_to(vmin + (vmax - vmin) * z, (nz, nx)).copy()
    if not background_only:
        v *= 1.0 + perturb * _smooth_random_field((nz, nx), sigma, seed)
        zc, xc = lens_centre[0] * (nz - 1), lens_centre[1] * (nx - 1)
        zz, xx = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
        inside = ((zz - zc) / lens_axes[0]) ** 2 + ((xx - xc) / lens_axes[1]) ** 2 <= 1.0
        v[inside] += lens_dv
    if vclip is not None:
        v = np.minimum(v, vclip)
    return v.astype(np.float32)


def layered_3d(n: int, seed: int, nlayers=8, vmin=1500.0, vmax=4000.0, blob_sigma=20.0,
               blob_amp=0.10, with_blob=True, shape=None) -> np.ndarray:
    """Flat layers vmin..vmax (equal thickness) with one Gaussian anomaly of
    relative amplitude +-blob_amp at a seeded centre."""
    nz, ny, nx = shape if shape is not None else (n, n, n)
    layer = np.minimum((np.arange(nz) * nlayers) // nz, nlayers - 1)
    vz = vmin + (vmax - vmin) * layer / max(nlayers - 1, 1)
    v = np.broadcast_to(vz[:, None, None], (nz, ny, nx)).astype(np.float64)
    if with_blob:
        rng = np.random.default_rng(seed)
        c = rng.uniform(0.3, 0.7, size=3) * np.array([nz, ny, nx])
        sign = 1.0 if rng.uniform() < 0.5 else -1.0
        zz = (np.arange(nz) - c[0])[:, None, None] ** 2
        yy = (np.arange(ny) - c[1])[None, :, None] ** 2
        xx = (np.arange(nx) - c[2])[None, None, :] ** 2
        v = v * (1.0 + sign * blob_amp * np.exp(-(zz + yy + xx) / (2.0 * blob_sigma ** 2)))
    return np.ascontiguousarray(v.astype(np.float32))


# ----------------------------------------------------------------- configs
def config1(seed: int = DEFAULT_SEED) -> Workload:
    """2-D 101x101 at 10 m, two layers 1.5/2.5 km/s (interface at 250 m, so
    that its reflection arrives at about 0.41 s, inside the 0.5 s record),
    nt=500, dt=1 ms, 10 Hz Ricker, source at (500 m, 20 m), 101 surface
    receivers, 4th order, r=4 Rademacher, probe window T=128.  Gradient
    taken at homogeneous 1.5 km/s."""
    nx = nz = 101
    nt, dt, f0 = 500, 1e-3, 10.0
    return Workload(
        name="2d_101x101_nt500_o4_r4", ndim=2, nx=nx, ny=1, nz=nz, h=10.0, dt=dt, nt=nt,
        order=4, f0=f0, nshots=1,
        src=flat_index(nx, 1, 2, 0, 50).reshape(1, 1),
        rec=surface_receivers_2d(nx).reshape(1, -1),
        vel_true=two_layer_2d(nz, nx, 1500.0, 2500.0, 25),
        vel0=np.full((nz, nx), 1500.0, np.float32),
        wavelet=_wavelets(1, 1, nt, dt, f0), r=4, probe_kind="rademacher", seed=seed, T=128)


def config2(seed: int = DEFAULT_SEED, nt: int = 3000, nshots: int = 16) -> Workload:
    """2-D 601x201 at 12.5 m, gradient background 1.5-4.5 km/s + 5 % smooth
    random perturbation + elliptic lens, nt=3000, dt=1 ms, 8 Hz, 16 shots at
    25 m depth, 601 surface receivers, 8th order, r=16 Gaussian probes,
    probe window T=128."""
    nx, nz, h, dt, f0 = 601, 201, 12.5, 1e-3, 8.0
    vclip = 0.9 * CFL_LIMIT[(2, 8)] * h / dt
    xs = np.round(np.linspace(0, nx - 1, nshots + 2)[1:-1]).astype(np.int64)
    return Workload(
        name=f"2d_601x201_nt{nt}_o8_r16_{nshots}shots", ndim=2, nx=nx, ny=1, nz=nz, h=h, dt=dt,
        nt=nt, order=8, f0=f0, nshots=nshots,
        src=flat_index(nx, 1, 2, 0, xs).reshape(nshots, 1),
        rec=np.broadcast_to(surface_receivers_2d(nx), (nshots, nx)).copy(),
        vel_true=gradient_lens_2d(nz, nx, seed, vclip=vclip),
        vel0=gradient_lens_2d(nz, nx, seed, vclip=vclip, background_only=True),
        wavelet=_wavelets(nshots, 1, nt, dt, f0), r=16, probe_kind="gaussian", seed=seed, T=128)


def config3(seed: int = DEFAULT_SEED, n: int = 256, nt: int = 2000, T: int = 32,
            r: int = 32, rec_stride: int = 1) -> Workload:
    """3-D n^3 at 10 m, 8 layers 1.5-4.0 km/s + seeded Gaussian anomaly
    (sigma 20 cells, +-10 %), nt=2000, dt=0.8 ms, 10 Hz, one shot at
    (n/2, n/2, depth 2), n x n surface receivers, 8th order, r=32
    Rademacher, window T=32.  Gradient taken at the layered model."""
    dt, f0 = 8e-4, 10.0
    return Workload(
        name=f"3d_{n}cubed_nt{nt}_o8_r{r}_T{T}", ndim=3, nx=n, ny=n, nz=n, h=10.0, dt=dt,
        nt=nt, order=8, f0=f0, nshots=1,
        src=flat_index(n, n, 2, n // 2, n // 2).reshape(1, 1),
        rec=surface_receivers_3d(n, n, stride=rec_stride).reshape(1, -1),
        vel_true=layered_3d(n, seed),
        vel0=layered_3d(n, seed, with_blob=False),
        wavelet=_wavelets(1, 1, nt, dt, f0), r=r, probe_kind="rademacher", seed=seed, T=T)


def config4(seed: int = DEFAULT_SEED, nt: int = 2500, nshots: int = 8) -> Workload:
    """Batch of 8 shots on 2-D 801x301 at 10 m, nt=2500, dt=1 ms, 8 Hz,
    8th order, r=16 Gaussian probes, probe window T=128, model generator of
    config 2."""
    nx, nz, h, dt, f0 = 801, 301, 10.0, 1e-3, 8.0
    vclip = 0.9 * CFL_LIMIT[(2, 8)] * h / dt
    xs = np.round(np.linspace(0, nx - 1, nshots + 2)[1:-1]).astype(np.int64)
    return Workload(
        name=f"2d_801x301_nt{nt}_o8_r16_{nshots}shots", ndim=2, nx=nx, ny=1, nz=nz, h=h, dt=dt,
        nt=nt, order=8, f0=f0, nshots=nshots,
        src=flat_index(nx, 1, 2, 0, xs).reshape(nshots, 1),
        rec=np.broadcast_to(surface_receivers_2d(nx), (nshots, nx)).copy(),
        vel_true=gradient_lens_2d(nz, nx, seed, vclip=vclip),
        vel0=gradient_lens_2d(nz, nx, seed, vclip=vclip, background_only=True),
        wavelet=_wavelets(nshots, 1, nt, dt, f0), r=16, probe_kind="gaussian", seed=seed, T=128)


def small_2d(nx=67, nz=45, nt=160, order=8, nshots=1, r=4, probe_kind="rademacher",
             h=10.0, dt=1e-3, f0=15.0, seed=DEFAULT_SEED, T=32, nrec=None) -> Workload:
    """Small 2-D case (several tiles, ragged edges) for checker-sized parity tests."""
    vclip = 0.8 * CFL_LIMIT[(2, order)] * h / dt
    vt = gradient_lens_2d(nz, nx, seed, vmin=1500.0, vmax=3000.0, lens_axes=(nz / 8, nx / 6),
                          sigma=2.0, vclip=vclip)
    v0 = gradient_lens_2d(nz, nx, seed, vmin=1500.0, vmax=3000.0, background_only=True, vclip=vclip)
    xs = np.round(np.linspace(0, nx - 1, nshots + 2)[1:-1]).astype(np.int64)
    rstride = 1 if nrec is None else max(1, nx // nrec)
    rec = surface_receivers_2d(nx, row=1, stride=rstride)
    return Workload(
        name=f"2d_{nx}x{nz}_nt{nt}_o{order}", ndim=2, nx=nx, ny=1, nz=nz, h=h, dt=dt, nt=nt,
        order=order, f0=f0, nshots=nshots, src=flat_index(nx, 1, 3, 0, xs).reshape(nshots, 1),
        rec=np.broadcast_to(rec, (nshots, rec.size)).copy(), vel_true=vt, vel0=v0,
        wavelet=_wavelets(nshots, 1, nt, dt, f0), r=r, probe_kind=probe_kind, seed=seed, T=T)


def small_3d(nx=36, ny=22, nz=28, nt=90, order=8, nshots=1, r=4, probe_kind="rademacher",
             h=10.0, dt=1e-3, f0=20.0, seed=DEFAULT_SEED, T=32, rec_stride=3) -> Workload:
    """Small 3-D case with unequal, ragged dimensions for checker-sized tests."""
    vclip = 0.8 * CFL_LIMIT[(3, order)] * h / dt
    vt = np.minimum(layered_3d(0, seed, nlayers=4, vmin=1500.0, vmax=3000.0,
                               blob_sigma=4.0, shape=(nz, ny, nx)), vclip).astype(np.float32)
    # background 5 % slow everywhere, so the residual is a physical signal from
    # the first arrival on (not only the anomaly's late reflection)
    v0 = (0.95 * np.minimum(layered_3d(0, seed, nlayers=4, vmin=1500.0, vmax=3000.0, with_blob=False,
                                       shape=(nz, ny, nx)), vclip)).astype(np.float32)
    pos = np.round(np.linspace(0, nx - 1, nshots + 2)[1:-1]).astype(np.int64)
    src = flat_index(nx, ny, 3, ny // 2, pos).reshape(nshots, 1)
    rec = surface_receivers_3d(nx, ny, row=1, stride=rec_stride)
    return Workload(
        name=f"3d_{nz}x{ny}x{nx}_nt{nt}_o{order}", ndim=3, nx=nx, ny=ny, nz=nz, h=h, dt=dt,
        nt=nt, order=order, f0=f0, nshots=nshots, src=src,
        rec=np.broadcast_to(rec, (nshots, rec.size)).copy(), vel_true=vt, vel0=v0,
        wavelet=_wavelets(nshots, 1, nt, dt, f0), r=r, probe_kind=probe_kind, seed=seed, T=T)


def synthetic_data(nshots: int, nt: int, nrec: int, seed: int, amp: float = 1e-3) -> np.ndarray:
    """Seeded band-limited pseudo-observed data [nshots, nt, nrec] (float32),
    for full-size runs whose observed data need not come from a model."""
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((nshots, nt, nrec))
    k = np.exp(-0.5 * (np.arange(-8, 9) / 3.0) ** 2)
    from scipy.ndimage import convolve1d
    d = convolve1d(d, k / k.sum(), axis=1, mode="constant")
    return (amp * d).astype(np.float32)


def sponge_eta_for(vmax: float, width: int, h: float, reflection: float = 1e-3) -> float:
    """Peak damping of a quadratic absorbing layer of `width` cells: the
    usual choice 3 v ln(1/R) / (2 L) for a target reflection R over a layer
    of thickness L = width * h."""
    return 3.0 * vmax * np.log(1.0 / reflection) / (2.0 * width * h)


def with_sponge(w: Workload, width: int, reflection: float = 1e-3) -> Workload:
    """The workload with an absorbing layer of `width` cells on every face but
    the top (the free surface, where sources and receivers sit)."""
    import dataclasses
    vmax = float(max(w.vel_true.max(), w.vel0.max()))
    return dataclasses.replace(w, sponge=int(width), sponge_eta=sponge_eta_for(vmax, width, w.h, reflection))
