"""The fp32 arithmetic form of the sweeps, checked on the CPU.

Emulating the sweeps' fp32 operation order in numpy (exact products, one
rounding per FMA, fp32 sums) on a 201 x 101 2-D case over 2000 steps, against
the FP64 oracle:
  * the centred form the kernels use, sum_k w_k (neighbour sum - 2 ndim u)
    with the -2 ndim u in one FMA, stays within the trace bound (1e-5), like
    the per-neighbour difference form;
  * the plain sum form with an fp32 w_0 drifts past 2e-5: the rounded
    weights leave a zero-order term that grows with the number of steps.
The GPU parity tests check the kernels themselves (configs 2 and 4 over
their full time axes)."""
import numpy as np
import pytest

import oracle
from paper_2104_00794_gb300 import workloads as wl

F32, F64 = np.float32, np.float64
R = H = 4
W32 = np.array([-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0], F32)


def _fma(a, b, c):  # one rounding to fp32 (the product of two fp32 values is exact in fp64)
    return (np.asarray(a, F64) * np.asarray(b, F64) + np.asarray(c, F64)).astype(F32)


def _neighbours(u, k, nz, nx):
    return (u[H:-H, H + k:nx + H + k], u[H:-H, H - k:nx + H - k],
            u[H + k:nz + H + k, H:-H], u[H - k:nz + H - k, H:-H])


def _centred(u, nz, nx):
    c = u[H:-H, H:-H]
    s = np.zeros_like(c)
    for k in range(1, R + 1):
        a, b, d, e = _neighbours(u, k, nz, nx)
        total = ((a + b).astype(F32) + (d + e).astype(F32)).astype(F32)
        s = _fma(W32[k], _fma(F32(-4), c, total), s)
    return s


def _difference(u, nz, nx):
    c = u[H:-H, H:-H]
    s = np.zeros_like(c)
    for k in range(1, R + 1):
        a, b, d, e = _neighbours(u, k, nz, nx)
        t = (((a - c) + (b - c)).astype(F32) + ((d - c) + (e - c)).astype(F32)).astype(F32)
        s = _fma(W32[k], t, s)
    return s


def _plain_sum(u, nz, nx):
    c = u[H:-H, H:-H]
    s = (W32[0] * F32(2) * c).astype(F32)
    for k in range(1, R + 1):
        a, b, d, e = _neighbours(u, k, nz, nx)
        s = _fma(W32[k], ((a + b).astype(F32) + (d + e).astype(F32)).astype(F32), s)
    return s


def _traces(w, form):
    """Leapfrog with the kernels' step order: c2 formed in fp64 and rounded
    once, res = fma(c2, S(u), 2u - u_old), then the source injection."""
    nz, nx, nt = w.nz, w.nx, w.nt
    vel = w.vel_true.astype(F64)
    c2 = (w.dt * w.dt * vel * vel / (w.h * w.h)).astype(F32)
    sz, sx = divmod(int(w.src[0, 0]), nx)
    cinj = F32(w.dt * w.dt * vel[sz, sx] ** 2)
    rz, rx = np.divmod(w.rec[0], nx)
    q = w.wavelet[0, :, 0].astype(F32)
    u0 = np.zeros((nz + 2 * H, nx + 2 * H), F32)
    u1 = u0.copy()
    d = np.zeros((nt, len(rx)))
    for t in range(1, nt - 1):
        c = u1[H:-H, H:-H]
        res = _fma(c2, form(u1, nz, nx), (F32(2) * c - u0[H:-H, H:-H]).astype(F32))
        res[sz, sx] = F32(res[sz, sx] + F32(cinj * q[t]))
        d[t] = u1[H + rz, H + rx]
        u2 = np.zeros_like(u1)
        u2[H:-H, H:-H] = res
        u0, u1 = u1, u2
    d[nt - 1] = u1[H + rz, H + rx]
    return d


@pytest.fixture(scope="module")
def case():
    w = wl.small_2d(nx=201, nz=101, nt=2000, order=8, nshots=1, h=12.5, dt=1e-3, f0=8.0)
    return w, oracle.batch_forward(w, w.vel_true)[0]


def _err(d, ref):
    return float(np.linalg.norm(d - ref) / np.linalg.norm(ref))


def test_centred_form_does_not_drift(case):
    w, ref = case
    e_cent = _err(_traces(w, _centred), ref)
    e_diff = _err(_traces(w, _difference), ref)
    assert e_cent <= 1e-5, e_cent
    assert e_cent <= 1.5 * e_diff, (e_cent, e_diff)


def test_plain_sum_form_drifts(case):
    w, ref = case
    e_sum = _err(_traces(w, _plain_sum), ref)
    assert e_sum >= 2e-5, e_sum  # the failure mode the centred form avoids
