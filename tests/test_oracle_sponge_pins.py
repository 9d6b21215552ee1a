"""Pins of the oracle's absorbing sponge (damping m*eta*du/dt on every face
but the top free surface).

What fixes them independently of the code under test:
  * the adjoint stays the exact transpose of the damped scheme (dot test);
  * the gradient, with the damping term eta*du/dt added to the second time
    derivative, is the derivative of the misfit (Taylor test, slopes 1 and
    2); identity probes and folded probes reproduce it exactly;
  * the layer absorbs: in a homogeneous medium the energy left in the grid
    after the direct wave has reached the damped faces is a small fraction
    of the energy left with the rigid (zero) boundary alone, and the wave is
    unchanged before it reaches the layer (the damping is local).
"""
import numpy as np
import pytest

import oracle
from paper_2104_00794_gb300 import workloads as wl


def _sponged(w, width=8):
    return wl.with_sponge(w, width)


@pytest.mark.parametrize("ndim,order", [(2, 4), (2, 8), (3, 8)])
def test_dot_product_adjoint_with_sponge(ndim, order):
    rng = np.random.default_rng(17)
    if ndim == 2:
        w = wl.small_2d(nx=37, nz=29, nt=150, order=order)
    else:
        w = wl.small_3d(nx=19, ny=15, nz=17, nt=90, order=order, rec_stride=4)
    w = _sponged(w, 6)
    g = oracle.grid_of(w)
    q = rng.standard_normal((w.nt, w.nsrc))
    d = rng.standard_normal((w.nt, w.nrec))
    Fq = oracle.forward(g, w.src[0], w.rec[0], w.vel_true, q)
    Ftd = oracle.adjoint(g, w.src[0], w.rec[0], w.vel_true, d)
    lhs, rhs = np.sum(Fq * d), np.sum(q * Ftd)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def test_taylor_gradient_with_sponge():
    w = _sponged(wl.small_2d(nx=41, nz=33, nt=220, order=8, nrec=20), 8)
    g = oracle.grid_of(w)
    d_obs = oracle.forward(g, w.src[0], w.rec[0], w.vel_true, w.wavelet[0])
    m0 = 1.0 / w.vel0.astype(np.float64) ** 2
    rng = np.random.default_rng(5)
    from scipy.ndimage import gaussian_filter
    dm = gaussian_filter(rng.standard_normal(m0.shape), 2.0)
    dm *= 0.05 * np.abs(m0).max() / np.abs(dm).max()

    def J(m):
        d = oracle.forward(g, w.src[0], w.rec[0], 1.0 / np.sqrt(m), w.wavelet[0])
        return 0.5 * np.sum((d - d_obs) ** 2)

    grad, J0 = oracle.gradient_full(g, w.src[0], w.rec[0], 1.0 / np.sqrt(m0), w.wavelet[0], d_obs)
    gdm = float(np.sum(grad.reshape(m0.shape) * dm))
    # the undamped scheme's gradient is a plausible wrong answer: the test must reject it
    g_nodamp, _ = oracle.gradient_full(oracle.grid_of(wl.small_2d(nx=41, nz=33, nt=220, order=8, nrec=20)),
                                       w.src[0], w.rec[0], 1.0 / np.sqrt(m0), w.wavelet[0], d_obs)
    gdm_bad = float(np.sum(g_nodamp.reshape(m0.shape) * dm))
    e1, e2, e2_bad = [], [], []
    for hh in [0.5 ** k for k in range(1, 6)]:
        Jh = J(m0 + hh * dm)
        e1.append(abs(Jh - J0))
        e2.append(abs(Jh - J0 - hh * gdm))
        e2_bad.append(abs(Jh - J0 - hh * gdm_bad))
    e1, e2, e2_bad = np.array(e1), np.array(e2), np.array(e2_bad)
    assert np.all(np.abs(np.log2(e1[:-1] / e1[1:]) - 1.0) < 0.2)
    assert np.all(np.abs(np.log2(e2[:-1] / e2[1:]) - 2.0) < 0.2), np.log2(e2[:-1] / e2[1:])
    assert np.all(np.log2(e2_bad[:-1] / e2_bad[1:]) < 1.3)  # measured slope ~1


def test_identity_and_folded_probes_with_sponge():
    w = _sponged(wl.small_2d(nx=37, nz=29, nt=120, order=8), 6)
    g = oracle.grid_of(w)
    d_obs = oracle.forward(g, w.src[0], w.rec[0], w.vel_true, w.wavelet[0])
    gf, _ = oracle.gradient_full(g, w.src[0], w.rec[0], w.vel0, w.wavelet[0], d_obs)
    Q = oracle.probes("identity", w.nt, w.nt, 0, 0)
    for form in (0, 1):
        gp, _ = oracle.gradient_probed(g, w.src[0], w.rec[0], w.vel0, w.wavelet[0], d_obs, Q, 1.0, form)
        assert np.max(np.abs(gp - gf)) <= 1e-9 * np.max(np.abs(gf))
    Q = oracle.probes("gaussian", w.nt, 6, 3, 0)
    g0, _ = oracle.gradient_probed(g, w.src[0], w.rec[0], w.vel0, w.wavelet[0], d_obs, Q, 1 / 6, 0)
    g1, _ = oracle.gradient_probed(g, w.src[0], w.rec[0], w.vel0, w.wavelet[0], d_obs, Q, 1 / 6, 1)
    assert np.max(np.abs(g0 - g1)) <= 1e-9 * np.max(np.abs(g0))


def test_sponge_absorbs():
    """Homogeneous 2-D medium, source in the middle: after the direct wave has
    crossed the damped faces, the energy left with the sponge is a small
    fraction of the energy left without it (where it reflects)."""
    nx = nz = 121
    h, dt, v = 10.0, 1e-3, 2000.0
    nt = 1300  # 1.3 s: the direct wave and its free-surface reflection have reached the damped faces
    vel = np.full((nz, nx), v)
    src = np.array([60 * nx + 60])
    rec = np.array([60 * nx + 60])
    q = wl.ricker(nt, dt, 15.0)[:, None]
    out = {}
    for width in (0, 25):
        eta = wl.sponge_eta_for(v, width, h) if width else 0.0
        g = oracle.make_grid(2, nx, 1, nz, h, dt, nt, 8, width, eta)
        _, U = oracle.forward(g, src, rec, vel, q, keep_history=True)
        out[width] = U
    e_rigid = np.sum(out[0][-1] ** 2)
    e_sponge = np.sum(out[25][-1] ** 2)
    assert e_sponge < 1e-3 * e_rigid, e_sponge / e_rigid  # measured 2.2e-4
    # before the wave reaches the layer (25 cells = 250 m from the source-side faces
    # minus the layer: ~0.18 s) the two runs agree: the damping is local
    assert np.allclose(out[25][120], out[0][120], rtol=0, atol=1e-12 * np.abs(out[0][120]).max())
