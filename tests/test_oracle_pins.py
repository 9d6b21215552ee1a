"""Pins of the FP64 oracle against what the paper and mathematics fix.

None of these compares the oracle with itself: each check is a textbook
value, a closed form, an exact algebraic identity or a statistical law that
a wrong term, sign, index or scale in ``oracle/tp_oracle.c`` would break.

  * FD weights           -> Fornberg (1988) table, polynomial exactness
  * SplitMix64           -> published reference outputs
  * F / F^T (Alg. 1 l.1, l.5) -> dot-product test <Fq, d> = <q, F^T d>
  * dJ/dm (Eq. 2, Eq. 3) -> Taylor test: remainder O(h^2)
  * amplitude/kinematics -> 3-D and 2-D homogeneous Green's functions
  * Algorithm 1 / Eq. 4  -> identity probes (Q = I, r = nt) give Eq. 3 exactly,
                            folded and unfolded forms agree,
                            unbiasedness with the closed-form variance (Eq. 1)
  * probes (Eq. 1)       -> E[z z^T] = I statistics, exact float32 values
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2104_00794_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]


# ------------------------------------------------------------------ weights
def test_fd_weights_match_published_table():
    for line in _golden_lines("fd_weights.txt"):
        head, vals = line.split(":")
        order = int(head.split()[1])
        expect = [float(Fraction(v)) for v in vals.split()]
        np.testing.assert_allclose(oracle.fd_weights(order), expect, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("ndim,order", [(2, 4), (2, 8), (3, 4), (3, 8)])
def test_laplacian_exact_on_polynomials(ndim, order):
    """A 2k-order centred stencil differentiates x^p exactly for p <= k+1."""
    R = order // 2
    nx, ny, nz = (21, 1, 19) if ndim == 2 else (17, 15, 13)
    h = 0.5
    g = oracle.make_grid(ndim, nx, ny, nz, h, 1e-3, 3, order)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X, Y, Z = (x - nx / 2) * h, (y - ny / 2) * h, (z - nz / 2) * h
    inner = ((x >= R) & (x < nx - R) & (z >= R) & (z < nz - R))
    if ndim == 3:
        inner &= (y >= R) & (y < ny - R)
    for p in range(0, order + 2):
        u = X ** p + 0.5 * Z ** p + ((0.25 * Y ** p) if ndim == 3 else 0.0)
        d2 = lambda A: p * (p - 1) * A ** (p - 2) if p >= 2 else 0.0 * A
        expect = d2(X) + 0.5 * d2(Z) + ((0.25 * d2(Y)) if ndim == 3 else 0.0)
        got = oracle.laplacian(g, u).reshape(u.shape)
        scale = max(1.0, float(np.max(np.abs(expect[inner]))))
        assert np.max(np.abs(got[inner] - expect[inner])) <= 1e-9 * scale, p
    # one degree more is no longer exact: the stencil order is exactly 2k
    p = order + 2
    u = X ** p
    got = oracle.laplacian(g, u).reshape(u.shape)
    expect = p * (p - 1) * X ** (p - 2)
    assert np.max(np.abs(got[inner] - expect[inner])) > 1e-6


# ------------------------------------------------------------------ probes
def test_splitmix64_reference_outputs():
    expect = [int(v) for v in _golden_lines("splitmix64_seed1234567.txt")]
    got = [oracle.splitmix64(1234567, n) for n in range(1, 6)]
    assert got == expect


def test_rademacher_probes():
    nt, r = 600, 16
    Z = oracle.probes("rademacher", nt, r, 7, 0)
    assert set(np.unique(Z)) == {-1.0, 1.0}
    # deterministic, shot-dependent, seed-dependent
    assert np.array_equal(Z, oracle.probes("rademacher", nt, r, 7, 0))
    assert not np.array_equal(Z, oracle.probes("rademacher", nt, r, 7, 1))
    assert not np.array_equal(Z, oracle.probes("rademacher", nt, r, 8, 0))
    # prefix property: row t does not depend on nt or on r
    assert np.array_equal(Z[:100, :4], oracle.probes("rademacher", 100, 4, 7, 0))
    # each column has a fair +-1 balance (|mean| < 4 sigma)
    assert np.all(np.abs(Z.mean(axis=0)) < 4.0 / math.sqrt(nt))


def test_gaussian_probes_irwin_hall_moments():
    nt, r = 4000, 32
    Z = oracle.probes("gaussian", nt, r, 11, 3)
    # every value is exactly a float32 and an odd multiple of 2^-21
    assert np.array_equal(Z.astype(np.float32).astype(np.float64), Z)
    k = Z * 2.0 ** 21
    assert np.array_equal(k, np.round(k)) and np.all(np.mod(np.round(k), 2) == 1)
    assert np.max(np.abs(Z)) <= 6.0
    n = Z.size
    assert abs(Z.mean()) < 4.0 / math.sqrt(n)
    assert abs(Z.var() - 1.0) < 4.0 * math.sqrt(2.0 / n)
    # Irwin-Hall(12) kurtosis 3 - 6/(5*12) = 2.9 (a sum of fewer or more
    # uniforms, or a true Gaussian, would give a different value)
    kurt = np.mean(Z ** 4) / np.mean(Z ** 2) ** 2
    assert abs(kurt - 2.9) < 0.04


def test_identity_probes():
    Z = oracle.probes("identity", 9, 9, 0, 0)
    assert np.array_equal(Z, np.eye(9))
    with pytest.raises(ValueError):
        oracle.probes("identity", 9, 8, 0, 0)


@pytest.mark.parametrize("kind,fourth", [("rademacher", 1.0), ("gaussian", 2.9)])
def test_probe_outer_product_crosstalk(kind, fourth):
    """||Z Z^T / r - I||_F^2 has expectation (nt^2 - nt)/r + nt (E z^4 - 1)/r
    (the cross-talk studied in the paper's probing-vector figure)."""
    nt = 200
    for r in (4, 16, 64):
        vals = []
        for seed in range(20):
            Z = oracle.probes(kind, nt, r, seed, 0)
            vals.append(np.sum((Z @ Z.T / r - np.eye(nt)) ** 2))
        expect = (nt * nt - nt) / r + nt * (fourth - 1.0) / r
        assert abs(np.mean(vals) / expect - 1.0) < 0.05, (r, np.mean(vals), expect)


# ------------------------------------------------------------------ operators
def _rand_case(ndim, order, nt=120, seed=0):
    rng = np.random.default_rng(seed)
    if ndim == 2:
        w = wl.small_2d(nx=33, nz=27, nt=nt, order=order, nrec=11)
    else:
        w = wl.small_3d(nx=17, ny=13, nz=15, nt=nt, order=order, rec_stride=4)
    return w, rng


@pytest.mark.parametrize("ndim,order", [(2, 4), (2, 8), (3, 4), (3, 8)])
def test_dot_product_adjoint(ndim, order):
    """<F q, d> = <q, F^T d> for random q, d: F^T is the exact transpose."""
    w, rng = _rand_case(ndim, order)
    g = oracle.grid_of(w)
    src = np.array([w.src[0, 0], w.src[0, 0] + 3, w.src[0, 0] + 5 * w.nx * w.ny])
    q = rng.standard_normal((w.nt, src.size))
    d = rng.standard_normal((w.nt, w.nrec))
    Fq = oracle.forward(g, src, w.rec[0], w.vel_true, q)
    Ftd = oracle.adjoint(g, src, w.rec[0], w.vel_true, d)
    lhs, rhs = np.sum(Fq * d), np.sum(q * Ftd)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def test_forward_is_linear_and_causal():
    w, rng = _rand_case(2, 8, nt=80)
    g = oracle.grid_of(w)
    q1 = rng.standard_normal((w.nt, 1))
    q2 = rng.standard_normal((w.nt, 1))
    d1 = oracle.forward(g, w.src[0], w.rec[0], w.vel_true, q1)
    d2 = oracle.forward(g, w.src[0], w.rec[0], w.vel_true, q2)
    d12 = oracle.forward(g, w.src[0], w.rec[0], w.vel_true, 2 * q1 - q2)
    np.testing.assert_allclose(d12, 2 * d1 - d2, rtol=1e-12, atol=1e-12 * np.abs(d12).max())
    # q[t] first reaches the data at level t+1 (two levels of zeros first)
    qi = np.zeros((w.nt, 1))
    qi[10, 0] = 1.0
    di, u = oracle.forward(g, w.src[0], w.rec[0], w.vel_true, qi, keep_history=True)
    assert np.all(u[:11] == 0.0)
    assert u[11, w.src[0, 0]] != 0.0


# ------------------------------------------------------------------ gradient
@pytest.mark.parametrize("order", [4, 8])
def test_taylor_gradient(order):
    """J(m + h dm) - J(m) - h <g, dm> = O(h^2) (g = dJ/dm of Eq. 2)."""
    w = wl.small_2d(nx=41, nz=33, nt=180, order=order, nrec=20)
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
    assert abs(J0 - J(m0)) <= 1e-12 * J0
    gdm = float(np.sum(grad.reshape(m0.shape) * dm))
    e1, e2 = [], []
    hs = [0.5 ** k for k in range(1, 6)]
    for hh in hs:
        Jh = J(m0 + hh * dm)
        e1.append(abs(Jh - J0))
        e2.append(abs(Jh - J0 - hh * gdm))
    e1, e2 = np.array(e1), np.array(e2)
    s1 = np.log2(e1[:-1] / e1[1:])
    s2 = np.log2(e2[:-1] / e2[1:])
    assert np.all(np.abs(s1 - 1.0) < 0.2), s1
    assert np.all(np.abs(s2 - 2.0) < 0.2), s2
    assert np.all(e2 < 0.2 * e1)


def test_gradient_sign_descends():
    """A small step along -g lowers the misfit (Eq. 3 carries a minus sign)."""
    w = wl.small_2d(nx=41, nz=33, nt=180, order=8, nrec=20)
    g = oracle.grid_of(w)
    d_obs = oracle.forward(g, w.src[0], w.rec[0], w.vel_true, w.wavelet[0])
    m0 = 1.0 / w.vel0.astype(np.float64).ravel() ** 2
    grad, J0 = oracle.gradient_full(g, w.src[0], w.rec[0], w.vel0, w.wavelet[0], d_obs)
    step = 1e-3 * np.abs(m0).max() / np.abs(grad).max()
    d = oracle.forward(g, w.src[0], w.rec[0], 1.0 / np.sqrt(m0 - step * grad), w.wavelet[0])
    assert 0.5 * np.sum((d - d_obs) ** 2) < J0


# ------------------------------------------------------------------ Green's functions
def _trace_error(num, ana):
    return np.linalg.norm(num - ana) / np.linalg.norm(ana)


@pytest.mark.parametrize("order,tol", [(8, 0.01), (4, 0.01)])
def test_green_3d_homogeneous(order, tol):
    """m u_tt - Lap u = h^3 q(t) delta(x): u = h^3 q(t - r/c) / (4 pi r)."""
    n, h, c, dt, f0, nt = 61, 10.0, 2000.0, 1e-3, 15.0, 230
    g = oracle.make_grid(3, n, n, n, h, dt, nt, order)
    ctr = n // 2
    src = wl.flat_index(n, n, ctr, ctr, ctr)
    dist = 10
    rec = np.array([wl.flat_index(n, n, ctr, ctr, ctr + dist), wl.flat_index(n, n, ctr + dist, ctr, ctr)])
    q = wl.ricker(nt, dt, f0)[:, None]
    d = oracle.forward(g, [src], rec, np.full(n ** 3, c), q)
    t = np.arange(nt) * dt
    rr = dist * h
    ana = h ** 3 * np.interp(t - rr / c, t, q[:, 0], left=0.0) / (4 * math.pi * rr)
    for j in range(2):
        assert _trace_error(d[:, j], ana) < tol
    # a velocity 2 % off already shifts the arrival by more than the tolerance
    ana_bad = h ** 3 * np.interp(t - rr / (1.02 * c), t, q[:, 0], left=0.0) / (4 * math.pi * rr)
    assert _trace_error(d[:, 0], ana_bad) > tol


@pytest.mark.parametrize("order,tol", [(8, 0.015), (4, 0.015)])
def test_green_2d_homogeneous(order, tol):
    """m u_tt - Lap u = h^2 q(t) delta(x):
    u = h^2/(2 pi) int_0^{acosh(ct/r)} q(t - (r/c) cosh s) ds."""
    n, h, c, dt, f0, nt = 161, 10.0, 2000.0, 1e-3, 15.0, 320
    g = oracle.make_grid(2, n, 1, n, h, dt, nt, order)
    ctr = n // 2
    dist = 20
    src = wl.flat_index(n, 1, ctr, 0, ctr)
    rec = np.array([wl.flat_index(n, 1, ctr, 0, ctr + dist), wl.flat_index(n, 1, ctr - dist, 0, ctr)])
    qw = wl.ricker(nt, dt, f0)
    d = oracle.forward(g, [src], rec, np.full(n * n, c), qw[:, None])
    rr = dist * h
    t0 = 1.0 / f0
    ricker = lambda tt: (1 - 2 * (math.pi * f0 * (tt - t0)) ** 2) * np.exp(-(math.pi * f0 * (tt - t0)) ** 2)
    ana = np.zeros(nt)
    for it in range(nt):
        tt = it * dt
        if c * tt <= rr:
            continue
        smax = math.acosh(c * tt / rr)
        s = np.linspace(0.0, smax, 4001)
        ana[it] = h ** 2 / (2 * math.pi) * np.trapezoid(ricker(tt - rr / c * np.cosh(s)), s)
    for j in range(2):
        assert _trace_error(d[:, j], ana) < tol


# ------------------------------------------------------------------ Algorithm 1
def _grad_case(ndim=2, order=8, nt=100):
    if ndim == 2:
        w = wl.small_2d(nx=29, nz=23, nt=nt, order=order, nrec=10)
    else:
        w = wl.small_3d(nx=15, ny=12, nz=13, nt=nt, order=order, rec_stride=3)
    g = oracle.grid_of(w)
    d_obs = oracle.forward(g, w.src[0], w.rec[0], w.vel_true, w.wavelet[0])
    return w, g, d_obs


@pytest.mark.parametrize("ndim,order", [(2, 4), (2, 8), (3, 8)])
def test_identity_probes_give_full_gradient(ndim, order):
    """With Q = I (r = nt) and scale 1, Eq. 4 is Eq. 3 exactly."""
    w, g, d_obs = _grad_case(ndim, order)
    gf, Jf = oracle.gradient_full(g, w.src[0], w.rec[0], w.vel0, w.wavelet[0], d_obs)
    Q = oracle.probes("identity", w.nt, w.nt, 0, 0)
    for form in (0, 1):
        gp, Jp = oracle.gradient_probed(g, w.src[0], w.rec[0], w.vel0, w.wavelet[0], d_obs, Q, 1.0,
                                        form)
        assert Jp == pytest.approx(Jf, rel=1e-14)
        assert np.max(np.abs(gp - gf)) <= 1e-9 * np.max(np.abs(gf))


@pytest.mark.parametrize("kind", ["rademacher", "gaussian"])
def test_folded_probes_equal_unfolded(kind):
    """Folding the second time difference into Q is an exact rewrite."""
    w, g, d_obs = _grad_case(2, 8)
    Q = oracle.probes(kind, w.nt, 6, 3, 0)
    g0, _, u0, v0 = oracle.gradient_probed(g, w.src[0], w.rec[0], w.vel0, w.wavelet[0], d_obs, Q,
                                           1 / 6, 0, keep_acc=True)
    g1, _, u1, v1 = oracle.gradient_probed(g, w.src[0], w.rec[0], w.vel0, w.wavelet[0], d_obs, Q,
                                           1 / 6, 1, keep_acc=True)
    assert np.array_equal(v0, v1)
    assert np.max(np.abs(u0 - u1)) <= 1e-9 * np.max(np.abs(u0))
    assert np.max(np.abs(g0 - g1)) <= 1e-9 * np.max(np.abs(g0))


@pytest.mark.parametrize("kind,fourth", [("rademacher", 1.0), ("gaussian", 2.9)])
def test_probed_estimator_unbiased_with_closed_form_variance(kind, fourth):
    """Eq. 1: E[(z.a)(z.b)] = a.b, with per-probe variance
    |a|^2|b|^2 + (a.b)^2 + (E z^4 - 3) sum a_k^2 b_k^2.  The mean over S
    seeds must sit within its standard error of Eq. 3 at every point."""
    w, g, d_obs = _grad_case(2, 8, nt=90)
    nt, r, S = w.nt, 4, 120
    gf, _ = oracle.gradient_full(g, w.src[0], w.rec[0], w.vel0, w.wavelet[0], d_obs)
    d, u = oracle.forward(g, w.src[0], w.rec[0], w.vel0, w.wavelet[0], keep_history=True)
    _, lam = oracle.adjoint(g, w.src[0], w.rec[0], w.vel0, d - d_obs, keep_history=True)
    a = np.zeros_like(u)
    a[2:] = (u[2:] - 2 * u[1:-1] + u[:-2]) / w.dt ** 2
    a, b = a[2:], lam[2:]                       # levels k = 2..nt-1
    ab = np.sum(a * b, axis=0)
    np.testing.assert_allclose(-ab, gf, rtol=1e-9, atol=1e-9 * np.abs(gf).max())
    var1 = (np.sum(a * a, 0) * np.sum(b * b, 0) + ab ** 2 + (fourth - 3.0) * np.sum(a * a * b * b, 0))
    est = np.zeros(w.N)
    for seed in range(S):
        Q = oracle.probes(kind, nt, r, 1000 + seed, 0)
        gp, _ = oracle.gradient_probed(g, w.src[0], w.rec[0], w.vel0, w.wavelet[0], d_obs, Q, 1.0 / r)
        est += gp / S
    sd = np.sqrt(var1 / (r * S))
    keep = sd > 1e-6 * sd.max()
    zsc = (est[keep] - gf[keep]) / sd[keep]
    assert 0.6 < np.mean(zsc ** 2) < 1.5, np.mean(zsc ** 2)
    assert np.mean(np.abs(zsc) > 4.5) < 0.01


# ------------------------------------------------------------------ Eq. 6 (QR probes)
def _record(nt=160, seed=4):
    w = wl.small_2d(nx=61, nz=41, nt=nt, order=8, nrec=30)
    return w, oracle.forward(oracle.grid_of(w), w.src[0], w.rec[0], w.vel_true, w.wavelet[0])


def test_qr_probes_orthonormal_and_span_the_range():
    w, D = _record()
    r = 8
    Z = oracle.probes("rademacher", w.nt, r, 5, 0)
    Q = oracle.qr_probes(D, Z)
    assert Q.shape == (w.nt, r)
    np.testing.assert_allclose(Q.T @ Q, np.eye(r), atol=1e-12)
    Y = D @ (D.T @ Z)
    assert np.linalg.norm(Y - Q @ (Q.T @ Y)) <= 1e-10 * np.linalg.norm(Y)
    P = Q @ Q.T
    np.testing.assert_allclose(P @ P, P, atol=1e-12)           # an orthogonal projector
    # R = Q^T Y is upper triangular with a positive diagonal (sign convention)
    R = Q.T @ Y
    assert np.all(np.abs(np.tril(R, -1)) <= 1e-10 * np.abs(R).max()) and np.all(np.diag(R) > 0)


def test_qr_probes_capture_the_dominant_range():
    """The range finder approximates the span of the top singular vectors of
    D D^T (Halko et al.): with r a few above the numerical rank of a low-rank
    record, Q spans it to rounding; random +-1 probes of the same r carry the
    identity's cross-talk instead."""
    rng = np.random.default_rng(2)
    nt, nrec, k, r = 200, 40, 5, 12
    U = np.linalg.qr(rng.standard_normal((nt, k)))[0]
    D = U @ np.diag([50.0, 20.0, 10.0, 5.0, 2.0]) @ rng.standard_normal((k, nrec))
    Q = oracle.qr_probes(D, oracle.probes("rademacher", nt, r, 9, 0))
    assert np.linalg.norm(U - Q @ (Q.T @ U)) <= 1e-10
    # trace of D D^T estimated with the QR probes (scale 1) is exact here,
    # with Rademacher probes (scale 1/r) it is not
    A = D @ D.T
    assert np.trace(Q.T @ A @ Q) == pytest.approx(np.trace(A), rel=1e-10)
    Zr = oracle.probes("rademacher", nt, r, 9, 0)
    assert abs(np.trace(Zr.T @ A @ Zr) / r - np.trace(A)) > 1e-3 * np.trace(A)
