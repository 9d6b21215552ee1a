"""Pins of the oracle's imaging conditions (§Imaging conditions, Eq. 5).

What fixes them independently of the code under test:
  * the centred first-derivative weights: the published values (Fornberg
    1988, Table 1) and exactness on polynomials up to the stencil's order;
    the same recursion at m = 2 reproduces the C oracle's second-derivative
    table (two implementations);
  * the derivative of a linear field is its slope away from the boundary;
  * Eq. 5 with Q = I (r = nt): the condition applied to the probed fields
    equals the condition applied at every time step -- two different code
    paths (per-step products vs. products of accumulated fields);
  * unbiasedness: the mean over many Rademacher draws converges to the
    per-step image at the 1/sqrt(draws) rate (a dropped scale, a lost time
    shift or a wrong index would leave a bias).
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2104_00794_gb300 import workloads as wl


def test_first_derivative_weights_published_values():
    assert np.allclose(oracle.fd_weights_first(4), [2 / 3, -1 / 12], rtol=0, atol=1e-15)
    assert np.allclose(oracle.fd_weights_first(8), [4 / 5, -1 / 5, 4 / 105, -1 / 280], rtol=0, atol=1e-15)


@pytest.mark.parametrize("order", [4, 8])
def test_first_derivative_exact_on_polynomials(order):
    c = oracle.fd_weights_first(order)
    R = c.size
    for p in range(order + 1):  # d/dx x^p at 0 is 1 for p = 1, else 0
        val = sum(c[k - 1] * (Fraction(k) ** p - Fraction(-k) ** p) for k in range(1, R + 1))
        assert abs(float(val) - (1.0 if p == 1 else 0.0)) < 1e-13, p


@pytest.mark.parametrize("order", [4, 8])
def test_second_derivative_recursion_matches_c_table(order):
    R = order // 2
    w = oracle.fornberg(2, 0.0, np.arange(-R, R + 1, dtype=np.float64))
    assert np.allclose(w[R:], oracle.fd_weights(order), rtol=0, atol=1e-13)


def test_derivative_of_linear_field():
    g = oracle.make_grid(3, 20, 14, 16, 5.0, 1e-3, 10, 8)
    z, y, x = np.meshgrid(np.arange(16), np.arange(14), np.arange(20), indexing="ij")
    f = 3.0 * z * g.h - 2.0 * y * g.h + 0.5 * x * g.h
    R = 4
    inner = (slice(R, -R),) * 3
    for ax, slope in enumerate([3.0, -2.0, 0.5]):
        d = oracle._derivative(g, f, ax)
        assert np.allclose(d[inner], slope, rtol=0, atol=1e-10)


def _case(ndim):
    if ndim == 2:
        w = wl.small_2d(nx=40, nz=30, nt=60, order=8, nshots=1)
    else:
        w = wl.small_3d(nx=18, ny=14, nz=16, nt=50, order=4, nshots=1)
    s = wl.synthetic_data(1, w.nt, w.nrec, seed=11)[0].astype(np.float64)
    return w, oracle.grid_of(w), s


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("cond", ["correlation", "gradient"])
def test_identity_probes_commute(ndim, cond):
    """Eq. 5 with Q = I: D applied to the probed fields = D applied per step."""
    w, g, s = _case(ndim)
    full = oracle.image_full(g, w.src[0], w.rec[0], w.vel0, w.wavelet[0], s, cond)
    Q = oracle.probes("identity", g.nt, g.nt, 0)
    probed = oracle.image_probed(g, w.src[0], w.rec[0], w.vel0, w.wavelet[0], s, Q, 1.0, cond)
    assert np.linalg.norm(full) > 0
    assert np.linalg.norm(probed - full) <= 1e-10 * np.linalg.norm(full)


@pytest.mark.parametrize("cond", ["correlation", "gradient"])
def test_probed_image_unbiased(cond):
    w, g, s = _case(2)
    full = oracle.image_full(g, w.src[0], w.rec[0], w.vel0, w.wavelet[0], s, cond)
    M, r = 120, 4
    draws = np.array([oracle.image_probed(g, w.src[0], w.rec[0], w.vel0, w.wavelet[0], s,
                                          oracle.probes("rademacher", g.nt, r, 1000 + m), 1.0 / r, cond)
                      for m in range(M)])
    single = np.sqrt(np.mean(np.sum((draws - full) ** 2, axis=1)))
    err_mean = np.linalg.norm(draws.mean(axis=0) - full)
    assert single > 0.05 * np.linalg.norm(full)  # a single draw is noisy
    assert err_mean <= 3.0 * single / np.sqrt(M)  # the mean converges to the per-step image
