"""The SPG optimiser of the FWI driver (host logic, numpy on the CPU).

On a box-constrained strictly convex quadratic the projected minimiser is
unique; SPG must reach it (checked against scipy's L-BFGS-B on the same
problem and by the projected-gradient optimality condition), its
nonmonotone line search must accept only points below the running maximum,
and a start at the solution must stop at once.
"""
import numpy as np
import pytest

from paper_2104_00794_gb300.fwi import spg


def _quadratic(n=40, seed=0):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, n))
    A = B @ B.T / n + 0.1 * np.eye(n)
    b = rng.standard_normal(n) * 3.0
    lo, hi = -0.5 * np.ones(n), 0.5 * np.ones(n)
    f = lambda x: 0.5 * x @ A @ x - b @ x
    fg = lambda x: (f(x), A @ x - b)
    proj = lambda x: np.clip(x, lo, hi)
    return A, b, lo, hi, f, fg, proj


def test_spg_reaches_the_box_constrained_minimiser():
    A, b, lo, hi, f, fg, proj = _quadratic()
    res = spg(np.zeros(A.shape[0]), fg, f, proj, np.dot, lambda a: np.max(np.abs(a)), iters=400)
    x = res.x
    g = A @ x - b
    assert np.max(np.abs(proj(x - g) - x)) < 1e-8  # projected-gradient stationarity
    scipy_opt = pytest.importorskip("scipy.optimize")
    ref = scipy_opt.minimize(f, np.zeros_like(x), jac=lambda x: A @ x - b, method="L-BFGS-B",
                             bounds=list(zip(lo, hi)), options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 10000}).x
    assert np.max(np.abs(x - ref)) < 1e-6
    assert np.sum((x == lo) | (x == hi)) > 0  # some bounds are active


def test_nonmonotone_acceptance_and_decrease():
    A, b, lo, hi, f, fg, proj = _quadratic(seed=3)
    M = 4
    res = spg(np.full(A.shape[0], 0.3), fg, f, proj, np.dot, lambda a: np.max(np.abs(a)), iters=60, memory=M)
    fh = res.f
    for k in range(1, len(fh)):
        assert fh[k] <= max(fh[max(0, k - M):k]) + 1e-12
    assert fh[-1] < fh[0]
    assert res.grads == len(fh) and res.evals >= res.grads


def test_start_at_solution_stops():
    A, b, lo, hi, f, fg, proj = _quadratic(seed=5)
    res = spg(np.zeros(A.shape[0]), fg, f, proj, np.dot, lambda a: np.max(np.abs(a)), iters=500)
    again = spg(res.x, fg, f, proj, np.dot, lambda a: np.max(np.abs(a)), iters=10)
    assert again.f[-1] <= res.f[-1] + 1e-12
    assert np.max(np.abs(again.x - res.x)) < 1e-8
