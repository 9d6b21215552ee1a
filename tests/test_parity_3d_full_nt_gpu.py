"""3-D parity over the whole time axis (Algorithm 1 lines 1 and 5 run for
thousands of fp32 steps), against the FP64 oracle.

Long fp32 runs are where rounding accumulates, so the 3-D path is checked at
the benchmark's own time axis, not only on truncated records:
  * the 256^3 benchmark grid, nt = 2000, forward traces within 1e-5;
  * a 96^3 grid with the benchmark's time axis, probes and window (nt = 2000,
    r = 32 Rademacher, T = 32): the probed gradient within 1e-4 of the
    oracle's estimator with the same probes, and the traces within 1e-5.
The oracle takes minutes here on the host cores."""
import pytest

import oracle
from paper_2104_00794_gb300 import api
from paper_2104_00794_gb300 import workloads as wl
from parity_util import host, oracle_dobs, problem, rel_l2, to_dev

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TRACE_TOL = 1e-5
GRAD_TOL = 1e-4


def test_config3_forward_full_nt():
    w = wl.config3()
    p = problem(w)
    d = host(p.forward(to_dev(w.vel_true), to_dev(w.wavelet)))
    ref = oracle.batch_forward(w, w.vel_true)
    err = rel_l2(d, ref)
    print(f"config 3 traces after {w.nt} steps: {err:.3e}")
    assert err <= TRACE_TOL, err


def test_probed_gradient_96cubed_full_nt():
    w = wl.config3(n=96)
    p = problem(w)
    dobs = oracle_dobs(w)
    d = host(p.forward(to_dev(w.vel0), to_dev(w.wavelet)))
    assert rel_l2(d, oracle.batch_forward(w, w.vel0)) <= TRACE_TOL
    spec = api.ProbeSpec(kind="rademacher", r=32, T=32, seed=w.seed)
    grad, sc = p.gradient_probed(to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs), spec)
    ref, J = oracle.batch_gradient_probed(w, w.vel0, dobs)
    err = rel_l2(host(grad), ref)
    print(f"96^3 probed gradient after {w.nt} steps: {err:.3e}")
    assert err <= GRAD_TOL, err
    print(f"misfit rel error {abs(host(sc)[0] - J) / J:.3e}")
    assert host(sc)[0] == pytest.approx(J, rel=1e-5)
