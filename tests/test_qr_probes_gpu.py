"""Range-finding probes (Eq. 6) on the GPU against the oracle's LAPACK QR of
the same D D^T Z, and the probed gradient with them (scale 1)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2104_00794_gb300 import api
from paper_2104_00794_gb300 import workloads as wl
from parity_util import host, oracle_dobs, problem, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _lib(cuda_lib):
    yield


@pytest.mark.parametrize("kind,r", [("rademacher", 8), ("gaussian", 16)])
def test_qr_probes_match_lapack(kind, r):
    w = wl.small_2d(nx=200, nz=60, nt=240, order=8, nshots=2)
    p = problem(w)
    dobs = oracle_dobs(w)
    Q = host(p.qr_probes(to_dev(dobs), r=r, seed=31, kind=kind)).astype(np.float64)
    for s in range(w.nshots):
        Z = oracle.probes(kind, w.nt, r, 31, s)
        ref = oracle.qr_probes(dobs[s], Z)
        np.testing.assert_allclose(Q[s].T @ Q[s], np.eye(r), atol=1e-5)
        assert np.max(np.abs(Q[s] - ref)) <= 1e-4, np.max(np.abs(Q[s] - ref))


def test_probed_gradient_with_qr_probes():
    w = wl.small_2d(nx=200, nz=60, nt=240, order=8, nshots=2)
    p = problem(w)
    dobs = oracle_dobs(w)
    r = 8
    Q = p.qr_probes(to_dev(dobs), r=r, seed=5)
    grad, _ = p.gradient_probed(to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs),
                                api.ProbeSpec(kind="user", r=r, T=32, Z_user=Q))
    g = oracle.grid_of(w)
    ref = np.zeros(w.N)
    for s in range(w.nshots):
        Qs = oracle.qr_probes(dobs[s], oracle.probes("rademacher", w.nt, r, 5, s))
        gs, _ = oracle.gradient_probed(g, w.src[s], w.rec[s], w.vel0, w.wavelet[s], dobs[s], Qs, 1.0)
        ref += gs
    assert rel_l2(host(grad), ref) <= 1e-4


def test_qr_probes_reject_bad_arguments():
    from paper_2104_00794_gb300 import native
    w = wl.small_2d(nx=64, nz=20, nt=40, order=8)
    p = problem(w)
    d = torch.zeros((1, w.nt, w.nrec), device="cuda")
    with pytest.raises((native.TprobeError, ValueError)):
        p.qr_probes(d, r=33)
    with pytest.raises(native.TprobeError):   # an all-zero record has no range
        p.qr_probes(d, r=4)
