"""GPU parity of the 128-level probe window (four 32-level sub-tiles whose
tcgen05 MMAs accumulate into one TMEM tile), with the ragged last window that
nt leaves, for every accumulator form.  Same bars as the 32- and 64-level
windows: relative L2 <= 1e-4 against the FP64 oracle with the same probes
(1.5e-4 for the bf16 value + compensation storage, whose rounding is a few
1e-5 per stored value)."""
import pytest

import oracle
from paper_2104_00794_gb300 import api, native
from paper_2104_00794_gb300 import workloads as wl
from parity_util import host, oracle_dobs, problem, rel_l2, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _lib(cuda_lib):
    yield


@pytest.mark.parametrize("mk,kind,r", [
    (lambda **k: wl.small_2d(nx=300, nz=70, nt=300, order=8, nshots=2, **k), "gaussian", 16),
    (lambda **k: wl.small_3d(nx=70, ny=37, nz=45, nt=170, order=8, nshots=1, **k), "rademacher", 8),
], ids=["2d", "3d"])
@pytest.mark.parametrize("acc,tol", [("f32", 1e-4), ("f32_fold", 1e-4), ("bf16_kahan", 1.5e-4)])
def test_window_128_matches_oracle(mk, kind, r, acc, tol):
    w = mk(r=r, probe_kind=kind)
    p = problem(w)
    dobs = oracle_dobs(w)
    g, sc = p.gradient_probed(to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs),
                              api.ProbeSpec(kind=kind, r=r, T=128, seed=w.seed, acc=acc))
    ref, J = oracle.batch_gradient_probed(w, w.vel0, dobs, kind=kind, r=r, seed=w.seed)
    assert rel_l2(host(g), ref) <= tol, rel_l2(host(g), ref)
    assert host(sc)[0] == pytest.approx(J, rel=1e-5)
    p.status(native.OP_GRADIENT_PROBED)
