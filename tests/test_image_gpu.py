"""GPU parity of the imaging conditions on probed fields (tp_probed_image).

The GPU applies D (identity or the spatial gradient) to the r probed fields
P_i (forward half) and V_i (an adjoint run driven by a seeded adjoint source)
and sums scale * <D P_i, D V_i>; the FP64 oracle does the same with the same
probes.  Both fields are fp32 sums over nt levels and D adds a few terms, so
the bar is the probed gradient's: relative L2 <= 1e-4.  With identity probes
the result is the condition applied at every time step (Eq. 5), checked
against the oracle's per-step image.
"""
import numpy as np
import pytest

import oracle
from paper_2104_00794_gb300 import api, native
from paper_2104_00794_gb300 import workloads as wl
from parity_util import host, problem, rel_l2, to_dev

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(autouse=True)
def _lib(cuda_lib):
    yield


def _run(w, spec, cond, adj):
    p = problem(w)
    vel, wav = to_dev(w.vel0), to_dev(w.wavelet)
    state = p.new_state(spec)
    p.probed_forward(vel, wav, spec, state)
    img = host(p.probed_image(vel, to_dev(adj), spec, state, cond))
    return img, p


@pytest.mark.parametrize("w_kw,kind,r,T", [
    (dict(nx=300, nz=70, nt=220, order=8, nshots=2), "rademacher", 8, 32),
    (dict(nx=67, nz=45, nt=160, order=4, nshots=1), "gaussian", 16, 64),
    (dict(nx=70, ny=37, nz=45, nt=90, order=8, nshots=2), "rademacher", 8, 32),
    (dict(nx=36, ny=22, nz=28, nt=80, order=4, nshots=1), "gaussian", 32, 64),
], ids=["2d_rad8", "2d_o4_gau16_T64", "3d_rad8", "3d_o4_gau32_T64"])
@pytest.mark.parametrize("cond", ["correlation", "gradient"])
def test_probed_image_matches_oracle(w_kw, kind, r, T, cond):
    w = (wl.small_3d if "ny" in w_kw else wl.small_2d)(**w_kw, r=r, probe_kind=kind)
    adj = wl.synthetic_data(w.nshots, w.nt, w.nrec, seed=23)
    spec = api.ProbeSpec(kind=kind, r=r, T=T, seed=w.seed)
    img, p = _run(w, spec, cond, adj)
    ref = oracle.batch_image(w, w.vel0, adj.astype(np.float64), cond, kind=kind, r=r, seed=w.seed)
    assert np.linalg.norm(ref) > 0
    assert rel_l2(img, ref) <= TOL, rel_l2(img, ref)
    p.status(native.OP_PROBED_BACKWARD)


@pytest.mark.parametrize("cond", ["correlation", "gradient"])
def test_identity_probes_give_the_per_step_image(cond):
    w = wl.small_2d(nx=67, nz=45, nt=96, order=4, nshots=1)
    adj = wl.synthetic_data(1, w.nt, w.nrec, seed=5)
    img, _ = _run(w, api.ProbeSpec(kind="identity", r=w.nt, T=32), cond, adj)
    ref = oracle.batch_image(w, w.vel0, adj.astype(np.float64), cond, probed=False)
    assert rel_l2(img, ref) <= TOL, rel_l2(img, ref)


def test_image_rejects_bad_arguments():
    w = wl.small_2d(nx=67, nz=45, nt=60, order=4, nshots=1)
    adj = to_dev(wl.synthetic_data(1, w.nt, w.nrec, seed=5))
    p = problem(w)
    spec = api.ProbeSpec(kind="rademacher", r=4, T=32, seed=1)
    state = p.new_state(spec)
    p.probed_forward(to_dev(w.vel0), to_dev(w.wavelet), spec, state)
    with pytest.raises(native.TprobeError, match="imaging condition"):
        img = p.probed_image(to_dev(w.vel0), adj, spec, state, "gradient")
        native.tp_probed_image(p.grid, p.geom, spec.to_c(), to_dev(w.vel0).data_ptr(), adj.data_ptr(), 7,
                               img.data_ptr(), state.data_ptr(), state.numel(),
                               *p.workspace(native.OP_PROBED_BACKWARD, spec), 0)
    bf = api.ProbeSpec(kind="rademacher", r=4, T=32, seed=1, acc="bf16")
    st_bf = p.new_state(bf)
    with pytest.raises(native.TprobeError, match="TP_ACC_F32"):
        p.probed_image(to_dev(w.vel0), adj, bf, st_bf, "gradient")
