"""The persistent 2-D cluster path (one thread-block cluster per shot, many
steps per launch) and the compensated forward, against the FP64 oracle.

  * compensated form (the default for 2-D grids that fit one cluster): F
    and F^T traces, full and probed gradients within the parity bounds, on
    ragged grids and both orders; its traces closer to FP64 than the levels
    form's after thousands of steps;
  * injection at coincident nodes: entries summed in index order, so two
    runs agree bit for bit, and both agree with the oracle;
  * a batch with more shots than clusters fit on the GPU at once (clusters
    step several shots in turn);
  * windows of 32, 64 and 128 levels with a ragged last window (the launches
    end where the window GEMMs close).
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2104_00794_gb300 import api
from paper_2104_00794_gb300 import workloads as wl
from parity_util import host, oracle_dobs, problem, rel_l2, to_dev

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-5
GRAD_TOL = 1e-4


@pytest.fixture(autouse=True)
def _lib(cuda_lib):
    yield


CASES = [
    dict(nx=300, nz=70, nt=220, order=8, nshots=2),
    dict(nx=67, nz=45, nt=160, order=4, nshots=1),
    dict(nx=129, nz=9, nt=90, order=8, nshots=3),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c['nz']}x{c['nx']}_o{c['order']}")
def test_compensated_traces_and_gradients(case):
    w = wl.small_2d(**case)
    p = problem(w, form="compensated")
    assert p.form == "compensated"
    d = host(p.forward(to_dev(w.vel_true), to_dev(w.wavelet)))
    assert rel_l2(d, oracle.batch_forward(w, w.vel_true)) <= TRACE_TOL
    s = wl.synthetic_data(w.nshots, w.nt, w.rec.shape[1], seed=9)
    q = host(p.adjoint(to_dev(w.vel0), to_dev(s)))
    g = oracle.grid_of(w)
    for k in range(w.nshots):
        ref = oracle.adjoint(g, w.src[k], w.rec[k], w.vel0, s[k])
        assert rel_l2(q[k], ref) <= TRACE_TOL
    dobs = oracle_dobs(w)
    args = (to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs))
    gf, _ = p.gradient_full(*args)
    ref_f, _ = oracle.batch_gradient_full(w, w.vel0, dobs)
    assert rel_l2(host(gf), ref_f) <= GRAD_TOL
    spec = api.ProbeSpec(kind=w.probe_kind, r=w.r, T=32, seed=w.seed)
    gp, sc = p.gradient_probed(*args, spec)
    ref_p, J = oracle.batch_gradient_probed(w, w.vel0, dobs)
    assert rel_l2(host(gp), ref_p) <= GRAD_TOL
    assert host(sc)[0] == pytest.approx(J, rel=1e-5)


def test_compensated_is_more_accurate_over_long_runs():
    """201 x 101, 2000 steps: both forms keep the traces within the bound,
    the compensated one closer to FP64."""
    w = wl.small_2d(nx=201, nz=101, nt=2000, order=8, nshots=1, h=12.5, dt=1e-3, f0=8.0)
    ref = oracle.batch_forward(w, w.vel_true)
    errs = {}
    for form in ("levels", "compensated"):
        p = problem(w, form=form)
        errs[form] = rel_l2(host(p.forward(to_dev(w.vel_true), to_dev(w.wavelet))), ref)
    assert errs["levels"] <= TRACE_TOL
    assert errs["compensated"] < errs["levels"], errs


@pytest.mark.parametrize("form", ["levels", "compensated"])
def test_coincident_points_are_deterministic(form):
    """Two sources on one node and receivers that repeat nodes (and sit on
    the source node): the injections at a node are summed in index order, so
    results repeat bit for bit, and they match the oracle."""
    w = wl.small_2d(nx=90, nz=40, nt=150, order=8, nshots=2)
    s0 = int(w.src[0, 0])
    src = np.array([[s0, s0], [s0 + 7, s0 + 7]])
    rec = np.concatenate([w.rec, w.rec[:, :25], np.array([[s0] * 3, [s0 + 7] * 3])], axis=1)
    wav = np.ascontiguousarray(np.repeat(w.wavelet, 2, axis=2) * np.array([1.0, 0.5], np.float32))
    w = dataclasses.replace(w, src=src, rec=rec, wavelet=wav)
    p = problem(w, form=form)
    d1 = host(p.forward(to_dev(w.vel_true), to_dev(w.wavelet)))
    d2 = host(p.forward(to_dev(w.vel_true), to_dev(w.wavelet)))
    assert np.array_equal(d1, d2)
    assert rel_l2(d1, oracle.batch_forward(w, w.vel_true)) <= TRACE_TOL
    s = wl.synthetic_data(w.nshots, w.nt, w.rec.shape[1], seed=4)
    q1 = host(p.adjoint(to_dev(w.vel0), to_dev(s)))
    q2 = host(p.adjoint(to_dev(w.vel0), to_dev(s)))
    assert np.array_equal(q1, q2)
    g = oracle.grid_of(w)
    for k in range(w.nshots):
        assert rel_l2(q1[k], oracle.adjoint(g, w.src[k], w.rec[k], w.vel0, s[k])) <= TRACE_TOL
    dobs = oracle_dobs(w)
    spec = api.ProbeSpec(kind="rademacher", r=4, T=32, seed=5)
    args = (to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs))
    ga, _ = p.gradient_probed(*args, spec)
    gb, _ = p.gradient_probed(*args, spec)
    assert np.array_equal(host(ga), host(gb))
    ref, _ = oracle.batch_gradient_probed(w, w.vel0, dobs, kind="rademacher", r=4, seed=5)
    assert rel_l2(host(ga), ref) <= GRAD_TOL


def test_more_shots_than_resident_clusters():
    """40 shots of 70 x 300: more clusters than fit on the GPU at once, so
    clusters step several shots in turn; every shot's traces against the
    oracle (the shots differ in their source position)."""
    w = wl.small_2d(nx=300, nz=70, nt=80, order=8, nshots=40)
    for form in ("levels", "compensated"):
        p = problem(w, form=form)
        d = host(p.forward(to_dev(w.vel_true), to_dev(w.wavelet)))
        ref = oracle.batch_forward(w, w.vel_true)
        for k in range(w.nshots):
            assert rel_l2(d[k], ref[k]) <= TRACE_TOL, (form, k)


@pytest.mark.parametrize("T", [32, 64, 128])
def test_windows_with_ragged_tail(T):
    """nt = 301: the windows of the probe GEMM end off the step grid of the
    launches; single and two accumulator sets."""
    w = wl.small_2d(nx=150, nz=60, nt=301, order=8, nshots=2, r=8)
    p = problem(w)
    dobs = oracle_dobs(w)
    ref, _ = oracle.batch_gradient_probed(w, w.vel0, dobs, kind="rademacher", r=8, seed=3)
    for acc in ("f32", "f32_fold"):
        spec = api.ProbeSpec(kind="rademacher", r=8, T=T, seed=3, acc=acc)
        g, _ = p.gradient_probed(to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs), spec)
        assert rel_l2(host(g), ref) <= GRAD_TOL, (T, acc)
