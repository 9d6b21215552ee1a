"""GPU parity with the absorbing sponge (tp_grid.sponge / sponge_eta).

Same bars as without it: traces of F and F^T within 1e-5 relative L2 of the
FP64 oracle, gradients within 1e-4, the GPU dot test within 1e-5.  The cases
run long enough for the wave to enter the damped layer, and one case puts a
source inside the layer (its injection coefficient carries the 1/(1+a) of
the damped step, while the gradient's source factor does not).
"""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2104_00794_gb300 import api, native
from paper_2104_00794_gb300 import workloads as wl
from parity_util import host, oracle_dobs, problem, rel_l2, to_dev

pytestmark = pytest.mark.gpu

TRACE_TOL = 1e-5
GRAD_TOL = 1e-4


@pytest.fixture(autouse=True)
def _lib(cuda_lib):
    yield


def _w2(**kw):
    return wl.with_sponge(wl.small_2d(nx=300, nz=70, nt=260, order=8, nshots=2, **kw), 12)


def _w3(**kw):
    return wl.with_sponge(wl.small_3d(nx=70, ny=37, nz=45, nt=120, order=8, nshots=2, **kw), 8)


def _source_in_layer(w):
    """Move the second shot's source to 3 cells from the left face (inside the layer)."""
    src = w.src.copy()
    z, x = 3, 3
    src[1, 0] = (z * w.ny + (w.ny // 2 if w.ndim == 3 else 0)) * w.nx + x
    return dataclasses.replace(w, src=src)


@pytest.mark.parametrize("form", ["levels", "increment"])
@pytest.mark.parametrize("mk", [_w2, _w3], ids=["2d", "3d"])
def test_forward_traces_with_sponge(mk, form):
    w = _source_in_layer(mk())
    d = host(problem(w, form=form).forward(to_dev(w.vel_true), to_dev(w.wavelet)))
    ref = oracle.batch_forward(w, w.vel_true)
    nosponge = oracle.batch_forward(dataclasses.replace(w, sponge=0, sponge_eta=0.0), w.vel_true)
    assert rel_l2(nosponge, ref) > 1e-3  # the layer changes the data
    assert rel_l2(d, ref) <= TRACE_TOL, rel_l2(d, ref)


@pytest.mark.parametrize("mk", [_w2, _w3], ids=["2d", "3d"])
def test_adjoint_and_dot_product_with_sponge(mk):
    w = _source_in_layer(mk())
    p = problem(w)
    rng = np.random.default_rng(3)
    s = rng.standard_normal((w.nshots, w.nt, w.nrec)).astype(np.float32)
    q = rng.standard_normal((w.nshots, w.nt, w.nsrc)).astype(np.float32)
    vel = to_dev(w.vel_true)
    qa = host(p.adjoint(vel, to_dev(s)))
    g = oracle.grid_of(w)
    ref = np.stack([oracle.adjoint(g, w.src[i], w.rec[i], w.vel_true, s[i]) for i in range(w.nshots)])
    assert rel_l2(qa, ref) <= TRACE_TOL
    fq = host(p.forward(vel, to_dev(q)))
    lhs = float(np.sum(fq.astype(np.float64) * s))
    rhs = float(np.sum(q.astype(np.float64) * qa))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))


@pytest.mark.parametrize("mk", [_w2, _w3], ids=["2d", "3d"])
def test_gradients_with_sponge(mk):
    w = _source_in_layer(mk(r=8))
    p = problem(w)
    dobs = oracle_dobs(w)
    args = (to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs))
    gf, _ = p.gradient_full(*args)
    ref_f, _ = oracle.batch_gradient_full(w, w.vel0, dobs)
    assert rel_l2(host(gf), ref_f) <= GRAD_TOL, rel_l2(host(gf), ref_f)
    ref_p, _ = oracle.batch_gradient_probed(w, w.vel0, dobs, kind="rademacher", r=8, seed=w.seed)
    for acc, T in (("f32", 32), ("f32_fold", 32), ("f32", 64), ("f32_fold", 64)):
        gp, _ = p.gradient_probed(*args, api.ProbeSpec(kind="rademacher", r=8, T=T, seed=w.seed, acc=acc))
        assert rel_l2(host(gp), ref_p) <= GRAD_TOL, (acc, T, rel_l2(host(gp), ref_p))
    p.status(native.OP_GRADIENT_PROBED)
