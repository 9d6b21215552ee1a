"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs, element by element.

Tolerances (stated by the hot-path contract, derived for fp32 arithmetic):
  * traces of F and F^T: relative L2 <= 1e-5 (fp32 leapfrog over <= 500
    steps accumulates a few 1e-7 per step of relative rounding);
  * gradients (full storage and probed with the same probes): relative L2
    <= 1e-4 (products of two fp32 wavefields summed over nt levels);
  * probes: bit-exact (integer hash, exactly representable values);
  * fp64 misfit: relative 1e-5 (inherits the fp32 trace error).
"""
import dataclasses

import numpy as np
import pytest
import torch

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


CASES_2D = [
    dict(nx=300, nz=70, nt=220, order=8, nshots=2),    # 3 x-strips, ragged tail
    dict(nx=67, nz=45, nt=160, order=4, nshots=1),
    dict(nx=129, nz=9, nt=90, order=8, nshots=3),      # one strip + 1 column
]
CASES_3D = [
    dict(nx=70, ny=37, nz=45, nt=90, order=8, nshots=2),  # 2 x-tiles, 3 y-tiles, ragged
    dict(nx=36, ny=22, nz=28, nt=80, order=4, nshots=1),
]


def _w(case, **kw):
    c = dict(case)
    c.update(kw)
    if "ny" in c:
        return wl.small_3d(**c)
    return wl.small_2d(**c)


# ------------------------------------------------------------------ probes
@pytest.mark.parametrize("kind,nt,r", [("rademacher", 500, 4), ("gaussian", 3000, 16), ("rademacher", 2000, 32),
                                       ("gaussian", 77, 5), ("identity", 64, 64)])
def test_probes_bit_exact(kind, nt, r):
    p = api.Problem(2, 8, 1, 8, 10.0, 1e-3, nt, 4, [[1]], [[2]], vmax=1500.0)
    for shot in (0, 3):
        spec = api.ProbeSpec(kind=kind, r=r, seed=2104 + shot)
        Z = host(p.probes(spec, shot))
        ref = oracle.probes(kind, nt, r, 2104 + shot, shot)
        assert np.array_equal(Z.astype(np.float64), ref)


# ------------------------------------------------------------------ F and F^T
@pytest.mark.parametrize("form", ["levels", "increment"])
@pytest.mark.parametrize("case", CASES_2D + CASES_3D, ids=lambda c: "x".join(str(c[k]) for k in ("nz", "ny", "nx") if k in c) + f"_o{c['order']}")
def test_forward_traces(case, form):
    w = _w(case)
    p = problem(w, form=form)
    d = host(p.forward(to_dev(w.vel_true), to_dev(w.wavelet)))
    ref = oracle.batch_forward(w, w.vel_true)
    assert d.shape == ref.shape
    assert np.all(d[:, :2] == 0.0)
    assert rel_l2(d, ref) <= TRACE_TOL, rel_l2(d, ref)
    for s in range(w.nshots):
        assert rel_l2(d[s], ref[s]) <= TRACE_TOL


@pytest.mark.parametrize("form", ["levels", "increment"])
@pytest.mark.parametrize("case", [CASES_2D[0], CASES_3D[0]], ids=["2d", "3d"])
def test_adjoint_traces_and_dot_product(case, form):
    w = _w(case)
    p = problem(w, form=form)
    rng = np.random.default_rng(3)
    s = rng.standard_normal((w.nshots, w.nt, w.nrec)).astype(np.float32)
    q = rng.standard_normal((w.nshots, w.nt, w.nsrc)).astype(np.float32)
    vel = to_dev(w.vel_true)
    qa = host(p.adjoint(vel, to_dev(s)))
    g = oracle.grid_of(w)
    ref = np.stack([oracle.adjoint(g, w.src[i], w.rec[i], w.vel_true, s[i]) for i in range(w.nshots)])
    assert rel_l2(qa, ref) <= TRACE_TOL
    assert np.all(qa[:, 0] == 0.0) and np.all(qa[:, -1] == 0.0)
    fq = host(p.forward(vel, to_dev(q)))
    lhs = float(np.sum(fq.astype(np.float64) * s))
    rhs = float(np.sum(q.astype(np.float64) * qa))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), abs(rhs))


# ------------------------------------------------------------------ gradients
@pytest.mark.parametrize("form", ["levels", "increment"])
@pytest.mark.parametrize("case", [CASES_2D[0], CASES_2D[1], CASES_3D[0]], ids=["2d_o8", "2d_o4", "3d_o8"])
def test_full_gradient(case, form):
    w = _w(case)
    p = problem(w, form=form)
    dobs = oracle_dobs(w)
    grad, sc = p.gradient_full(to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs))
    grad, sc = host(grad), host(sc)
    ref, J = oracle.batch_gradient_full(w, w.vel0, dobs)
    assert rel_l2(grad, ref) <= GRAD_TOL, rel_l2(grad, ref)
    assert sc[0] == pytest.approx(J, rel=1e-5)
    assert sc[1] == pytest.approx(np.linalg.norm(grad.astype(np.float64)), rel=1e-6)


@pytest.mark.parametrize("form", ["levels", "increment"])
def test_full_gradient_3d_imaging_in_the_adjoint_sweep(form):
    """3-D, levels form: the imaging condition runs inside the adjoint step's
    sweep (one launch per step, no separate imaging sweep); the increment form
    keeps the separate sweep.  Both within the parity bound (ragged tiles:
    70 x 21 x 37)."""
    w = _w(dict(CASES_3D[0], nx=70, ny=21, nz=37))
    p = problem(w, form=form)
    dobs = oracle_dobs(w)
    args = (to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs))
    p.gradient_full(*args)  # allocation and setup outside the profile
    torch.cuda.synchronize()
    native.tp_profile_begin()
    grad, _ = p.gradient_full(*args)
    kern = native.tp_profile_end()
    steps = w.nt - 2
    if form == "levels":
        assert kern["step_imaging_fused"]["launches"] == steps and kern["imaging_sweep"]["launches"] == 0
        assert kern["stencil_step"]["launches"] == steps  # the forward's
    else:
        assert kern["step_imaging_fused"]["launches"] == 0 and kern["imaging_sweep"]["launches"] == steps
    ref, _ = oracle.batch_gradient_full(w, w.vel0, dobs)
    assert rel_l2(host(grad), ref) <= GRAD_TOL


@pytest.mark.parametrize("case,kind,r,T", [
    (CASES_2D[0], "rademacher", 4, 32),
    (CASES_2D[0], "gaussian", 16, 64),
    (CASES_2D[1], "gaussian", 5, 32),
    (CASES_2D[2], "rademacher", 32, 32),
    (CASES_3D[0], "rademacher", 8, 32),
    (CASES_3D[1], "gaussian", 16, 64),
], ids=["2d_rad4", "2d_gau16_T64", "2d_o4_gau5", "2d_3shots_r32", "3d_rad8", "3d_o4_gau16_T64"])
@pytest.mark.parametrize("form", ["levels", "increment"])
def test_probed_gradient_same_probes(case, kind, r, T, form):
    w = _w(case, r=r, probe_kind=kind, T=T)
    p = problem(w, form=form)
    dobs = oracle_dobs(w)
    spec = api.ProbeSpec(kind=kind, r=r, T=T, seed=w.seed)
    grad, sc = p.gradient_probed(to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs), spec)
    grad, sc = host(grad), host(sc)
    ref, J = oracle.batch_gradient_probed(w, w.vel0, dobs, kind=kind, r=r, seed=w.seed)
    assert rel_l2(grad, ref) <= GRAD_TOL, rel_l2(grad, ref)
    assert sc[0] == pytest.approx(J, rel=1e-5)
    assert sc[1] == pytest.approx(np.linalg.norm(grad.astype(np.float64)), rel=1e-6)
    p.status(native.OP_GRADIENT_PROBED)


def test_identity_probes_reproduce_full_gradient():
    """Q = I (r = nt): the probed path computes Eq. 3 exactly (to rounding)."""
    w = _w(CASES_2D[1], nt=96)
    p = problem(w)
    dobs = oracle_dobs(w)
    args = (to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs))
    gp, _ = p.gradient_probed(*args, api.ProbeSpec(kind="identity", r=w.nt, T=32))
    gf, _ = p.gradient_full(*args)
    ref, _ = oracle.batch_gradient_full(w, w.vel0, dobs)
    assert rel_l2(host(gp), host(gf)) <= 1e-5
    assert rel_l2(host(gp), ref) <= GRAD_TOL


# ------------------------------------------------------------------ edge cases
def test_minimum_nt_gives_zero_gradient():
    w = _w(CASES_2D[1], nt=3)
    p = problem(w)
    dobs = np.zeros((1, 3, w.nrec), np.float32)
    g, sc = p.gradient_probed(to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs), api.ProbeSpec(r=4))
    assert np.all(host(g) == 0.0) and host(sc)[0] == 0.0
    g, sc = p.gradient_full(to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs))
    assert np.all(host(g) == 0.0)


def test_tiny_grid_and_coincident_points():
    """A 5 x 3 grid, source at a corner, a receiver on the source node."""
    nx, nz, nt = 5, 3, 40
    vel = np.full((nz, nx), 1500.0, np.float32)
    src = np.array([[0]])
    rec = np.array([[0, 4, 14]])
    wav = wl.ricker(nt, 1e-3, 30.0).astype(np.float32)[None, :, None]
    p = api.Problem(2, nx, 1, nz, 10.0, 1e-3, nt, 8, src, rec, vmax=1500.0)
    d = host(p.forward(to_dev(vel), to_dev(wav)))
    g = oracle.make_grid(2, nx, 1, nz, 10.0, 1e-3, nt, 8)
    ref = oracle.forward(g, src[0], rec[0], vel, wav[0])
    assert rel_l2(d[0], ref) <= TRACE_TOL


@pytest.mark.parametrize("nx,ny,nz", [(5, 3, 2), (9, 1, 6), (131, 2, 1)], ids=["5x3x2", "ny1", "nz1_2xtiles"])
def test_degenerate_3d_grids(nx, ny, nz):
    """3-D grids thinner than the stencil radius in y or z, and one plane
    wider than one 128-point GEMM row: the TMA boxes overhang the fields on
    every side.  Traces, the full and the probed gradient against the
    oracle."""
    nt = 48
    rng = np.random.default_rng(nx * 100 + ny * 10 + nz)
    vel_true = (1500.0 + 300.0 * rng.random((nz, ny, nx))).astype(np.float32)
    vel0 = np.full((nz, ny, nx), 1650.0, np.float32)
    N = nx * ny * nz
    src = np.array([[((nz // 2) * ny + ny // 2) * nx + nx // 2]])
    rec = np.array([[0, src[0, 0] - 1, src[0, 0] + 1, N - 1]])  # two next to the source: 48 steps reach few cells
    wav = wl.ricker(nt, 1e-3, 30.0).astype(np.float32)[None, :, None]
    p = api.Problem(3, nx, ny, nz, 10.0, 1e-3, nt, 8, src, rec, vmax=1800.0)
    g = oracle.make_grid(3, nx, ny, nz, 10.0, 1e-3, nt, 8)
    d = host(p.forward(to_dev(vel_true), to_dev(wav)))
    dobs = oracle.forward(g, src[0], rec[0], vel_true, wav[0])
    assert rel_l2(d[0], dobs) <= TRACE_TOL
    dobs32 = dobs.astype(np.float32)[None]
    args = (to_dev(vel0), to_dev(wav), to_dev(dobs32))
    gf, _ = p.gradient_full(*args)
    ref_f, _ = oracle.gradient_full(g, src[0], rec[0], vel0, wav[0], dobs32[0])
    assert np.linalg.norm(ref_f) > 0
    assert rel_l2(host(gf), ref_f) <= GRAD_TOL
    Q = oracle.probes("rademacher", nt, 4, 11, 0)
    ref_p, _ = oracle.gradient_probed(g, src[0], rec[0], vel0, wav[0], dobs32[0], Q, 0.25)
    gp, _ = p.gradient_probed(*args, api.ProbeSpec(kind="rademacher", r=4, T=32, seed=11))
    assert rel_l2(host(gp), ref_p) <= GRAD_TOL


def test_errors_are_reported():
    w = _w(CASES_2D[1])
    p = problem(w)
    vel = to_dev(w.vel0)
    with pytest.raises(native.TprobeError) as e:   # CFL violation
        bad = api.Problem(2, w.nx, 1, w.nz, w.h, 0.01, w.nt, w.order, w.src, w.rec)
        bad.forward(vel, to_dev(w.wavelet))
    assert e.value.status == native.TP_ERR_UNSTABLE
    with pytest.raises(native.TprobeError) as e:   # receiver outside the grid (checked with vmax = 0)
        bad = api.Problem(2, w.nx, 1, w.nz, w.h, w.dt, w.nt, w.order, w.src, np.array([[0, w.N + 5]]))
        bad.forward(vel, to_dev(w.wavelet))
    assert e.value.status == native.TP_ERR_ARG
    # with vmax given the call does not synchronise: the kernels skip the bad entry (its trace
    # is zero), the valid one is sampled as usual, and the status read reports the index
    vmax = float(w.vel0.max())
    bad = api.Problem(2, w.nx, 1, w.nz, w.h, w.dt, w.nt, w.order, w.src, np.array([[int(w.rec[0, 3]), w.N + 5]]),
                      vmax=vmax)
    d = host(bad.forward(vel, to_dev(w.wavelet)))
    with pytest.raises(native.TprobeError) as e:
        bad.status(native.OP_FORWARD)
    assert e.value.status == native.TP_ERR_ARG
    assert not d[0, :, 1].any()
    good = api.Problem(2, w.nx, 1, w.nz, w.h, w.dt, w.nt, w.order, w.src, w.rec[:, 3:4], vmax=vmax)
    assert np.array_equal(d[0, :, 0], host(good.forward(vel, to_dev(w.wavelet)))[0, :, 0])
    bad.status(native.OP_FORWARD)  # the read cleared the flag
    with pytest.raises(native.TprobeError) as e:   # workspace too small
        native.tp_forward(p.grid, p.geom, vel.data_ptr(), vel.data_ptr(), vel.data_ptr(), vel.data_ptr(), 256,
                          torch.cuda.current_stream().cuda_stream)
    assert e.value.status == native.TP_ERR_NOMEM


# ------------------------------------------------------------------ full-size grid
@pytest.mark.slow
def test_full_size_3d_grid_truncated_time():
    """The 256^3 bench grid in the bench's launch configuration, with nt cut
    to 48 so that the oracle finishes: traces and the probed gradient."""
    w = wl.config3(nt=48)
    p = problem(w)
    dobs = wl.synthetic_data(1, w.nt, w.nrec, seed=5)
    d = host(p.forward(to_dev(w.vel_true), to_dev(w.wavelet)))
    ref = oracle.batch_forward(w, w.vel_true)
    assert rel_l2(d, ref) <= TRACE_TOL
    gref, _ = oracle.batch_gradient_probed(w, w.vel0, dobs)
    # every window length at full size: 2 windows of 32, 1 of 64, 1 of 128 (ragged: 45 levels);
    # two accumulator sets and the single-accumulator form
    for T in (32, 64, 128):
        for acc in ("f32", "f32_fold"):
            spec = api.ProbeSpec(kind="rademacher", r=32, T=T, seed=w.seed, acc=acc)
            grad, _ = p.gradient_probed(to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs), spec)
            assert rel_l2(host(grad), gref) <= GRAD_TOL, (T, acc, rel_l2(host(grad), gref))
            p.release()


# ------------------------------------------------------------------ the named configurations
def test_config1_exact_size():
    """101 x 101, nt = 500, order 4, r = 4 Rademacher: traces, full and probed
    gradients against the oracle at the configuration's own size."""
    w = wl.config1()
    p = problem(w)
    dobs = oracle_dobs(w)
    d = host(p.forward(to_dev(w.vel0), to_dev(w.wavelet)))
    assert rel_l2(d, oracle.batch_forward(w, w.vel0)) <= TRACE_TOL
    args = (to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs))
    gf, _ = p.gradient_full(*args)
    ref_f, _ = oracle.batch_gradient_full(w, w.vel0, dobs)
    assert rel_l2(host(gf), ref_f) <= GRAD_TOL
    gp, _ = p.gradient_probed(*args, api.ProbeSpec(kind="rademacher", r=4, T=32, seed=w.seed))
    ref_p, _ = oracle.batch_gradient_probed(w, w.vel0, dobs)
    assert rel_l2(host(gp), ref_p) <= GRAD_TOL


@pytest.mark.slow
@pytest.mark.parametrize("cfg", ["config2", "config4"])
def test_config_2_4_shot_subset_full_nt(cfg):
    """601 x 201 (order 8, r = 16 Gaussian, nt = 3000) and 801 x 301 (nt =
    2500): two of the shots at the full time axis, in the batched launch,
    with the library's default form for these grids (the compensated
    forward).  Traces and the probed gradient meet the contract's bounds.

    Why the compensated forward: the probed gradient applies the Laplacian
    to the probed forward field, which amplifies the grid-scale rounding
    noise that fp32 levels collect over thousands of steps (config 4's
    gradient sat at 1.07e-4 with the levels form although its traces were
    within 7.5e-6); carrying the rounding of the levels as a bf16 low part
    removes that noise."""
    w = getattr(wl, cfg)()
    k = [0, w.nshots - 1]
    w = dataclasses.replace(w, nshots=2, src=w.src[k], rec=w.rec[k], wavelet=np.ascontiguousarray(w.wavelet[k]))
    p = api.Problem.from_workload(w)
    assert p.form == "compensated"
    dobs = oracle_dobs(w)
    d = host(p.forward(to_dev(w.vel0), to_dev(w.wavelet)))
    assert rel_l2(d, oracle.batch_forward(w, w.vel0)) <= TRACE_TOL  # thousands of fp32 steps
    gp, sc = p.gradient_probed(to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs),
                               api.ProbeSpec(kind="gaussian", r=16, T=32, seed=w.seed))
    ref, J = oracle.batch_gradient_probed(w, w.vel0, dobs)
    err = rel_l2(host(gp), ref)
    pl = api.Problem.from_workload(w, form="levels")
    gl, _ = pl.gradient_probed(to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs),
                               api.ProbeSpec(kind="gaussian", r=16, T=32, seed=w.seed))
    err_levels = rel_l2(host(gl), ref)
    print(f"{cfg}: probed gradient {err:.3e} (levels form {err_levels:.3e}) after {w.nt} steps")
    assert err <= GRAD_TOL, err
    assert err < err_levels


@pytest.mark.slow
@pytest.mark.parametrize("cfg", ["config2", "config4"])
def test_config_2_4_every_shot_full_nt(cfg):
    """All 16 (config 2) and 8 (config 4) shots at the full time axis, in the
    batched launch the bench times: every shot's traces against the oracle;
    and, since batched shots are independent, the batch's probed gradient and
    misfit against the sums over the shots computed one shot per call (each
    with the batch's probes of that shot, passed as user probes).  The
    two-shot test above pins the gradient itself to the oracle."""
    w = getattr(wl, cfg)()
    p = api.Problem.from_workload(w)
    vel, wav = to_dev(w.vel0), to_dev(w.wavelet)
    d = host(p.forward(vel, wav))
    ref = oracle.batch_forward(w, w.vel0)
    errs = [rel_l2(d[s], ref[s]) for s in range(w.nshots)]
    print(f"{cfg}: worst shot's traces {max(errs):.3e}")
    assert max(errs) <= TRACE_TOL, errs
    dobs = to_dev(oracle_dobs(w))
    spec = api.ProbeSpec(kind="gaussian", r=16, T=32, seed=w.seed)
    gb, sb = p.gradient_probed(vel, wav, dobs, spec)
    gb, sb = host(gb).astype(np.float64), host(sb)
    p.release()
    gsum, jsum = np.zeros_like(gb), 0.0
    for s in range(w.nshots):
        ws = dataclasses.replace(w, nshots=1, src=w.src[s:s + 1], rec=w.rec[s:s + 1],
                                 wavelet=np.ascontiguousarray(w.wavelet[s:s + 1]))
        ps = api.Problem.from_workload(ws)
        Z = p.probes(spec, s)[None].contiguous()
        user = api.ProbeSpec(kind="user", r=16, T=32, Z_user=Z, scale=1.0 / 16)
        g, sc = ps.gradient_probed(vel, wav[s:s + 1].contiguous(), dobs[s:s + 1].contiguous(), user)
        gsum += host(g).astype(np.float64)
        jsum += float(host(sc)[0])
        ps.release()
    err = rel_l2(gb, gsum)
    print(f"{cfg}: batch gradient against the sum of {w.nshots} single-shot gradients {err:.3e}")
    assert err <= 2e-6, err
    assert sb[0] == pytest.approx(jsum, rel=1e-9)


@pytest.mark.parametrize("sponge", [0, 6], ids=["rigid", "sponge"])
def test_coincident_points_per_step_path_deterministic(sponge):
    """3-D (and a 2-D grid with an absorbing layer): the per-step path.  Two
    sources on one node and receivers repeating nodes: entries alone at a
    node inject in parallel, the others one after the other in index order,
    so runs repeat bit for bit; traces and the probed gradient match the
    oracle."""
    import dataclasses
    if sponge:
        w = wl.with_sponge(wl.small_2d(nx=90, nz=50, nt=140, order=8, nshots=2), sponge)
    else:
        w = wl.small_3d(nx=36, ny=22, nz=28, nt=80, order=8, nshots=2)
    s0 = w.src[:, :1]
    w = dataclasses.replace(w, src=np.concatenate([s0, s0], axis=1),
                            rec=np.concatenate([w.rec, w.rec[:, :5], w.rec[:, 2:4], s0], axis=1),
                            wavelet=np.ascontiguousarray(np.repeat(w.wavelet, 2, axis=2) * np.array([1.0, -0.3], np.float32)))
    p = problem(w)
    d1 = host(p.forward(to_dev(w.vel_true), to_dev(w.wavelet)))
    d2 = host(p.forward(to_dev(w.vel_true), to_dev(w.wavelet)))
    assert np.array_equal(d1, d2)
    assert rel_l2(d1, oracle.batch_forward(w, w.vel_true)) <= TRACE_TOL
    dobs = oracle_dobs(w)
    spec = api.ProbeSpec(kind="rademacher", r=4, T=32, seed=5)
    args = (to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs))
    ga, _ = p.gradient_probed(*args, spec)
    gb, _ = p.gradient_probed(*args, spec)
    assert np.array_equal(host(ga), host(gb))
    ref, _ = oracle.batch_gradient_probed(w, w.vel0, dobs, kind="rademacher", r=4, seed=5)
    assert rel_l2(host(ga), ref) <= GRAD_TOL
