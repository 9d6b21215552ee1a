"""The graphed public call (api.GraphedGradient): one capture, replays with new
inputs.  Every kernel is deterministic (fixed work split, fixed-order
reductions), so a replay must equal the eager call bit for bit, for host
(pinned) and device inputs, for consecutive calls with different models, and
for the probed and the full-storage gradient.  The probed form runs as its
halves with tp_residual between them (d_obs uploaded beside the forward
half), which must give tp_gradient_probed's result bit for bit."""
import numpy as np
import pytest
import torch

from paper_2104_00794_gb300 import api, native
from paper_2104_00794_gb300 import workloads as wl
from parity_util import oracle_dobs, problem, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _lib(cuda_lib):
    yield


@pytest.mark.parametrize("full", [False, True], ids=["probed", "full"])
@pytest.mark.parametrize("mk", [lambda: wl.small_2d(nx=300, nz=70, nt=220, order=8, nshots=2, r=8),
                                lambda: wl.small_3d(nx=70, ny=37, nz=45, nt=90, order=8, nshots=2, r=8)],
                         ids=["2d", "3d"])
def test_graphed_gradient_equals_eager(mk, full):
    w = mk()
    p = problem(w)
    dobs = oracle_dobs(w)
    spec = api.ProbeSpec(kind="rademacher", r=8, T=32, seed=w.seed)
    gg = api.GraphedGradient(p, None if full else spec, full=full)
    h_out = torch.empty(p.shape, dtype=torch.float32).pin_memory()
    h_sc = torch.empty(2, dtype=torch.float64).pin_memory()
    for vel in (w.vel0, w.vel_true):  # two calls in a row with different inputs
        h_vel = torch.from_numpy(np.ascontiguousarray(vel)).pin_memory()
        h_wav = torch.from_numpy(np.ascontiguousarray(w.wavelet)).pin_memory()
        h_d = torch.from_numpy(np.ascontiguousarray(dobs)).pin_memory()
        gg(h_vel, h_wav, h_d, grad_out=h_out, scalars_out=h_sc)
        torch.cuda.synchronize()
        args = (to_dev(vel), to_dev(w.wavelet), to_dev(dobs))
        ge, se = p.gradient_full(*args) if full else p.gradient_probed(*args, spec)
        assert torch.equal(h_out, ge.cpu())
        assert torch.equal(h_sc, se.cpu())
        gd, sd = gg(*args)  # device inputs, static outputs
        assert torch.equal(gd, ge) and torch.equal(sd, se)


def test_graphed_gradient_survives_problem_release():
    """The graph holds the workspace: releasing the Problem's cache does not free it."""
    w = wl.small_2d(nx=300, nz=70, nt=120, order=8, nshots=1, r=8)
    p = problem(w)
    dobs = oracle_dobs(w)
    spec = api.ProbeSpec(kind="rademacher", r=8, T=32, seed=w.seed)
    gg = api.GraphedGradient(p, spec)
    args = (to_dev(w.vel0), to_dev(w.wavelet), to_dev(dobs))
    g1, _ = gg(*args)
    g1 = g1.clone()
    p.release()
    junk = torch.full((1 << 24,), 7.0, device="cuda")  # reuse freed memory if any was freed
    g2, _ = gg(*args)
    assert torch.equal(g1, g2)
    del junk


def test_graphed_gradient_needs_vmax():
    w = wl.small_2d(nx=67, nz=45, nt=60, order=4)
    p = api.Problem.from_workload(w, vmax=0.0)
    with pytest.raises(ValueError, match="vmax"):
        api.GraphedGradient(p, api.ProbeSpec(r=4))


def test_residual_entry_point():
    """tp_residual (Eq. 2): d - d_obs in place, 1/2 |d - d_obs|^2 in fp64."""
    rng = np.random.default_rng(5)
    n = 3 * 1000 * 601 + 7
    d_h = rng.standard_normal(n).astype(np.float32)
    o_h = rng.standard_normal(n).astype(np.float32)
    d, o = to_dev(d_h), to_dev(o_h)
    J = torch.zeros(1, dtype=torch.float64, device="cuda")
    nb = native.tp_residual_workspace_bytes()
    buf = torch.empty(nb + 256, dtype=torch.uint8, device="cuda")
    ws = buf.data_ptr() + (-buf.data_ptr()) % 256
    s = torch.cuda.current_stream().cuda_stream
    native.tp_residual(d.data_ptr(), o.data_ptr(), n, J.data_ptr(), ws, nb, s)
    res = d_h - o_h  # fp32, exact IEEE subtraction on both sides
    assert np.array_equal(d.cpu().numpy(), res)
    ref = 0.5 * float(np.sum(res.astype(np.float64) ** 2))
    assert abs(float(J.item()) - ref) <= 1e-12 * ref
    with pytest.raises(native.TprobeError) as e:
        native.tp_residual(d.data_ptr(), o.data_ptr(), n, J.data_ptr(), ws, nb - 8, s)
    assert e.value.status == native.TP_ERR_NOMEM
    with pytest.raises(native.TprobeError) as e:
        native.tp_residual(d.data_ptr(), o.data_ptr(), 0, J.data_ptr(), ws, nb, s)
    assert e.value.status == native.TP_ERR_ARG
