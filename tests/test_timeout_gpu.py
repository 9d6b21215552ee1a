"""The timeout path of the bounded device-side waits (TP_ERR_TIMEOUT).

A wait that gives up must not fault or hang the GPU: the kernel sets an
error bit, lets its own copies land and returns, and the host reads the
status.  tp_set_wait_limit shortens the role waits of the 3-D sweep's
copy pipeline below a copy's latency, so they run out on an ordinary call;
the call must then report TP_ERR_TIMEOUT through tp_workspace_status with a
NaN misfit, and the next call with the default limit must give the result
of a call that never timed out, bit for bit."""
import numpy as np
import pytest

from paper_2104_00794_gb300 import api, native
from paper_2104_00794_gb300 import workloads as wl
from parity_util import host, problem, to_dev

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["probed", "full"])
def test_short_wait_limit_times_out_and_recovers(cuda_lib, kind):
    """The probed gradient (leapfrog sweeps) and the full-storage gradient,
    whose 3-D adjoint steps run the sweep with the imaging condition inside
    (two staged fields per plane)."""
    w = wl.small_3d(nx=70, ny=37, nz=45, nt=40, order=8, nshots=1)
    p = problem(w)
    vel0, wav = to_dev(w.vel0), to_dev(w.wavelet)
    dobs = to_dev(wl.synthetic_data(1, w.nt, w.rec.shape[1], seed=3))
    spec = api.ProbeSpec(kind="rademacher", r=4, T=32, seed=11)
    op = native.OP_GRADIENT_PROBED if kind == "probed" else native.OP_GRADIENT_FULL

    def run():
        if kind == "probed":
            return p.gradient_probed(vel0, wav, dobs, spec)
        return p.gradient_full(vel0, wav, dobs)

    g_ref, s_ref = run()
    g_ref, s_ref = host(g_ref).copy(), host(s_ref).copy()
    p.status(op)

    native.tp_set_wait_limit(64)  # cycles: far below the latency of one tensor copy
    try:
        _, s_bad = run()
        s_bad = host(s_bad).copy()
        with pytest.raises(native.TprobeError) as ei:
            p.status(op)
        assert ei.value.status == native.TP_ERR_TIMEOUT
        assert np.isnan(s_bad[0])
    finally:
        native.tp_set_wait_limit(0)

    g, s = run()
    g, s = host(g), host(s)
    p.status(op)  # the flag was cleared by the read above
    assert np.array_equal(g, g_ref)
    assert np.array_equal(s, s_ref)


def test_wait_limit_rejects_negative(cuda_lib):
    with pytest.raises(native.TprobeError) as ei:
        native.tp_set_wait_limit(-1)
    assert ei.value.status == native.TP_ERR_ARG
