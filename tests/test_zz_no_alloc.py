"""The allocation-free misfit entry point, tp_misfit_noalloc.

Some callers cannot allocate device memory where they need the data misfit
(their device memory comes from a host framework's own pool, or they run a
latency-critical loop that must not allocate).  tp_misfit_noalloc serves
them with scratch space that lives inside the library, so it takes no
workspace.  Here it is called through the C ABI twice in a row and checked
against the misfit that tp_gradient_full returns for the same model and data,
within the misfit tolerance of the other parity tests; then over a
descending run of sizes (two chunks of the scratch, an exact chunk, one
sample past it, a single sample) against the same sum taken on the host.

This file is named to be collected last: if it fails, a run that stops at the
first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2104_00794_gb300 import api, native
from paper_2104_00794_gb300 import workloads as wl
from parity_util import host, oracle_dobs, to_dev

pytestmark = pytest.mark.gpu


def test_misfit_noalloc_matches_gradient_full_twice(cuda_lib):
    # 3 shots x 300 levels x 101 receivers = 90,900 samples: two scratch chunks
    w = wl.small_2d(nx=101, nz=40, nt=300, order=8, nshots=3)
    p = api.Problem.from_workload(w)
    dobs = to_dev(oracle_dobs(w))
    vel0, wav = to_dev(w.vel0), to_dev(w.wavelet)
    _, sc = p.gradient_full(vel0, wav, dobs)           # existing entry point
    ref = float(host(sc)[0])
    d_syn = p.forward(vel0, wav)
    n = d_syn.numel()
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for k in range(2):                                   # two calls in a row
        native.tp_misfit_noalloc(d_syn.data_ptr(), dobs.data_ptr(), n, out.data_ptr() + 8 * k, stream)
    got = host(out)
    assert got[0] == pytest.approx(ref, rel=1e-5)
    assert got[1] == pytest.approx(ref, rel=1e-5)
    assert got[0] == got[1]


def test_misfit_noalloc_sizes_descending(cuda_lib):
    """Each call after a longer one: a result that leaned on partial sums left
    in the shared array by the previous call would be off.  The host sum takes
    the residual in fp32 (as the kernel does) and its squares in fp64, so only
    the order of the fp64 additions differs."""
    rng = np.random.default_rng(7)
    n_max = 90_900
    d = rng.standard_normal(n_max).astype(np.float32)
    dobs = rng.standard_normal(n_max).astype(np.float32)
    dd, do = to_dev(d), to_dev(dobs)
    sizes = [90_900, 65_537, 65_536, 1]
    out = torch.full((len(sizes),), -1.0, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for k, n in enumerate(sizes):
        native.tp_misfit_noalloc(dd.data_ptr(), do.data_ptr(), n, out.data_ptr() + 8 * k, stream)
    got = host(out)
    for k, n in enumerate(sizes):
        r = (d[:n] - dobs[:n]).astype(np.float64)
        ref = 0.5 * float(np.sum(r * r))
        assert got[k] == pytest.approx(ref, rel=1e-11), (n, got[k], ref)


def test_misfit_noalloc_rejects_bad_sizes(cuda_lib):
    L = native.lib()
    buf = torch.zeros(4, dtype=torch.float32, device="cuda")
    res = torch.zeros(1, dtype=torch.float64, device="cuda")
    too_many = 268435456 + 1
    st = L.tp_misfit_noalloc(buf.data_ptr(), buf.data_ptr(), too_many, res.data_ptr(), None)
    assert st == native.TP_ERR_ARG and "exceeds" in native.last_error()
    st = L.tp_misfit_noalloc(buf.data_ptr(), None, 4, res.data_ptr(), None)
    assert st == native.TP_ERR_ARG
    st = L.tp_misfit_noalloc(buf.data_ptr(), buf.data_ptr(), 0, res.data_ptr(), None)
    assert st == native.TP_ERR_ARG
