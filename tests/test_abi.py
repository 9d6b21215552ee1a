"""CPU-side checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point that include/tprobe.h declares; host-only logic
(argument validation, workspace sizes, memory model) behaves as documented.
No kernel is launched here."""
import ctypes
import os
import re

import pytest

from paper_2104_00794_gb300 import build, native
from paper_2104_00794_gb300 import workloads as wl


@pytest.fixture(scope="module")
def L():
    return native.lib()


def _grid(w, nt=None, vmax=0.0):
    return native.tp_grid(w.ndim, w.nx, w.ny, w.nz, w.h, w.dt, w.nt if nt is None else nt, w.order, vmax)


def _geom(w, fake_ptr=0x1000):
    return native.tp_geom(w.nshots, w.nsrc, fake_ptr, w.nrec, fake_ptr)


def test_library_exports_every_declared_symbol(L):
    declared = native.exported_symbols()
    assert {"tp_forward", "tp_adjoint", "tp_gradient_probed", "tp_gradient_full",
            "tp_workspace_bytes"} <= set(declared)
    for name in declared:
        assert hasattr(L, name), name
    # the library is built for sm_103a only
    objdir = os.path.join(build.LIBDIR, "obj")
    assert os.path.exists(build.LIB)
    assert set(os.listdir(objdir)) >= {s.replace(".cu", ".o") for s in build.SOURCES}


def test_header_declares_extern_c_and_cites_the_paper():
    with open(os.path.join(build.INCLUDE, "tprobe.h")) as f:
        text = f.read()
    assert 'extern "C"' in text
    for cite in ("Algorithm 1", "Eq. 2", "Eq. 3", "Eq. 4"):
        assert cite in text


def test_workspace_sizes_follow_the_memory_model(L):
    w = wl.config3()
    g, geo = _grid(w), _geom(w)
    pr = native.tp_probe(0, 32, 32, 1, None, 0.0)
    full = native.tp_workspace_bytes(native.OP_GRADIENT_FULL, g, geo)
    probed = native.tp_workspace_bytes(native.OP_GRADIENT_PROBED, g, geo, pr)
    N, nt = w.N, w.nt
    # full storage holds the N x nt history (padded layout adds < 25 %)
    assert 4 * N * nt <= full <= 1.25 * 4 * N * nt + 2 * 4 * w.nt * w.nrec + (1 << 30)
    # probed: 2 N r accumulators + (T + 2) ring levels (+ padding), >= 10x less
    assert probed >= 4 * N * (2 * 32 + 34)
    assert full / probed >= 10.0
    # window 64 costs 32 more ring levels
    pr64 = native.tp_probe(0, 32, 64, 1, None, 0.0)
    p64 = native.tp_workspace_bytes(native.OP_GRADIENT_PROBED, g, geo, pr64)
    assert p64 > probed
    # forward/adjoint need three levels only
    fwd = native.tp_workspace_bytes(native.OP_FORWARD, g, geo)
    assert fwd < probed / 10


def test_folded_accumulators_halve_the_accumulator_memory(L):
    """TP_ACC_F32_FOLD keeps one N r accumulator set instead of two: the
    probed workspace drops by exactly the vbar block (nshots r padded
    fields), the state is unchanged, and r > 32 is rejected."""
    w = wl.config3()
    g, geo = _grid(w), _geom(w)
    r = 16
    two = native.tp_probe(0, r, 32, 1, None, 0.0, native.ACC_TYPES["f32"])
    one = native.tp_probe(0, r, 32, 1, None, 0.0, native.ACC_TYPES["f32_fold"])
    for op in (native.OP_GRADIENT_PROBED, native.OP_PROBED_BACKWARD):
        b2 = native.tp_workspace_bytes(op, g, geo, two)
        b1 = native.tp_workspace_bytes(op, g, geo, one)
        vbar = b2 - b1
        # one padded field per probe and shot, 4 bytes per value
        assert w.nshots * r * 4 * w.N <= vbar <= 1.25 * w.nshots * r * 4 * w.N
    assert (native.tp_probed_state_bytes(g, geo, two) == native.tp_probed_state_bytes(g, geo, one))
    big = native.tp_probe(0, 33, 32, 1, None, 0.0, native.ACC_TYPES["f32_fold"])
    n = L.tp_workspace_bytes(native.OP_GRADIENT_PROBED, ctypes.byref(g), ctypes.byref(geo), ctypes.byref(big))
    assert n == 0 and "r <= 32" in native.last_error()


def test_window_128_needs_at_most_32_probes(L):
    w = wl.small_2d(nt=300)
    g, geo = _grid(w), _geom(w)
    ok = native.tp_probe(0, 32, 128, 1, None, 0.0)
    n128 = native.tp_workspace_bytes(native.OP_GRADIENT_PROBED, g, geo, ok)
    n64 = native.tp_workspace_bytes(native.OP_GRADIENT_PROBED, g, geo, native.tp_probe(0, 32, 64, 1, None, 0.0))
    assert n128 > n64  # a ring of T + 2 levels
    bad = native.tp_probe(0, 33, 128, 1, None, 0.0)
    n = L.tp_workspace_bytes(native.OP_GRADIENT_PROBED, ctypes.byref(g), ctypes.byref(geo), ctypes.byref(bad))
    assert n == 0 and "T = 128" in native.last_error()


@pytest.mark.parametrize("mutate,msg", [
    (lambda g, p: setattr(g, "ndim", 4), "ndim"),
    (lambda g, p: setattr(g, "order", 6), "order"),
    (lambda g, p: setattr(g, "nt", 2), "nt"),
    (lambda g, p: setattr(g, "ny", 3), "ny"),
    (lambda g, p: setattr(g, "h", -1.0), "positive"),
    (lambda g, p: setattr(g, "sponge", -1), "sponge"),
    (lambda g, p: setattr(g, "sponge_eta", float("nan")), "sponge"),
    (lambda g, p: setattr(p, "r", 0), "r must"),
    (lambda g, p: setattr(p, "r", 300), "r must"),
    (lambda g, p: setattr(p, "T", 48), "window"),
    (lambda g, p: setattr(p, "kind", 2), "identity"),
    (lambda g, p: setattr(p, "kind", 3), "Z_user"),
    (lambda g, p: setattr(p, "kind", 9), "kind"),
])
def test_invalid_arguments_are_rejected(L, mutate, msg):
    w = wl.small_2d()
    g, geo = _grid(w), _geom(w)
    pr = native.tp_probe(0, 4, 32, 1, None, 0.0)
    mutate(g, pr)
    n = L.tp_workspace_bytes(native.OP_GRADIENT_PROBED, ctypes.byref(g), ctypes.byref(geo), ctypes.byref(pr))
    assert n == 0
    assert msg in native.last_error()


def test_null_geometry_and_counts_rejected(L):
    w = wl.small_2d()
    g = _grid(w)
    geo = native.tp_geom(1, 1, None, 3, 0x1000)
    assert L.tp_workspace_bytes(native.OP_FORWARD, ctypes.byref(g), ctypes.byref(geo), None) == 0
    geo = native.tp_geom(0, 1, 0x1000, 3, 0x1000)
    assert L.tp_workspace_bytes(native.OP_FORWARD, ctypes.byref(g), ctypes.byref(geo), None) == 0
    # a call with a NULL workspace fails before touching the device
    geo = _geom(w)
    st = L.tp_forward(ctypes.byref(g), ctypes.byref(geo), 0x1000, 0x1000, 0x1000, None, 0, None)
    assert st == native.TP_ERR_ARG
    st = L.tp_forward(ctypes.byref(g), ctypes.byref(geo), 0x1000, 0x1000, 0x1000, 0x1000, 16, None)
    assert st == native.TP_ERR_NOMEM and "needed" in native.last_error()


def test_residual_arguments_checked_before_the_device(L):
    nb = L.tp_residual_workspace_bytes()
    assert nb >= 1024 * 8  # fp64 partial sums
    # NULL pointers, n < 1, misaligned or small workspaces fail before any CUDA call
    assert L.tp_residual(None, 0x1000, 10, 0x1000, 0x1000, nb, None) == native.TP_ERR_ARG
    assert L.tp_residual(0x1000, 0x1000, 0, 0x1000, 0x1000, nb, None) == native.TP_ERR_ARG
    assert L.tp_residual(0x1000, 0x1000, 10, 0x1000, 0x1008, nb, None) == native.TP_ERR_ARG
    assert "aligned" in native.last_error()
    assert L.tp_residual(0x1000, 0x1000, 10, 0x1000, 0x1000, nb - 8, None) == native.TP_ERR_NOMEM


def test_kernel_names(L):
    names = [L.tp_kernel_name(k).decode() for k in range(native.KERNEL_KINDS)]
    assert names[0] == "stencil_step" and "probe_gemm_tcgen05" in names
    assert L.tp_kernel_name(99).decode() == "unknown"


def test_no_cpu_fallback_in_product_path():
    """The product package never imports the checker."""
    pkg = os.path.dirname(native.__file__)
    for root, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                with open(os.path.join(root, f)) as fh:
                    src = fh.read()
                assert not re.search(r"^\s*(import|from)\s+oracle", src, re.M), f
                assert "tp_oracle" not in src, f


def test_form_supported_and_compensated_workspace(L):
    """The compensated form runs 2-D grids whose shot fits one thread-block
    cluster and no absorbing layer; elsewhere tp_form_supported (and every
    sizing call) rejects it, and the levels form stays available."""
    comp = native.TIME_FORMS["compensated"]
    w4 = wl.config4()
    g4 = _grid(w4)
    g4.form = comp
    assert native.tp_form_supported(g4, _geom(w4))
    ws_comp = native.tp_workspace_bytes(native.OP_FORWARD, g4, _geom(w4))
    g4.form = native.TIME_FORMS["levels"]
    ws_lev = native.tp_workspace_bytes(native.OP_FORWARD, g4, _geom(w4))
    assert ws_comp > ws_lev  # two bf16 low-part levels per shot
    w3 = wl.config3(n=64, nt=10)
    g3 = _grid(w3)
    g3.form = comp
    assert not native.tp_form_supported(g3, _geom(w3))
    assert "2-D" in native.last_error()
    assert L.tp_workspace_bytes(native.OP_FORWARD, ctypes.byref(g3), ctypes.byref(_geom(w3)), None) == 0
    g4.form = comp
    g4.sponge, g4.sponge_eta = 10, 50.0
    assert not native.tp_form_supported(g4, _geom(w4))
    big = native.tp_grid(2, 4000, 1, 3000, 10.0, 1e-3, 100, 8, 0.0, comp)
    assert not native.tp_form_supported(big, native.tp_geom(1, 1, 0x1000, 10, 0x1000))
    many = native.tp_geom(1, 1, 0x1000, 1025, 0x1000)  # more receivers per shot than one list holds
    assert native.tp_form_supported(_grid(w4), many)  # the levels form takes any count
    g4.sponge, g4.sponge_eta = 0, 0.0
    assert not native.tp_form_supported(g4, many)


def test_wait_limit_validation(L):
    assert L.tp_set_wait_limit(-5) == native.TP_ERR_ARG
    assert L.tp_set_wait_limit(0) == native.TP_OK
