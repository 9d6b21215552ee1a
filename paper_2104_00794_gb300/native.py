"""ctypes binding of the C ABI in include/tprobe.h (libtprobe.so).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the library.  The names mirror the C entry points.  If the
library cannot be built or loaded this module raises; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

TP_OK, TP_ERR_ARG, TP_ERR_UNSTABLE, TP_ERR_NOMEM, TP_ERR_CUDA, TP_ERR_TIMEOUT = range(6)
STATUS_NAMES = {0: "TP_OK", 1: "TP_ERR_ARG", 2: "TP_ERR_UNSTABLE", 3: "TP_ERR_NOMEM", 4: "TP_ERR_CUDA",
                5: "TP_ERR_TIMEOUT"}
PROBE_KINDS = {"rademacher": 0, "gaussian": 1, "identity": 2, "user": 3}
OP_FORWARD, OP_ADJOINT, OP_GRADIENT_PROBED, OP_GRADIENT_FULL, OP_PROBED_FORWARD, OP_PROBED_BACKWARD = range(6)
ACC_TYPES = {"f32": 0, "bf16": 1, "bf16_kahan": 2, "f32_fold": 3}
IMAGE_CONDS = {"correlation": 0, "gradient": 1}
TIME_FORMS = {"levels": 0, "increment": 1, "compensated": 2}
KERNEL_KINDS = 7


class tp_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_float), ("dt", ctypes.c_float), ("nt", ctypes.c_int), ("order", ctypes.c_int),
                ("vmax", ctypes.c_float), ("form", ctypes.c_int), ("sponge", ctypes.c_int),
                ("sponge_eta", ctypes.c_float)]


class tp_geom(ctypes.Structure):
    _fields_ = [("nshots", ctypes.c_int), ("nsrc", ctypes.c_int), ("src", ctypes.c_void_p),
                ("nrec", ctypes.c_int), ("rec", ctypes.c_void_p)]


class tp_probe(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("r", ctypes.c_int), ("T", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("Z_user", ctypes.c_void_p), ("scale", ctypes.c_float), ("acc", ctypes.c_int)]


class TprobeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def lib_path() -> str:
    return _build.LIB


def lib():
    """Loads libtprobe.so, building it in-tree first if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        L = ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
        vp, sz, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int
        G, E, Pr = ctypes.POINTER(tp_grid), ctypes.POINTER(tp_geom), ctypes.POINTER(tp_probe)
        L.tp_workspace_bytes.argtypes = [i32, G, E, Pr]
        L.tp_workspace_bytes.restype = sz
        L.tp_forward.argtypes = [G, E, vp, vp, vp, vp, sz, vp]
        L.tp_adjoint.argtypes = [G, E, vp, vp, vp, vp, sz, vp]
        L.tp_gradient_probed.argtypes = [G, E, Pr, vp, vp, vp, vp, vp, vp, vp, sz, vp]
        L.tp_gradient_full.argtypes = [G, E, vp, vp, vp, vp, vp, vp, vp, sz, vp]
        L.tp_probes.argtypes = [Pr, i32, i32, vp, vp]
        L.tp_workspace_status.argtypes = [vp, sz, vp]
        L.tp_misfit_noalloc.argtypes = [vp, vp, ctypes.c_int64, vp, vp]
        L.tp_qr_workspace_bytes.argtypes = [i32, i32, i32, i32]
        L.tp_qr_workspace_bytes.restype = sz
        L.tp_qr_probes.argtypes = [Pr, i32, i32, i32, vp, vp, vp, sz, vp]
        L.tp_probed_state_bytes.argtypes = [G, E, Pr]
        L.tp_probed_state_bytes.restype = sz
        L.tp_probed_forward.argtypes = [G, E, Pr, vp, vp, vp, vp, sz, vp, sz, vp]
        L.tp_probed_backward.argtypes = [G, E, Pr, vp, vp, vp, i32, vp, vp, vp, sz, vp, sz, vp]
        L.tp_probed_image.argtypes = [G, E, Pr, vp, vp, i32, vp, vp, sz, vp, sz, vp]
        L.tp_residual_workspace_bytes.argtypes = []
        L.tp_residual_workspace_bytes.restype = sz
        L.tp_residual.argtypes = [vp, vp, ctypes.c_int64, vp, vp, sz, vp]
        L.tp_last_error.restype = ctypes.c_char_p
        L.tp_profile_begin.argtypes = [i32]
        L.tp_profile_end.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)]
        L.tp_set_wait_limit.argtypes = [ctypes.c_int64]
        L.tp_form_supported.argtypes = [G, E]
        L.tp_kernel_name.argtypes = [i32]
        L.tp_kernel_name.restype = ctypes.c_char_p
        for f in ("tp_forward", "tp_adjoint", "tp_gradient_probed", "tp_gradient_full", "tp_probes",
                  "tp_workspace_status", "tp_profile_begin", "tp_profile_end", "tp_misfit_noalloc",
                  "tp_probed_forward", "tp_probed_backward", "tp_qr_probes", "tp_probed_image", "tp_residual",
                  "tp_set_wait_limit", "tp_form_supported"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
        return L


def _check(status: int):
    if status != TP_OK:
        raise TprobeError(status, lib().tp_last_error().decode())


def last_error() -> str:
    return lib().tp_last_error().decode()


# ---------------------------------------------------------------- entry points
def tp_workspace_bytes(op: int, grid: tp_grid, geom: tp_geom, probe: tp_probe | None = None) -> int:
    n = lib().tp_workspace_bytes(op, ctypes.byref(grid), ctypes.byref(geom),
                                 ctypes.byref(probe) if probe is not None else None)
    if n == 0:
        raise TprobeError(TP_ERR_ARG, last_error())
    return int(n)


def tp_forward(grid, geom, vel, wavelet, d_out, ws, ws_bytes, stream):
    _check(lib().tp_forward(ctypes.byref(grid), ctypes.byref(geom), vel, wavelet, d_out, ws, ws_bytes, stream))


def tp_adjoint(grid, geom, vel, d_in, q_out, ws, ws_bytes, stream):
    _check(lib().tp_adjoint(ctypes.byref(grid), ctypes.byref(geom), vel, d_in, q_out, ws, ws_bytes, stream))


def tp_gradient_probed(grid, geom, probe, vel, wavelet, d_obs, grad, misfit, gnorm, ws, ws_bytes, stream):
    _check(lib().tp_gradient_probed(ctypes.byref(grid), ctypes.byref(geom), ctypes.byref(probe), vel, wavelet,
                                    d_obs, grad, misfit, gnorm, ws, ws_bytes, stream))


def tp_gradient_full(grid, geom, vel, wavelet, d_obs, grad, misfit, gnorm, ws, ws_bytes, stream):
    _check(lib().tp_gradient_full(ctypes.byref(grid), ctypes.byref(geom), vel, wavelet, d_obs, grad, misfit,
                                  gnorm, ws, ws_bytes, stream))


def tp_probed_state_bytes(grid, geom, probe) -> int:
    n = lib().tp_probed_state_bytes(ctypes.byref(grid), ctypes.byref(geom), ctypes.byref(probe))
    if n == 0:
        raise TprobeError(TP_ERR_ARG, last_error())
    return int(n)


def tp_probed_forward(grid, geom, probe, vel, wavelet, d_out, state, state_bytes, ws, ws_bytes, stream):
    _check(lib().tp_probed_forward(ctypes.byref(grid), ctypes.byref(geom), ctypes.byref(probe), vel, wavelet, d_out,
                                   state, state_bytes, ws, ws_bytes, stream))


def tp_probed_backward(grid, geom, probe, vel, wavelet, adj_src, wrt_velocity, grad, gnorm, state, state_bytes, ws,
                       ws_bytes, stream):
    _check(lib().tp_probed_backward(ctypes.byref(grid), ctypes.byref(geom), ctypes.byref(probe), vel, wavelet,
                                    adj_src, int(wrt_velocity), grad, gnorm, state, state_bytes, ws, ws_bytes,
                                    stream))


def tp_qr_workspace_bytes(nt, nrec, nshots, r) -> int:
    n = lib().tp_qr_workspace_bytes(nt, nrec, nshots, r)
    if n == 0:
        raise TprobeError(TP_ERR_ARG, "invalid sizes for range-finding probes")
    return int(n)


def tp_probed_image(grid, geom, probe, vel, adj_src, cond, image, state, state_bytes, ws, ws_bytes, stream):
    _check(lib().tp_probed_image(ctypes.byref(grid), ctypes.byref(geom), ctypes.byref(probe), vel, adj_src,
                                 int(cond), image, state, state_bytes, ws, ws_bytes, stream))


def tp_qr_probes(probe, nt, nrec, nshots, d_obs, Q, ws, ws_bytes, stream):
    _check(lib().tp_qr_probes(ctypes.byref(probe), nt, nrec, nshots, d_obs, Q, ws, ws_bytes, stream))


def tp_probes(probe, nt, shot, Z, stream):
    _check(lib().tp_probes(ctypes.byref(probe), nt, shot, Z, stream))


def tp_residual_workspace_bytes() -> int:
    return int(lib().tp_residual_workspace_bytes())


def tp_residual(d, d_obs, n, misfit, ws, ws_bytes, stream):
    """d -= d_obs in place (the adjoint source) and J = 1/2 sum (d - d_obs)^2
    into the device double at `misfit` (Eq. 2, the fused call's reduction)."""
    _check(lib().tp_residual(d, d_obs, n, misfit, ws, ws_bytes, stream))


def tp_misfit_noalloc(d_syn, d_obs, n, misfit, stream):
    """J = 1/2 sum (d_syn - d_obs)^2 into the device double at `misfit`,
    using the library's fixed scratch instead of a workspace (for callers
    that cannot allocate device memory at that point)."""
    _check(lib().tp_misfit_noalloc(d_syn, d_obs, n, misfit, stream))


def tp_workspace_status(ws, ws_bytes, stream):
    _check(lib().tp_workspace_status(ws, ws_bytes, stream))


def tp_form_supported(grid, geom) -> bool:
    """Whether the library can run `grid` (its time form in particular) for
    batches with geom's counts (no device work)."""
    return lib().tp_form_supported(ctypes.byref(grid), ctypes.byref(geom)) == TP_OK


def tp_set_wait_limit(cycles: int):
    """Spin limit (SM cycles) of the pipelined kernels' role waits for the
    launches that follow; 0 restores the default (about one second)."""
    _check(lib().tp_set_wait_limit(int(cycles)))


def tp_profile_begin(max_launches: int = 0):
    _check(lib().tp_profile_begin(max_launches))


def tp_profile_end() -> dict:
    ms = (ctypes.c_double * KERNEL_KINDS)()
    n = (ctypes.c_int64 * KERNEL_KINDS)()
    _check(lib().tp_profile_end(ms, n))
    return {lib().tp_kernel_name(k).decode(): {"ms": ms[k], "launches": int(n[k])} for k in range(KERNEL_KINDS)}


def exported_symbols() -> list[str]:
    """Names of the tp_* functions declared in include/tprobe.h."""
    import re
    hdr = os.path.join(_build.INCLUDE, "tprobe.h")
    with open(hdr) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(tp_[a-z_0-9]+)\s*\(", text)))
