"""FP64 CPU oracle for the probed FWI gradient (arXiv 2104.00794).

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The CUDA
library never calls it and shares no code with it.

The arithmetic lives in ``tp_oracle.c`` (plain double-precision loops with
OpenMP over grid points); this module compiles it with gcc on first use and
wraps each entry point for numpy arrays.  Every function cites the passage of
the paper it follows in ``tp_oracle.c``:

  forward          F(m; q): Eq. 2 and Algorithm 1 line 1
  adjoint          F^T: Algorithm 1 line 5 (exact discrete transpose)
  gradient_full    Eq. 3, full forward history stored
  gradient_probed  Algorithm 1 / Eq. 4 (form 0 as printed, form 1 with the
                   second time difference folded into the probes)
  probes           Eq. 1 probing vectors from SplitMix64 (Rademacher,
                   Irwin-Hall Gaussian, identity)
  qr_probes        Eq. 6 range-finding probes qr(D D^T Z) (numpy / LAPACK)
  fd_weights       Fornberg (1988) centred second-derivative weights
  image_full       imaging conditions applied to every time step (numpy)
  image_probed     the same conditions applied to the probed fields (Eq. 5)
  fd_weights_first Fornberg (1988) centred first-derivative weights (numpy)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tp_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

PROBE_KINDS = {"rademacher": 0, "gaussian": 1, "identity": 2}


class Grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nz", ctypes.c_int), ("nt", ctypes.c_int), ("order", ctypes.c_int),
                ("h", ctypes.c_double), ("dt", ctypes.c_double),
                ("sponge", ctypes.c_int), ("sponge_eta", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile tp_oracle.c into oracle/lib/liboracle.so (gcc, -O2, OpenMP)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_LIBDIR, exist_ok=True)
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.POINTER
    d, i64, i32 = P(ctypes.c_double), P(ctypes.c_int64), ctypes.c_int
    g = P(Grid)
    lib.oracle_fd_weights.argtypes = [i32, d]
    lib.oracle_laplacian.argtypes = [g, d, d]
    lib.oracle_laplacian.restype = None
    lib.oracle_forward.argtypes = [g, i32, i64, i32, i64, d, d, d, d]
    lib.oracle_adjoint.argtypes = [g, i32, i64, i32, i64, d, d, d, d]
    lib.oracle_gradient_full.argtypes = [g, i32, i64, i32, i64, d, d, d, d, d]
    lib.oracle_gradient_probed.argtypes = [g, i32, i64, i32, i64, d, d, d, i32, d,
                                           ctypes.c_double, i32, d, d, d, d]
    lib.oracle_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    lib.oracle_splitmix64.restype = ctypes.c_uint64
    lib.oracle_probes.argtypes = [i32, i32, i32, ctypes.c_uint64, i32, d]
    _lib = lib
    return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _i64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int64).ravel())


def make_grid(ndim, nx, ny, nz, h, dt, nt, order, sponge=0, sponge_eta=0.0) -> Grid:
    """sponge / sponge_eta: width (cells) and peak damping [1/s] of the
    absorbing layer on every face (0: none)."""
    return Grid(int(ndim), int(nx), int(ny), int(nz), int(nt), int(order), float(h), float(dt),
                int(sponge), float(sponge_eta))


def grid_of(w, nt=None) -> Grid:
    """Grid of a ``workloads.Workload`` (optionally with a truncated nt)."""
    return make_grid(w.ndim, w.nx, w.ny, w.nz, w.h, w.dt, w.nt if nt is None else nt, w.order,
                     getattr(w, "sponge", 0), getattr(w, "sponge_eta", 0.0))


def fd_weights(order: int) -> np.ndarray:
    w = np.zeros(order // 2 + 1)
    if _load().oracle_fd_weights(order, _dp(w)) != 0:
        raise ValueError(f"unsupported order {order}")
    return w


def laplacian(g: Grid, u) -> np.ndarray:
    u = _f64(u).ravel()
    out = np.empty_like(u)
    _load().oracle_laplacian(ctypes.byref(g), _dp(u), _dp(out))
    return out


def forward(g: Grid, src, rec, vel, q, keep_history=False):
    """Data d [nt, nrec] (and the history [nt, N] if asked) for one shot."""
    src, rec, vel, q = _i64(src), _i64(rec), _f64(vel).ravel(), _f64(q)
    N = g.nx * g.ny * g.nz
    d = np.zeros((g.nt, rec.size))
    hist = np.zeros((g.nt, N)) if keep_history else None
    rc = _load().oracle_forward(ctypes.byref(g), src.size, _ip(src), rec.size, _ip(rec), _dp(vel),
                                _dp(q), _dp(d), _dp(hist))
    if rc:
        raise MemoryError("oracle_forward failed")
    return (d, hist) if keep_history else d


def adjoint(g: Grid, src, rec, vel, s, keep_history=False):
    """F^T s: [nt, nsrc] (and lambda history [nt, N] if asked) for one shot."""
    src, rec, vel, s = _i64(src), _i64(rec), _f64(vel).ravel(), _f64(s)
    N = g.nx * g.ny * g.nz
    q = np.zeros((g.nt, src.size))
    hist = np.zeros((g.nt, N)) if keep_history else None
    rc = _load().oracle_adjoint(ctypes.byref(g), src.size, _ip(src), rec.size, _ip(rec), _dp(vel),
                                _dp(s), _dp(q), _dp(hist))
    if rc:
        raise MemoryError("oracle_adjoint failed")
    return (q, hist) if keep_history else q


def gradient_full(g: Grid, src, rec, vel, q, dobs):
    """(dJ/dm [N], J) with the full forward history, one shot."""
    src, rec, vel, q, dobs = _i64(src), _i64(rec), _f64(vel).ravel(), _f64(q), _f64(dobs)
    grad = np.zeros(g.nx * g.ny * g.nz)
    J = ctypes.c_double(0.0)
    rc = _load().oracle_gradient_full(ctypes.byref(g), src.size, _ip(src), rec.size, _ip(rec),
                                      _dp(vel), _dp(q), _dp(dobs), _dp(grad), ctypes.byref(J))
    if rc:
        raise MemoryError("oracle_gradient_full failed")
    return grad, J.value


def gradient_probed(g: Grid, src, rec, vel, q, dobs, Q, scale, form=0, keep_acc=False):
    """(probed dJ/dm estimate [N], J[, ubar, vbar]) for one shot (Algorithm 1)."""
    src, rec, vel, q, dobs, Q = (_i64(src), _i64(rec), _f64(vel).ravel(), _f64(q), _f64(dobs),
                                 _f64(Q))
    N = g.nx * g.ny * g.nz
    r = Q.shape[1]
    assert Q.shape[0] == g.nt
    grad = np.zeros(N)
    J = ctypes.c_double(0.0)
    ub = np.zeros((N, r)) if keep_acc else None
    vb = np.zeros((N, r)) if keep_acc else None
    rc = _load().oracle_gradient_probed(ctypes.byref(g), src.size, _ip(src), rec.size, _ip(rec),
                                        _dp(vel), _dp(q), _dp(dobs), r, _dp(Q), float(scale),
                                        int(form), _dp(grad), ctypes.byref(J), _dp(ub), _dp(vb))
    if rc:
        raise MemoryError("oracle_gradient_probed failed")
    return (grad, J.value, ub, vb) if keep_acc else (grad, J.value)


def splitmix64(state: int, n: int) -> int:
    return int(_load().oracle_splitmix64(ctypes.c_uint64(state & (2**64 - 1)), ctypes.c_uint64(n)))


def probes(kind: str, nt: int, r: int, seed: int, shot: int = 0) -> np.ndarray:
    Z = np.zeros((nt, r))
    if _load().oracle_probes(PROBE_KINDS[kind], nt, r, ctypes.c_uint64(seed), shot, _dp(Z)) != 0:
        raise ValueError("bad probe specification")
    return Z


def qr_probes(dobs_shot, Z):
    """Range-finding probes of Eq. 6: [Q, ~] = qr(A Z) with A = D_obs D_obs^T,
    D_obs the shot record as an nt x nrec matrix (time x receivers), Z the
    nt x r random probes.  Householder QR (LAPACK) in fp64; the column signs
    are fixed so that diag(R) > 0 (the QR factorisation is unique then)."""
    D = np.asarray(dobs_shot, dtype=np.float64)
    Y = D @ (D.T @ np.asarray(Z, dtype=np.float64))
    Q, R = np.linalg.qr(Y)
    sgn = np.sign(np.diag(R))
    sgn[sgn == 0] = 1.0
    return Q * sgn[None, :]


def default_scale(kind: str, r: int) -> float:
    """Eq. 1 normalisation: 1/r for random probes, 1 for the identity."""
    return 1.0 if kind == "identity" else 1.0 / r


# ------------------------------------------------------------------ batches
def batch_gradient_probed(w, vel, dobs, kind=None, r=None, seed=None, form=0, nt=None):
    """Sum over the workload's shots of the probed gradient (per-shot probes
    drawn with shot index s), plus the summed misfit."""
    kind = kind or w.probe_kind
    r = r or w.r
    seed = w.seed if seed is None else seed
    g = grid_of(w, nt)
    total = np.zeros(w.N)
    J = 0.0
    for s in range(w.nshots):
        Q = probes(kind, g.nt, r, seed, s)
        gs, js = gradient_probed(g, w.src[s], w.rec[s], vel, w.wavelet[s][: g.nt], dobs[s], Q,
                                 default_scale(kind, r), form)
        total += gs
        J += js
    return total, J


def batch_gradient_full(w, vel, dobs, nt=None):
    g = grid_of(w, nt)
    total = np.zeros(w.N)
    J = 0.0
    for s in range(w.nshots):
        gs, js = gradient_full(g, w.src[s], w.rec[s], vel, w.wavelet[s][: g.nt], dobs[s])
        total += gs
        J += js
    return total, J


def batch_forward(w, vel, nt=None):
    g = grid_of(w, nt)
    return np.stack([forward(g, w.src[s], w.rec[s], vel, w.wavelet[s][: g.nt])
                     for s in range(w.nshots)])


# ------------------------------------------------------------------ imaging conditions
IMAGE_CONDS = {"correlation": 0, "gradient": 1}


def fornberg(m: int, x0: float, xs) -> np.ndarray:
    """Weights of the m-th derivative at x0 on the nodes xs, by Fornberg's
    (1988) recursion over the nodes (weights of every order up to m are built
    together, one node at a time)."""
    xs = np.asarray(xs, dtype=np.float64)
    n = xs.size
    c = np.zeros((n, m + 1))
    c[0, 0] = 1.0
    prod_prev = 1.0
    d_prev = xs[0] - x0
    for i in range(1, n):
        kmax = min(i, m)
        prod = 1.0
        d_old = d_prev
        d_prev = xs[i] - x0
        for j in range(i):
            diff = xs[i] - xs[j]
            prod *= diff
            if j == i - 1:
                for k in range(kmax, 0, -1):
                    c[i, k] = prod_prev * (k * c[i - 1, k - 1] - d_old * c[i - 1, k]) / prod
                c[i, 0] = -prod_prev * d_old * c[i - 1, 0] / prod
            for k in range(kmax, 0, -1):
                c[j, k] = (d_prev * c[j, k] - k * c[j, k - 1]) / diff
            c[j, 0] = d_prev * c[j, 0] / diff
        prod_prev = prod
    return c[:, m]


def fd_weights_first(order: int) -> np.ndarray:
    """c_1..c_R of the centred first derivative of order 2R = `order`:
    f'(x) ~ sum_k c_k (f(x + k h) - f(x - k h)) / h."""
    R = order // 2
    w = fornberg(1, 0.0, np.arange(-R, R + 1, dtype=np.float64))
    return w[R + 1:]


def _field(g: Grid, f) -> np.ndarray:
    f = np.asarray(f, dtype=np.float64)
    return f.reshape((g.nz, g.ny, g.nx)) if g.ndim == 3 else f.reshape((g.nz, g.nx))


def _derivative(g: Grid, f: np.ndarray, axis: int) -> np.ndarray:
    """Centred first difference of the grid's order along `axis`, with zero
    values outside the grid (the modelling's Dirichlet boundary)."""
    c = fd_weights_first(g.order)
    R = c.size
    pad = [(0, 0)] * f.ndim
    pad[axis] = (R, R)
    fp = np.pad(f, pad)
    n = f.shape[axis]
    out = np.zeros_like(f)
    for k in range(1, R + 1):
        plus = np.take(fp, np.arange(R + k, R + k + n), axis=axis)
        minus = np.take(fp, np.arange(R - k, R - k + n), axis=axis)
        out += c[k - 1] * (plus - minus)
    return out / g.h


def image_of_fields(g: Grid, a, b, cond: str) -> np.ndarray:
    """<D a, D b> at every grid point: D = identity ("correlation") or the
    spatial gradient ("gradient", the products summed over the axes)."""
    A, B = _field(g, a), _field(g, b)
    if cond == "correlation":
        return (A * B).ravel()
    return sum(_derivative(g, A, ax) * _derivative(g, B, ax) for ax in range(A.ndim)).ravel()


def image_full(g: Grid, src, rec, vel, q, s, cond: str) -> np.ndarray:
    """The imaging condition applied at every time step, without probing:
    sum_{j=2}^{nt-2} <D u[j], D lambda[j+1]>, u the forward wavefield of q,
    lambda the adjoint wavefield driven by s [nt, nrec]."""
    _, U = forward(g, src, rec, vel, q, keep_history=True)
    _, Lam = adjoint(g, src, rec, vel, s, keep_history=True)
    img = np.zeros(g.nx * g.ny * g.nz)
    for j in range(2, g.nt - 1):
        img += image_of_fields(g, U[j], Lam[j + 1], cond)
    return img


def image_probed(g: Grid, src, rec, vel, q, s, Q, scale: float, cond: str) -> np.ndarray:
    """Eq. 5: the same condition applied to the r probed fields
    P_i = sum_{j=2}^{nt-2} Q[j+1, i] u[j] and V_i = sum_{k=2}^{nt-1} Q[k, i] lambda[k],
    image = scale * sum_i <D P_i, D V_i>."""
    Q = np.asarray(Q, dtype=np.float64)
    _, U = forward(g, src, rec, vel, q, keep_history=True)
    _, Lam = adjoint(g, src, rec, vel, s, keep_history=True)
    nt = g.nt
    P = Q[3:nt].T @ U[2:nt - 1]   # [r, N]
    V = Q[2:nt].T @ Lam[2:nt]     # [r, N]
    img = np.zeros(g.nx * g.ny * g.nz)
    for i in range(Q.shape[1]):
        img += image_of_fields(g, P[i], V[i], cond)
    return scale * img


def batch_image(w, vel, s_all, cond, kind=None, r=None, seed=None, probed=True, nt=None):
    """Sum over the workload's shots of image_probed (per-shot probes drawn
    with shot index s) or of image_full."""
    kind = kind or w.probe_kind
    r = r or w.r
    seed = w.seed if seed is None else seed
    g = grid_of(w, nt)
    total = np.zeros(w.N)
    for sh in range(w.nshots):
        q = w.wavelet[sh][: g.nt]
        if probed:
            Q = probes(kind, g.nt, r, seed, sh)
            total += image_probed(g, w.src[sh], w.rec[sh], vel, q, s_all[sh], Q, default_scale(kind, r), cond)
        else:
            total += image_full(g, w.src[sh], w.rec[sh], vel, q, s_all[sh], cond)
    return total
