"""FP64 CPU oracle for the batched 2D panel method (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  The CUDA
library never does, and this package imports nothing from it.

The arithmetic lives in ``panel_oracle.c`` (plain C, IEEE double, OpenMP only
across airfoils); this module compiles it with gcc on first use and wraps it
with ctypes.  Function names follow Section 2 of the paper: the panel integral
F_i, the bordered collocation + Kutta system, its LU solve, and the forces.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "panel_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIBS = {"double": os.path.join(_BUILD, "liboracle.so"),
         "long": os.path.join(_BUILD, "liboracle_ld.so")}
_lock = threading.Lock()
_loaded = {}
_current = threading.local()

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int32)
_INT = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile panel_oracle.c twice (gcc -O2, OpenMP): working type double
    (liboracle.so) and long double (liboracle_ld.so)."""
    os.makedirs(_BUILD, exist_ok=True)
    for kind, path in _LIBS.items():
        if (not force and os.path.exists(path)
                and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
            continue
        tmp = path + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        if kind == "long":
            cmd.insert(1, "-DORACLE_LONG_DOUBLE")
        subprocess.run(cmd, check=True)
        os.replace(tmp, path)
    return _LIBS["double"]


def _bind(lib):
    lib.oracle_is_extended.restype = ctypes.c_int
    lib.oracle_is_extended.argtypes = []
    lib.oracle_signed_area.restype = ctypes.c_double
    lib.oracle_signed_area.argtypes = [ctypes.c_int, _D]
    lib.oracle_panel_integral.restype = ctypes.c_double
    lib.oracle_panel_integral.argtypes = [ctypes.c_double] * 6
    lib.oracle_panel_integral_dual.restype = None
    lib.oracle_panel_integral_dual.argtypes = [_D, _D, _D]
    lib.oracle_assemble.restype = None
    lib.oracle_assemble.argtypes = [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double, _D, _D]
    lib.oracle_lu_factor.restype = ctypes.c_int
    lib.oracle_lu_factor.argtypes = [ctypes.c_int, _D, _INT]
    lib.oracle_lu_solve.restype = None
    lib.oracle_lu_solve.argtypes = [ctypes.c_int, _D, _INT, _D]
    lib.oracle_lu_solve_transposed.restype = None
    lib.oracle_lu_solve_transposed.argtypes = [ctypes.c_int, _D, _INT, _D]
    lib.oracle_forces.restype = None
    lib.oracle_forces.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_double,
                                  ctypes.c_double, _D, _D]
    lib.oracle_evaluate.restype = ctypes.c_int
    lib.oracle_evaluate.argtypes = [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, _D, _D, _D]
    lib.oracle_cl_gradient.restype = ctypes.c_int
    lib.oracle_cl_gradient.argtypes = [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, _D]
    lib.oracle_vjp.restype = ctypes.c_int
    lib.oracle_vjp.argtypes = [ctypes.c_int, _D, ctypes.c_double, ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, _D, _D, _D]
    lib.oracle_evaluate_batch.restype = None
    lib.oracle_evaluate_batch.argtypes = [ctypes.c_int, _D, _I64, _D, _D, _D, _D, _D, _D,
                                          _D, _D, _I32, ctypes.c_int]
    lib.oracle_cl_gradient_batch.restype = None
    lib.oracle_cl_gradient_batch.argtypes = [ctypes.c_int, _D, _I64, _D, _D, _D, _D, _I32,
                                             ctypes.c_int]
    lib.oracle_cl_gradient_strided_batch.restype = None
    lib.oracle_cl_gradient_strided_batch.argtypes = [ctypes.c_int, _D, _I64, _D, _D, _D,
                                                     ctypes.c_int, _D, _I32, ctypes.c_int]
    lib.oracle_max_threads.restype = ctypes.c_int
    lib.oracle_max_threads.argtypes = []
    return lib


def _load(kind=None):
    kind = kind or getattr(_current, "kind", "double")
    with _lock:
        if kind not in _loaded:
            build()
            _loaded[kind] = _bind(ctypes.CDLL(_LIBS[kind]))
        return _loaded[kind]


class extended:
    """Context manager: inside ``with oracle.extended():`` every oracle call of
    this thread uses the long double build of the same source."""

    def __enter__(self):
        self._prev = getattr(_current, "kind", "double")
        _current.kind = "long"
        return self

    def __exit__(self, *exc):
        _current.kind = self._prev
        return False


def is_extended() -> bool:
    return bool(_load().oracle_is_extended())


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------------
# Single-airfoil functions (Section 2)
# --------------------------------------------------------------------------

def signed_area(nodes) -> float:
    nodes = _f64(nodes)
    return _load().oracle_signed_area(len(nodes), _dp(nodes))


def panel_integral(p, a, b) -> float:
    """F_i(p)/gamma_i for the panel a -> b, the printed closed form (Section 2)."""
    return _load().oracle_panel_integral(float(p[0]), float(p[1]), float(a[0]), float(a[1]),
                                         float(b[0]), float(b[1]))


def panel_integral_dual(inputs6, seed6):
    """(value, directional derivative) of the panel integral with dual numbers."""
    i6 = _f64(inputs6)
    s6 = _f64(seed6)
    out = np.zeros(2)
    _load().oracle_panel_integral_dual(_dp(i6), _dp(s6), _dp(out))
    return float(out[0]), float(out[1])


def assemble(nodes, alpha: float, vinf: float = 1.0):
    """Bordered (n+1)x(n+1) matrix M and right-hand side b (collocation + Kutta)."""
    nodes = _f64(nodes)
    n = len(nodes)
    M = np.zeros((n + 1, n + 1))
    b = np.zeros(n + 1)
    _load().oracle_assemble(n, _dp(nodes), float(alpha), float(vinf), _dp(M), _dp(b))
    return M, b


def lu_factor(A):
    """In-place-style LU with partial pivoting; returns (LU, piv, info)."""
    LU = _f64(A).copy()
    m = LU.shape[0]
    piv = np.zeros(m, dtype=np.intc)
    info = _load().oracle_lu_factor(m, _dp(LU), piv.ctypes.data_as(_INT))
    return LU, piv, info


def lu_solve(LU, piv, rhs, transposed: bool = False):
    x = _f64(rhs).copy()
    LU = _f64(LU)
    piv = np.ascontiguousarray(piv, dtype=np.intc)
    fn = _load().oracle_lu_solve_transposed if transposed else _load().oracle_lu_solve
    fn(LU.shape[0], _dp(LU), piv.ctypes.data_as(_INT), _dp(x))
    return x


def forces(nodes, u, alpha: float, vinf: float = 1.0, chord: float = 1.0):
    """(cp[n], Cl, Cl_p, Cd_p) from the solved strengths u = (gamma, C)."""
    nodes = _f64(nodes)
    u = _f64(u)
    n = len(nodes)
    cp = np.zeros(n)
    out = np.zeros(3)
    _load().oracle_forces(n, _dp(nodes), _dp(u), float(alpha), float(vinf), float(chord),
                          _dp(cp), _dp(out))
    return cp, float(out[0]), float(out[1]), float(out[2])


def evaluate(nodes, alpha: float, vinf: float = 1.0, chord: float = 1.0):
    """Full solve of one airfoil: dict(u, gamma, C, cp, cl, cl_p, cd_p, info)."""
    nodes = _f64(nodes)
    n = len(nodes)
    u = np.zeros(n + 1)
    cp = np.zeros(n)
    out = np.full(3, np.nan)
    info = _load().oracle_evaluate(n, _dp(nodes), float(alpha), float(vinf), float(chord),
                                   _dp(u), _dp(cp), _dp(out))
    return dict(u=u, gamma=u[:n], C=u[n], cp=cp, cl=out[0], cl_p=out[1], cd_p=out[2],
                info=info)


def cl_gradient(nodes, alpha: float, vinf: float = 1.0, chord: float = 1.0):
    """dCl/d(node coordinates) [n][2] by forward tangents; returns (grad, info)."""
    nodes = _f64(nodes)
    n = len(nodes)
    g = np.zeros((n, 2))
    info = _load().oracle_cl_gradient(n, _dp(nodes), float(alpha), float(vinf), float(chord),
                                      _dp(g))
    return g, info


def vjp(nodes, alpha: float, w_cl: float = 0.0, w_u=None, w_cp=None, vinf: float = 1.0,
        chord: float = 1.0):
    """Gradient w.r.t. the nodes [n][2] of w_cl Cl + w_u . u + w_cp . Cp by forward
    tangents, u = (gamma, C) (w_u of length n + 1); returns (grad, info)."""
    nodes = _f64(nodes)
    n = len(nodes)
    g = np.zeros((n, 2))
    wg = None if w_u is None else _f64(w_u)
    wc = None if w_cp is None else _f64(w_cp)
    info = _load().oracle_vjp(n, _dp(nodes), float(alpha), float(vinf), float(chord),
                              float(w_cl), _dp(wg), _dp(wc), _dp(g))
    return g, info


# --------------------------------------------------------------------------
# Ragged batches
# --------------------------------------------------------------------------

def evaluate_batch(nodes, offsets, alpha, vinf=None, chord=None, nthreads: int = 0):
    """Evaluate a ragged batch; u packed at offsets[b] + b (n_b + 1 values each)."""
    nodes = _f64(nodes)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    alpha = _f64(alpha)
    B = len(offsets) - 1
    total = int(offsets[-1])
    u = np.zeros(total + B)
    cp = np.zeros(total)
    cl = np.zeros(B)
    clp = np.zeros(B)
    cdp = np.zeros(B)
    info = np.zeros(B, dtype=np.int32)
    vinf = _f64(vinf) if vinf is not None else None
    chord = _f64(chord) if chord is not None else None
    _load().oracle_evaluate_batch(B, _dp(nodes), offsets.ctypes.data_as(_I64), _dp(alpha),
                                  _dp(vinf), _dp(chord), _dp(u), _dp(cp), _dp(cl), _dp(clp),
                                  _dp(cdp), info.ctypes.data_as(_I32), int(nthreads))
    return dict(u=u, cp=cp, cl=cl, cl_p=clp, cd_p=cdp, info=info)


def cl_gradient_batch(nodes, offsets, alpha, vinf=None, chord=None, nthreads: int = 0):
    nodes = _f64(nodes)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    alpha = _f64(alpha)
    B = len(offsets) - 1
    grad = np.zeros_like(nodes)
    info = np.zeros(B, dtype=np.int32)
    vinf = _f64(vinf) if vinf is not None else None
    chord = _f64(chord) if chord is not None else None
    _load().oracle_cl_gradient_batch(B, _dp(nodes), offsets.ctypes.data_as(_I64), _dp(alpha),
                                     _dp(vinf), _dp(chord), _dp(grad),
                                     info.ctypes.data_as(_I32), int(nthreads))
    return grad, info


def cl_gradient_strided_batch(nodes, offsets, alpha, node_stride: int, vinf=None, chord=None,
                              nthreads: int = 0):
    """dCl/d(nodes) of the nodes k = 0, s, 2s, ... of every airfoil only (the
    other rows of the result are 0): a bounded sample of the gradient's work."""
    nodes = _f64(nodes)
    offsets = np.ascontiguousarray(offsets, dtype=np.int64)
    alpha = _f64(alpha)
    B = len(offsets) - 1
    grad = np.zeros_like(nodes)
    info = np.zeros(B, dtype=np.int32)
    vinf = _f64(vinf) if vinf is not None else None
    chord = _f64(chord) if chord is not None else None
    _load().oracle_cl_gradient_strided_batch(B, _dp(nodes), offsets.ctypes.data_as(_I64),
                                             _dp(alpha), _dp(vinf), _dp(chord), int(node_stride),
                                             _dp(grad), info.ctypes.data_as(_I32), int(nthreads))
    return grad, info


def max_threads() -> int:
    return int(_load().oracle_max_threads())
