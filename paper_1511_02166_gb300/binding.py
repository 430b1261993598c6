"""Thin ctypes binding of the C ABI in include/panel.h.

Argument marshalling only: torch CUDA tensors become device pointers, the
current torch stream becomes the cudaStream_t, numpy arrays become host
pointers for ``panel_plan``.  Every step of the computation runs in the CUDA
library; if the library cannot be loaded, the call raises (there is no CPU
fallback).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

PANEL_OK, PANEL_EINVAL, PANEL_ENOTSUP, PANEL_ECUDA, PANEL_ESCRATCH = 0, 1, 2, 3, 4
PANEL_NOALLOC_SCRATCH_BYTES = 32 * 1024 * 1024
PANEL_FP64 = 0x1
PANEL_MIXED = 0x2
PANEL_WITH_ADJOINT = 0x10
PANEL_FACTOR_ONLY = 0x20
PANEL_REUSE_FACTOR = 0x40
PANEL_INVERSE = 0x80
PANEL_TUNE_IR_SHIFT = 8
PANEL_TUNE_ROUNDS_SHIFT = 12
PANEL_TUNE_LU_SHIFT = 16


def PANEL_TUNE_IR(shape: int) -> int:
    """Refinement block shape field of the flags: 0 by size, 1..5 = 128 x 8, 256 x 4,
    512 x 2, 1024 x 1, 256 x 3 (threads per block x blocks per SM)."""
    return int(shape) << PANEL_TUNE_IR_SHIFT


def PANEL_TUNE_ROUNDS(sel: int) -> int:
    """Assembly field of the flags: 0 by size, 1 near-field pairs inline, 2..5 =
    queued after 4, 8, 16, 32 pairs per thread, 6 = both entries of a pair of
    control points at once."""
    return int(sel) << PANEL_TUNE_ROUNDS_SHIFT


def PANEL_TUNE_LU(kind: int) -> int:
    """FP32 LU field of the flags (n_b < 224): 0 by size, 1 trailing matrix
    through L2, 2 whole matrix in shared memory."""
    return int(kind) << PANEL_TUNE_LU_SHIFT
PANEL_N_MAX = 2048

INFO_FEW_NODES = -1
INFO_ORIENTATION = -2
INFO_ZERO_PANEL = -3
INFO_NONFINITE = -4
INFO_NOCONV = -5
INFO_TOO_LARGE = -6
INFO_DEVICE_TIMEOUT = -7

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

#: symbol -> (restype, argtypes); mirrors include/panel.h
SIGNATURES = {
    "panel_plan": (_I, [_I, _P, _P, _P, _P]),
    "panel_workspace_size": (ctypes.c_size_t, [_I, _P, _I]),
    "panel_assemble": (_I, [_I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "panel_solve": (_I, [_I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                         _I, _D, _P, _P, _P]),
    "panel_forces": (_I, [_I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "panel_viscous": (_I, [_I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                           _P]),
    "panel_adjoint": (_I, [_I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                           _P, _P, _P, _I, _D, _P, _P]),
    "panel_polar": (_I, [_I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _I, _P, _P, _P,
                         _P, _I, _D, _P, _P, _P]),
    "panel_vjp": (_I, [_I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                       _P, _P, _I, _D, _P, _P]),
    "panel_ga_sample": (_I, [_I, _I, _I, _P, _P, _P, _P]),
    "panel_ga_step": (_I, [_I, _I, _I, _D, _D, _P, _P, _P, _P, _P, _P, _P, _P]),
    "panel_ga_genome_grad": (_I, [_I, _I, _I, _P, _D, _P, _P, _P, _P, _P]),
    "panel_df_eval": (_I, [_I, _I, _P, _P, _P, _P]),
    "panel_solve_noalloc": (_I, [_I, _I, _I, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P,
                                 _P, _I, _D, _P, _P, _P]),
    "panel_debug_wait_limit": (ctypes.c_int64, [ctypes.c_int64]),
    "panel_strerror": (ctypes.c_char_p, [_I]),
    "panel_version": (ctypes.c_char_p, []),
}


class PanelError(RuntimeError):
    pass


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libpanel.so (building it first if needed); raises if that fails."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path) or not _build.up_to_date():
            if not build_if_missing:
                raise PanelError("libpanel.so is missing: run paper_1511_02166_gb300.build")
            _build.build()
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream
    import torch
    return torch.cuda.current_stream().cuda_stream


def _check(status: int, what: str):
    if status != PANEL_OK:
        msg = load().panel_strerror(status).decode()
        raise PanelError("%s failed: %s (%d)" % (what, msg, status))


def panel_plan(node_offsets: np.ndarray):
    """Host plan: (mat_offsets[B+1] i64, order[B] i32, n_max)."""
    node_offsets = np.ascontiguousarray(node_offsets, dtype=np.int64)
    B = len(node_offsets) - 1
    mat = np.zeros(B + 1, dtype=np.int64)
    order = np.zeros(max(B, 1), dtype=np.int32)
    nmax = np.zeros(1, dtype=np.int32)
    _check(load().panel_plan(B, _ptr(node_offsets), _ptr(mat), _ptr(order), _ptr(nmax)),
           "panel_plan")
    return mat, order[:B], int(nmax[0])


def panel_workspace_size(node_offsets: np.ndarray, flags: int) -> int:
    """Host: bytes of the planes, factor, pivots, rhs and lambda of a batch."""
    node_offsets = np.ascontiguousarray(node_offsets, dtype=np.int64)
    n = load().panel_workspace_size(len(node_offsets) - 1, _ptr(node_offsets), int(flags))
    if n == ctypes.c_size_t(-1).value:
        raise ValueError("panel_workspace_size: invalid offsets or flags")
    return int(n)


def panel_assemble(B, n_max, flags, nodes, node_offsets, mat_offsets, order, alpha, vinf,
                   A64, A_hi, A_lo, rhs, info, stream=None):
    _check(load().panel_assemble(B, n_max, flags, _ptr(nodes), _ptr(node_offsets),
                                 _ptr(mat_offsets), _ptr(order), _ptr(alpha), _ptr(vinf),
                                 _ptr(A64), _ptr(A_hi), _ptr(A_lo), _ptr(rhs), _ptr(info),
                                 _stream(stream)), "panel_assemble")


def panel_solve(B, n_max, flags, nodes, node_offsets, mat_offsets, order, A64, A_hi, A_lo,
                LU, piv, rhs, vinf, chord, u, lam, max_iter, tol, info, iters, stream=None):
    _check(load().panel_solve(B, n_max, flags, _ptr(nodes), _ptr(node_offsets),
                              _ptr(mat_offsets), _ptr(order), _ptr(A64), _ptr(A_hi), _ptr(A_lo),
                              _ptr(LU), _ptr(piv), _ptr(rhs), _ptr(vinf), _ptr(chord), _ptr(u),
                              _ptr(lam), int(max_iter), float(tol), _ptr(info), _ptr(iters),
                              _stream(stream)), "panel_solve")


def panel_solve_noalloc(B, n_max, flags, node_offsets_host, nodes, node_offsets, mat_offsets,
                        order, A64, A_hi, A_lo, rhs, vinf, chord, u, lam, max_iter, tol, info,
                        iters, stream=None):
    """panel_solve with the factor and pivots in the library's static device array
    (for callers that cannot allocate); node_offsets_host is a host int64 array."""
    node_offsets_host = np.ascontiguousarray(node_offsets_host, dtype=np.int64)
    _check(load().panel_solve_noalloc(B, n_max, flags, _ptr(node_offsets_host), _ptr(nodes),
                                      _ptr(node_offsets), _ptr(mat_offsets), _ptr(order),
                                      _ptr(A64), _ptr(A_hi), _ptr(A_lo), _ptr(rhs), _ptr(vinf),
                                      _ptr(chord), _ptr(u), _ptr(lam), int(max_iter), float(tol),
                                      _ptr(info), _ptr(iters), _stream(stream)),
           "panel_solve_noalloc")


def panel_forces(B, nodes, node_offsets, u, alpha, vinf, chord, info, cp, cl, cl_p, cd_p,
                 stream=None):
    _check(load().panel_forces(B, _ptr(nodes), _ptr(node_offsets), _ptr(u), _ptr(alpha),
                               _ptr(vinf), _ptr(chord), _ptr(info), _ptr(cp), _ptr(cl),
                               _ptr(cl_p), _ptr(cd_p), _stream(stream)), "panel_forces")


def panel_adjoint(B, n_max, flags, nodes, node_offsets, mat_offsets, order, A64, A_hi, A_lo,
                  LU, piv, u, lambda_in, lambda_out, alpha, vinf, chord, grad_cl, grad_nodes,
                  max_iter, tol, info, stream=None):
    _check(load().panel_adjoint(B, n_max, flags, _ptr(nodes), _ptr(node_offsets),
                                _ptr(mat_offsets), _ptr(order), _ptr(A64), _ptr(A_hi),
                                _ptr(A_lo), _ptr(LU), _ptr(piv), _ptr(u), _ptr(lambda_in),
                                _ptr(lambda_out), _ptr(alpha), _ptr(vinf), _ptr(chord),
                                _ptr(grad_cl), _ptr(grad_nodes), int(max_iter), float(tol),
                                _ptr(info), _stream(stream)), "panel_adjoint")


def panel_viscous(B, nodes, node_offsets, u, alpha, vinf, chord, reynolds, info, cl, ld, cd,
                  cd_f=None, theta=None, cf=None, sep=None, stream=None):
    _check(load().panel_viscous(B, _ptr(nodes), _ptr(node_offsets), _ptr(u), _ptr(alpha),
                                _ptr(vinf), _ptr(chord), _ptr(reynolds), _ptr(info), _ptr(cl),
                                _ptr(ld), _ptr(cd), _ptr(cd_f), _ptr(theta), _ptr(cf), _ptr(sep),
                                _stream(stream)),
           "panel_viscous")


def panel_polar(B, n_max, flags, nodes, node_offsets, mat_offsets, order, A_hi, A_lo, LU, piv,
                vinf, chord, K, alphas, u_y, u_x, cl, max_iter, tol, info, iters, stream=None):
    _check(load().panel_polar(B, n_max, flags, _ptr(nodes), _ptr(node_offsets),
                              _ptr(mat_offsets), _ptr(order), _ptr(A_hi), _ptr(A_lo), _ptr(LU),
                              _ptr(piv), _ptr(vinf), _ptr(chord), int(K), _ptr(alphas),
                              _ptr(u_y), _ptr(u_x), _ptr(cl), int(max_iter), float(tol),
                              _ptr(info), _ptr(iters), _stream(stream)), "panel_polar")


def panel_vjp(B, n_max, flags, nodes, node_offsets, mat_offsets, order, A_hi, A_lo, LU, piv, u,
              alpha, vinf, chord, w_cl, w_u, w_cp, lam, grad_nodes, max_iter, tol, info,
              stream=None):
    _check(load().panel_vjp(B, n_max, flags, _ptr(nodes), _ptr(node_offsets), _ptr(mat_offsets),
                            _ptr(order), _ptr(A_hi), _ptr(A_lo), _ptr(LU), _ptr(piv), _ptr(u),
                            _ptr(alpha), _ptr(vinf), _ptr(chord), _ptr(w_cl), _ptr(w_u),
                            _ptr(w_cp), _ptr(lam), _ptr(grad_nodes), int(max_iter), float(tol),
                            _ptr(info), _stream(stream)), "panel_vjp")


def panel_ga_sample(B, P, n, ctrl_x, genome, nodes, stream=None):
    _check(load().panel_ga_sample(int(B), int(P), int(n), _ptr(ctrl_x), _ptr(genome),
                                  _ptr(nodes), _stream(stream)), "panel_ga_sample")


def panel_ga_genome_grad(B, P, n, grad_nodes, lr, lo, hi, genome, grad_genome, stream=None):
    _check(load().panel_ga_genome_grad(B, P, n, _ptr(grad_nodes), float(lr), _ptr(lo), _ptr(hi),
                                       _ptr(genome), _ptr(grad_genome), _stream(stream)),
           "panel_ga_genome_grad")


def panel_ga_step(B, P, k, p, pm, lo, hi, sigma, genome_in, fitness, rand, genome_out,
                  stream=None):
    _check(load().panel_ga_step(int(B), int(P), int(k), float(p), float(pm), _ptr(lo), _ptr(hi),
                                _ptr(sigma), _ptr(genome_in), _ptr(fitness), _ptr(rand),
                                _ptr(genome_out), _stream(stream)), "panel_ga_step")


def panel_df_eval(op, count, a, b, out, stream=None):
    _check(load().panel_df_eval(int(op), int(count), _ptr(a), _ptr(b), _ptr(out),
                                _stream(stream)), "panel_df_eval")


def panel_debug_wait_limit(polls: int) -> int:
    """Polls after which a pipeline wait of the large-airfoil tensor-core update
    gives up (diagnostic; <= 0 restores the default).  Returns the previous value."""
    return int(load().panel_debug_wait_limit(int(polls)))


def panel_strerror(status: int) -> str:
    return load().panel_strerror(int(status)).decode()


def panel_version() -> str:
    return load().panel_version().decode()
