"""C-ABI checks that need no GPU: the library builds, loads and exports every
symbol include/panel.h declares; the host planner and argument validation work."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1511_02166_gb300 import binding as bd
from paper_1511_02166_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "panel.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(panel_[a-z0-9_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(build.build())
    syms = declared_symbols()
    assert "panel_assemble" in syms and "panel_adjoint" in syms
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) <= set(bd.SIGNATURES)


def test_constants_match_header():
    txt = open(os.path.join(ROOT, "include", "panel.h")).read()
    for name, val in [("PANEL_FP64", bd.PANEL_FP64), ("PANEL_MIXED", bd.PANEL_MIXED),
                      ("PANEL_WITH_ADJOINT", bd.PANEL_WITH_ADJOINT),
                      ("PANEL_N_MAX", bd.PANEL_N_MAX),
                      ("PANEL_FACTOR_ONLY", bd.PANEL_FACTOR_ONLY),
                      ("PANEL_REUSE_FACTOR", bd.PANEL_REUSE_FACTOR),
                      ("PANEL_INVERSE", bd.PANEL_INVERSE)]:
        m = re.search(r"#define %s\s+(0x[0-9a-fA-F]+|\d+)" % name, txt)
        assert m and int(m.group(1), 0) == val, name
    for name, val in [("PANEL_INFO_FEW_NODES", bd.INFO_FEW_NODES),
                      ("PANEL_INFO_ORIENTATION", bd.INFO_ORIENTATION),
                      ("PANEL_INFO_ZERO_PANEL", bd.INFO_ZERO_PANEL),
                      ("PANEL_INFO_NONFINITE", bd.INFO_NONFINITE),
                      ("PANEL_INFO_NOCONV", bd.INFO_NOCONV),
                      ("PANEL_INFO_TOO_LARGE", bd.INFO_TOO_LARGE),
                      ("PANEL_INFO_DEVICE_TIMEOUT", bd.INFO_DEVICE_TIMEOUT)]:
        m = re.search(r"#define %s \((-\d+)\)" % name, txt)
        assert m and int(m.group(1)) == val, name


def test_plan_offsets_and_order():
    sizes = np.array([5, 200, 3, 200, 17, 0])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    mat, order, nmax = bd.panel_plan(off)
    assert nmax == 200
    assert list(mat) == list(np.concatenate([[0], np.cumsum((sizes + 1) ** 2)]))
    assert list(order) == [1, 3, 4, 0, 2, 5]  # decreasing size, stable
    empty, order0, _ = bd.panel_plan(np.zeros(1, np.int64))
    assert list(empty) == [0] and len(order0) == 0


def test_plan_rejects_bad_offsets():
    with pytest.raises(bd.PanelError):
        bd.panel_plan(np.array([0, 5, 3], np.int64))
    with pytest.raises(bd.PanelError):
        bd.panel_plan(np.array([0, bd.PANEL_N_MAX + 1], np.int64))


def test_argument_validation_before_any_launch():
    lib = bd.load()
    # negative batch, bad flags and missing pointers are rejected on the host
    assert lib.panel_assemble(-1, 10, bd.PANEL_FP64, *([None] * 11), None) == bd.PANEL_EINVAL
    assert lib.panel_assemble(1, 10, 0x3, *([None] * 11), None) == bd.PANEL_EINVAL
    assert lib.panel_assemble(1, 10, bd.PANEL_FP64, *([None] * 11), None) == bd.PANEL_EINVAL
    assert lib.panel_assemble(1, bd.PANEL_N_MAX + 1, bd.PANEL_FP64, *([None] * 11),
                              None) == bd.PANEL_EINVAL
    assert lib.panel_solve(1, 10, 0x40 | bd.PANEL_FP64, *([None] * 14), 3, 1e-12, None, None,
                           None) == bd.PANEL_EINVAL
    assert lib.panel_forces(1, *([None] * 11), None) == bd.PANEL_EINVAL
    assert lib.panel_adjoint(1, 10, bd.PANEL_MIXED, *([None] * 17), 3, 1e-12, None,
                             None) == bd.PANEL_EINVAL
    # factor/reuse stages are mixed-mode only and exclusive
    assert lib.panel_solve(1, 10, bd.PANEL_FP64 | bd.PANEL_FACTOR_ONLY, *([None] * 14), 3, 1e-12,
                           None, None, None) == bd.PANEL_EINVAL
    assert lib.panel_solve(1, 10, bd.PANEL_MIXED | bd.PANEL_FACTOR_ONLY | bd.PANEL_REUSE_FACTOR,
                           *([None] * 14), 3, 1e-12, None, None, None) == bd.PANEL_EINVAL
    # polars: mixed path only, pointers checked, an empty batch is a no-op
    args = [None] * 10 + [0, None, None, None, None, 3, 1e-12, None, None, None]
    assert lib.panel_polar(1, 10, bd.PANEL_FP64, *args) == bd.PANEL_ENOTSUP
    assert lib.panel_polar(1, 10, bd.PANEL_MIXED, *args) == bd.PANEL_EINVAL
    assert lib.panel_polar(1, 10, bd.PANEL_MIXED | bd.PANEL_INVERSE, *args) == bd.PANEL_EINVAL
    assert lib.panel_polar(0, 10, bd.PANEL_MIXED, *args) == bd.PANEL_OK
    # viscous correction: required pointers, cl required with ld
    assert lib.panel_viscous(1, *([None] * 16)) == bd.PANEL_EINVAL
    assert lib.panel_viscous(-1, *([None] * 16)) == bd.PANEL_EINVAL
    assert lib.panel_viscous(0, *([None] * 16)) == bd.PANEL_OK
    # genetic algorithm: sizes, probabilities and buffers checked before any launch
    assert lib.panel_ga_sample(1, 3, 10, None, None, None, None) == bd.PANEL_EINVAL
    assert lib.panel_ga_sample(65535 * 64 + 1, 18, 10, None, None, None, None) == bd.PANEL_EINVAL
    assert lib.panel_ga_sample(0, 18, 10, None, None, None, None) == bd.PANEL_OK
    ga = [None] * 8
    assert lib.panel_ga_step(3, 18, 4, 0.8, 0.3, *ga) == bd.PANEL_EINVAL  # odd population
    assert lib.panel_ga_step(4, 18, 17, 0.8, 0.3, *ga) == bd.PANEL_EINVAL  # tournament > 16
    assert lib.panel_ga_step(4, 18, 4, 1.5, 0.3, *ga) == bd.PANEL_EINVAL
    assert lib.panel_ga_step(4, 18, 4, 0.8, -0.1, *ga) == bd.PANEL_EINVAL
    assert lib.panel_ga_step(4, 18, 4, 0.8, 0.3, *ga) == bd.PANEL_EINVAL  # NULL buffers
    assert lib.panel_ga_step(0, 18, 4, 0.8, 0.3, *ga) == bd.PANEL_OK
    # genome gradient: sizes, NaN step, and the buffers each mode needs
    gg = lambda B, P, n, lr, *ptrs: lib.panel_ga_genome_grad(B, P, n, None, lr, *ptrs, None)
    assert gg(1, 3, 10, 0.0, None, None, None, None) == bd.PANEL_EINVAL      # P < 4
    assert gg(1, 18, 2, 0.0, None, None, None, None) == bd.PANEL_EINVAL      # n < 3
    assert gg(1, 18, 10, float("nan"), None, None, None, None) == bd.PANEL_EINVAL
    assert gg(1, 18, 10, 0.0, None, None, None, None) == bd.PANEL_EINVAL     # no node gradient
    assert gg(0, 18, 10, 0.0, None, None, None, None) == bd.PANEL_OK
    # vector-Jacobian products: mixed path only, pointers checked
    vj = [None] * 17 + [3, 1e-12, None, None]
    assert lib.panel_vjp(1, 10, bd.PANEL_FP64, *vj) == bd.PANEL_ENOTSUP
    assert lib.panel_vjp(1, 10, bd.PANEL_MIXED | bd.PANEL_INVERSE, *vj) == bd.PANEL_EINVAL
    assert lib.panel_vjp(1, 10, bd.PANEL_MIXED, *vj) == bd.PANEL_EINVAL
    assert lib.panel_vjp(1, bd.PANEL_N_MAX + 1, bd.PANEL_MIXED, *vj) == bd.PANEL_EINVAL
    assert lib.panel_vjp(0, 10, bd.PANEL_MIXED, *vj) == bd.PANEL_OK
    # an empty batch is a no-op
    assert lib.panel_forces(0, *([None] * 11), None) == bd.PANEL_OK
    assert bd.panel_strerror(bd.PANEL_EINVAL) == "invalid argument"
    assert "sm_103a" in bd.panel_version()


def test_workspace_size_counts_the_work_arrays():
    offs = np.array([0, 100, 300, 303], dtype=np.int64)
    m = np.diff(offs) + 1
    mat, vec = int((m * m).sum()), int(m.sum())
    assert bd.panel_workspace_size(offs, bd.PANEL_MIXED) == mat * 12 + vec * 20
    assert bd.panel_workspace_size(offs, bd.PANEL_FP64) == mat * 16 + vec * 20
    assert bd.panel_workspace_size(np.zeros(1, dtype=np.int64), bd.PANEL_MIXED) == 0
    with pytest.raises(ValueError):
        bd.panel_workspace_size(offs, 0)
    with pytest.raises(ValueError):
        bd.panel_workspace_size(np.array([0, bd.PANEL_N_MAX + 1]), bd.PANEL_MIXED)


def test_debug_wait_limit_is_host_state_with_a_default():
    # the tensor-core update's wait bound is a host-side setting: set, read back
    # through the previous value, restored by a non-positive argument
    default = bd.panel_debug_wait_limit(0)
    assert default == 1 << 22
    assert bd.panel_debug_wait_limit(5) == default
    assert bd.panel_debug_wait_limit(-1) == 5
    assert bd.panel_debug_wait_limit(0) == default


def test_tuning_fields_of_the_flags_are_validated():
    # the launch-shape fields are accepted in range and rejected out of range, on
    # the host, before anything is launched (null device pointers: nothing runs)
    lib = bd.load()
    offs = np.array([0, 10], dtype=np.int64)
    mat, order, nmax = bd.panel_plan(offs)
    p = ctypes.c_void_p(1)  # never dereferenced: validation fails or B = 0 returns first
    for f, want in [(bd.PANEL_MIXED | bd.PANEL_TUNE_IR(6), bd.PANEL_EINVAL),
                    (bd.PANEL_MIXED | bd.PANEL_TUNE_IR(5), bd.PANEL_OK),
                    (bd.PANEL_MIXED | bd.PANEL_TUNE_ROUNDS(7), bd.PANEL_EINVAL),
                    (bd.PANEL_MIXED | bd.PANEL_TUNE_ROUNDS(6), bd.PANEL_OK),
                    (bd.PANEL_MIXED | bd.PANEL_TUNE_LU(3), bd.PANEL_EINVAL),
                    (bd.PANEL_MIXED | bd.PANEL_TUNE_LU(2) | bd.PANEL_TUNE_IR(1), bd.PANEL_OK),
                    (bd.PANEL_MIXED | bd.PANEL_TUNE_IR(4) | bd.PANEL_TUNE_ROUNDS(5), bd.PANEL_OK)]:
        st = lib.panel_assemble(0, 10, f, p, p, p, p, p, None, None, p, p, p, p, None)
        assert st == want, (f, st)
