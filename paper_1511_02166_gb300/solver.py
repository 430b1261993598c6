"""Device-resident batches and the torch autograd wrapper over the C ABI.

``PanelBatch`` owns the torch tensors of one ragged population (inputs,
matrices, factors, solutions, forces and gradients) and runs the four library
calls on the current torch stream.  A ragged population is cut into size
buckets (contiguous runs of the size-sorted launch order), each launched with
its own size bound so that small airfoils get small shared-memory footprints;
``autotune()`` times the bucket width, and per bucket the assembly's near-field
rounds, the factorisation (LU, or the Gauss-Jordan inverse) and the
refinement's block shape, and remembers the fastest; ``capture()`` records a
whole step into a CUDA graph.  ``PanelCl`` is
a ``torch.autograd.Function`` mapping node coordinates to Cl whose backward is
``panel_adjoint``.  Everything numerical happens in the CUDA library.
"""
from __future__ import annotations

import json
import os
import threading

import numpy as np
import torch

from . import binding as bd

_tune_lock = threading.Lock()


def _tune_cache_path():
    return os.environ.get("PANEL_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "panel_gb300",
                                       "autotune.json"))


def _load_tune_cache():
    try:
        with open(_tune_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_tune_cache(cache):
    path = _tune_cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def size_buckets(sorted_sizes, width, min_count=1):
    """Contiguous runs of the (descending) sizes with equal ceil(n / width):
    a list of (start, count, n_max).  Runs shorter than ``min_count`` airfoils
    are merged with the following ones (a launch of a few blocks would leave
    most SMs idle), and a short last run joins the one before it."""
    runs = []
    start = 0
    B = len(sorted_sizes)
    while start < B:
        key = -(-int(sorted_sizes[start]) // width)
        end = start + 1
        while end < B and -(-int(sorted_sizes[end]) // width) == key:
            end += 1
        runs.append((start, end - start, max(int(sorted_sizes[start]), 3)))
        start = end
    out = []
    for r in runs:
        if out and out[-1][1] < min_count:
            s0, c0, n0 = out[-1]
            out[-1] = (s0, c0 + r[1], n0)
        else:
            out.append(r)
    if len(out) > 1 and out[-1][1] < min_count:
        s0, c0, n0 = out[-2]
        out[-2:] = [(s0, c0 + out[-1][1], n0)]
    return out

MODES = {"fp64": bd.PANEL_FP64, "mixed": bd.PANEL_MIXED}
GJ_MAX_M = 288  # largest m = n + 1 that the library factors by Gauss-Jordan
LU_SMEM_MAX_M = 224  # largest m whose LU the library can run in shared memory


def _require_cuda(device):
    dev = torch.device(device)
    if dev.type != "cuda" or not torch.cuda.is_available():
        raise RuntimeError("the panel library runs on a CUDA device only (no CPU fallback)")
    return dev


class PanelBatch:
    """A population resident in device memory, with its workspace.

    nodes [sum n_b][2] float64, offsets [B+1] int64 (host or device), alpha [B]
    float64 radians.  mode 'mixed' (double-float assembly, FP32 LU, refined) or
    'fp64' (plain FP64 path).
    """

    def __init__(self, nodes, offsets, alpha, mode: str = "mixed", vinf=None, chord=None,
                 device="cuda", max_iter: int = 10, tol: float = 1e-12,
                 bucket_width: int | None = 192, bucket_min: int = 608):
        self.device = _require_cuda(device)
        if mode not in MODES:
            raise ValueError("mode must be one of %s" % sorted(MODES))
        self.mode = mode
        self.flags = MODES[mode]
        self.max_iter = int(max_iter)
        self.tol = float(tol)
        offsets_h = np.ascontiguousarray(
            offsets.cpu().numpy() if torch.is_tensor(offsets) else offsets, dtype=np.int64)
        self.mat_offsets_h, order_h, self.n_max = bd.panel_plan(offsets_h)
        self.offsets_h = offsets_h
        self.B = len(offsets_h) - 1
        total = int(offsets_h[-1])
        self.total_nodes = total
        self.total_vec = total + self.B
        self.total_mat = int(self.mat_offsets_h[-1])
        dev = self.device
        f64 = dict(dtype=torch.float64, device=dev)
        i32 = dict(dtype=torch.int32, device=dev)
        self.nodes = torch.as_tensor(nodes, dtype=torch.float64).to(dev).contiguous()
        if self.nodes.shape != (total, 2):
            raise ValueError("nodes must be [%d][2]" % total)
        self.node_offsets = torch.as_tensor(offsets_h).to(dev)
        self.mat_offsets = torch.as_tensor(self.mat_offsets_h).to(dev)
        self.order = torch.as_tensor(order_h).to(dev)
        self.alpha = torch.as_tensor(alpha, dtype=torch.float64).to(dev).contiguous()
        self.vinf = None if vinf is None else torch.as_tensor(vinf, **f64).contiguous()
        self.chord = None if chord is None else torch.as_tensor(chord, **f64).contiguous()
        if self.flags == bd.PANEL_FP64:
            self.A64 = torch.empty(self.total_mat, **f64)
            self.A_hi = self.A_lo = None
            self.LU = torch.empty(self.total_mat, **f64)
        else:
            self.A64 = None
            self.A_hi = torch.empty(self.total_mat, dtype=torch.float32, device=dev)
            self.A_lo = torch.empty(self.total_mat, dtype=torch.float32, device=dev)
            self.LU = torch.empty(self.total_mat, dtype=torch.float32, device=dev)
        self.piv = torch.empty(self.total_vec, **i32)
        self.rhs = torch.empty(self.total_vec, **f64)
        self.u = torch.empty(self.total_vec, **f64)
        self.lam = torch.empty(self.total_vec, **f64)
        self.info = torch.zeros(self.B, **i32)
        self.iters = torch.zeros(self.B, **i32)
        self.cp = torch.empty(total, **f64)
        self.cl = torch.empty(self.B, **f64)
        self.cl_p = torch.empty(self.B, **f64)
        self.cd_p = torch.empty(self.B, **f64)
        self.grad = torch.empty(total, 2, **f64)
        self.reynolds = torch.full((self.B,), 1.0e6, **f64)
        self.cd = torch.empty(self.B, **f64)
        self.cd_f = torch.empty(self.B, **f64)
        self.ld = torch.empty(self.B, **f64)
        self.theta = torch.empty(total, **f64)
        self.cf = torch.empty(total, **f64)
        self.sep = torch.empty(self.B, 2, **i32)
        self.have_lambda = False
        sizes = np.diff(offsets_h)
        sorted_sizes = sizes[order_h] if self.B else sizes
        self.bucket_min = int(bucket_min)
        self.bucket_width = bucket_width
        if bucket_width is None or self.B == 0:
            self.buckets = [(0, self.B, self.n_max)] if self.B else []
        else:
            self.buckets = size_buckets(sorted_sizes, int(bucket_width), int(bucket_min))
        self._reset_tuning()
        self.graph = None

    def _reset_tuning(self):
        """Per bucket: the factorisation (Gauss-Jordan inverse or LU, and the
        LU's kernel), the refinement's block shape and the assembly's near-field
        rounds (0 = the library's choice by size)."""
        self.inverse = [False] * len(self.buckets)
        self.lu_kind = [0] * len(self.buckets)
        self.ir_shape = [0] * len(self.buckets)
        self.rounds = [0] * len(self.buckets)

    def set_bucket_width(self, width):
        """Cut the population into buckets of `width` panels (None: one bucket)
        and forget the per-bucket tuning."""
        sizes = np.diff(self.offsets_h)
        order_h = self.order.cpu().numpy()
        if width is None or self.B == 0:
            self.buckets = [(0, self.B, self.n_max)] if self.B else []
        else:
            self.buckets = size_buckets(sizes[order_h], int(width), self.bucket_min)
        self.bucket_width = width
        self._reset_tuning()
        self.graph = None

    # -- the four library calls (per size bucket) --------------------------------
    def assemble(self):
        for k, (start, cnt, nmax) in enumerate(self.buckets):
            bd.panel_assemble(cnt, nmax, self.flags | self._asm_tune(k), self.nodes,
                              self.node_offsets, self.mat_offsets, self.order[start:],
                              self.alpha, self.vinf, self.A64, self.A_hi, self.A_lo, self.rhs,
                              self.info)

    def _asm_tune(self, k):
        return bd.PANEL_TUNE_ROUNDS(self.rounds[k]) if self.flags == bd.PANEL_MIXED else 0

    def _solve_bucket(self, k, start, cnt, nmax, with_adjoint, stage, stream=None):
        f = self.flags | (bd.PANEL_WITH_ADJOINT if with_adjoint else 0)
        f |= {"all": 0, "factor": bd.PANEL_FACTOR_ONLY, "refine": bd.PANEL_REUSE_FACTOR}[stage]
        if self.flags == bd.PANEL_MIXED:
            f |= bd.PANEL_TUNE_IR(self.ir_shape[k])
            if not self.inverse[k]:
                f |= bd.PANEL_TUNE_LU(self.lu_kind[k])
        if self.inverse[k] and stage != "refine":
            f |= bd.PANEL_INVERSE
        bd.panel_solve(cnt, nmax, f, self.nodes, self.node_offsets, self.mat_offsets,
                       self.order[start:], self.A64, self.A_hi, self.A_lo, self.LU,
                       self.piv, self.rhs, self.vinf, self.chord, self.u,
                       self.lam if with_adjoint else None, self.max_iter, self.tol,
                       self.info, self.iters, stream=stream)

    def solve(self, with_adjoint: bool = False, stage: str = "all"):
        """stage 'all' (factor + refine), 'factor' (LU only) or 'refine' (reuse the
        stored LU; mixed mode only)."""
        for k, (start, cnt, nmax) in enumerate(self.buckets):
            self._solve_bucket(k, start, cnt, nmax, with_adjoint, stage)
        if stage != "factor":
            self.have_lambda = with_adjoint

    def forces(self):
        bd.panel_forces(self.B, self.nodes, self.node_offsets, self.u, self.alpha, self.vinf,
                        self.chord, self.info, self.cp, self.cl, self.cl_p, self.cd_p)

    def viscous(self, reynolds=None):
        """Thwaites's boundary layer on the solved surface speed (after forces()):
        cd (Squire-Young), cd_f (skin friction), ld = cl / cd, theta and cf at the
        control points, sep (separating control point per surface, -1 attached).
        `reynolds` (scalar or [B], v_inf c / nu) replaces the stored values."""
        if reynolds is not None:
            self.reynolds.copy_(torch.as_tensor(reynolds, dtype=torch.float64).expand(self.B))
        bd.panel_viscous(self.B, self.nodes, self.node_offsets, self.u, self.alpha, self.vinf,
                         self.chord, self.reynolds, self.info, self.cl, self.ld, self.cd,
                         self.cd_f, self.theta, self.cf, self.sep)

    def _adjoint_bucket(self, start, cnt, nmax, gc, have_lambda, stream=None):
        bd.panel_adjoint(cnt, nmax, self.flags, self.nodes, self.node_offsets,
                         self.mat_offsets, self.order[start:], self.A64, self.A_hi,
                         self.A_lo, self.LU, self.piv, self.u,
                         self.lam if have_lambda else None,
                         None if have_lambda else self.lam, self.alpha, self.vinf,
                         self.chord, gc, self.grad, self.max_iter, self.tol, self.info,
                         stream=stream)

    def adjoint(self, grad_cl=None):
        gc = None if grad_cl is None else torch.as_tensor(
            grad_cl, dtype=torch.float64, device=self.device).contiguous()
        for start, cnt, nmax in self.buckets:
            self._adjoint_bucket(start, cnt, nmax, gc, self.have_lambda)
        self.have_lambda = True

    def polar(self, alphas, factor: bool = True):
        """Cl at K angles per airfoil, alphas [B][K] radians (by airfoil index),
        from one factorisation: the two basis systems (right-hand sides v m_y
        and -v m_x) are refined with the stored factor and combined,
        Cl(a) = cos(a) Cl_y + sin(a) Cl_x.  Returns cl [B][K] (and keeps the basis
        strengths in self.u_y, self.u_x).  factor=False reuses the factor of an
        earlier solve of the same matrices."""
        if self.flags != bd.PANEL_MIXED:
            raise ValueError("polars need the mixed-precision path")
        al = torch.as_tensor(alphas, dtype=torch.float64, device=self.device).contiguous()
        if al.dim() != 2 or al.shape[0] != self.B:
            raise ValueError("alphas must be [B][K]")
        K = int(al.shape[1])
        if factor:
            self.assemble()
            self.solve(stage="factor")
        if getattr(self, "u_y", None) is None:
            self.u_y = torch.empty_like(self.u)
            self.u_x = torch.empty_like(self.u)
        cl = torch.empty(self.B, K, dtype=torch.float64, device=self.device)
        for start, cnt, nmax in self.buckets:
            bd.panel_polar(cnt, nmax, self.flags, self.nodes, self.node_offsets,
                           self.mat_offsets, self.order[start:], self.A_hi, self.A_lo, self.LU,
                           self.piv, self.vinf, self.chord, K, al, self.u_y, self.u_x, cl,
                           self.max_iter, self.tol, self.info, self.iters)
        return cl

    def vjp(self, w_cl=None, w_u=None, w_cp=None):
        """Gradient w.r.t. the nodes of sum w_cl Cl + w_u . u + w_cp . Cp (w_cl [B],
        w_u [sum m] packed like self.u = (gamma, C) per airfoil, w_cp [sum n]
        packed like the nodes; None = 0), after run() of the mixed path; returns
        self.grad [sum n][2]."""
        if self.flags != bd.PANEL_MIXED:
            raise ValueError("vector-Jacobian products need the mixed-precision path")

        def dev(w):
            return None if w is None else torch.as_tensor(
                w, dtype=torch.float64, device=self.device).contiguous()
        wc, wg, wp = dev(w_cl), dev(w_u), dev(w_cp)
        for start, cnt, nmax in self.buckets:
            bd.panel_vjp(cnt, nmax, self.flags, self.nodes, self.node_offsets, self.mat_offsets,
                         self.order[start:], self.A_hi, self.A_lo, self.LU, self.piv, self.u,
                         self.alpha, self.vinf, self.chord, wc, wg, wp, self.lam, self.grad,
                         self.max_iter, self.tol, self.info)
        self.have_lambda = False  # lambda now belongs to this product
        return self.grad

    def run(self, with_grad: bool = False):
        """Assemble, solve, forces (and the adjoint for unit upstream gradient)."""
        self.assemble()
        self.solve(with_adjoint=with_grad)
        self.forces()
        if with_grad:
            self.adjoint()
        return self

    def step(self, with_grad: bool = True):
        """One pass of the whole hot path; replays the captured graph if there is one."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self.run(with_grad=with_grad)

    def launches_per_step(self, with_grad: bool = True) -> int:
        """Kernel launches of one step: per bucket assemble, factor, refine and
        adjoint, plus one forces launch.  The mixed factor launches one kernel
        per size class the bucket may hold (Gauss-Jordan in shared memory and in
        global memory, or the one-block LU in shared memory and through L2) and,
        for m > 640 with T 128-column blocks, the step-synchronous LU: the tiled
        copy, T diagonal LUs, one CUDA-core and T - 1 tensor-core triangular
        solves, T - 1 updates, the untranspose of the U tiles and the inversion
        of the diagonal blocks; the adjoint of n > 256 adds a zeroing launch."""
        n = 1  # forces
        for k, (start, cnt, nmax) in enumerate(self.buckets):
            m = nmax + 1
            n += 1  # assemble
            if self.flags == bd.PANEL_MIXED:
                if self.inverse[k]:
                    n += 1 + (m > 230) + (m > GJ_MAX_M)
                else:
                    n += (self.lu_kind[k] != 1) + (m > LU_SMEM_MAX_M or self.lu_kind[k] == 1)
                if m > 640:
                    blocks = -(-m // 128)
                    n += 3 + blocks + 2 * (blocks - 1)
                n += 1  # refine
            else:
                n += 1
            if with_grad:
                n += 1 + (nmax > 256 and self.flags == bd.PANEL_MIXED)
        return n

    # -- autotuning and graph capture -------------------------------------------
    BUCKET_WIDTHS = (96, 128, 192, 256, None)

    def _time(self, fn, reps):
        fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    def autotune(self, reps: int = 3, use_cache: bool = True, widths=BUCKET_WIDTHS):
        """Pick the launch configuration by timing it (mixed mode):
          1. the bucket width, when the population's sizes differ: each width of
             `widths` (None = one bucket) times a whole step (assemble, solve with
             the transposed system, forces, adjoint);
          2. per bucket, the assembly (PANEL_TUNE_ROUNDS 0..6: near-field rounds, or
             both entries of a pair at once);
          3. per bucket, the solve (factor + refinement of both systems): the LU
             (for m <= 224 with the matrix in shared memory or through L2,
             PANEL_TUNE_LU 2 / 1) or the Gauss-Jordan inverse (m <= 288), each
             with each refinement block shape (PANEL_TUNE_IR 0..5).
        Choices are cached by device, size bound and batch class
        ($PANEL_AUTOTUNE_CACHE).  Returns {key: choice}."""
        if self.flags != bd.PANEL_MIXED or not self.buckets:
            return dict()
        dev = torch.cuda.get_device_name(self.device)
        with _tune_lock:
            cache = _load_tune_cache() if use_cache else {}
        chosen = {}
        bclass = lambda cnt: min(cnt, 1024) // 152 * 152
        sizes = np.diff(self.offsets_h)
        # 1. bucket width
        if len(set(sizes.tolist())) > 1 and widths:
            sig = "%s|width|B%d|n%d-%d|w%s" % (dev, self.B, int(sizes.min()), int(sizes.max()),
                                               ",".join(str(w) for w in widths))
            if sig in cache:
                best = cache[sig]
            else:
                times = {}
                for w in widths:
                    self.set_bucket_width(w)
                    times[str(w)] = self._time(lambda: self.run(with_grad=True), reps)
                best = min(times, key=times.get)
                cache[sig] = best
            self.set_bucket_width(None if best == "None" else int(best))
            chosen[sig] = best
        self.assemble()
        torch.cuda.synchronize(self.device)
        for k, (start, cnt, nmax) in enumerate(self.buckets):
            # 2. assembly rounds
            key = "%s|asm-rounds|n%d|b%d" % (dev, nmax, bclass(cnt))
            if key not in cache:
                times = []
                for r in range(7):
                    f = bd.PANEL_MIXED | bd.PANEL_TUNE_ROUNDS(r)

                    def call(f=f, start=start, cnt=cnt, nmax=nmax):
                        bd.panel_assemble(cnt, nmax, f, self.nodes, self.node_offsets,
                                          self.mat_offsets, self.order[start:], self.alpha,
                                          self.vinf, None, self.A_hi, self.A_lo, self.rhs,
                                          self.info)
                    times.append(self._time(call, reps))
                # the library's choice (0) unless another is at least 1 % faster
                best = 0
                for r in range(1, 7):
                    if times[r] < 0.99 * times[best]:
                        best = r
                cache[key] = best
            self.rounds[k] = int(cache[key])
            chosen[key] = self.rounds[k]
            # 3. factorisation and refinement shape
            key = "%s|solve-lu|n%d|b%d" % (dev, nmax, bclass(cnt))
            if key not in cache:
                best, best_t = None, None
                factors = [(False, 2), (False, 1)] if nmax + 1 <= LU_SMEM_MAX_M else [(False, 0)]
                if nmax + 1 <= GJ_MAX_M:
                    factors.append((True, 0))
                for inverse, lu in factors:
                    for shape in range(6):
                        f = (bd.PANEL_MIXED | bd.PANEL_WITH_ADJOINT | bd.PANEL_TUNE_IR(shape) |
                             (bd.PANEL_INVERSE if inverse else bd.PANEL_TUNE_LU(lu)))

                        def call(f=f, start=start, cnt=cnt, nmax=nmax):
                            bd.panel_solve(cnt, nmax, f, self.nodes, self.node_offsets,
                                           self.mat_offsets, self.order[start:], None,
                                           self.A_hi, self.A_lo, self.LU, self.piv, self.rhs,
                                           self.vinf, self.chord, self.u, self.lam,
                                           self.max_iter, self.tol, self.info, self.iters)
                        t = self._time(call, reps)
                        # candidates in order, the library's choice first: a later
                        # one wins only by at least 1 % (shapes that do not fit the
                        # size fall back to the choice by size and time the same)
                        if best_t is None or t < 0.99 * best_t:
                            best, best_t = [bool(inverse), shape, lu], t
                cache[key] = best
            c = cache[key]
            self.inverse[k], self.ir_shape[k] = bool(c[0]), int(c[1])
            self.lu_kind[k] = int(c[2]) if len(c) > 2 else 0
            chosen[key] = [self.inverse[k], self.ir_shape[k], self.lu_kind[k]]
        if use_cache:
            with _tune_lock:
                merged = _load_tune_cache()
                merged.update(cache)
                _store_tune_cache(merged)
        self.info.zero_()
        return chosen

    def tuning(self):
        """The launch configuration in use: bucket width and, per bucket, its
        size bound and count, factorisation, refinement shape and assembly rounds."""
        return {"bucket_width": self.bucket_width,
                "buckets": [{"n_max": int(nmax), "count": int(cnt),
                             "factor": "gauss-jordan" if self.inverse[k] else
                             ["lu", "lu (L2)", "lu (shared memory)"][self.lu_kind[k]],
                             "refine_shape": ["by size", "128x8", "256x4", "512x2",
                                              "1024x1", "256x3"][self.ir_shape[k]],
                             "assembly_rounds": ["by size", "inline", 4, 8, 16, 32,
                                                 "pairs"][self.rounds[k]]}
                            for k, (start, cnt, nmax) in enumerate(self.buckets)]}

    def capture(self, with_grad: bool = True):
        """Record one step into a CUDA graph (after a warm-up step outside it)."""
        self.graph = None
        self.run(with_grad=with_grad)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.run(with_grad=with_grad)
        self.graph = g
        return g

    # -- views -----------------------------------------------------------------
    def vec(self, t, b):
        o = int(self.offsets_h[b]) + b
        return t[o:o + int(self.offsets_h[b + 1] - self.offsets_h[b]) + 1]

    def matrix(self, b):
        """Airfoil b's assembled matrix as float64 (A64, or A_hi + A_lo)."""
        o = int(self.mat_offsets_h[b])
        m = int(self.offsets_h[b + 1] - self.offsets_h[b]) + 1
        if self.A64 is not None:
            return self.A64[o:o + m * m].view(m, m)
        return (self.A_hi[o:o + m * m].double() + self.A_lo[o:o + m * m].double()).view(m, m)

    def gamma(self, b):
        return self.vec(self.u, b)[:-1]


class PanelSolve(torch.autograd.Function):
    """Strengths, Cp and Cl of every airfoil of a batch as differentiable
    functions of the nodes (mixed path).

    forward(nodes [sum n][2] f64 cuda, offsets (host int64 [B+1]), alpha [B])
    -> (u [sum (n+1)] = (gamma, C) per airfoil, packed at offsets[b] + b;
        cp [sum n]; cl [B]).  backward is one panel_vjp: a transposed solve with
    the stored factor for dL/du assembled from all three upstream gradients,
    then the dM/dx contraction.
    """

    @staticmethod
    def forward(ctx, nodes, offsets, alpha):
        pb = PanelBatch(nodes.detach(), offsets, alpha.detach(), mode="mixed",
                        device=nodes.device)
        pb.run(with_grad=False)
        ctx.pb = pb
        return pb.u.clone(), pb.cp.clone(), pb.cl.clone()

    @staticmethod
    def backward(ctx, g_u, g_cp, g_cl):
        grad = ctx.pb.vjp(w_cl=g_cl, w_u=g_u, w_cp=g_cp)
        return grad.clone(), None, None


class PanelCl(torch.autograd.Function):
    """Cl of every airfoil of a batch as a differentiable function of the nodes.

    forward(nodes [sum n][2] f64 cuda, offsets (host int64 [B+1]), alpha [B], mode)
    -> cl [B].  backward maps dL/dCl to dL/dnodes with panel_adjoint (a
    transposed solve with the stored LU and the dM/dx contraction).
    """

    @staticmethod
    def forward(ctx, nodes, offsets, alpha, mode="mixed"):
        pb = PanelBatch(nodes.detach(), offsets, alpha.detach(), mode=mode, device=nodes.device)
        pb.run(with_grad=False)
        ctx.pb = pb
        return pb.cl.clone()

    @staticmethod
    def backward(ctx, grad_cl):
        pb = ctx.pb
        pb.adjoint(grad_cl.contiguous())
        return pb.grad.clone(), None, None, None
