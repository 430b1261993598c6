#!/usr/bin/env python
"""Benchmark: airfoil solves/s and dCl/dx gradients/s on one GB300.

One step = the whole hot path over one batch resident in device memory:
panel_assemble (geometry + influence matrix + Kutta row), panel_solve (LU +
refinement, with the transposed system for the adjoint), panel_forces
(Cp, Cl) and panel_adjoint (dCl/d(nodes)).  Every airfoil of the batch gets
Cl and its node gradient, so `value` counts airfoils (solve + gradient) per
second over all ranks; `solves_per_s` is the same batch without the gradient.

The headline workload is the largest one, 1024 airfoils of 1024..2048 panels
(`--config` picks another).  The other workloads are measured in the same run
and reported under `configs`: 64 x 100 panels on the plain FP64 path and mixed,
4096 x 200 mixed and plain FP64 (the mixed path against the plain FP64 path),
10 000 airfoils of 64..512 panels, and 4096 x 256 panels.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config NAME]
                  [--mode mixed|fp64] [--impl ours|reference] [--no-extra-configs]

--impl reference times the FP64 CPU oracle (the plain C restatement of the
method) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "airfoil solves/sec and dCl/dx gradients/sec on 1 GB300 at <=1e-10 Cl error"
DEFAULT_CONFIG = "large_b1024_n1024_2048"
# measured besides the headline workload: (workload, precision mode)
EXTRA_CONFIGS = [("naca_b64_n100", "fp64"), ("naca_b64_n100", "mixed"),
                 ("naca_b4096_n200", "mixed"), ("naca_b4096_n200", "fp64"),
                 ("uneven_b10000_n64_512", "mixed"), ("adjoint_b4096_n256", "mixed")]
# workload whose measurement also times polars, vector-Jacobian products, the
# viscous correction and GA generations
EXTRAS_ON = "naca_b4096_n200"
L2_BYTES = 135528448

# Algorithmic work per unit:
#  * assembly: one (control point, panel) pair = the FP32 flops (FMA = 2) of the
#    double-float far-field evaluation, ASSEMBLY_FLOP_PER_PAIR;
#  * factor: 2/3 m^3 FP32 flops per airfoil (m = n + 1);
#  * refine: 8 bytes per matrix entry for the initial solves (the FP32 factor,
#    once per system) + 16 per refinement step (both planes once, the factor
#    once per system);
#  * adjoint contraction: one pair = ADJOINT_FLOP_PER_PAIR FP32 flops;
#  * viscous correction: VISCOUS_BYTES_PER_NODE per node;
#  * plain FP64 path: FP64 flops of the same formulas (ASSEMBLY_F64_FLOP_PER_PAIR,
#    2/3 m^3 for the LU, ADJOINT_F64_FLOP_PER_PAIR).
ASSEMBLY_FLOP_PER_PAIR = 350
ADJOINT_FLOP_PER_PAIR = 480
ASSEMBLY_F64_FLOP_PER_PAIR = 90
# viscous correction: per node the node (16 B) and its strength (8 B) read, theta
# and cf (16 B) written
VISCOUS_BYTES_PER_NODE = 40
ADJOINT_F64_FLOP_PER_PAIR = 110
# FP32 peak from unit counts and the maximum clock: 152 SMs x 128 lanes x 2 x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = 1.25
# nominal dense TF32 / bf16 tensor rates of the GB300 (1.1 and 2.25 PFLOP/s)
TF32_OVER_BF16 = 1.1 / 2.25
# what `roofline.achieved` counts for each call (the method's work) ...
ROOF_WORK = {
    "mixed": {"assemble": "%d FP64-class flops per (control point, panel) pair"
                          % ASSEMBLY_F64_FLOP_PER_PAIR,
              "factor": "2/3 m^3 flops per airfoil (m = n + 1)",
              "refine": "8 B per matrix entry + 16 B per entry and refinement step",
              "forces": "40 B per node",
              "adjoint": "%d FP64-class flops per pair" % ADJOINT_F64_FLOP_PER_PAIR},
    "fp64": {"assemble": "%d FP64 flops per pair" % ASSEMBLY_F64_FLOP_PER_PAIR,
             "solve": "2/3 m^3 FP64 flops per airfoil",
             "forces": "40 B per node",
             "adjoint": "%d FP64 flops per pair" % ADJOINT_F64_FLOP_PER_PAIR},
}
# ... and what `roofline.issue_frac` counts (the work the kernels execute)
ROOF_IMPL_WORK = {
    "assemble": "%d FP32 flops per pair of the double-float evaluation" % ASSEMBLY_FLOP_PER_PAIR,
    "adjoint": "%d FP32 flops per pair of the double-float evaluation" % ADJOINT_FLOP_PER_PAIR,
    "factor": "3 TF32 products per multiply-add (3xTF32) in the tensor-core update",
}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.proc = None
        self.lines = []
        self.dev = device_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


TRAFFIC_TABLE = os.path.join(ROOT, "profiles", "dram_traffic.txt")


CALL_SOURCES = {
    "mixed": {"assemble": ["k_assemble_df.cu"],
              "factor": ["k_solve_mixed.cu", "k_gj_mixed.cu"],
              "factor-large": ["k_solve_mixed.cu", "k_gj_mixed.cu", "k_lu_large.cu",
                               "k_update_tc.cu"],
              "refine": ["k_solve_mixed.cu"],
              "forces": ["k_forces.cu"],
              "adjoint": ["k_adjoint_df.cu"]},
    "fp64": {"assemble": ["k_assemble_f64.cu"], "solve": ["k_solve_f64.cu"],
             "forces": ["k_forces.cu"], "adjoint": ["k_solve_f64.cu"]},
}


def kernel_source_digest(call=None, mode="mixed", large=False) -> str:
    """sha256 over the CUDA sources of the kernels one library call launches
    (the .cu files and the csrc headers they include, transitively; the mixed
    factor of airfoils above 639 panels, `large`, adds the step-synchronous
    LU's), or over every source when `call` is None: a DRAM-traffic figure
    recorded with another digest was taken on different kernels."""
    import hashlib
    import glob
    import re
    csrc = os.path.join(ROOT, "paper_1511_02166_gb300", "csrc")
    if call is None:
        files = sorted(os.path.basename(f) for f in
                       glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")))
    else:
        key = "factor-large" if (call == "factor" and large and mode == "mixed") else call
        todo, seen = list(CALL_SOURCES[mode][key]), set()
        while todo:
            f = todo.pop()
            if f in seen:
                continue
            seen.add(f)
            with open(os.path.join(csrc, f)) as fh:
                for inc in re.findall(r'^#include "([^"/]+)"', fh.read(), flags=re.M):
                    todo.append(inc)
        files = sorted(seen)
    h = hashlib.sha256()
    for f in files:
        h.update(f.encode())
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(call, workload, mode, batch, digest):
    """DRAM bytes per launch of `call` from the table in profiles/ (one ncu
    capture per row, scaled to `batch` airfoils as the row says), or None if
    there is no row for this call and workload or the kernels have changed."""
    try:
        with open(TRAFFIC_TABLE) as f:
            lines = f.read().splitlines()
    except OSError:
        return None
    for ln in lines:
        cells = [c.strip().strip("`") for c in ln.strip().strip("|").split("|")]
        if len(cells) < 7 or cells[0] != call or cells[1] != workload or cells[2] != mode:
            continue
        try:
            cap_batch = int(cells[3])
            per_airfoil = float(cells[5]) / cap_batch
        except ValueError:
            continue
        return per_airfoil * batch if cells[6] == digest else None
    return None


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_population_spec(spec, rank):
    """Weak scaling: rank r evaluates its own population of the configured size
    (the seed index shifted by 1000 r); airfoils are independent, so no data
    crosses ranks."""
    from paper_1511_02166_gb300 import inputs
    return inputs.PopulationSpec(spec.name, spec.batch, spec.n_min, spec.n_max, spec.perturbed,
                                 spec.seed_index + 1000 * rank)


def max_over_ranks(x, device=None):
    """The largest x over the ranks of the default process group (x itself
    without one): the slowest rank sets the whole job's time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, units_per_rank, ms):
    """Units per second of the whole job: every rank's units over the slowest
    rank's time."""
    return world * units_per_rank / (ms * 1e-3)


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------
def gradient_stride(n_max):
    """Node stride of the oracle's sampled gradient: 1 (the whole gradient) up to
    640 panels; above, about 96 nodes per airfoil (the forward-tangent gradient
    costs O(n^3) per airfoil, a minute and more at 1500-2000 panels)."""
    return 1 if n_max <= 640 else max(2, int(n_max) // 96)


def oracle_time(sub, stride):
    """Wall seconds of the FP64 oracle on the airfoils of `sub` (OpenMP across
    airfoils): the solve (oracle.evaluate_batch) and the forward-tangent dCl/dx.

    With stride 1 both are timed as they are.  With stride s > 1 the gradient is
    timed on the nodes k = 0, s, 2s, ... only, once with stride s and once with
    2s: each node's two tangents cost the same and are independent, so the
    gradient's time is F + G / s (F the assembly, LU and solve inside the
    gradient call, G the tangents of all nodes), and the two timings give F and
    G.  Returns (measured seconds, seconds of the solve + whole gradient)."""
    import oracle
    t0 = time.perf_counter()
    oracle.evaluate_batch(sub.nodes, sub.offsets, sub.alpha)
    t_eval = time.perf_counter() - t0
    if stride <= 1:
        t0 = time.perf_counter()
        oracle.cl_gradient_batch(sub.nodes, sub.offsets, sub.alpha)
        t_grad = time.perf_counter() - t0
        return t_eval + t_grad, t_eval + t_grad
    t0 = time.perf_counter()
    oracle.cl_gradient_strided_batch(sub.nodes, sub.offsets, sub.alpha, stride)
    t1 = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.cl_gradient_strided_batch(sub.nodes, sub.offsets, sub.alpha, 2 * stride)
    t2 = time.perf_counter() - t0
    G = max(2.0 * stride * (t1 - t2), 0.0)
    F = max(t1 - G / stride, 0.0)
    return t_eval + t1 + t2, t_eval + F + G


def _sample_text(sub, spec, config, stride, threads, measured, full):
    what = ("%d of %d airfoils of %s (solve + forward-tangent dCl/dx), %d threads"
            % (sub.batch, spec.batch, config, threads))
    if stride > 1:
        what += ("; the gradient timed on every %d-th and every %d-th node and extended "
                 "linearly to all nodes (each node's tangents cost the same): %.1f s "
                 "measured for an estimated %.1f s of whole-gradient work"
                 % (stride, 2 * stride, measured, full))
    else:
        what += ", %.1f s" % measured
    return what


def cpu_baseline(config, seconds=15.0, max_airfoils=None):
    import oracle
    from paper_1511_02166_gb300 import inputs

    spec = inputs.SPECS[config]
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    threads = oracle.max_threads()
    stride = gradient_stride(spec.n_max)
    # grow the sample until it takes about `seconds` (one airfoil per thread at
    # least)
    k = threads if stride > 1 else 4 * threads
    pop_all = inputs.make_population(spec, batch=min(spec.batch, max_airfoils or spec.batch))
    while True:
        sub = pop_all.subset(np.arange(min(k, pop_all.batch)))
        measured, full = oracle_time(sub, stride)
        if measured > seconds / 4 or sub.batch >= pop_all.batch:
            break
        k = min(pop_all.batch, int(k * max(2.0, seconds / 4 / max(measured, 1e-3))))
    # library-solve reference: LAPACK (numpy.linalg.solve) on the oracle's assembled
    # matrices of the first airfoils of the sample, the solve alone
    ls = pop_all.subset(np.arange(min(64, sub.batch, pop_all.batch)))
    mats = []
    for b in range(ls.batch):
        s0, s1 = ls.offsets[b], ls.offsets[b + 1]
        mats.append(oracle.assemble(ls.nodes[s0:s1], float(ls.alpha[b])))
    t0 = time.perf_counter()
    for M, rhs in mats:
        np.linalg.solve(M, rhs)
    lapack = ls.batch / (time.perf_counter() - t0)
    return {"value": sub.batch / full, "unit": "airfoils/s", "cores": int(threads),
            "host_cores": int(cores), "kind": "oracle",
            "sample": _sample_text(sub, spec, config, stride, threads, measured, full),
            "lapack_solves_per_s": lapack,
            "lapack_sample": "numpy.linalg.solve of the oracle's assembled systems, first %d "
                             "airfoils" % ls.batch}


def run_reference(args):
    """The oracle as it stands on the host cores: W untimed and K timed steps,
    each the solve and forward-tangent gradient of the same bounded sample of
    the workload (sized so that the whole run takes about args.ref_seconds;
    above 640 panels the gradient is sampled by node and extended as
    oracle_time describes).  `value` is airfoils per second of the whole work,
    `ms_per_step` the measured wall time of a step.  Under torchrun only rank 0
    runs; the other ranks exit without work."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_1511_02166_gb300 import inputs
    spec = inputs.SPECS[args.config]
    threads = oracle.max_threads()
    stride = gradient_stride(spec.n_max)
    pop_all = inputs.make_population(spec)
    per_step = max(1.0, args.ref_seconds / max(args.steps + args.warmup, 1))

    # size the sample: grow it until one step takes about per_step seconds
    # (one airfoil per thread at least)
    k = threads if stride > 1 else 2 * threads
    while True:
        sub = pop_all.subset(np.arange(min(k, pop_all.batch)))
        measured, _ = oracle_time(sub, stride)
        if measured > per_step / 2 or sub.batch >= pop_all.batch:
            break
        k = min(pop_all.batch, int(k * max(2.0, per_step / max(measured, 1e-3))))
    for _ in range(args.warmup):
        oracle_time(sub, stride)
    runs = [oracle_time(sub, stride) for _ in range(args.steps)]
    measured = float(np.mean([r[0] for r in runs]))
    full = float(np.mean([r[1] for r in runs]))
    value = sub.batch / full
    sample = _sample_text(sub, spec, args.config, stride, threads, measured, full)
    out = {"metric": METRIC, "value": value, "unit": "airfoils/s", "impl": "reference",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": measured * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.config, "batch_per_step": int(sub.batch),
                      "gradient_node_stride": stride,
                      "whole_work_s_per_step": full},
           "cpu_baseline": {"value": value, "unit": "airfoils/s", "cores": int(threads),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "airfoils/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def call_work(mode, sizes, iters_mean):
    """Per library call: (bound, algorithmic work of the method, implementation
    work or None, unit of the work) for one batch with panel counts `sizes`.

    The method's work: the panel integral's pairs at the FP64-class flop count
    of its formulas (ASSEMBLY_F64_FLOP_PER_PAIR, ADJOINT_F64_FLOP_PER_PAIR),
    2/3 m^3 flops for the LU, the refinement's and the forces' bytes.  The
    implementation's work (issue efficiency of the mixed path): the FP32 flops
    the double-float kernels execute per pair, and three TF32 products per
    multiply-add in the tensor-core update of airfoils above 640 panels."""
    sizes = np.asarray(sizes, dtype=np.float64)
    m = sizes + 1
    pairs = float((sizes ** 2).sum())
    m2 = float((m ** 2).sum())
    m3_small = float((m[m <= 640] ** 3).sum())
    m3_large = float((m[m > 640] ** 3).sum())
    lu = 2.0 / 3.0 * (m3_small + m3_large)
    if mode == "mixed":
        factor_bound = "tensor" if m3_large > m3_small else "alu"
        return {"assemble": ("alu", pairs * ASSEMBLY_F64_FLOP_PER_PAIR,
                             pairs * ASSEMBLY_FLOP_PER_PAIR),
                "factor": (factor_bound, lu,
                           2.0 / 3.0 * (m3_small + 3.0 * m3_large)),
                "refine": ("hbm", m2 * (8.0 + 16.0 * iters_mean), None),
                "forces": ("hbm", float(sizes.sum()) * 40.0, None),
                "adjoint": ("alu", pairs * ADJOINT_F64_FLOP_PER_PAIR,
                            pairs * ADJOINT_FLOP_PER_PAIR)}
    return {"assemble": ("alu", pairs * ASSEMBLY_F64_FLOP_PER_PAIR, None),
            "solve": ("alu", lu, None),
            "forces": ("hbm", float(sizes.sum()) * 40.0, None),
            "adjoint": ("alu", pairs * ADJOINT_F64_FLOP_PER_PAIR, None)}


def peaks_by_bound(mode):
    """Roofline denominators: (value, unit, source) per bound."""
    pk = _peaks()
    hbm = float(pk.get("hbm_gbs", 6800.0))
    bf16 = pk.get("bf16_tflops")
    if bf16:
        tf32 = float(bf16) * TF32_OVER_BF16
        tsrc = ("TF32 dense = measured cuBLAS bf16 burst (MEASURED_PEAKS.json bf16_tflops "
                "%.1f) x nominal TF32/bf16 ratio 1.1/2.25, of measured" % float(bf16))
    else:
        tf32 = 1900.0 * TF32_OVER_BF16
        tsrc = "TF32 dense = fallback bf16 1.9 PFLOP/s x nominal 1.1/2.25, of fallback"
    alu = (FP32_PEAK_TFLOPS, "TFLOP/s",
           "FP32 pipe: 152 SMs x 128 lanes x 2 flop x 2.07 GHz (from unit counts)")
    if mode == "fp64":
        alu = (FP64_PEAK_TFLOPS, "TFLOP/s", "FP64 nominal 1.25 TFLOP/s")
    return {"alu": alu, "tensor": (tf32, "TFLOP/s", tsrc),
            "hbm": (hbm, "GB/s", "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)")}


class Timer:
    """CUDA-event timing on the launching stream, with the L2 flushed (a write
    of twice its size) before every timed call, outside the events."""

    def __init__(self, torch, dev, stream):
        self.torch = torch
        self.stream = stream
        self.flush_buf = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def flush(self):
        self.flush_buf.zero_()

    def times(self, fn, reps, warmup):
        torch = self.torch
        ts = []
        for it in range(warmup + reps):
            self.flush()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            fn()
            e1.record(self.stream)
            e1.synchronize()
            if it >= warmup:
                ts.append(e0.elapsed_time(e1))
        return ts

    def mean(self, fn, reps, warmup):
        return float(np.mean(self.times(fn, reps, warmup)))


def measure_workload(name, mode, args, ctx, headline=False, extras=False):
    """Time one workload: the whole step (solve + dCl/dx) and the solve alone
    (assemble, solve, forces), each replayed from a captured CUDA graph, plus a
    per-call breakdown from eager steps with events around every library call.
    The headline workload also gets the clock record and the end-to-end figure
    through host buffers; `extras` adds the polar, vector-Jacobian, viscous and
    GA timings."""
    import torch

    from paper_1511_02166_gb300 import inputs
    from paper_1511_02166_gb300.solver import PanelBatch

    world, rank, dev, timer = ctx["world"], ctx["rank"], ctx["dev"], ctx["timer"]
    spec_r = rank_population_spec(inputs.SPECS[name], rank)
    pop = inputs.make_population(spec_r, batch=args.batch if headline else None)
    B = pop.batch
    pb = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode=mode, device=dev,
                    max_iter=args.max_iter, tol=args.tol)
    tuned = pb.autotune() if (args.autotune and mode == "mixed") else {}
    if mode == "mixed":
        names = ["assemble", "factor", "refine", "forces", "adjoint"]
        fns = [pb.assemble, lambda: pb.solve(stage="factor"),
               lambda: pb.solve(with_adjoint=True, stage="refine"), pb.forces, pb.adjoint]
    else:
        names = ["assemble", "solve", "forces", "adjoint"]
        fns = [pb.assemble, lambda: pb.solve(with_adjoint=True), pb.forces, pb.adjoint]
    stream = timer.stream

    def eager_step(evs=None):
        for k, fn in enumerate(fns):
            if evs is not None:
                evs[k][0].record(stream)
            fn()
            if evs is not None:
                evs[k][1].record(stream)

    for _ in range(args.warmup):
        eager_step()
    torch.cuda.synchronize()
    info = pb.info.cpu().numpy()
    iters = pb.iters.cpu().numpy()

    # per-call breakdown (events around every library call of eager steps)
    kern = {nm: [] for nm in names}
    for _ in range(max(2, args.steps // 2)):
        timer.flush()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in names]
        eager_step(evs)
        torch.cuda.synchronize()
        for k, nm in enumerate(names):
            kern[nm].append(evs[k][0].elapsed_time(evs[k][1]))

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # the solve alone (assemble + solve + forces), replayed from its own graph
    if args.graph:
        pb.capture(with_grad=False)
        solve_step = pb.step
    else:
        def solve_step():
            pb.run(with_grad=False)
    barrier()
    ms_solve = max_over_ranks(timer.mean(solve_step, args.steps, args.warmup), dev)

    # the whole step (solve + dCl/dx)
    if args.graph:
        pb.capture(with_grad=True)
        run_step = pb.step
    else:
        run_step = eager_step
    for _ in range(args.warmup):
        run_step()
    torch.cuda.synchronize()
    clk = None
    if headline:
        clk = ClockSampler(ctx["local"])
        clk.start()
    barrier()
    totals = timer.times(run_step, args.steps, 0)
    barrier()
    clocks = clk.stop() if clk is not None else None
    ms = max_over_ranks(float(np.mean(totals)), dev)

    out = {"workload": name, "mode": mode, "batch_per_gpu": B,
           "n_min": int(pop.sizes.min()), "n_max": int(pop.sizes.max()),
           "ms_per_step": ms, "solves_and_gradients_per_s": whole_job_rate(world, B, ms),
           "ms_per_solve_step": ms_solve, "solves_per_s": whole_job_rate(world, B, ms_solve),
           "size_buckets": len(pb.buckets), "inverse_buckets": int(sum(pb.inverse)),
           "tuning": pb.tuning(),
           "refinement_iters": {"mean": float(iters.mean()), "max": int(iters.max())}
           if mode == "mixed" else None,
           "info_nonzero": int((info != 0).sum()),
           "launches_per_step": pb.launches_per_step(with_grad=True)}

    # rooflines of every call, on the method's work (and the implementation's
    # issue efficiency where it differs)
    kms = {nm: float(np.mean(v)) for nm, v in kern.items()}
    work = call_work(mode, pop.sizes, float(iters.mean()) if mode == "mixed" else 0.0)
    pk = peaks_by_bound(mode)
    kernels = {}
    for nm in names:
        bound, w, w_impl = work[nm]
        sec = kms[nm] * 1e-3
        peak, unit, _ = pk[bound]
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        ent = {"ms": kms[nm], "bound": bound, "achieved": w / sec / scale, "peak": peak,
               "unit": unit, "frac": w / sec / scale / peak}
        if w_impl is not None and w_impl != w:
            ent["issue_frac"] = w_impl / sec / scale / peak
        kernels[nm] = ent
    out["kernels"] = kernels
    dom = max(kms, key=kms.get)
    dk = kernels[dom]
    digest = kernel_source_digest(dom, mode, large=int(pop.sizes.max()) + 1 > 640)
    # the traffic row of the kernels in use: the factor's LU kernel as tuned
    tkey = dom
    if dom == "factor" and mode == "mixed":
        kinds = {"lu" if bk["factor"] == "lu (shared memory)" else bk["factor"]
                 for bk in pb.tuning()["buckets"]}
        if len(kinds) == 1 and kinds != {"lu"}:
            tkey = "factor:" + kinds.pop()
    roof = {"kernel": dom, "bound": dk["bound"], "achieved": dk["achieved"], "peak": dk["peak"],
            "unit": dk["unit"], "frac": dk["frac"],
            "traffic": recorded_traffic(tkey, name, mode, B, digest),
            "traffic_unit": "bytes per launch", "kernel_digest": digest,
            "work": ROOF_WORK[mode][dom], "peak_source": pk[dk["bound"]][2]}
    if "issue_frac" in dk:
        roof["issue_frac"] = dk["issue_frac"]
        roof["issue_work"] = ROOF_IMPL_WORK[dom]
    out["roofline"] = roof

    if headline:
        out["clocks"] = clocks
        # ---- e2e through the public API with host buffers ----
        nodes_h = torch.from_numpy(pop.nodes).pin_memory()
        alpha_h = torch.from_numpy(pop.alpha).pin_memory()
        cl_h = torch.empty(B, dtype=torch.float64).pin_memory()
        grad_h = torch.empty(pop.nodes.shape, dtype=torch.float64).pin_memory()
        h2d = nodes_h.numel() * 8 + alpha_h.numel() * 8
        d2h = cl_h.numel() * 8 + grad_h.numel() * 8
        e2e_ms = []
        for it in range(args.warmup + args.steps):
            timer.flush()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pb.nodes.copy_(nodes_h, non_blocking=True)
            pb.alpha.copy_(alpha_h, non_blocking=True)
            run_step()
            cl_h.copy_(pb.cl, non_blocking=True)
            grad_h.copy_(pb.grad, non_blocking=True)
            torch.cuda.synchronize()
            if it >= args.warmup:
                e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e = max_over_ranks(float(np.mean(e2e_ms)), dev)
        out["e2e"] = {"value": whole_job_rate(world, B, e2e), "unit": "airfoils/s",
                      "ms_per_step": e2e, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h)}
        out["autotuned"] = tuned
    if extras and mode == "mixed":
        out.update(measure_extras(pb, pop, args, ctx))
    del pb
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return out


def profile_step(args):
    """One eager mixed step of a workload prefix, nothing timed: the command
    that per-kernel ncu captures (profiles/dram_traffic.txt) run."""
    import torch

    from paper_1511_02166_gb300 import inputs
    from paper_1511_02166_gb300.solver import PanelBatch
    pop = inputs.make_population(args.config, batch=args.batch)
    pb = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode="mixed", max_iter=args.max_iter,
                    tol=args.tol)
    pb.lu_kind = [args.lu_kind] * len(pb.buckets)
    pb.assemble()
    pb.solve(with_adjoint=True)
    pb.forces()
    pb.adjoint()
    torch.cuda.synchronize()
    bad = int((pb.info != 0).sum())
    print(json.dumps({"profile_step": args.config, "batch": pop.batch, "lu_kind": args.lu_kind,
                      "info_nonzero": bad, "tuning": pb.tuning()}))
    if bad:
        sys.exit(1)


def measure_extras(pb, pop, args, ctx):
    """Polars, vector-Jacobian products, the viscous correction and GA
    generations on a solved population (the calls of the library beyond the
    solve and the Cl gradient)."""
    import torch
    world, rank, dev, timer = ctx["world"], ctx["rank"], ctx["dev"], ctx["timer"]
    B = pop.batch
    reps = max(2, args.steps // 2)
    res = {}
    pb.graph = None
    if args.polar > 0:
        K = int(args.polar)
        alphas = torch.linspace(math.radians(-4.0), math.radians(10.0), K, dtype=torch.float64,
                                device=dev).repeat(B, 1).contiguous()
        pb.polar(alphas)
        torch.cuda.synchronize()
        pm = timer.mean(lambda: pb.polar(alphas), reps, args.warmup)
        res["polar"] = {"angles": K, "ms": pm, "cl_per_s": world * B * K / (pm * 1e-3),
                        "airfoil_polars_per_s": world * B / (pm * 1e-3),
                        "what": "panel_assemble + panel_solve(factor) + panel_polar per step"}
    if args.vjp:
        gen = torch.Generator(device=dev)
        gen.manual_seed(1511)
        w_cl = torch.randn(B, dtype=torch.float64, device=dev, generator=gen)
        w_u = torch.randn(pb.total_vec, dtype=torch.float64, device=dev, generator=gen)
        w_cp = torch.randn(pb.total_nodes, dtype=torch.float64, device=dev, generator=gen)
        pb.run()
        pb.vjp(w_cl, w_u, w_cp)
        torch.cuda.synchronize()
        vm = timer.mean(lambda: pb.vjp(w_cl, w_u, w_cp), reps, args.warmup)
        res["vjp"] = {"ms": vm, "products_per_s": world * B / (vm * 1e-3),
                      "what": "panel_vjp of w_cl.Cl + w_u.u + w_cp.Cp per airfoil, after a solve"}
    if args.viscous:
        pb.run()
        pb.viscous(1.0e6)
        torch.cuda.synchronize()
        vm_ = timer.mean(pb.viscous, reps, args.warmup)
        vbytes = float(pop.sizes.sum()) * VISCOUS_BYTES_PER_NODE
        sep = pb.sep.cpu().numpy()
        res["viscous"] = {"ms": vm_, "airfoils_per_s": world * B / (vm_ * 1e-3),
                          "reynolds": 1.0e6, "bound": "hbm",
                          "achieved_gbs": vbytes / (vm_ * 1e-3) / 1e9,
                          "attached_surfaces": float((sep == -1).mean()),
                          "what": "panel_viscous: Thwaites march, separation, Squire-Young and "
                                  "friction drag, L/D per airfoil, after a solve"}
    if args.ga > 0:
        from paper_1511_02166_gb300.ga import GeneticOptimizer
        n_ga = int(np.clip(int(pop.sizes.max()), 16, 1024))
        opt = GeneticOptimizer(B=B - (B % 2), n=n_ga, alpha=math.radians(4.0), seed=1511 + rank,
                               device=dev)
        opt.evaluate()
        if args.autotune:
            opt.pb.autotune()
        for _ in range(args.warmup):
            opt.evaluate()
            opt.step()
        torch.cuda.synchronize()

        def generation():
            opt.evaluate()  # panel_ga_sample + assemble + solve + forces + viscous
            opt.step()      # uniforms + panel_ga_step

        gts = timer.times(generation, int(args.ga), 0)
        gm = float(np.mean(gts))
        best = float(torch.nan_to_num(opt.evaluate(), nan=-np.inf).max())
        res["ga"] = {"population": opt.B, "nodes": n_ga, "control_points": opt.P,
                     "generations": len(gts), "fitness": "lift over drag (Re 1e6, alpha 4 deg)",
                     "best_fitness": best, "ms_per_generation": gm,
                     "generations_per_s": 1e3 / gm,
                     "airfoils_per_s": world * opt.B / (gm * 1e-3),
                     "what": "panel_ga_sample + assemble + solve + forces + panel_viscous + "
                             "panel_ga_step per generation"}
        del opt
    return res


def run_ours(args):
    import torch

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = {"world": world, "rank": rank, "local": local, "dev": dev,
           "timer": Timer(torch, dev, torch.cuda.current_stream())}

    head = measure_workload(args.config, args.mode, args, ctx, headline=True,
                            extras=args.extras_on == args.config)
    configs = {}
    if args.extra_configs:
        for name, mode in EXTRA_CONFIGS:
            if (name, mode) == (args.config, args.mode):
                continue
            configs["%s/%s" % (name, mode)] = measure_workload(
                name, mode, args, ctx, extras=(args.extras_on == name and mode == "mixed"))
        c2m, c2f = configs.get("naca_b4096_n200/mixed"), configs.get("naca_b4096_n200/fp64")
        if c2m and c2f:
            configs["naca_b4096_n200/mixed_over_fp64"] = {
                "solves_and_gradients": c2m["solves_and_gradients_per_s"]
                / c2f["solves_and_gradients_per_s"],
                "solves": c2m["solves_per_s"] / c2f["solves_per_s"]}

    B = head["batch_per_gpu"]
    value = head["solves_and_gradients_per_s"]
    out = {"metric": METRIC, "value": value, "unit": "airfoils/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+df32" if args.mode == "mixed" else "f64", "data": "synthetic",
           "config": {"workload": args.config, "batch_per_gpu": B, "mode": args.mode,
                      "subset": args.batch is not None,
                      "n_min": head["n_min"], "n_max": head["n_max"],
                      "l2": "flushed before every timed step (%d MB write)"
                            % (ctx["timer"].flush_buf.numel() * 4 // 2**20),
                      "max_iter": args.max_iter, "tol": args.tol,
                      "graph": bool(args.graph), "size_buckets": head["size_buckets"],
                      "inverse_buckets": head["inverse_buckets"],
                      "tuning": head["tuning"],
                      "parallelism": "dp%d (independent airfoils)" % world},
           "what": "value: airfoils per second with Cl and dCl/dx (assemble, LU, refinement of "
                   "the forward and transposed systems, forces, adjoint contraction); "
                   "solves_per_s: assemble, LU, refinement, forces only",
           "solves_per_s": head["solves_per_s"],
           "gradients_per_s": value,
           "ms_per_solve_step": head["ms_per_solve_step"],
           "kernels": head["kernels"],
           "refinement_iters": head["refinement_iters"],
           "info_nonzero": head["info_nonzero"],
           "e2e": head["e2e"],
           "roofline": head["roofline"],
           "gpu_launches": head["launches_per_step"] * args.steps,
           "clocks": head["clocks"],
           "configs": configs}
    for k in ("polar", "vjp", "viscous", "ga"):
        if k in head:
            out[k] = head[k]
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.config, seconds=args.cpu_seconds)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default=DEFAULT_CONFIG)
    ap.add_argument("--mode", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--max-iter", type=int, default=10)
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0,
                    help="--impl reference: about this many seconds for the whole run")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--polar", type=int, default=16,
                    help="also time Cl at this many angles per airfoil from one factorisation "
                         "(0: skip)")
    ap.add_argument("--no-vjp", dest="vjp", action="store_false",
                    help="skip timing the vector-Jacobian product of (Cl, u, Cp)")
    ap.add_argument("--no-viscous", dest="viscous", action="store_false",
                    help="skip timing the viscous correction (boundary layer and drag)")
    ap.add_argument("--ga", type=int, default=5,
                    help="also time this many generations of the device genetic optimiser on a "
                         "population of the configured batch (0: skip)")
    ap.add_argument("--no-extra-configs", dest="extra_configs", action="store_false",
                    help="measure only the --config workload")
    ap.add_argument("--extras-on", default=EXTRAS_ON,
                    help="workload on which polars, vector-Jacobian products, the viscous "
                         "correction and the GA are timed")
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="launch the calls one by one instead of replaying a CUDA graph")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--profile-step", action="store_true",
                    help="run one eager mixed step (assemble, solve with the transposed "
                         "system, forces, adjoint) of --config/--batch with the library's "
                         "launch choices and exit: the driver of per-kernel ncu captures")
    ap.add_argument("--lu-kind", type=int, default=0,
                    help="with --profile-step: PANEL_TUNE_LU of every bucket (0 by size)")
    ap.add_argument("--batch", type=int, default=None,
                    help="evaluate only the first BATCH airfoils of the workload (profiling)")
    args = ap.parse_args()
    if args.profile_step:
        profile_step(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
