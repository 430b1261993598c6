#!/usr/bin/env python
"""Benchmark: airfoil solves/s and dCl/dx gradients/s on one GB300.

One step = the whole hot path over one batch resident in device memory:
panel_assemble (geometry + influence matrix + Kutta row), panel_solve (LU +
refinement, with the transposed system for the adjoint), panel_forces
(Cp, Cl) and panel_adjoint (dCl/d(nodes)).  Every airfoil of the batch gets
Cl and its node gradient, so `value` counts airfoils (solve + gradient) per
second over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config NAME]
                  [--mode mixed|fp64] [--impl ours|reference]

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
DEFAULT_CONFIG = "naca_b4096_n200"
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
              "factor": ["k_solve_mixed.cu", "k_gj_mixed.cu", "k_lu_large.cu", "k_update_tc.cu"],
              "refine": ["k_solve_mixed.cu"],
              "forces": ["k_forces.cu"],
              "adjoint": ["k_adjoint_df.cu"]},
    "fp64": {"assemble": ["k_assemble_f64.cu"], "solve": ["k_solve_f64.cu"],
             "forces": ["k_forces.cu"], "adjoint": ["k_solve_f64.cu"]},
}


def kernel_source_digest(call=None, mode="mixed") -> str:
    """sha256 over the CUDA sources of the kernels one library call launches
    (the .cu files and the csrc headers they include, transitively), or over
    every source when `call` is None: a DRAM-traffic figure recorded with
    another digest was taken on different kernels."""
    import hashlib
    import glob
    import re
    csrc = os.path.join(ROOT, "paper_1511_02166_gb300", "csrc")
    if call is None:
        files = sorted(os.path.basename(f) for f in
                       glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh")))
    else:
        todo, seen = list(CALL_SOURCES[mode][call]), set()
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
def cpu_baseline(config, seconds=15.0, max_airfoils=None):
    import oracle
    from paper_1511_02166_gb300 import inputs

    spec = inputs.SPECS[config]
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    threads = oracle.max_threads()
    # grow the sample until it takes about `seconds`
    k = 4 * threads
    done, elapsed = 0, 0.0
    pop_all = inputs.make_population(spec, batch=min(spec.batch, max_airfoils or spec.batch))
    while True:
        sub = pop_all.subset(np.arange(min(k, pop_all.batch)))
        t0 = time.perf_counter()
        oracle.evaluate_batch(sub.nodes, sub.offsets, sub.alpha)
        oracle.cl_gradient_batch(sub.nodes, sub.offsets, sub.alpha)
        dt = time.perf_counter() - t0
        done, elapsed = sub.batch, dt
        if dt > seconds / 4 or sub.batch >= pop_all.batch:
            break
        k = min(pop_all.batch, int(k * max(2.0, seconds / 4 / max(dt, 1e-3))))
    # library-solve reference: LAPACK (numpy.linalg.solve) on the oracle's assembled
    # matrices of the first airfoils of the sample, the solve alone
    ls = pop_all.subset(np.arange(min(64, pop_all.batch)))
    mats = []
    for b in range(ls.batch):
        s0, s1 = ls.offsets[b], ls.offsets[b + 1]
        mats.append(oracle.assemble(ls.nodes[s0:s1], float(ls.alpha[b])))
    t0 = time.perf_counter()
    for M, rhs in mats:
        np.linalg.solve(M, rhs)
    lapack = ls.batch / (time.perf_counter() - t0)
    return {"value": done / elapsed, "unit": "airfoils/s", "cores": int(threads),
            "host_cores": int(cores), "kind": "oracle",
            "sample": "%d of %d airfoils of %s (solve + forward-tangent gradient), %.1f s"
                      % (done, spec.batch, config, elapsed),
            "lapack_solves_per_s": lapack,
            "lapack_sample": "numpy.linalg.solve of the oracle's assembled systems, first %d "
                             "airfoils" % ls.batch}


def run_reference(args):
    """The oracle as it stands on the host cores: W untimed and K timed steps,
    each the solve and forward-tangent gradient of the same bounded sample of
    the workload (sized so that the whole run takes about args.ref_seconds).
    Under torchrun only rank 0 runs; the other ranks exit without work."""
    world, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from paper_1511_02166_gb300 import inputs
    spec = inputs.SPECS[args.config]
    threads = oracle.max_threads()
    pop_all = inputs.make_population(spec)
    per_step = max(1.0, args.ref_seconds / max(args.steps + args.warmup, 1))

    def one(sub):
        t0 = time.perf_counter()
        oracle.evaluate_batch(sub.nodes, sub.offsets, sub.alpha)
        oracle.cl_gradient_batch(sub.nodes, sub.offsets, sub.alpha)
        return time.perf_counter() - t0

    # size the sample: grow it until one step takes about per_step seconds
    k = 2 * threads
    while True:
        sub = pop_all.subset(np.arange(min(k, pop_all.batch)))
        dt = one(sub)
        if dt > per_step / 2 or sub.batch >= pop_all.batch:
            break
        k = min(pop_all.batch, int(k * max(2.0, per_step / max(dt, 1e-3))))
    for _ in range(args.warmup):
        one(sub)
    times = [one(sub) for _ in range(args.steps)]
    sec = float(np.mean(times))
    value = sub.batch / sec
    sample = ("%d of %d airfoils of %s per step (solve + forward-tangent gradient), "
              "%d threads" % (sub.batch, spec.batch, args.config, threads))
    out = {"metric": METRIC, "value": value, "unit": "airfoils/s", "impl": "reference",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.config, "batch_per_step": int(sub.batch)},
           "cpu_baseline": {"value": value, "unit": "airfoils/s", "cores": int(threads),
                            "kind": "oracle", "sample": sample},
           "e2e": {"value": value, "unit": "airfoils/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    from paper_1511_02166_gb300 import binding as bd
    from paper_1511_02166_gb300 import inputs
    from paper_1511_02166_gb300.solver import PanelBatch

    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    spec_r = rank_population_spec(inputs.SPECS[args.config], rank)
    pop = inputs.make_population(spec_r, batch=args.batch)
    pb = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode=args.mode, device=dev,
                    max_iter=args.max_iter, tol=args.tol)
    tuned = pb.autotune() if (args.autotune and args.mode == "mixed") else {}
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def timed_ms(fn, reps, warmup):
        """Mean CUDA-event time of fn() on the launching stream over `reps` calls
        after `warmup` untimed ones, with the L2 flushed before each call."""
        ts = []
        for it in range(warmup + reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            if it >= warmup:
                ts.append(e0.elapsed_time(e1))
        return float(np.mean(ts)), len(ts)

    if args.mode == "mixed":
        names = ["assemble", "factor", "refine", "forces", "adjoint"]
        fns = [pb.assemble, lambda: pb.solve(stage="factor"),
               lambda: pb.solve(with_adjoint=True, stage="refine"), pb.forces, pb.adjoint]
    else:
        names = ["assemble", "solve", "forces", "adjoint"]
        fns = [pb.assemble, lambda: pb.solve(with_adjoint=True), pb.forces, pb.adjoint]

    def step(evs=None):
        for k, fn in enumerate(fns):
            if evs is not None:
                evs[k][0].record(stream)
            fn()
            if evs is not None:
                evs[k][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    info = pb.info.cpu().numpy()
    iters = pb.iters.cpu().numpy()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # per-call breakdown (CUDA events around every library call), untimed for `value`
    kern = {nm: [] for nm in names}
    for _ in range(max(2, args.steps // 2)):
        flush.zero_()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in names]
        step(evs)
        torch.cuda.synchronize()
        for k, nm in enumerate(names):
            kern[nm].append(evs[k][0].elapsed_time(evs[k][1]))

    if args.graph:
        pb.capture(with_grad=True)
        run_step = pb.step
    else:
        run_step = step
    for _ in range(args.warmup):
        run_step()
    torch.cuda.synchronize()

    clk = ClockSampler(local)
    clk.start()
    totals = []
    barrier()
    for _ in range(args.steps):
        flush.zero_()  # L2 flush outside the timed events
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        run_step()
        e1.record(stream)
        e1.synchronize()
        totals.append(e0.elapsed_time(e1))
    barrier()
    clocks = clk.stop()
    ms = max_over_ranks(float(np.mean(totals)), dev)
    B = pop.batch
    value = whole_job_rate(world, B, ms)

    # ---- e2e through the public API with host buffers ----
    nodes_h = torch.from_numpy(pop.nodes).pin_memory()
    alpha_h = torch.from_numpy(pop.alpha).pin_memory()
    cl_h = torch.empty(B, dtype=torch.float64).pin_memory()
    grad_h = torch.empty(pop.nodes.shape, dtype=torch.float64).pin_memory()
    h2d = nodes_h.numel() * 8 + alpha_h.numel() * 8
    d2h = cl_h.numel() * 8 + grad_h.numel() * 8
    e2e_ms = []
    for it in range(args.warmup + args.steps):
        flush.zero_()
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

    # ---- polar: Cl at POLAR_ANGLES angles per airfoil from one factorisation ----
    polar = None
    if args.mode == "mixed" and args.polar > 0:
        K = int(args.polar)
        alphas = torch.linspace(math.radians(-4.0), math.radians(10.0), K, dtype=torch.float64,
                                device=dev).repeat(B, 1).contiguous()
        pb.polar(alphas)
        torch.cuda.synchronize()
        # assemble + factor + two basis refinements + combination
        pm, _ = timed_ms(lambda: pb.polar(alphas), max(2, args.steps // 2), args.warmup)
        polar = {"angles": K, "ms": pm, "cl_per_s": world * B * K / (pm * 1e-3),
                 "airfoil_polars_per_s": world * B / (pm * 1e-3),
                 "what": "panel_assemble + panel_solve(factor) + panel_polar per step"}

    # ---- vector-Jacobian product of (Cl, u, Cp) on the solved population ----
    vjp = None
    if args.mode == "mixed" and args.vjp:
        gen = torch.Generator(device=dev)
        gen.manual_seed(1511)
        w_cl = torch.randn(B, dtype=torch.float64, device=dev, generator=gen)
        w_u = torch.randn(pb.total_vec, dtype=torch.float64, device=dev, generator=gen)
        w_cp = torch.randn(pb.total_nodes, dtype=torch.float64, device=dev, generator=gen)
        pb.run()
        pb.vjp(w_cl, w_u, w_cp)
        torch.cuda.synchronize()
        # transposed refinement + dM/dx contraction
        vm, _ = timed_ms(lambda: pb.vjp(w_cl, w_u, w_cp), max(2, args.steps // 2), args.warmup)
        vjp = {"ms": vm, "products_per_s": world * B / (vm * 1e-3),
               "what": "panel_vjp of w_cl.Cl + w_u.u + w_cp.Cp per airfoil, after a solve"}

    # ---- viscous correction (Thwaites boundary layer, drag, L/D) on the solved population ----
    viscous = None
    if args.mode == "mixed" and args.viscous:
        pb.run()
        pb.viscous(1.0e6)
        torch.cuda.synchronize()
        vm_, _ = timed_ms(pb.viscous, max(2, args.steps // 2), args.warmup)
        vbytes = float(pop.sizes.sum()) * VISCOUS_BYTES_PER_NODE
        sep = pb.sep.cpu().numpy()
        viscous = {"ms": vm_, "airfoils_per_s": world * B / (vm_ * 1e-3),
                   "reynolds": 1.0e6, "bound": "hbm", "achieved_gbs": vbytes / (vm_ * 1e-3) / 1e9,
                   "attached_surfaces": float((sep == -1).mean()),
                   "what": "panel_viscous: Thwaites march, separation, Squire-Young and friction "
                           "drag, L/D per airfoil, after a solve"}

    # ---- genetic optimisation: sample -> evaluate -> select/crossover/mutate on the device ----
    ga = None
    if args.mode == "mixed" and args.ga > 0:
        from paper_1511_02166_gb300.ga import GeneticOptimizer
        n_ga = int(np.clip(int(pop.sizes.max()), 16, 1024))
        opt = GeneticOptimizer(B=B - (B % 2), n=n_ga, alpha=math.radians(4.0), seed=1511 + rank,
                               device=dev)
        opt.evaluate()  # nodes of the first population, then pick each bucket's factorisation
        if args.autotune:
            opt.pb.autotune()
        for _ in range(args.warmup):
            opt.evaluate()
            opt.step()
        torch.cuda.synchronize()

        def generation():
            opt.evaluate()  # panel_ga_sample + assemble + solve + forces + viscous
            opt.step()      # uniforms + panel_ga_step

        gm, ngen = timed_ms(generation, int(args.ga), 0)
        best = float(torch.nan_to_num(opt.evaluate(), nan=-np.inf).max())
        ga = {"population": opt.B, "nodes": n_ga, "control_points": opt.P, "generations": ngen,
              "fitness": "lift over drag (Re 1e6, alpha 4 deg)", "best_fitness": best,
              "ms_per_generation": gm, "generations_per_s": 1e3 / gm,
              "airfoils_per_s": world * opt.B / (gm * 1e-3),
              "what": "panel_ga_sample + assemble + solve + forces + panel_viscous + "
                      "panel_ga_step per generation"}

    # ---- roofline of the dominant kernel ----
    kms = {nm: float(np.mean(v)) for nm, v in kern.items()}
    sizes = pop.sizes.astype(np.float64)
    pairs = float((sizes ** 2).sum())
    m2 = float(((sizes + 1) ** 2).sum())
    m3 = float(((sizes + 1) ** 3).sum())
    peaks = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    it_mean = float(iters.mean())
    if args.mode == "mixed":
        work = {"assemble": ("alu", pairs * ASSEMBLY_FLOP_PER_PAIR),
                "factor": ("alu", 2.0 / 3.0 * m3),
                "refine": ("hbm", m2 * (8.0 + 16.0 * it_mean)),
                "forces": ("hbm", float(sizes.sum()) * 40.0),
                "adjoint": ("alu", pairs * ADJOINT_FLOP_PER_PAIR)}
        alu_peak, alu_src = FP32_PEAK_TFLOPS, "FP32 pipe: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"
    else:
        work = {"assemble": ("alu", pairs * ASSEMBLY_F64_FLOP_PER_PAIR),
                "solve": ("alu", 2.0 / 3.0 * m3),
                "forces": ("hbm", float(sizes.sum()) * 40.0),
                "adjoint": ("alu", pairs * ADJOINT_F64_FLOP_PER_PAIR)}
        alu_peak, alu_src = FP64_PEAK_TFLOPS, "FP64 nominal 1.25 TFLOP/s"
    kernels = {}
    for nm in names:
        bound, w = work[nm]
        sec = kms[nm] * 1e-3
        if bound == "alu":
            ach, peak, unit = w / sec / 1e12, alu_peak, "TFLOP/s"
        else:
            ach, peak, unit = w / sec / 1e9, hbm, "GB/s"
        kernels[nm] = {"ms": kms[nm], "bound": bound, "achieved": ach, "peak": peak,
                       "unit": unit, "frac": ach / peak}
    dom = max(kms, key=kms.get)
    dk = kernels[dom]
    digest = kernel_source_digest(dom, args.mode)
    traffic = recorded_traffic(dom, args.config, args.mode, B, digest)
    roofline = {"kernel": dom, "bound": dk["bound"], "achieved": dk["achieved"],
                "peak": dk["peak"], "unit": dk["unit"], "frac": dk["frac"],
                "traffic": traffic, "traffic_unit": "bytes per launch",
                "kernel_digest": digest,
                "peak_source": alu_src if dk["bound"] == "alu"
                else "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"}
    launches_per_step = pb.launches_per_step(with_grad=True)
    out = {"metric": METRIC, "value": value, "unit": "airfoils/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f32+df32" if args.mode == "mixed" else "f64", "data": "synthetic",
           "config": {"workload": args.config, "batch_per_gpu": B, "mode": args.mode,
                      "subset": args.batch is not None,
                      "n_min": int(sizes.min()), "n_max": int(sizes.max()),
                      "l2": "flushed before every timed step (%d MB write)"
                            % (flush.numel() * 4 // 2**20),
                      "max_iter": args.max_iter, "tol": args.tol,
                      "graph": bool(args.graph), "size_buckets": len(pb.buckets),
                      "inverse_buckets": int(sum(pb.inverse)),
                      "parallelism": "dp%d (independent airfoils)" % world},
           "gradients_per_s": value,
           "polar": polar,
           "vjp": vjp,
           "ga": ga,
           "viscous": viscous,
           "kernels": kernels,
           "refinement_iters": {"mean": float(iters.mean()), "max": int(iters.max())},
           "info_nonzero": int((info != 0).sum()),
           "e2e": {"value": whole_job_rate(world, B, e2e), "unit": "airfoils/s",
                   "ms_per_step": e2e, "h2d_bytes_per_step": int(h2d),
                   "d2h_bytes_per_step": int(d2h)},
           "roofline": roofline,
           "gpu_launches": launches_per_step * args.steps,
           "clocks": clocks}
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
    ap.add_argument("--no-graph", dest="graph", action="store_false",
                    help="launch the calls one by one instead of replaying a CUDA graph")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false")
    ap.add_argument("--batch", type=int, default=None,
                    help="evaluate only the first BATCH airfoils of the workload (profiling)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
