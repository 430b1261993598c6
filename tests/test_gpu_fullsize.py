"""GPU parity at the workloads' full sizes, in the launch configuration that
bench.py times (size buckets, autotuned factorisation, the step captured in a
CUDA graph and replayed): sampled airfoils against the oracle computed one by
one.  Tolerances as in test_gpu_mixed.py: strengths and Cl within 1e-10
(|dCl| / max(|Cl|, 1)), gradients within 1e-9 relative (inf norm)."""
import numpy as np
import pytest

import oracle
from paper_1511_02166_gb300 import inputs
from tests.gpu_util import cl_err, need_gpu, rel_inf

pytestmark = pytest.mark.gpu


def _bench_step(pop):
    import torch
    from paper_1511_02166_gb300.solver import PanelBatch
    pb = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode="mixed")
    pb.autotune()
    pb.run(with_grad=True)          # warm-up (shared-memory attributes) before capture
    pb.capture(with_grad=True)
    pb.step()
    torch.cuda.synchronize()
    return pb


def _sample(pop, k, seed):
    return np.sort(np.random.default_rng(seed).choice(pop.batch, k, replace=False))


@pytest.mark.parametrize("config,k", [("naca_b4096_n200", 24), ("adjoint_b4096_n256", 12)])
def test_full_batch_graph_replay_samples(config, k):
    need_gpu()
    pop = inputs.make_population(config)
    pb = _bench_step(pop)
    info = pb.info.cpu().numpy()
    assert np.all(info == 0)
    u, cl, g = pb.u.cpu().numpy(), pb.cl.cpu().numpy(), pb.grad.cpu().numpy()
    idx = _sample(pop, k, 11)
    sub = pop.subset(idx)
    ref = oracle.evaluate_batch(sub.nodes, sub.offsets, sub.alpha)
    gref, ginfo = oracle.cl_gradient_batch(sub.nodes, sub.offsets, sub.alpha)
    assert np.all(ginfo == 0)
    for s, b in enumerate(idx):
        n = pop.offsets[b + 1] - pop.offsets[b]
        o, os_ = pop.offsets[b] + b, sub.offsets[s] + s
        assert rel_inf(u[o:o + n], ref["u"][os_:os_ + n]) < 1e-10, b
        gs = slice(pop.offsets[b], pop.offsets[b + 1])
        gr = slice(sub.offsets[s], sub.offsets[s + 1])
        assert rel_inf(g[gs], gref[gr]) < 1e-9, b
    assert cl_err(cl[idx], ref["cl"]) < 1e-10


def test_uneven_full_population_samples():
    # all 10 000 airfoils of 64..512 panels in their size buckets; the reference
    # is the long double oracle (some of these systems are too ill conditioned
    # for the FP64 evaluation itself, see test_gpu_mixed.py)
    need_gpu()
    pop = inputs.make_population("uneven_b10000_n64_512")
    pb = _bench_step(pop)
    assert np.all(pb.info.cpu().numpy() == 0)
    idx = _sample(pop, 24, 12)
    sub = pop.subset(idx)
    with oracle.extended():
        ref = oracle.evaluate_batch(sub.nodes, sub.offsets, sub.alpha)
    ref64 = oracle.evaluate_batch(sub.nodes, sub.offsets, sub.alpha)
    gref, ginfo = oracle.cl_gradient_batch(sub.nodes, sub.offsets, sub.alpha)
    assert np.all(ginfo == 0)
    u, g = pb.u.cpu().numpy(), pb.grad.cpu().numpy()
    for s, b in enumerate(idx):
        n = pop.offsets[b + 1] - pop.offsets[b]
        o, os_ = pop.offsets[b] + b, sub.offsets[s] + s
        e64 = rel_inf(ref64["u"][os_:os_ + n], ref["u"][os_:os_ + n])
        assert rel_inf(u[o:o + n], ref["u"][os_:os_ + n]) < max(1e-10, 3 * e64), b
        # the gradient against the FP64 tangent oracle; on the systems whose FP64
        # evaluation is itself off by e64 in the strengths, the oracle's gradient
        # carries the same conditioning, so the bound follows it
        gs = slice(pop.offsets[b], pop.offsets[b + 1])
        gr = slice(sub.offsets[s], sub.offsets[s + 1])
        eg = rel_inf(g[gs], gref[gr])
        print("uneven airfoil %d n=%d: gradient deviation %.2e (FP64 strength deviation %.2e)"
              % (b, n, eg, e64))
        assert eg < max(1e-9, 10 * e64), b
    assert cl_err(pb.cl.cpu().numpy()[idx], ref["cl"]) < 1e-10


def _large_golden():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "large_gradient_extended.npz")
    return np.load(path)


def _large_solution_golden():
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "large_solution_extended.npz")
    return np.load(path)


def test_large_full_population_samples():
    # all 1024 airfoils of 1024..2048 panels (the step-synchronous factor with
    # the tcgen05 update, the 1024-thread refinement of both systems, the
    # column-split adjoint contraction) in the bench's launch configuration.
    # Strengths, Cl and the backward error as in test_gpu_large.py: gamma of the
    # three stored airfoils within 1e-10 of the extended-precision oracle
    # (tests/golden/large_solution_extended.npz), of the other samples within
    # 5e-9 of the FP64 oracle (itself off by up to ~2e-9 at these condition
    # numbers), backward error against the oracle's matrix in long double
    # within 4 x the refinement's tolerance 1e-12, Cl within 1e-10.  dCl/dx within 1e-9
    # (inf norm relative) of extended-precision oracle gradients stored in
    # tests/golden (the FP64 oracle's own gradient is off by up to ~4e-10 at
    # these condition numbers, see make_large_gradient_golden.py): the smallest
    # airfoil, the one nearest 1537 panels and the largest, whose exact node
    # coordinates are put into the population first.
    need_gpu()
    from tests.test_gpu_large import _backward_error
    gold = _large_golden()
    pop = inputs.make_population("large_b1024_n1024_2048")
    gidx = [int(b) for b in gold["index"]]
    for b in gidx:
        x = gold["nodes_%d" % b]
        assert x.shape == pop.airfoil(b).shape
        pop.nodes[pop.offsets[b]:pop.offsets[b + 1]] = x
        pop.alpha[b] = float(gold["alpha_%d" % b])
    pb = _bench_step(pop)
    assert np.all(pb.info.cpu().numpy() == 0)
    g = pb.grad.cpu().numpy()
    step = int(gold["node_step"])
    for b in gidx:
        gs = g[pop.offsets[b]:pop.offsets[b + 1]][::step]
        eg = float(np.max(np.abs(gs - gold["grad_%d" % b])) / float(gold["scale_%d" % b]))
        print("large airfoil %d n=%d: gradient deviation from the extended oracle %.2e "
              "(FP64 oracle's own %.2e)" % (b, pop.sizes[b], eg, float(gold["fp64_dev_%d" % b])))
        assert eg < 1e-9, (b, eg)
    idx = np.array(sorted(set(gidx) | set(int(i) for i in _sample(pop, 2, 13))))
    sub = pop.subset(idx)
    ref = oracle.evaluate_batch(sub.nodes, sub.offsets, sub.alpha)
    u = pb.u.cpu().numpy()
    sol = _large_solution_golden()
    assert [int(i) for i in sol["c5_index"]] == gidx
    for s, b in enumerate(gidx):
        n = pop.offsets[b + 1] - pop.offsets[b]
        o, oe = pop.offsets[b] + b, sol["c5_offsets"][s] + s
        dev = rel_inf(u[o:o + n], sol["c5_u"][oe:oe + n])
        print("large airfoil %d n=%d: gamma deviation from the extended oracle %.2e" % (b, n, dev))
        assert dev < 1e-10, (b, dev)
    for s, b in enumerate(idx):
        n = pop.offsets[b + 1] - pop.offsets[b]
        o, os_ = pop.offsets[b] + b, sub.offsets[s] + s
        assert rel_inf(u[o:o + n], ref["u"][os_:os_ + n]) < 5e-9, b
        gs = slice(pop.offsets[b], pop.offsets[b + 1])
        assert _backward_error(pop.nodes[gs], pop.alpha[b], u[o:o + n + 1]) < 4e-12, b
    assert cl_err(pb.cl.cpu().numpy()[idx], ref["cl"]) < 1e-10


def test_adjoint_workload_gradient_against_central_differences_of_the_device_cl():
    # the adjoint workload's own check: central differences (h = 1e-6 chord) of
    # the device's Cl against the device's dCl/dx, within 1e-5 relative to the
    # gradient's inf norm, on three airfoils of the 4096 x 256 workload and eight
    # coordinates each (trailing edge, both surfaces, leading edge region)
    need_gpu()
    import torch
    from paper_1511_02166_gb300.solver import PanelBatch
    pop = inputs.make_population("adjoint_b4096_n256", batch=64)
    idx = np.array([0, 17, 63])
    sub = pop.subset(idx)
    pb = PanelBatch(sub.nodes, sub.offsets, sub.alpha, mode="mixed")
    pb.run(with_grad=True)
    torch.cuda.synchronize()
    assert np.all(pb.info.cpu().numpy() == 0)
    g = pb.grad.cpu().numpy()
    h = 1e-6
    coords = [(0, 0), (0, 1), (40, 1), (100, 0), (128, 1), (129, 0), (200, 1), (255, 1)]
    air, alpha = [], []
    for s in range(sub.batch):
        base = sub.nodes[sub.offsets[s]:sub.offsets[s + 1]]
        for (k, c) in coords:
            for sgn in (1.0, -1.0):
                x = base.copy()
                x[k, c] += sgn * h
                air.append(x)
                alpha.append(sub.alpha[s])
    fd = inputs.pack(air, np.array(alpha))
    pf = PanelBatch(fd.nodes, fd.offsets, fd.alpha, mode="mixed")
    pf.run()
    torch.cuda.synchronize()
    assert np.all(pf.info.cpu().numpy() == 0)
    cl = pf.cl.cpu().numpy().reshape(sub.batch, len(coords), 2)
    for s in range(sub.batch):
        gs = g[sub.offsets[s]:sub.offsets[s + 1]]
        scale = np.max(np.abs(gs))
        for q, (k, c) in enumerate(coords):
            d = (cl[s, q, 0] - cl[s, q, 1]) / (2 * h)
            assert abs(d - gs[k, c]) <= 1e-5 * scale, (s, k, c, d, gs[k, c])
