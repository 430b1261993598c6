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
    u = pb.u.cpu().numpy()
    for s, b in enumerate(idx):
        n = pop.offsets[b + 1] - pop.offsets[b]
        o, os_ = pop.offsets[b] + b, sub.offsets[s] + s
        e64 = rel_inf(ref64["u"][os_:os_ + n], ref["u"][os_:os_ + n])
        assert rel_inf(u[o:o + n], ref["u"][os_:os_ + n]) < max(1e-10, 3 * e64), b
    assert cl_err(pb.cl.cpu().numpy()[idx], ref["cl"]) < 1e-10


def test_large_full_population_samples():
    # all 1024 airfoils of 1024..2048 panels (the step-synchronous factor with
    # the tcgen05 update, the 1024-thread refinement); tolerances of
    # test_gpu_large.py: gamma within 5e-9, the backward error against the
    # oracle's matrix (long double) within 1e-13, Cl within 1e-10
    need_gpu()
    from tests.test_gpu_large import _backward_error
    pop = inputs.make_population("large_b1024_n1024_2048")
    pb = _bench_step(pop)
    assert np.all(pb.info.cpu().numpy() == 0)
    idx = _sample(pop, 3, 13)
    sub = pop.subset(idx)
    ref = oracle.evaluate_batch(sub.nodes, sub.offsets, sub.alpha)
    u = pb.u.cpu().numpy()
    for s, b in enumerate(idx):
        n = pop.offsets[b + 1] - pop.offsets[b]
        o, os_ = pop.offsets[b] + b, sub.offsets[s] + s
        assert rel_inf(u[o:o + n], ref["u"][os_:os_ + n]) < 5e-9, b
        gs = slice(pop.offsets[b], pop.offsets[b + 1])
        assert _backward_error(pop.nodes[gs], pop.alpha[b], u[o:o + n + 1]) < 1e-13, b
    assert cl_err(pb.cl.cpu().numpy()[idx], ref["cl"]) < 1e-10
