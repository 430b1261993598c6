"""GPU tests of the batching layer: size buckets, the two factorisations chosen by
autotuning, and CUDA-graph replay with new inputs written into the captured
buffers.  Every result is checked against the oracle (long double build, as in
the ragged tests: gamma within 1e-10, Cl within 1e-10)."""
import numpy as np
import pytest

import oracle
from paper_1511_02166_gb300 import inputs
from tests.gpu_util import cl_err, need_gpu, rel_inf

pytestmark = pytest.mark.gpu


def _ragged(seed, sizes):
    rng = np.random.default_rng(seed)
    air = [inputs.naca4(rng.uniform(0, .06), rng.uniform(.2, .6), rng.uniform(.08, .18), n)
           for n in sizes]
    return inputs.pack(air, rng.uniform(-0.07, 0.17, len(air)))


def _check(pop, u, cl, tol=1e-10):
    with oracle.extended():
        ref = oracle.evaluate_batch(pop.nodes, pop.offsets, pop.alpha)
    for b in range(pop.batch):
        o = pop.offsets[b] + b
        n = pop.offsets[b + 1] - pop.offsets[b]
        assert rel_inf(u[o:o + n], ref["u"][o:o + n]) < tol, b
    assert cl_err(cl, ref["cl"]) < tol


SIZES = [512, 500, 449, 300, 257, 231, 229, 200, 130, 129, 128, 64, 63, 33, 3]


def test_buckets_match_single_launch():
    need_gpu()
    import torch
    from paper_1511_02166_gb300.solver import PanelBatch
    pop = _ragged(5, SIZES)
    one = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode="mixed", bucket_width=None)
    many = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode="mixed", bucket_width=64,
                      bucket_min=1)
    assert len(one.buckets) == 1 and len(many.buckets) == 6
    one.run(with_grad=True)
    many.run(with_grad=True)
    torch.cuda.synchronize()
    assert np.all(many.info.cpu().numpy() == 0)
    u1, u2 = one.u.cpu().numpy(), many.u.cpu().numpy()
    for b in range(pop.batch):
        o = pop.offsets[b] + b
        n = pop.offsets[b + 1] - pop.offsets[b]
        assert rel_inf(u2[o:o + n + 1], u1[o:o + n + 1]) < 1e-12, b
    g1, g2 = one.grad.cpu().numpy(), many.grad.cpu().numpy()
    for b in range(pop.batch):
        s = slice(pop.offsets[b], pop.offsets[b + 1])
        assert rel_inf(g2[s], g1[s]) < 1e-11, b
    _check(pop, u2, many.cl.cpu().numpy())


def test_inverse_in_every_bucket():
    need_gpu()
    import torch
    from paper_1511_02166_gb300.solver import PanelBatch
    pop = _ragged(6, SIZES)
    pb = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode="mixed", bucket_width=64,
                    bucket_min=1)
    pb.inverse = [True] * len(pb.buckets)
    pb.run(with_grad=False)
    torch.cuda.synchronize()
    assert np.all(pb.info.cpu().numpy() == 0)
    _check(pop, pb.u.cpu().numpy(), pb.cl.cpu().numpy())


def test_autotune_then_graph_replay_with_new_inputs(tmp_path, monkeypatch):
    need_gpu()
    import torch
    from paper_1511_02166_gb300.solver import PanelBatch
    monkeypatch.setenv("PANEL_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    sizes = [64 + (37 * k) % 449 for k in range(40)]
    pop = _ragged(7, sizes)
    pb = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode="mixed", bucket_min=4)
    chosen = pb.autotune(reps=1)
    assert (tmp_path / "tune.json").exists() and len(chosen) >= 1
    pb.capture(with_grad=True)
    # same sizes, new shapes and angles written into the captured input buffers
    pop2 = _ragged(8, sizes)
    pb.nodes.copy_(torch.from_numpy(pop2.nodes))
    pb.alpha.copy_(torch.from_numpy(pop2.alpha))
    pb.step()
    torch.cuda.synchronize()
    assert np.all(pb.info.cpu().numpy() == 0)
    _check(pop2, pb.u.cpu().numpy(), pb.cl.cpu().numpy())
    ref, info = oracle.cl_gradient_batch(pop2.nodes, pop2.offsets, pop2.alpha)
    g = pb.grad.cpu().numpy()
    for b in range(0, pop2.batch, 7):
        s = slice(pop2.offsets[b], pop2.offsets[b + 1])
        assert rel_inf(g[s], ref[s]) < 1e-9, b
    # a second instance reads the cached choice instead of timing again
    pb2 = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode="mixed", bucket_min=4)
    assert pb2.autotune(reps=1) == chosen and pb2.inverse == pb.inverse


def test_inverse_small_airfoils_with_static_shared_memory():
    # n = 100: the Gauss-Jordan kernel's dynamic shared memory (41 KB) plus its
    # static arrays cross the default 48 KB, so the launch needs the opt-in
    need_gpu()
    import torch
    from paper_1511_02166_gb300.solver import PanelBatch
    pop = inputs.make_population("naca_b64_n100", batch=16)
    pb = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode="mixed")
    pb.inverse = [True] * len(pb.buckets)
    pb.run()
    torch.cuda.synchronize()
    assert np.all(pb.info.cpu().numpy() == 0)
    _check(pop, pb.u.cpu().numpy(), pb.cl.cpu().numpy())


def test_empty_batch_is_a_no_op():
    # B = 0 through every call of the Python layer: nothing launched, nothing raised
    need_gpu()
    import torch
    from paper_1511_02166_gb300.solver import PanelBatch
    pb = PanelBatch(np.zeros((0, 2)), np.zeros(1, dtype=np.int64), np.zeros(0), mode="mixed")
    pb.run(with_grad=True)
    pb.viscous(1.0e6)
    assert pb.cl.numel() == 0 and pb.grad.numel() == 0 and pb.cd.numel() == 0
    torch.cuda.synchronize()


def test_every_launch_shape_gives_the_oracle_result():
    # the autotuner's search space: every refinement block shape, every assembly
    # near-field setting, the three factorisations (LU through L2, LU in shared
    # memory, Gauss-Jordan inverse), with buckets of several widths;
    # each combination is a layout of the same computation and matches the
    # oracle (long double) to 1e-10
    need_gpu()
    import torch
    from paper_1511_02166_gb300.solver import PanelBatch
    pop = _ragged(31, [300, 257, 200, 130, 64, 3])
    with oracle.extended():
        ref = oracle.evaluate_batch(pop.nodes, pop.offsets, pop.alpha)
    for width in (None, 128):
        for inverse, lu in ((False, 1), (False, 2), (True, 0)):
            for shape in range(6):
                for rounds in (0, 1, 2, 5, 6):
                    pb = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode="mixed",
                                    bucket_width=width, bucket_min=1)
                    pb.inverse = [inverse] * len(pb.buckets)
                    pb.lu_kind = [lu] * len(pb.buckets)
                    pb.ir_shape = [shape] * len(pb.buckets)
                    pb.rounds = [rounds] * len(pb.buckets)
                    pb.run()
                    torch.cuda.synchronize()
                    assert np.all(pb.info.cpu().numpy() == 0), (width, inverse, shape, rounds)
                    u = pb.u.cpu().numpy()
                    for b in range(pop.batch):
                        o = pop.offsets[b] + b
                        n = pop.offsets[b + 1] - pop.offsets[b]
                        assert rel_inf(u[o:o + n], ref["u"][o:o + n]) < 1e-10, (b, shape)
                    assert cl_err(pb.cl.cpu().numpy(), ref["cl"]) < 1e-10


def test_assembly_kernels_give_the_same_matrix():
    # the pair-at-once assembly (both entries of a pair of control points from
    # one evaluation of |P|^2, 1/|P|^2, log|P| and P^2) performs the same
    # operations for every entry as the row-by-row assembly, inline or with the
    # near-field queue: the planes agree bit for bit, across 32 x 32 tile edges
    need_gpu()
    import torch
    from paper_1511_02166_gb300.solver import PanelBatch
    pop = _ragged(33, [1100, 700, 200, 100, 64, 33, 32, 31, 3])
    planes = []
    for rounds in (1, 4, 6):
        pb = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode="mixed", bucket_width=None)
        pb.rounds = [rounds] * len(pb.buckets)
        pb.assemble()
        torch.cuda.synchronize()
        assert np.all(pb.info.cpu().numpy() == 0)
        planes.append((pb.A_hi.cpu().numpy().view(np.uint32).copy(),
                       pb.A_lo.cpu().numpy().view(np.uint32).copy(), pb.rhs.cpu().numpy().copy()))
    for k in (1, 2):
        assert np.array_equal(planes[0][0], planes[k][0]), k
        assert np.array_equal(planes[0][1], planes[k][1]), k
        assert np.array_equal(planes[0][2], planes[k][2]), k


def test_lu_kernels_give_the_same_factor():
    # the LU with the trailing matrix through L2 and the LU with the whole matrix
    # in shared memory perform the same operations in the same order: the stored
    # factors and pivots agree bit for bit (sizes across the 32-column panels and
    # up to the largest shared-memory size, 223 panels, and one above it)
    need_gpu()
    import torch
    from paper_1511_02166_gb300.solver import PanelBatch
    pop = _ragged(32, [230, 223, 222, 200, 131, 96, 64, 33, 32, 31, 3])
    out = []
    for lu in (1, 2):
        pb = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode="mixed")
        pb.lu_kind = [lu] * len(pb.buckets)
        pb.assemble()
        pb.solve(stage="factor")
        torch.cuda.synchronize()
        assert np.all(pb.info.cpu().numpy() == 0)
        out.append((pb.LU.cpu().numpy().copy(), pb.piv.cpu().numpy().copy()))
    assert np.array_equal(out[0][1], out[1][1])
    assert np.array_equal(out[0][0].view(np.uint32), out[1][0].view(np.uint32))


def test_autotuner_records_a_configuration_per_bucket(tmp_path, monkeypatch):
    # the broadened search picks a bucket width for a ragged population and,
    # per bucket, rounds, factorisation and refinement shape; a second batch of
    # the same population reads the same choices from the cache
    need_gpu()
    import torch
    from paper_1511_02166_gb300.solver import PanelBatch
    monkeypatch.setenv("PANEL_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    pop = inputs.make_population("uneven_b10000_n64_512", batch=1216)
    pb = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode="mixed")
    chosen = pb.autotune(reps=1)
    t = pb.tuning()
    assert len(t["buckets"]) == len(pb.buckets) >= 1
    assert any("|width|" in k for k in chosen)
    pb.run(with_grad=True)
    torch.cuda.synchronize()
    assert np.all(pb.info.cpu().numpy() == 0)
    pb2 = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode="mixed")
    assert pb2.autotune(reps=1) == chosen and pb2.tuning() == t
