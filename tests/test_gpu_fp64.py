"""GPU parity of the plain FP64 path against the FP64 oracle (element by element).

Tolerances: strengths |dgamma|_inf/|gamma|_inf <= 1e-10, |dC| <= 1e-10 |C|,
Cl <= 1e-10 (relative to max(|Cl|, 1)), matrix entries <= 1e-13 absolute,
gradients <= 1e-9 relative (inf norm).
"""
import math

import numpy as np
import pytest

import oracle
from paper_1511_02166_gb300 import inputs
from tests.gpu_util import cl_err, need_gpu, rel_inf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small_pop():
    need_gpu()
    return inputs.make_population("naca_b64_n100")


def _run(pop, mode="fp64", grad=False):
    from paper_1511_02166_gb300.solver import PanelBatch
    pb = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode=mode)
    pb.run(with_grad=grad)
    import torch
    torch.cuda.synchronize()
    return pb


def test_fp64_matrix_entries_match_oracle(small_pop):
    pb = _run(small_pop)
    for b in (0, 17, 63):
        M_ref, b_ref = oracle.assemble(small_pop.airfoil(b), small_pop.alpha[b])
        M = pb.matrix(b).cpu().numpy()
        assert np.max(np.abs(M - M_ref)) < 1e-13
        assert np.max(np.abs(pb.vec(pb.rhs, b).cpu().numpy() - b_ref)) < 1e-15


def test_fp64_solution_and_forces_match_oracle(small_pop):
    pb = _run(small_pop)
    ref = oracle.evaluate_batch(small_pop.nodes, small_pop.offsets, small_pop.alpha)
    assert np.all(pb.info.cpu().numpy() == 0)
    u = pb.u.cpu().numpy()
    for b in range(small_pop.batch):
        o = small_pop.offsets[b] + b
        n = small_pop.offsets[b + 1] - small_pop.offsets[b]
        assert rel_inf(u[o:o + n], ref["u"][o:o + n]) < 1e-10
        assert abs(u[o + n] - ref["u"][o + n]) <= 1e-10 * abs(ref["u"][o + n])
    assert cl_err(pb.cl.cpu().numpy(), ref["cl"]) < 1e-10
    assert np.max(np.abs(pb.cp.cpu().numpy() - ref["cp"])) < 1e-9
    assert np.max(np.abs(pb.cl_p.cpu().numpy() - ref["cl_p"])) < 1e-9
    assert np.max(np.abs(pb.cd_p.cpu().numpy() - ref["cd_p"])) < 1e-9


def test_fp64_gradient_matches_tangent_oracle(small_pop):
    sub = small_pop.subset([0, 5, 9])
    pb = _run(sub, grad=True)
    g = pb.grad.cpu().numpy()
    ref, info = oracle.cl_gradient_batch(sub.nodes, sub.offsets, sub.alpha)
    assert np.all(info == 0)
    for b in range(sub.batch):
        s = slice(sub.offsets[b], sub.offsets[b + 1])
        assert rel_inf(g[s], ref[s]) < 1e-9


def test_fp64_ragged_and_degenerate_batch():
    need_gpu()
    good = [inputs.naca4(0.02, 0.4, 0.12, n) for n in (3, 4, 7, 33, 64, 129)]
    cyl = inputs.cylinder(40)
    bad_cw = good[4][::-1].copy()
    two = good[3][:2].copy()
    zero = good[3].copy()
    zero[5] = zero[4]
    nan = good[3].copy()
    nan[7, 1] = np.nan
    airfoils = good + [cyl, bad_cw, two, zero, nan]
    alphas = [0.05 * k for k in range(len(airfoils))]
    pop = inputs.pack(airfoils, alphas)
    pb = _run(pop)
    info = pb.info.cpu().numpy()
    assert list(info[-4:]) == [-2, -1, -3, -4]
    assert np.all(info[:-4] == 0)
    ref = oracle.evaluate_batch(pop.nodes, pop.offsets, pop.alpha)
    u = pb.u.cpu().numpy()
    for b in range(len(good) + 1):
        o = pop.offsets[b] + b
        n = pop.offsets[b + 1] - pop.offsets[b]
        assert rel_inf(u[o:o + n + 1], ref["u"][o:o + n + 1]) < 1e-10
    assert np.all(np.isnan(pb.cl.cpu().numpy()[-4:]))


def test_fp64_cylinder_lift():
    need_gpu()
    al = math.radians(5.0)
    pop = inputs.pack([inputs.cylinder(256)], [al])
    pb = _run(pop)
    assert abs(pb.cl.item() - 4 * math.pi * math.sin(al)) < 2e-4
