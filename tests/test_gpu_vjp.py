"""GPU parity of panel_vjp -- the gradient w.r.t. the nodes of
w_cl . Cl + w_u . u + w_cp . Cp (u = (gamma, C) per airfoil) -- against the
forward-tangent oracle of the same objective: 1e-9 relative (inf norm), the
tolerance of the Cl gradient.  Also: with w_cl alone it reproduces panel_adjoint,
and PanelSolve's autograd backward is the same product."""
import numpy as np
import pytest

import oracle
from paper_1511_02166_gb300 import inputs
from tests.gpu_util import need_gpu, rel_inf

pytestmark = pytest.mark.gpu


def _weights(pop, seed):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=pop.batch), rng.normal(size=pop.offsets[-1] + pop.batch),
            rng.normal(size=pop.offsets[-1]))


def _check(pop, w_cl, w_u, w_cp, g):
    for b in range(pop.batch):
        s = slice(pop.offsets[b], pop.offsets[b + 1])
        o, n = pop.offsets[b] + b, pop.offsets[b + 1] - pop.offsets[b]
        ref, info = oracle.vjp(pop.nodes[s], pop.alpha[b], w_cl[b], w_u[o:o + n + 1], w_cp[s])
        assert info == 0
        assert rel_inf(g[s], ref) < 1e-9, b


@pytest.mark.parametrize("sizes", [[200, 200, 120], [40, 229, 300, 700]])
def test_vjp_matches_tangent_oracle(sizes):
    # small and large airfoils: the one-block and the column-split contractions
    need_gpu()
    import torch
    from paper_1511_02166_gb300.solver import PanelBatch
    rng = np.random.default_rng(len(sizes))
    air = [inputs.naca4(rng.uniform(0, .06), rng.uniform(.2, .6), rng.uniform(.08, .18), n)
           for n in sizes]
    pop = inputs.pack(air, rng.uniform(-0.07, 0.17, len(air)))
    pb = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode="mixed")
    pb.run()
    w_cl, w_u, w_cp = _weights(pop, 3)
    g = pb.vjp(w_cl, w_u, w_cp).cpu().numpy()
    torch.cuda.synchronize()
    assert np.all(pb.info.cpu().numpy() == 0)
    _check(pop, w_cl, w_u, w_cp, g)


def test_vjp_cl_alone_equals_adjoint():
    need_gpu()
    import torch
    from paper_1511_02166_gb300.solver import PanelBatch
    pop = inputs.make_population("naca_b4096_n200", batch=8)
    pb = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode="mixed")
    pb.run(with_grad=True)
    g_adj = pb.grad.cpu().numpy().copy()
    w_cl = np.linspace(0.5, 2.0, pop.batch)
    g = pb.vjp(w_cl=w_cl).cpu().numpy()
    torch.cuda.synchronize()
    for b in range(pop.batch):
        s = slice(pop.offsets[b], pop.offsets[b + 1])
        assert rel_inf(g[s], w_cl[b] * g_adj[s]) < 1e-11, b


def test_panel_solve_autograd_backward():
    need_gpu()
    import torch
    from paper_1511_02166_gb300.solver import PanelSolve
    pop = inputs.make_population("adjoint_b4096_n256", batch=3)
    x = torch.tensor(pop.nodes, device="cuda", requires_grad=True)
    al = torch.tensor(pop.alpha, device="cuda")
    u, cp, cl = PanelSolve.apply(x, pop.offsets, al)
    w_cl, w_u, w_cp = _weights(pop, 9)
    loss = ((cl * torch.tensor(w_cl, device="cuda")).sum() +
            (u * torch.tensor(w_u, device="cuda")).sum() +
            (cp * torch.tensor(w_cp, device="cuda")).sum())
    loss.backward()
    _check(pop, w_cl, w_u, w_cp, x.grad.cpu().numpy())
