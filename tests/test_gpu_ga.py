"""GPU parity of the genetic algorithm: the B-spline sampler against the
oracle's (scipy) evaluation within 1e-14, one generation step bit-exact
against the oracle given the same genomes, fitness and random numbers (integer
decisions from comparisons; the mutation rounded as written on both sides), and
a device-resident generation whose fitness matches the panel oracle."""
import numpy as np
import pytest

import oracle
from oracle import ga as oga
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("B,n", [(5, 137), (130, 64), (67, 3)])
def test_sampler_matches_oracle(B, n):
    # tiles of 64 nodes x 64 airfoils: ragged in both directions, one exact tile, n = 3
    need_gpu()
    import torch
    from paper_1511_02166_gb300 import binding as bd
    from paper_1511_02166_gb300.ga import default_bounds, default_control_x
    cx = default_control_x()
    lo, hi = default_bounds(cx)
    rng = np.random.default_rng(4)
    g = lo + rng.random((B, len(cx))) * (hi - lo)
    out = torch.empty(B * n, 2, dtype=torch.float64, device="cuda")
    bd.panel_ga_sample(B, len(cx), n, torch.tensor(cx, device="cuda"),
                       torch.tensor(g, device="cuda"), out)
    ref = oga.sample(cx, g, n)
    assert np.max(np.abs(out.cpu().numpy() - ref)) < 1e-14


@pytest.mark.parametrize("k,p,pm", [(4, 0.8, 0.3), (2, 1.0, 1.0), (7, 0.35, 0.0)])
def test_step_bit_exact(k, p, pm):
    need_gpu()
    import torch
    from paper_1511_02166_gb300 import binding as bd
    rng = np.random.default_rng(k)
    B, P = 64, 18
    lo, hi = np.full(P, -0.1), np.full(P, 0.12)
    sig = rng.random(P) * 0.02
    g = lo + rng.random((B, P)) * (hi - lo)
    fit = rng.normal(size=B)
    fit[::7] = np.nan
    fit[5] = fit[9] = fit[11]  # ties
    rand = rng.random((B // 2, 4 * k + 5))
    dev = {k_: torch.tensor(v, device="cuda") for k_, v in
           dict(lo=lo, hi=hi, sig=sig, g=g, fit=fit, rand=rand).items()}
    out = torch.empty_like(dev["g"])
    bd.panel_ga_step(B, P, k, p, pm, dev["lo"], dev["hi"], dev["sig"], dev["g"], dev["fit"],
                     dev["rand"], out)
    ref = oga.step(g, fit, rand, k, p, pm, lo, hi, sig)
    assert np.array_equal(out.cpu().numpy(), ref)


@pytest.mark.parametrize("fitness", ["cl", "ld"])
def test_device_generation_matches_oracle(fitness):
    need_gpu()
    import torch
    from oracle import viscous as ov
    from paper_1511_02166_gb300.ga import GeneticOptimizer
    alpha, Re = np.radians(2.0), 1.0e6
    opt = GeneticOptimizer(B=16, n=120, alpha=alpha, seed=7, fitness=fitness, reynolds=Re)
    fit0 = opt.evaluate().cpu().numpy().copy()
    g0 = opt.genome.cpu().numpy().copy()
    cx = opt.ctrl_x.cpu().numpy()
    nodes = oga.sample(cx, g0, opt.n)
    offs = np.arange(opt.B + 1, dtype=np.int64) * opt.n
    al = np.full(opt.B, alpha)
    ref = oracle.evaluate_batch(nodes, offs, al)
    want = ref["cl"].copy()
    if fitness == "ld":
        want = want / ov.viscous_batch(nodes, offs, ref["u"], al, Re, info=ref["info"])["cd"]
    want[ref["info"] != 0] = np.nan
    ok = np.isfinite(want)
    assert ok.sum() >= opt.B // 2
    assert np.array_equal(ok, np.isfinite(fit0))
    assert np.max(np.abs(fit0[ok] - want[ok]) / np.maximum(np.abs(want[ok]), 1)) < 1e-9
    rand = opt.step()
    nxt = oga.step(g0, fit0, rand.cpu().numpy(), opt.k, opt.p, opt.pm, opt.lo.cpu().numpy(),
                   opt.hi.cpu().numpy(), opt.sigma.cpu().numpy())
    assert np.array_equal(opt.genome.cpu().numpy(), nxt)
    torch.cuda.synchronize()


@pytest.mark.parametrize("n,lr", [(120, 0.0), (301, 1e-3)])
def test_genome_gradient_and_ascent_step(n, lr):
    # the transpose of the sampler on the device against scipy's design matrix;
    # with lr != 0 the clamped ascent step on the genome
    need_gpu()
    import torch
    from paper_1511_02166_gb300 import binding as bd
    from paper_1511_02166_gb300.ga import default_bounds, default_control_x
    cx = default_control_x()
    lo, hi = default_bounds(cx)
    rng = np.random.default_rng(n)
    B, P = 9, len(cx)
    g = lo + rng.random((B, P)) * (hi - lo)
    w = rng.normal(size=(B * n, 2)) * 50.0
    ref = oga.genome_grad(cx, w, n)
    dev = lambda a: torch.tensor(a, device="cuda")
    gd, out = dev(g), torch.empty(B, P, dtype=torch.float64, device="cuda")
    bd.panel_ga_genome_grad(B, P, n, dev(w), lr, dev(lo), dev(hi), gd, out)
    torch.cuda.synchronize()
    assert np.max(np.abs(out.cpu().numpy() - ref)) <= 1e-13 * np.max(np.abs(ref))
    want = oga.ascent_step(g, ref, lr, lo, hi) if lr else g
    assert np.max(np.abs(gd.cpu().numpy() - want)) <= 1e-14


def test_ascent_step_leaves_genomes_with_nan_gradients_unchanged():
    # an airfoil whose solve failed has NaN node gradients: its genome keeps its
    # values instead of being clamped to a bound, the others take the step
    need_gpu()
    import torch
    from paper_1511_02166_gb300 import binding as bd
    from paper_1511_02166_gb300.ga import default_bounds, default_control_x
    cx = default_control_x()
    lo, hi = default_bounds(cx)
    rng = np.random.default_rng(3)
    B, P, n, lr = 6, len(cx), 90, 2e-3
    g = lo + rng.random((B, P)) * (hi - lo)
    w = rng.normal(size=(B * n, 2)) * 20.0
    w[2 * n:3 * n] = np.nan            # airfoil 2 failed
    ref = oga.genome_grad(cx, w, n)
    want = oga.ascent_step(g, ref, lr, lo, hi)
    assert np.array_equal(want[2], g[2])
    dev = lambda a: torch.tensor(a, device="cuda")
    gd, out = dev(g), torch.empty(B, P, dtype=torch.float64, device="cuda")
    bd.panel_ga_genome_grad(B, P, n, dev(w), lr, dev(lo), dev(hi), gd, out)
    torch.cuda.synchronize()
    got = gd.cpu().numpy()
    assert np.array_equal(got[2], g[2])
    assert np.array_equal(np.isnan(out.cpu().numpy()), np.isnan(ref))
    assert np.max(np.abs(got - want)) <= 1e-14


def test_gradient_refined_generation_raises_lift():
    # one refinement step on Cl (adjoint gradient through the sampler) raises the
    # population's lift where the bounds allow, and its fitness is the oracle's Cl
    need_gpu()
    from paper_1511_02166_gb300.ga import GeneticOptimizer
    opt = GeneticOptimizer(B=32, n=120, alpha=np.radians(3.0), seed=5, fitness="cl")
    f0 = opt.evaluate().cpu().numpy().copy()
    f1 = opt.refine(2e-3).cpu().numpy()
    ok = np.isfinite(f0) & np.isfinite(f1)
    assert ok.sum() >= 24 and np.mean(f1[ok] > f0[ok]) > 0.9
    nodes = oga.sample(opt.ctrl_x.cpu().numpy(), opt.genome.cpu().numpy(), opt.n)
    offs = np.arange(opt.B + 1, dtype=np.int64) * opt.n
    ref = oracle.evaluate_batch(nodes, offs, np.full(opt.B, np.radians(3.0)))
    good = ok & (ref["info"] == 0)
    assert np.max(np.abs(f1[good] - ref["cl"][good]) / np.maximum(np.abs(ref["cl"][good]), 1)) < 1e-9
