"""Pins of the genetic-algorithm oracle (oracle/ga.py) against what the
operators' definitions fix, independently of its own code paths: the textbook
Cox-de Boor recursion for the sampler, partition of unity and clamped ends,
exact selection for p = 1, the acceptance law p (1-p)^j, segment structure of
one-point crossover, and the mutation's single-gene, bounded change."""
import math

import numpy as np

from oracle import ga
from paper_1511_02166_gb300.ga import default_bounds, default_control_x


def _cox_de_boor(i, p, t, kn):
    # the recursive definition, with the right end of the last span closed
    if p == 0:
        last = kn[i + 1] == kn[-1] and kn[i] < kn[i + 1]
        return 1.0 if (kn[i] <= t < kn[i + 1] or (last and t == kn[-1])) else 0.0
    a = 0.0 if kn[i + p] == kn[i] else (t - kn[i]) / (kn[i + p] - kn[i]) * _cox_de_boor(
        i, p - 1, t, kn)
    b = 0.0 if kn[i + p + 1] == kn[i + 1] else (kn[i + p + 1] - t) / (
        kn[i + p + 1] - kn[i + 1]) * _cox_de_boor(i + 1, p - 1, t, kn)
    return a + b


def test_sampler_against_recursive_definition():
    cx = default_control_x()
    rng = np.random.default_rng(1)
    lo, hi = default_bounds(cx)
    y = lo + rng.random(len(cx)) * (hi - lo)
    n = 41
    nodes = ga.sample(cx, y, n)
    kn = ga.knots(len(cx))
    for i, t in enumerate(ga.sample_parameters(n)):
        N = np.array([_cox_de_boor(j, 3, t, kn) for j in range(len(cx))])
        assert abs(N.sum() - 1.0) < 1e-14
        assert abs(nodes[i, 0] - N @ cx) < 1e-14 and abs(nodes[i, 1] - N @ y) < 1e-14


def test_sampler_partition_of_unity_and_clamped_start():
    cx = default_control_x()
    nodes = ga.sample(cx, np.full(len(cx), 0.37), 30)
    assert np.max(np.abs(nodes[:, 1] - 0.37)) < 1e-15
    y = np.linspace(0.0, 1.0, len(cx))
    nodes = ga.sample(cx, y, 30)
    assert np.array_equal(nodes[0], [cx[0], y[0]])  # clamped: the curve starts at P_0
    t = ga.sample_parameters(30)
    assert t[0] == 0.0 and abs(t[15] - 0.5) < 1e-15 and np.all(np.diff(t) > 0)


def test_tournament_picks_best_when_p_is_one_and_follows_the_acceptance_law():
    rng = np.random.default_rng(2)
    B, k = 50, 5
    fit = rng.normal(size=B)
    for _ in range(200):
        u = rng.random(2 * k - 1)
        cands = [min(int(math.floor(x * B)), B - 1) for x in u[:k]]
        assert ga.tournament(fit, k, 1.0, u) == max(cands, key=lambda c: (fit[c], -c))
    # distinct candidates 0..k-1 with decreasing fitness: rank j with p (1-p)^j
    p = 0.6
    fit2 = np.arange(k, 0, -1, dtype=float)
    counts = np.zeros(k)
    trials = 20000
    for _ in range(trials):
        u = np.concatenate([(np.arange(k) + 0.5) / k, rng.random(k - 1)])
        counts[ga.tournament(fit2[:k], k, p, u)] += 1
    expect = np.array([p * (1 - p) ** j for j in range(k - 1)] + [(1 - p) ** (k - 1)])
    assert np.max(np.abs(counts / trials - expect)) < 0.015


def test_nan_fitness_never_preferred():
    fit = np.array([np.nan, 0.2, np.nan, 0.1])
    u = np.array([0.0, 0.6, 0.26, 0.9, 0.1, 0.1, 0.1])  # candidates 0, 2, 1, 3
    assert ga.tournament(fit, 4, 1.0, u) == 1


def test_crossover_segments_and_mutation_bounds():
    rng = np.random.default_rng(3)
    B, P, k = 6, 9, 3
    g = 0.2 + 0.6 * rng.random((B, P))  # inside the bounds, so clamping only shortens a move
    fit = rng.random(B)
    lo, hi, sig = np.full(P, 0.2), np.full(P, 0.8), np.full(P, 0.05)
    rand = rng.random((B // 2, 4 * k + 5))
    out0 = ga.step(g, fit, rand, k, 0.7, 0.0, lo, hi, sig)  # no mutation
    for pair in range(B // 2):
        u = rand[pair]
        a = ga.tournament(fit, k, 0.7, u[:2 * k - 1])
        b = ga.tournament(fit, k, 0.7, u[2 * k - 1:4 * k - 2])
        c = min(1 + int(math.floor(u[4 * k - 2] * (P - 1))), P - 1)
        assert np.array_equal(out0[2 * pair], np.concatenate([g[a, :c], g[b, c:]]))
        assert np.array_equal(out0[2 * pair + 1], np.concatenate([g[b, :c], g[a, c:]]))
    out1 = ga.step(g, fit, rand, k, 0.7, 1.0, lo, hi, sig)  # every child mutated once
    diff = out1 != out0
    assert np.all(diff.sum(axis=1) <= 1)
    changed = out1[diff]
    assert np.all((changed >= 0.2) & (changed <= 0.8))
    assert np.all(np.abs(out1 - out0) <= 0.05 + 1e-15)


def test_genome_gradient_is_the_adjoint_of_the_sampler():
    # the sampler is linear in the genome: the gradient of L = <w, y(g)> is J^T w,
    # checked by central differences of L and by the partition of unity
    # (sum over control points of dL/dg = sum over nodes of dL/dy)
    cx = default_control_x()
    lo, hi = default_bounds(cx)
    rng = np.random.default_rng(21)
    n, B = 57, 3
    g = lo + rng.random((B, len(cx))) * (hi - lo)
    w = rng.normal(size=(B * n, 2))
    grad = ga.genome_grad(cx, w, n)
    L = lambda gg: float(np.sum(w[:, 1] * ga.sample(cx, gg, n)[:, 1]))
    h = 1e-6
    for b in range(B):
        for r in range(len(cx)):
            gp, gm = g.copy(), g.copy()
            gp[b, r] += h
            gm[b, r] -= h
            assert abs((L(gp) - L(gm)) / (2 * h) - grad[b, r]) < 1e-8 * max(1.0, abs(grad[b, r]))
    assert np.allclose(grad.sum(axis=1), w[:, 1].reshape(B, n).sum(axis=1), rtol=1e-13, atol=1e-13)


def test_ascent_step_moves_along_the_gradient_within_bounds_and_skips_non_finite():
    # the step increases every unclamped gene by exactly lr times its gradient
    # (first-order ascent), never leaves [lo, hi], and leaves a gene with a
    # non-finite gradient untouched (a failed solve's NaN gradient must not snap
    # the genome to a bound)
    cx = default_control_x()
    lo, hi = default_bounds(cx)
    rng = np.random.default_rng(7)
    B, P = 5, len(cx)
    g = lo + rng.random((B, P)) * (hi - lo)
    d = rng.normal(size=(B, P))
    d[1, :] = np.nan
    d[3, 2] = np.inf
    lr = 1e-3
    out = ga.ascent_step(g, d, lr, lo, hi)
    assert np.array_equal(out[1], g[1])
    assert out[3, 2] == g[3, 2]
    assert np.all(out >= lo) and np.all(out <= hi)
    inside = np.isfinite(d) & (g + lr * d > lo) & (g + lr * d < hi)
    assert inside.sum() > 0.8 * np.isfinite(d).sum()
    assert np.allclose(out[inside] - g[inside], lr * d[inside], rtol=0, atol=1e-15)
    big = ga.ascent_step(g, np.where(np.isfinite(d), np.sign(d) * 1e9, d), 1.0, lo, hi)
    fin = np.isfinite(d)
    assert np.all(big[fin & (d > 0)] == np.broadcast_to(hi, (B, P))[fin & (d > 0)])
    assert np.all(big[fin & (d < 0)] == np.broadcast_to(lo, (B, P))[fin & (d < 0)])
