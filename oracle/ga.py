"""Genetic-algorithm oracle (test infrastructure): the B-spline genome sampler,
the genome gradient of a node-gradient (gradient-refined steps), and one
generation of tournament selection, one-point crossover and mutation,
written from the genetic optimisation of Section 2 with plain numpy / scipy and
Python loops.  Only tests/ (and the CPU legs of bench.py) use it; it shares no
code with the CUDA library.

The paper fixes the operators' kind (B-spline genome from the trailing edge
over the upper surface to the leading edge and back; tournament of k with the
j-th best taken with probability p (1-p)^j; one-point crossover into two
children; a mutation of one coefficient with some probability) but not the
spline, the sampling, the constants or the order of the random draws; those
readings are the library's and are restated here:
  * clamped uniform cubic B-spline over P control points (x fixed, genome = y);
  * node i of n at t_i = (1 - cos(pi i / n_u)) / 4 for i <= n_u = ceil(n/2), else
    1/2 + (1 - cos(pi (i - n_u) / (n - n_u))) / 4;
  * per pair of children, 4k + 5 uniforms: for each tournament k candidate
    draws floor(u B) and k - 1 acceptance draws (accept rank j at the first draw
    below p, the last rank if none), the crossover point 1 + floor(u (P - 1)),
    then per child: mutate if u < pm, gene floor(u P), amount sigma (2u - 1),
    clamped to [lo, hi];
  * ranking: higher fitness first, NaN last, ties by lower index, then by draw
    order.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.interpolate import BSpline


def sample_parameters(n: int) -> np.ndarray:
    nu = (n + 1) // 2
    t = np.empty(n)
    for i in range(n):
        if i <= nu:
            t[i] = 0.25 * (1.0 - math.cos(math.pi * i / nu))
        else:
            t[i] = 0.5 + 0.25 * (1.0 - math.cos(math.pi * (i - nu) / (n - nu)))
    return t


def knots(P: int) -> np.ndarray:
    segs = P - 3
    return np.concatenate([np.zeros(3), np.arange(segs + 1) / segs, np.ones(3)])


def sample(ctrl_x, genome, n: int) -> np.ndarray:
    """Nodes [B*n][2] of the B-spline airfoils genome [B][P] (scipy's BSpline)."""
    ctrl_x = np.asarray(ctrl_x, dtype=np.float64)
    genome = np.atleast_2d(np.asarray(genome, dtype=np.float64))
    P = len(ctrl_x)
    t = sample_parameters(n)
    kn = knots(P)
    out = np.empty((genome.shape[0] * n, 2))
    for b, y in enumerate(genome):
        curve = BSpline(kn, np.stack([ctrl_x, y], axis=1), 3, extrapolate=False)
        pts = curve(np.minimum(t, 1.0))
        out[b * n:(b + 1) * n] = pts
    return out


def genome_grad(ctrl_x, grad_nodes, n: int) -> np.ndarray:
    """dL/dgenome [B][P] from dL/dnodes [B*n][2]: the nodes' y coordinates are
    the B-spline's design matrix (scipy) times the genome, x is fixed."""
    P = len(ctrl_x)
    t = np.minimum(sample_parameters(n), 1.0)
    J = BSpline.design_matrix(t, knots(P), 3).toarray()  # [n][P]
    gy = np.asarray(grad_nodes, dtype=np.float64)[:, 1].reshape(-1, n)
    return gy @ J


def ascent_step(genome, grad_genome, lr: float, lo, hi) -> np.ndarray:
    """One clamped gradient-ascent step of the genomes [B][P]:
    g <- min(max(g + lr dL/dg, lo), hi) for every gene whose gradient is
    finite; a gene with a non-finite gradient (an airfoil whose solve failed)
    keeps its value (the library's reading; the paper has no gradient steps)."""
    g = np.array(genome, dtype=np.float64, copy=True)
    d = np.asarray(grad_genome, dtype=np.float64)
    out = g.copy()
    B, P = g.shape
    for b in range(B):
        for r in range(P):
            if math.isfinite(d[b, r]):
                out[b, r] = min(max(g[b, r] + lr * d[b, r], lo[r]), hi[r])
    return out


def _rank_key(fitness, idx, pos):
    f = fitness[idx]
    return (1, 0.0, idx, pos) if math.isnan(f) else (0, -f, idx, pos)


def tournament(fitness, k: int, p: float, u) -> int:
    B = len(fitness)
    cands = [(min(int(math.floor(u[j] * B)), B - 1), j) for j in range(k)]
    ranked = sorted(cands, key=lambda c: _rank_key(fitness, c[0], c[1]))
    for j in range(k - 1):
        if u[k + j] < p:
            return ranked[j][0]
    return ranked[k - 1][0]


def step(genome, fitness, rand, k: int, p: float, pm: float, lo, hi, sigma) -> np.ndarray:
    """One generation: genome [B][P], fitness [B], rand [B/2][4k + 5]."""
    genome = np.asarray(genome, dtype=np.float64)
    fitness = np.asarray(fitness, dtype=np.float64)
    B, P = genome.shape
    out = np.empty_like(genome)
    for pair in range(B // 2):
        u = rand[pair]
        a = tournament(fitness, k, p, u[:2 * k - 1])
        b = tournament(fitness, k, p, u[2 * k - 1:4 * k - 2])
        c = min(1 + int(math.floor(u[4 * k - 2] * (P - 1))), P - 1)
        c1 = np.concatenate([genome[a, :c], genome[b, c:]])
        c2 = np.concatenate([genome[b, :c], genome[a, c:]])
        for ch, child in enumerate((c1, c2)):
            um = u[4 * k - 1 + 3 * ch:4 * k + 2 + 3 * ch]
            if um[0] < pm:
                g = min(int(math.floor(um[1] * P)), P - 1)
                child[g] = min(max(child[g] + sigma[g] * (2.0 * um[2] - 1.0), lo[g]), hi[g])
        out[2 * pair] = c1
        out[2 * pair + 1] = c2
    return out
