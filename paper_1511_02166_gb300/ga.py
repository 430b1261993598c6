"""Genetic optimisation around the batched evaluator (the genetic optimisation
of Section 2): a population of B-spline airfoils lives on the device, each
generation is panel_ga_sample -> the panel method (assemble, solve, forces) ->
panel_ga_step.  Fitness is the lift-to-drag ratio at the population's angle
of attack and Reynolds number (Section 3's fitness; the drag from the viscous
correction, panel_viscous), or the lift coefficient alone.  An airfoil the
library flags -- invalid geometry, no convergence, no stagnation point -- has
fitness NaN and is never preferred.  Random numbers are drawn on the
device from a seeded torch generator and passed to the library as inputs."""
from __future__ import annotations

import numpy as np
import torch

from . import binding as bd
from .solver import PanelBatch


def default_control_x(half: int = 7) -> np.ndarray:
    """Control-point x coordinates: trailing edge, `half` stations over the
    upper surface (cosine-spaced), the leading edge twice (a vertical tangent),
    `half` stations over the lower surface, trailing edge: P = 2 half + 4."""
    s = 0.5 * (1.0 + np.cos(np.pi * np.arange(1, half + 1) / (half + 1)))
    return np.concatenate([[1.0], s, [0.0, 0.0], s[::-1], [1.0]])


def default_bounds(ctrl_x: np.ndarray):
    """y bounds per control point: 0 at the two trailing-edge points, an upper
    band over the first half and a lower band over the second, both narrowing
    linearly towards the trailing edge (|y| <= 0.25 (1 - x) above, 0.2 (1 - x)
    below, sign-definite behind x = 0.8).  The narrowing keeps the
    trailing-edge angle small: the drag of the viscous correction is taken at
    the trailing edge, where a blunt edge would drive the inviscid speed, and
    with it the drag estimate, to zero."""
    ctrl_x = np.asarray(ctrl_x, dtype=np.float64)
    P = len(ctrl_x)
    lo = np.zeros(P)
    hi = np.zeros(P)
    for j in range(1, P - 1):
        taper = 1.0 - ctrl_x[j]
        aft = ctrl_x[j] > 0.8
        if j < P // 2:
            lo[j], hi[j] = (0.0 if aft else 0.005), min(0.12, 0.25 * taper)
        else:
            lo[j], hi[j] = max(-0.10, -0.2 * taper), (0.0 if aft else 0.02)
    return lo, hi


class GeneticOptimizer:
    def __init__(self, B: int, n: int, alpha: float, ctrl_x=None, lo=None, hi=None, sigma=None,
                 k: int = 4, p: float = 0.8, pm: float = 0.3, seed: int = 0, device="cuda",
                 fitness: str = "ld", reynolds: float = 1.0e6):
        if B % 2:
            raise ValueError("the population size must be even")
        if fitness not in ("ld", "cl"):
            raise ValueError("fitness is 'ld' (lift over drag) or 'cl'")
        self.fitness_kind = fitness
        self.device = torch.device(device)
        self.B, self.n = int(B), int(n)
        cx = default_control_x() if ctrl_x is None else np.asarray(ctrl_x, dtype=np.float64)
        dlo, dhi = default_bounds(cx)
        lo = dlo if lo is None else np.asarray(lo, dtype=np.float64)
        hi = dhi if hi is None else np.asarray(hi, dtype=np.float64)
        sigma = 0.1 * (hi - lo) if sigma is None else np.asarray(sigma, dtype=np.float64)
        self.P = len(cx)
        self.k, self.p, self.pm = int(k), float(p), float(pm)
        f64 = dict(dtype=torch.float64, device=self.device)
        self.ctrl_x = torch.as_tensor(cx, **f64)
        self.lo = torch.as_tensor(lo, **f64)
        self.hi = torch.as_tensor(hi, **f64)
        self.sigma = torch.as_tensor(sigma, **f64)
        self.gen = torch.Generator(device=self.device)
        self.gen.manual_seed(seed)
        u = torch.rand(self.B, self.P, generator=self.gen, **f64)
        self.genome = self.lo + u * (self.hi - self.lo)
        self.genome_next = torch.empty_like(self.genome)
        offsets = np.arange(self.B + 1, dtype=np.int64) * self.n
        self.pb = PanelBatch(np.zeros((self.B * self.n, 2)), offsets, np.full(self.B, alpha),
                             mode="mixed", device=self.device)
        self.pb.reynolds.fill_(float(reynolds))
        self.fitness = None
        self.generation = 0

    def evaluate(self):
        bd.panel_ga_sample(self.B, self.P, self.n, self.ctrl_x, self.genome, self.pb.nodes)
        self.pb.info.zero_()
        self.pb.run(with_grad=False)
        if self.fitness_kind == "ld":
            self.pb.viscous()
            self.fitness = self.pb.ld
        else:
            self.fitness = self.pb.cl
        return self.fitness

    def refine(self, lr: float):
        """One gradient-ascent step of every genome on Cl (gradient-refined GA
        step): dCl/dnodes by the adjoint, mapped to the genome by the transpose
        of the B-spline sampling, g <- clamp(g + lr dCl/dg, lo, hi), then the
        fitness of the refined population.  Needs fitness 'cl'."""
        if self.fitness_kind != "cl":
            raise ValueError("gradient refinement follows dCl/dgenome: use fitness='cl'")
        bd.panel_ga_sample(self.B, self.P, self.n, self.ctrl_x, self.genome, self.pb.nodes)
        self.pb.info.zero_()
        self.pb.run(with_grad=True)
        bd.panel_ga_genome_grad(self.B, self.P, self.n, self.pb.grad, float(lr), self.lo,
                                self.hi, self.genome, None)
        return self.evaluate()

    def draw(self):
        return torch.rand(self.B // 2, 4 * self.k + 5, generator=self.gen, dtype=torch.float64,
                          device=self.device)

    def step(self, rand=None):
        """One generation from the current fitness (evaluate() first)."""
        rand = self.draw() if rand is None else rand
        bd.panel_ga_step(self.B, self.P, self.k, self.p, self.pm, self.lo, self.hi, self.sigma,
                         self.genome, self.fitness, rand, self.genome_next)
        self.genome, self.genome_next = self.genome_next, self.genome
        self.generation += 1
        return rand

    def run(self, generations: int, refine_lr: float = 0.0):
        """`generations` steps; with refine_lr > 0 each generation first takes
        one gradient-ascent step on Cl (refine())."""
        best = []
        for _ in range(generations):
            f = self.refine(refine_lr) if refine_lr > 0 else self.evaluate()
            best.append(float(torch.nan_to_num(f, nan=-np.inf).max()))
            self.step()
        self.evaluate()
        return best
