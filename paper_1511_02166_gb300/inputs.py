"""Seeded synthetic airfoil populations and analytic test shapes.

This module only makes inputs: node polygons, angles of attack and batch
offsets.  It holds none of the panel method's arithmetic, so both the CUDA path
and the FP64 oracle can be fed from it.

Node convention (Section 2, Figure 1 of the paper): n distinct nodes per
airfoil, counter-clockwise, x_0 at the trailing edge, the closing node x_n = x_0
implied.  For NACA shapes the upper surface comes first (trailing edge ->
leading edge), then the lower surface (leading edge -> trailing edge), which is
the genome order the paper describes for its B-spline knots (Section 2).

The populations stand in for the paper's genetic-algorithm generations
(Section 3, Table 2: thousands of candidate airfoils of about 200 panels): NACA
4-digit sections with camber m ~ U[0, 0.06], camber position p ~ U[0.2, 0.6],
thickness t ~ U[0.08, 0.18] and angle of attack alpha ~ U[-4, 10] degrees,
cosine-spaced nodes and a closed trailing edge.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 1511021660

#: trailing-edge-closed NACA 4-digit thickness coefficients (last one -0.1036)
_T_COEF = (0.2969, -0.1260, -0.3516, 0.2843, -0.1036)


def _thickness(x: np.ndarray, t: float) -> np.ndarray:
    a0, a1, a2, a3, a4 = _T_COEF
    return 5.0 * t * (a0 * np.sqrt(x) + a1 * x + a2 * x**2 + a3 * x**3 + a4 * x**4)


def _camber(x: np.ndarray, m: float, p: float):
    if m == 0.0:
        return np.zeros_like(x), np.zeros_like(x)
    fore = x < p
    yc = np.where(fore, m / p**2 * (2 * p * x - x**2),
                  m / (1 - p)**2 * ((1 - 2 * p) + 2 * p * x - x**2))
    dyc = np.where(fore, 2 * m / p**2 * (p - x), 2 * m / (1 - p)**2 * (p - x))
    return yc, dyc


def cosine_stations(n: int):
    """x-stations of the upper (TE->LE, inclusive) and lower (LE->TE, exclusive) sides.

    The upper side gets ceil(n/2) panels and the lower floor(n/2); they share
    the leading-edge node, and the trailing edge is node 0.
    """
    if n < 3:
        raise ValueError("an airfoil needs at least 3 nodes")
    nu, nl = (n + 1) // 2, n // 2
    xu = 0.5 * (1.0 + np.cos(np.pi * np.arange(nu + 1) / nu))
    xl = 0.5 * (1.0 - np.cos(np.pi * np.arange(1, nl) / nl))
    return xu, xl


def naca4(m: float, p: float, t: float, n: int, dy_camber=None, dy_thick=None) -> np.ndarray:
    """Closed-trailing-edge NACA 4-digit section with n cosine-spaced nodes.

    ``dy_camber`` / ``dy_thick`` are optional callables of the station x that
    add a vertical camber / half-thickness perturbation (used by the uneven
    population).  Returns float64 nodes [n][2], counter-clockwise, x_0 at the TE.
    """
    xu, xl = cosine_stations(n)
    out = []
    for xs, sign in ((xu, 1.0), (xl, -1.0)):
        yt = _thickness(xs, t)
        yc, dyc = _camber(xs, m, p)
        th = np.arctan(dyc)
        X = xs - sign * yt * np.sin(th)
        Y = yc + sign * yt * np.cos(th)
        if dy_camber is not None:
            Y = Y + dy_camber(xs)
        if dy_thick is not None:
            Y = Y + sign * dy_thick(xs)
        out.append(np.stack([X, Y], axis=1))
    nodes = np.concatenate(out, axis=0)
    assert nodes.shape == (n, 2)
    return nodes


def cylinder(n: int, radius: float = 0.5, center=(0.5, 0.0)) -> np.ndarray:
    """Circle of n nodes at uniform angles, node 0 at angle 0 (the rear point)."""
    th = 2.0 * np.pi * np.arange(n) / n
    return np.stack([center[0] + radius * np.cos(th), center[1] + radius * np.sin(th)], axis=1)


@dataclasses.dataclass(frozen=True)
class Joukowski:
    """Joukowski section z = zeta + 1/zeta of the circle through zeta = 1.

    Circle centre mu = (-eps, (1 + eps) tan(beta)), radius R = |1 - mu|; the
    trailing edge is z = 2 (zeta = 1).
    """
    eps: float = 0.1
    beta: float = math.radians(5.0)

    @property
    def mu(self) -> complex:
        return complex(-self.eps, (1.0 + self.eps) * math.tan(self.beta))

    @property
    def radius(self) -> float:
        return abs(1.0 - self.mu)

    def zeta(self, phi):
        """Circle point at angle phi (measured from the centre, 0 = +x)."""
        return self.mu + self.radius * np.exp(1j * np.asarray(phi))

    def phi_te(self) -> float:
        return math.atan2(-(self.mu.imag), 1.0 - self.mu.real)

    def nodes(self, n: int) -> np.ndarray:
        phi = self.phi_te() + 2.0 * np.pi * np.arange(n) / n
        zeta = self.zeta(phi)
        zeta[0] = 1.0  # the trailing edge exactly
        z = zeta + 1.0 / zeta
        return np.stack([z.real, z.imag], axis=1)


# --------------------------------------------------------------------------
# Batched populations
# --------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class PopulationSpec:
    name: str
    batch: int
    n_min: int
    n_max: int
    perturbed: bool = False
    seed_index: int = 0

    @property
    def seed(self) -> int:
        return SEED_BASE + self.seed_index


#: The five workloads: small FP64 case, GA generation, uneven batch, adjoint, large N.
SPECS = {
    "naca_b64_n100": PopulationSpec("naca_b64_n100", 64, 100, 100, False, 0),
    "naca_b4096_n200": PopulationSpec("naca_b4096_n200", 4096, 200, 200, False, 1),
    "uneven_b10000_n64_512": PopulationSpec("uneven_b10000_n64_512", 10000, 64, 512, True, 2),
    "adjoint_b4096_n256": PopulationSpec("adjoint_b4096_n256", 4096, 256, 256, False, 3),
    "large_b1024_n1024_2048": PopulationSpec("large_b1024_n1024_2048", 1024, 1024, 2048,
                                             False, 4),
}


@dataclasses.dataclass
class Population:
    """A ragged batch: nodes [sum n_b][2] f64, offsets [B+1] i64, alpha [B] f64 (rad)."""
    nodes: np.ndarray
    offsets: np.ndarray
    alpha: np.ndarray
    params: np.ndarray  # [B][3] = (m, p, t)

    @property
    def batch(self) -> int:
        return len(self.offsets) - 1

    @property
    def sizes(self) -> np.ndarray:
        return np.diff(self.offsets)

    def airfoil(self, b: int) -> np.ndarray:
        return self.nodes[self.offsets[b]:self.offsets[b + 1]]

    def subset(self, idx) -> "Population":
        idx = np.asarray(idx, dtype=np.int64)
        parts = [self.airfoil(int(b)) for b in idx]
        sizes = np.array([len(p) for p in parts], dtype=np.int64)
        offsets = np.zeros(len(idx) + 1, dtype=np.int64)
        np.cumsum(sizes, out=offsets[1:])
        nodes = np.concatenate(parts, axis=0) if parts else np.zeros((0, 2))
        return Population(np.ascontiguousarray(nodes), offsets, self.alpha[idx].copy(),
                          self.params[idx].copy())


def _perturbations(rng: np.random.Generator, t: float, n: int):
    """Eight cosine-mode perturbations (4 camber, 4 thickness), amplitudes N(0, 0.005).

    In the cosine variable beta (x = (1 - cos beta)/2): dy_c = sum a_k sin(k beta),
    dy_t = sum b_k sin(k beta) sin(beta), k = 1..4.  Redrawn from the same stream
    until the perturbed half-thickness stays >= half of the base one.
    """
    xu, xl = cosine_stations(n)
    xs = np.concatenate([xu, xl])
    xs = xs[(xs > 0.0) & (xs < 1.0)]  # the perturbations vanish at the LE and TE
    k = np.arange(1, 5)[:, None]
    for _ in range(1000):
        a = rng.normal(0.0, 0.005, 4)
        b = rng.normal(0.0, 0.005, 4)

        def dyc(x, a=a):
            beta = np.arccos(np.clip(1.0 - 2.0 * x, -1.0, 1.0))
            return (a[:, None] * np.sin(k * beta)).sum(0)

        def dyt(x, b=b):
            beta = np.arccos(np.clip(1.0 - 2.0 * x, -1.0, 1.0))
            return (b[:, None] * np.sin(k * beta)).sum(0) * np.sin(beta)

        if np.all(dyt(xs) >= -0.5 * _thickness(xs, t)):
            return dyc, dyt
    raise RuntimeError("could not draw an admissible perturbation")


def make_population(spec: PopulationSpec | str, batch: int | None = None) -> Population:
    """Draw a seeded population.  Per airfoil the draw order is m, p, t, alpha,
    then n (uneven batches), then the perturbation amplitudes.  ``batch`` draws
    only the first ``batch`` airfoils of the same stream."""
    if isinstance(spec, str):
        spec = SPECS[spec]
    B = spec.batch if batch is None else int(batch)
    rng = np.random.Generator(np.random.PCG64(spec.seed))
    parts, sizes, alpha, params = [], [], [], []
    for _ in range(B):
        m = rng.uniform(0.0, 0.06)
        p = rng.uniform(0.2, 0.6)
        t = rng.uniform(0.08, 0.18)
        a = math.radians(rng.uniform(-4.0, 10.0))
        n = int(rng.integers(spec.n_min, spec.n_max + 1)) if spec.n_max > spec.n_min else spec.n_min
        if spec.perturbed:
            dyc, dyt = _perturbations(rng, t, n)
            nodes = naca4(m, p, t, n, dyc, dyt)
        else:
            nodes = naca4(m, p, t, n)
        parts.append(nodes)
        sizes.append(n)
        alpha.append(a)
        params.append((m, p, t))
    offsets = np.zeros(B + 1, dtype=np.int64)
    np.cumsum(np.asarray(sizes, dtype=np.int64), out=offsets[1:])
    nodes = np.ascontiguousarray(np.concatenate(parts, axis=0)) if parts else np.zeros((0, 2))
    return Population(nodes, offsets, np.asarray(alpha, dtype=np.float64),
                      np.asarray(params, dtype=np.float64).reshape(B, 3))


def pack(airfoils, alphas) -> Population:
    """Pack a list of node arrays and angles into a ragged Population."""
    sizes = np.array([len(a) for a in airfoils], dtype=np.int64)
    offsets = np.zeros(len(airfoils) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    nodes = (np.ascontiguousarray(np.concatenate([np.asarray(a, np.float64) for a in airfoils]))
             if len(airfoils) else np.zeros((0, 2)))
    return Population(nodes, offsets, np.asarray(alphas, dtype=np.float64),
                      np.zeros((len(airfoils), 3)))
