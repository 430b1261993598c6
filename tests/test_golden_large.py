"""Consistency of the stored extended-precision large-airfoil strengths
(tests/golden/large_solution_extended.npz, written by
make_large_solution_golden.py from the long double oracle): the stored nodes
are those of the seeded NACA 4-digit populations, and on the airfoils small
enough to solve here in FP64 the FP64 oracle reproduces the stored strengths
within the deviation recorded beside them."""
import os

import numpy as np

import oracle
from paper_1511_02166_gb300 import inputs

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                    "large_solution_extended.npz")
SETS = {"ragged": (11, [640, 641, 767, 768, 1025, 1300, 2048]),
        "mixed": (12, [1500, 700, 639, 300, 229, 100, 3])}


def _population(seed, sizes):
    rng = np.random.default_rng(seed)
    air = [inputs.naca4(rng.uniform(0, .06), rng.uniform(.2, .6), rng.uniform(.08, .18), n)
           for n in sizes]
    return inputs.pack(air, rng.uniform(-0.07, 0.17, len(air)))


def test_stored_nodes_are_the_seeded_populations():
    g = np.load(GOLD)
    for name, (seed, sizes) in SETS.items():
        pop = _population(seed, sizes)
        assert np.array_equal(g[name + "_offsets"], pop.offsets)
        np.testing.assert_allclose(g[name + "_nodes"], pop.nodes, rtol=0, atol=1e-15)
        np.testing.assert_allclose(g[name + "_alpha"], pop.alpha, rtol=0, atol=1e-15)
        assert g[name + "_u"].shape == (pop.offsets[-1] + pop.batch,)


def test_fp64_oracle_reproduces_small_stored_strengths():
    g = np.load(GOLD)
    nodes, offs, alpha = g["mixed_nodes"], g["mixed_offsets"], g["mixed_alpha"]
    dev = g["mixed_fp64_dev"]
    for b in range(len(offs) - 1):
        n = int(offs[b + 1] - offs[b])
        if n > 300:
            continue
        s = slice(offs[b], offs[b + 1])
        r = oracle.evaluate(nodes[s], float(alpha[b]))
        o = int(offs[b]) + b
        ue = g["mixed_u"][o:o + n]
        d = np.max(np.abs(r["u"][:n] - ue)) / np.max(np.abs(ue))
        assert d <= max(3 * dev[b], 1e-15), (n, d, dev[b])
        assert dev[b] < 1e-10
