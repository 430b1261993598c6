"""Write tests/golden/large_solution_extended.npz: extended-precision reference
strengths (gamma_1..gamma_n and the constant C of the bordered system) for
large airfoils, against which the GPU's refined solutions are compared.

Why stored values.  Above ~600 panels the bordered systems have condition
numbers of 1e6..4e6 (inf norm), so the FP64 oracle's own strengths are off by
up to ~1e-9 (relative, inf norm) from the exact discrete solution, the same
order as the tolerance the GPU path is held to.  The long double build of the
oracle (oracle.extended(): assembly, factor and refinement all in long double)
is the reference.  On the GPU host long double is a software binary128 type,
far too slow for 2000-panel systems, so this script computes the strengths once
on a host whose long double is the x87 80-bit type and stores them with the
exact node coordinates they belong to (libm differs in the last bit between
hosts, and at these condition numbers one ulp of a node moves gamma by ~1e-9).
It also stores the FP64 oracle's deviation from them, which sets each
airfoil's tolerance: max(1e-10, 3 x that deviation).

Only the oracle and the seeded input generators are called.  Sets:
  ragged     NACA 4-digit airfoils of 640, 641, 767, 768, 1025, 1300 and 2048
             panels (seed 11): the edges of the 128-wide blocks of the
             step-synchronous factor;
  mixed      1500, 700, 639, 300, 229, 100 and 3 panels (seed 12): all
             factorisations in one launch;
  c5         the three airfoils of the 1024..2048-panel workload that
             large_gradient_extended.npz holds (their stored nodes).

    python tests/golden/make_large_solution_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1511_02166_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "large_solution_extended.npz")
RAGGED = {"ragged": (11, [640, 641, 767, 768, 1025, 1300, 2048]),
          "mixed": (12, [1500, 700, 639, 300, 229, 100, 3])}


def ragged_population(seed, sizes):
    """The NACA 4-digit test populations of the large-airfoil GPU tests."""
    rng = np.random.default_rng(seed)
    air = [inputs.naca4(rng.uniform(0, .06), rng.uniform(.2, .6), rng.uniform(.08, .18), n)
           for n in sizes]
    return inputs.pack(air, rng.uniform(-0.07, 0.17, len(air)))


def solve_set(nodes, offsets, alpha):
    with oracle.extended():
        assert oracle.is_extended()
        ext = oracle.evaluate_batch(nodes, offsets, alpha)
    assert np.all(ext["info"] == 0)
    f64 = oracle.evaluate_batch(nodes, offsets, alpha)
    assert np.all(f64["info"] == 0)
    dev = []
    for b in range(len(offsets) - 1):
        n = int(offsets[b + 1] - offsets[b])
        o = int(offsets[b]) + b
        ue = ext["u"][o:o + n]
        dev.append(float(np.max(np.abs(f64["u"][o:o + n] - ue)) / np.max(np.abs(ue))))
    return ext["u"], np.array(dev)


def main():
    out = {}
    for name, (seed, sizes) in RAGGED.items():
        pop = ragged_population(seed, sizes)
        u, dev = solve_set(pop.nodes, pop.offsets, pop.alpha)
        out[name + "_nodes"] = pop.nodes.copy()
        out[name + "_offsets"] = pop.offsets.copy()
        out[name + "_alpha"] = pop.alpha.copy()
        out[name + "_u"] = u
        out[name + "_fp64_dev"] = dev
        for n, d in zip(sizes, dev):
            print("%s n=%d: FP64 oracle gamma deviation %.2e" % (name, n, d))
    gold = np.load(os.path.join(HERE, "large_gradient_extended.npz"))
    idx = [int(b) for b in gold["index"]]
    air = [gold["nodes_%d" % b] for b in idx]
    offsets = np.concatenate([[0], np.cumsum([len(a) for a in air])]).astype(np.int64)
    alpha = np.array([float(gold["alpha_%d" % b]) for b in idx])
    u, dev = solve_set(np.concatenate(air), offsets, alpha)
    out["c5_index"] = np.array(idx, dtype=np.int64)
    out["c5_offsets"] = offsets
    out["c5_u"] = u
    out["c5_fp64_dev"] = dev
    for b, d in zip(idx, dev):
        print("c5 airfoil %d: FP64 oracle gamma deviation %.2e" % (b, d))
    np.savez_compressed(OUT, **out)
    print("wrote", OUT, os.path.getsize(OUT), "bytes")


if __name__ == "__main__":
    main()
