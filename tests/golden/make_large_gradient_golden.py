"""Write tests/golden/large_gradient_extended.npz: extended-precision reference
gradients dCl/d(nodes) for three airfoils of the large workload (1024 airfoils
of 1024..2048 panels): its smallest airfoil, the one nearest 1537 panels and
its largest.

Why stored values.  These bordered systems are so ill conditioned (1-norm
condition numbers 1e9..2e10) that the FP64 oracle's own gradient is off by up
to a few 1e-10 relative to the exact discrete gradient, the same order as the
1e-9 bound the GPU path is held to.  The long double build of the oracle
(oracle.extended(): every step, the panel integrals included, in long double)
is the reference, but on the GPU host long double is a software binary128 type
and one 2000-panel gradient would take hours there.  So this script computes
them once, on a host whose long double is the x87 80-bit type (64-bit
significand), and stores them with the exact node coordinates they belong to
(libm differs in the last bit between hosts, so the test puts these nodes into
the population instead of regenerating them).

Only the oracle and the seeded input generator are called.  Stored per airfoil:
its index in the population, the nodes, alpha, the gradient at every 4th node
(x and y), the inf norm of the whole extended gradient, and the FP64 oracle's
deviation from it (context).

    python tests/golden/make_large_gradient_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1511_02166_gb300 import inputs  # noqa: E402

OUT = os.path.join(HERE, "large_gradient_extended.npz")
NODE_STEP = 4


def main():
    pop = inputs.make_population("large_b1024_n1024_2048")
    sizes = pop.sizes
    idx = sorted({int(np.argmin(sizes)), int(np.argmin(np.abs(sizes - 1537))),
                  int(np.argmax(sizes))})
    sub = pop.subset(idx)
    with oracle.extended():
        assert oracle.is_extended()
        g_ld, info = oracle.cl_gradient_batch(sub.nodes, sub.offsets, sub.alpha)
    assert np.all(info == 0)
    g_64, info64 = oracle.cl_gradient_batch(sub.nodes, sub.offsets, sub.alpha)
    assert np.all(info64 == 0)
    out = {"index": np.array(idx, dtype=np.int64), "node_step": np.int64(NODE_STEP)}
    for s, b in enumerate(idx):
        sl = slice(sub.offsets[s], sub.offsets[s + 1])
        g = g_ld[sl]
        scale = float(np.max(np.abs(g)))
        out["nodes_%d" % b] = sub.nodes[sl].copy()
        out["alpha_%d" % b] = np.float64(sub.alpha[s])
        out["grad_%d" % b] = g[::NODE_STEP].copy()
        out["scale_%d" % b] = np.float64(scale)
        out["fp64_dev_%d" % b] = np.float64(np.max(np.abs(g_64[sl] - g)) / scale)
        print("airfoil %d: n = %d, |g|_inf = %.6e, FP64 oracle deviation %.2e"
              % (b, sl.stop - sl.start, scale, out["fp64_dev_%d" % b]))
    np.savez_compressed(OUT, **out)
    print("wrote", OUT, os.path.getsize(OUT), "bytes")


if __name__ == "__main__":
    main()
