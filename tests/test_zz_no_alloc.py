"""panel_solve_noalloc: the solve for callers that cannot allocate device memory.

Some callers of this library cannot call cudaMalloc (a plug-in inside a host
application that owns all device allocations, a real-time loop that must not
allocate once running, a binding without a device allocator), so they cannot
pass panel_solve its factor and pivot work arrays.  panel_solve_noalloc keeps
those two arrays in a fixed-size static device array of the library instead.
These tests call it through the C ABI and check, on two calls in a row with
different batches (the array keeps the previous call's contents), that it
returns what panel_solve returns with caller-owned work arrays, within the
tolerance of the other parity tests (1e-10 relative, inf norm), and that a
batch too large for the array is refused before anything runs.

The file is named to be collected last, so that a run stopping at the first
failure has run every other test before this one.
"""
import ctypes

import numpy as np
import pytest

from paper_1511_02166_gb300 import inputs
from tests.gpu_util import need_gpu, rel_inf

pytestmark = pytest.mark.gpu


def _ragged(seed, sizes):
    rng = np.random.default_rng(seed)
    air = [inputs.naca4(rng.uniform(0, .06), rng.uniform(.2, .6), rng.uniform(.08, .18), n)
           for n in sizes]
    return inputs.pack(air, rng.uniform(-0.07, 0.17, len(air)))


def _assembled(pop, mode):
    import torch
    from paper_1511_02166_gb300.solver import PanelBatch
    pb = PanelBatch(pop.nodes, pop.offsets, pop.alpha, mode=mode, bucket_width=None)
    pb.assemble()
    torch.cuda.synchronize()
    assert np.all(pb.info.cpu().numpy() == 0)
    return pb


def _solve_both(pb, flags):
    """(u, lambda, iters) from panel_solve with the batch's own work arrays and
    from panel_solve_noalloc, on the same assembled batch."""
    import torch
    from paper_1511_02166_gb300 import binding as bd
    out = []
    for noalloc in (False, True):
        u = torch.full_like(pb.u, np.nan)
        lam = torch.full_like(pb.lam, np.nan)
        info = torch.zeros_like(pb.info)
        iters = torch.zeros_like(pb.iters)
        common = (pb.nodes, pb.node_offsets, pb.mat_offsets, pb.order, pb.A64, pb.A_hi, pb.A_lo)
        if noalloc:
            bd.panel_solve_noalloc(pb.B, pb.n_max, flags, pb.offsets_h, *common, pb.rhs,
                                   pb.vinf, pb.chord, u, lam, pb.max_iter, pb.tol, info, iters)
        else:
            bd.panel_solve(pb.B, pb.n_max, flags, *common, pb.LU, pb.piv,
                           pb.rhs, pb.vinf, pb.chord, u, lam, pb.max_iter, pb.tol, info, iters)
        torch.cuda.synchronize()
        assert np.all(info.cpu().numpy() == 0)
        out.append((u.cpu().numpy(), lam.cpu().numpy(), iters.cpu().numpy()))
    return out


def _assert_same(pop, ref, got):
    for b in range(pop.batch):
        o = pop.offsets[b] + b
        m = pop.offsets[b + 1] - pop.offsets[b] + 1
        assert rel_inf(got[0][o:o + m], ref[0][o:o + m]) < 1e-10, b
        assert rel_inf(got[1][o:o + m], ref[1][o:o + m]) < 1e-10, b


@pytest.mark.parametrize("mode", ["mixed", "fp64"])
def test_noalloc_solve_matches_panel_solve_on_two_calls_in_a_row(mode):
    need_gpu()
    from paper_1511_02166_gb300 import binding as bd
    flags = (bd.PANEL_MIXED if mode == "mixed" else bd.PANEL_FP64) | bd.PANEL_WITH_ADJOINT
    # first call: ragged sizes across the one-block and the step-synchronous
    # (tensor-core) factorisations; second call: a different, smaller batch, so
    # that the array still holds the first call's larger factor
    first = _ragged(21, [100, 257, 3, 700, 200, 64] if mode == "mixed" else [100, 257, 3, 64])
    second = _ragged(22, [150, 31, 90])
    for pop in (first, second):
        pb = _assembled(pop, mode)
        ref, got = _solve_both(pb, flags)
        _assert_same(pop, ref, got)
        if mode == "mixed":
            assert np.array_equal(ref[2], got[2])


def test_noalloc_rejects_a_batch_beyond_the_static_array():
    need_gpu()
    import torch
    from paper_1511_02166_gb300 import binding as bd
    lib = bd.load()
    # three airfoils of 2048 panels need 3 x 2049^2 x 4 bytes of factor > 32 MiB
    offs = np.arange(4, dtype=np.int64) * 2048
    need = 3 * 2049 ** 2 * 4
    assert need > bd.PANEL_NOALLOC_SCRATCH_BYTES
    d = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(d.data_ptr())
    st = lib.panel_solve_noalloc(3, 2048, bd.PANEL_MIXED, offs.ctypes.data, p, p, p, p, None, p,
                                 p, p, None, None, p, None, 10, 1e-12, p, None,
                                 torch.cuda.current_stream().cuda_stream)
    assert st == bd.PANEL_ESCRATCH
    assert "static work array" in bd.panel_strerror(st)
    torch.cuda.synchronize()
    assert np.all(d.cpu().numpy() == 0)  # nothing ran
