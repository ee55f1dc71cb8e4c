"""Handle life cycle on the GPU (C ABI): many handles alive at once, created on
two streams and solved out of creation order, then destroyed and created again.

This exercises what the create hands from one handle to the next: the pooled
set-up streams and events, the page-locked staging arena passed on through an
event (a create returns before its device work has finished), the arrays carved
from per-handle chunks of the memory pool, and the deferred operator check.
Every solution is compared with the dense oracle solve (relative L2 <= 1e-6).
"""
import numpy as np
import pytest

from oracle import bem
from paper_1910_10863_gb300 import workloads as W
from tests.gpu_common import ensure_built, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    ensure_built()
    from paper_1910_10863_gb300 import pfmbem
    return pfmbem


def test_many_live_handles_solve_out_of_order(pf):
    import torch
    w = W.square_2x2_n64()
    pb = bem.problem(w)
    psi_ref = np.linalg.solve(bem.operator_rows(pb), bem.rhs(pb))
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    hs = []
    for i in range(12):
        s = pf.Solver(w, precision=pf.MIXED, stream=streams[i % 2].cuda_stream)
        hs.append(s)
    # the plan is readable straight after create (it waits for the set-up)
    assert hs[-1].plan().near_blocks > 0
    for i in (7, 0, 11, 4):
        psi = np.zeros(2 * hs[i].E, dtype=np.complex128)
        info = hs[i].solve(psi, tol=1e-8, maxit=500)
        assert info.rel_residual <= 1e-8
        assert rel(psi, psi_ref) < 1e-6
    for s in reversed(hs):
        s.close()
    torch.cuda.synchronize()
    # a create after the others were released reuses their streams, events and memory
    s = pf.Solver(w, precision=pf.FP64)
    psi = np.zeros(2 * s.E, dtype=np.complex128)
    info = s.solve(psi, tol=1e-8, maxit=500)
    s.close()
    assert info.rel_residual <= 1e-8
    assert rel(psi, psi_ref) < 1e-6
