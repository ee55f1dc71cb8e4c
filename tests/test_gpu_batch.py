"""Batched lockstep solve (band-gap sweep) against dense LU of the oracle, with
uneven element counts and one CUDA stream per instance."""
import math

import numpy as np
import pytest

from oracle import bem
from paper_1910_10863_gb300 import workloads as W
from tests.gpu_common import ensure_built, rel

pytestmark = pytest.mark.gpu


def test_batch_solve_matches_dense_lu():
    ensure_built()
    import torch

    from paper_1910_10863_gb300 import pfmbem as pf
    ws = [W.square_block(2, 2, 1.0, 0.3, 24, 2.0, math.radians(30), name="b0"),
          W.square_block(2, 2, 1.0, 0.25, 40, 3.3, math.radians(11), name="b1"),
          W.hexagon_block(2, 2, 1.0, 0, 1.7, math.radians(52), seed=9, n_of_r=lambda rf: 20 + int(60 * rf), name="b2")]
    streams = [torch.cuda.Stream() for _ in ws]
    solvers = [pf.Solver(w, precision=pf.MIXED, stream=s.cuda_stream) for w, s in zip(ws, streams)]
    psis = [np.zeros(2 * s.E, dtype=np.complex128) for s in solvers]
    st, infos = pf.pfmbem_solve_batch([s.h for s in solvers], psis, tol=1e-9, maxit=2000)
    assert st == 0
    for w, psi, info in zip(ws, psis, infos):
        assert info.rel_residual <= 1e-9
        pb = bem.problem(w)
        ref = np.linalg.solve(bem.operator_rows(pb), bem.rhs(pb))
        assert rel(psi, ref) < 1e-6
