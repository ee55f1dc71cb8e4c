"""Outputs of Sec. 4 through the C ABI: the x1-derivative of the scattered field
and the energy transmission coefficient ETC against the oracle (the stop bands
of Table 3 are in test_gpu_table3.py)."""
import numpy as np
import pytest

from oracle import bem
from paper_1910_10863_gb300 import workloads as W
from tests.gpu_common import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    ensure_built()
    from paper_1910_10863_gb300 import pfmbem
    return pfmbem


def test_field_x1_derivative_and_etc_match_oracle(pf):
    w = W.square_2x2_n64()
    pb = bem.problem(w)
    M = bem.operator_rows(pb)
    psi = np.linalg.solve(M, bem.rhs(pb))
    s = pf.Solver(w)
    pts = np.array([[1.0, 0.13], [0.95, 0.61], [-0.05, 0.37], [0.5, 0.5]])
    u = np.zeros(len(pts), dtype=np.complex128)
    du = np.zeros(len(pts), dtype=np.complex128)
    pf.pfmbem_field_dx1(s.h, psi, pts, u, du)
    hstep = 1e-5
    ref = (bem.potential(pb, psi, pts + [hstep, 0]) - bem.potential(pb, psi, pts - [hstep, 0])) / (2 * hstep)
    assert np.max(np.abs(u - bem.potential(pb, psi, pts))) < 1e-8 * np.max(np.abs(u))
    assert np.max(np.abs(du - ref)) < 1e-6 * np.max(np.abs(ref))
    # ETC on the block's right edge (x1 = 1, 0.1 to the right of the fibers):
    # midpoint rule on the GPU against the oracle's Rayleigh expansion on the same
    # points (x2 = H (j + 1/2) / npts; the root box starts at y0 = 0 here).  The GPU
    # field takes the images |m| >= 2 from the root's local expansion, whose
    # truncation at p0 leaves ~1e-6 of max|du| at the two ends of the line (the root
    # box's corners, 0.71 H from its centre) and ~1e-8 elsewhere: ETC agrees to ~1e-8.
    etc = pf.pfmbem_etc(s.h, psi, 1.0, 512)
    etc_ref = bem.etc(pb, psi, nmax=60, npts=512, x1=1.0)
    assert abs(etc - etc_ref) < 1e-6 * etc_ref
