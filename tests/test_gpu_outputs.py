"""Outputs of Sec. 4 through the C ABI: the x1-derivative of the scattered field
and the energy transmission coefficient ETC against the oracle, and the stop
band of the water/mercury crystal of Table 3."""
import os

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


def _golden_gap(scatterer, lattice, fill):
    path = os.path.join(os.path.dirname(__file__), "golden", "table3_band_gaps.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        if f[0] == scatterer and f[1] == lattice and abs(float(f[2]) - fill) < 1e-9:
            return [float(x) for x in f[3:]]
    raise KeyError((scatterer, lattice, fill))


def test_table3_first_stop_band_circles_in_square_lattice(pf):
    """Table 3, circular scatterers in a square lattice, filling fraction 35 %:
    ETC < 3 % inside the printed first gap and above it below the gap."""
    lo, hi, _, _ = _golden_gap("circular", "square", 0.35)
    inside = [lo + 0.25 * (hi - lo), 0.5 * (lo + hi), lo + 0.7 * (hi - lo)]
    outside = [0.1, 0.14]
    for ka in inside + outside:
        # stay away from the Wood anomalies ka/2pi = n/6 of normal incidence
        assert min(abs(ka - n / 6) for n in range(1, 10)) > 0.01
    for ka, expect_gap in [(k, True) for k in inside] + [(k, False) for k in outside]:
        w = W.table3_square(ka, f=0.35)
        s = pf.Solver(w, precision=pf.MIXED)
        psi = np.zeros(2 * s.E, dtype=np.complex128)
        info = s.solve(psi, tol=1e-6, check=False)
        assert info.rel_residual <= 1e-6
        etc = pf.pfmbem_etc(s.h, psi, 2.0, 256)
        assert (etc < 0.03) == expect_gap, (ka, etc)
