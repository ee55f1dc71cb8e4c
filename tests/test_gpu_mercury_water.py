"""The last experiment of Sec. 4 on the GPU path: the mercury/water crystal
(mercury cylinders in water, square lattice a = 0.5, filling 35 %, 256 elements
per circle, normal incidence).  The paper reports that its stop band is not
visible with M_L = 4 columns and becomes visible, with sharper edges, with
M_L = 10.

The 10-column block (width 5) is wider than the crystal's period 6a = 3 along y,
so the fundamental block is taken two periods tall (12 rows, H = 6): the same
crystal, whose field at normal incidence is 3-periodic and hence 6-periodic.  The
first test checks that reading: the 4-column crystal's ETC from the one-period
and the two-period blocks agree, and so does the 10-column crystal's from the
two-period block and from the one-period block, which is wider than its period
(two root squares)."""
import numpy as np
import pytest

from paper_1910_10863_gb300 import workloads as W
from tests.gpu_common import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    ensure_built()
    from paper_1910_10863_gb300 import pfmbem
    return pfmbem


def etc(pf, ka, ml, rows=12, tol=1e-6):
    w = W.mercury_water_block(ka, f=0.35, ml=ml, rows=rows)
    s = pf.Solver(w, precision=pf.MIXED)
    psi = np.zeros(2 * s.E, dtype=np.complex128)
    info = s.solve(psi, tol=tol, maxit=3000, check=False)
    assert info.rel_residual <= tol, (ka, ml, rows, info.rel_residual)
    e = pf.pfmbem_etc(s.h, psi, ml * 0.5, 256)
    s.close()
    return e


def test_one_period_and_two_period_blocks_agree(pf):
    for ka in (0.21, 0.37):
        a, b = etc(pf, ka, 4, rows=6, tol=1e-9), etc(pf, ka, 4, rows=12, tol=1e-9)
        assert abs(a - b) < 1e-7 * max(1.0, abs(a)), (ka, a, b)
    for ka in (0.34, 0.47):
        a, b = etc(pf, ka, 10, rows=6, tol=1e-9), etc(pf, ka, 10, rows=12, tol=1e-9)
        assert abs(a - b) < 1e-6 * max(1.0, abs(a)), (ka, a, b)


def test_stop_band_visible_with_ten_columns_only(pf):
    inside = (0.40, 0.47, 0.55)
    e4 = {ka: etc(pf, ka, 4) for ka in (0.34,) + inside}
    e10 = {ka: etc(pf, ka, 10) for ka in (0.34,) + inside}
    # M_L = 4: no stop band (ETC stays above 3 %); M_L = 10: ETC below 3 %
    assert all(e4[ka] > 0.03 for ka in inside), e4
    assert all(e10[ka] < 0.03 for ka in inside), e10
    # the lower band edge is much sharper with ten columns: the fall of ETC from
    # 0.34 to 0.40 is more than ten times larger
    assert e10[0.34] / e10[0.40] > 10 * (e4[0.34] / e4[0.40]), (e4, e10)
