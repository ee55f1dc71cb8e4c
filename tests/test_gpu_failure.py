"""Status codes of the solve's failure paths, made on the host (no GPU fault):

* ENOCONV: a tolerance that maxit products cannot reach; psi still holds the
  best iterate (its residual is below that of the zero start).
* ENUMERIC: a right-hand side with a NaN entry makes the residual non-finite.
* The handle stays usable after either: the next solve succeeds.
(ETIMEOUT, a device-side wait that runs out, is in test_gpu_flow.py.)
"""
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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_enoconv_writes_best_iterate(pf, precision):
    w = W.hexagon_8x8_n256()
    s = pf.Solver(w, precision=pf.FP64 if precision == "fp64" else pf.MIXED)
    psi = np.zeros(2 * s.E, dtype=np.complex128)
    info = s.solve(psi, tol=1e-14, maxit=3, check=False)
    assert info.status == 6                      # PFMBEM_ENOCONV
    assert 0 < info.rel_residual < 1.0
    assert np.all(np.isfinite(psi)) and np.linalg.norm(psi) > 0
    psi2 = np.zeros_like(psi)
    ok = s.solve(psi2, tol=1e-6, maxit=500)
    assert ok.rel_residual <= 1e-6


def test_enumeric_on_non_finite_rhs(pf):
    w = W.square_2x2_n64()
    s = pf.Solver(w)
    B = np.ones(2 * s.E, dtype=np.complex128)
    B[7] = np.nan
    psi = np.zeros_like(B)
    with pytest.raises(pf.PfmbemError) as e:
        s.solve(psi, B=B, tol=1e-8, maxit=100)
    assert e.value.status == 8                   # PFMBEM_ENUMERIC
    psi2 = np.zeros_like(B)
    ok = s.solve(psi2, tol=1e-8, maxit=300)
    assert ok.rel_residual <= 1e-8
