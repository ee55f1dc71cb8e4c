"""Status codes of the solve's failure paths, made on the host (no GPU fault):

* ENOCONV: a tolerance that maxit products cannot reach; psi still holds the
  best iterate (its residual is below that of the zero start).
* ENUMERIC: a right-hand side with a NaN entry makes the residual non-finite.
* The handle stays usable after either: the next solve succeeds.
* ETIMEOUT: a device-wide barrier wait bounded by 1 us runs out.
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


def test_device_wait_that_runs_out_returns_etimeout(pf):
    """Every device-wide barrier wait of the single-launch product is bounded by
    options.wait_us; a 1 us bound runs out on the 8x8 hexagon block.  The call that
    reads the result returns PFMBEM_ETIMEOUT (no trap, no unbounded wait), the next
    product on the handle starts from cleared barrier words, and a handle with the
    default bound gives the per-stage kernels' product."""
    from tests.gpu_common import rel
    w = W.hexagon_8x8_n256()
    s = pf.Solver(w, wait_us=1)
    x = W.density_vector(w.E, 2)
    y = np.zeros_like(x)
    for _ in range(2):
        with pytest.raises(pf.PfmbemError) as e:
            s.matvec(x, y, pf.MIXED)
        assert e.value.status == 7                # PFMBEM_ETIMEOUT
    psi = np.zeros_like(x)
    with pytest.raises(pf.PfmbemError) as e:
        s.solve(psi, tol=1e-6, maxit=50)
    assert e.value.status == 7
    s.close()
    ok = pf.Solver(w)
    y2 = np.zeros_like(x)
    ok.matvec(x, y2, pf.FP64)
    ref = pf.Solver(w, launch=1)                  # per-stage kernels: no device-wide waits
    y3 = np.zeros_like(x)
    ref.matvec(x, y3, pf.FP64)
    assert rel(y2, y3) < 1e-12
