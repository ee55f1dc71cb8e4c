"""Blocks wider than the period H (Sec. 2 allows any block width L): a row of
root squares of side H, coupled at the top by explicit root-to-root M2L for the
images |m| < m0 and a super root over the row whose lattice sums (Sec. 3.3) take
the images |m| >= m0.  Against the dense CPU oracle, which has no tree: the FP64
and mixed products on random and smooth densities, the solution, the Bragg
coefficients and ETC on the right block edge."""
import math

import numpy as np
import pytest

from oracle import bem
from paper_1910_10863_gb300 import workloads as W
from tests.gpu_common import ensure_built, rel

pytestmark = pytest.mark.gpu

CASES = [
    # (workload, options, roots)
    (lambda: W.square_block(3, 2, 1.0, 0.3, 20, 3.0, math.radians(20), name="wide_3x2_kH3"), {}, 2),
    (lambda: W.square_block(5, 2, 1.0, 0.3, 20, 2.2, math.radians(35), name="wide_5x2_kH2.2"), {}, 3),
    (lambda: W.square_block(5, 2, 1.0, 0.3, 20, 2.2, math.radians(35), name="wide_5x2_kH2.2_d3"), {"depth": 3}, 3),
]
_cache = {}


@pytest.fixture(scope="module")
def pf():
    ensure_built()
    from paper_1910_10863_gb300 import pfmbem
    return pfmbem


def oracle(w):
    if w.name not in _cache:
        pb = bem.problem(w)
        A = bem.operator_rows(pb)
        B = bem.rhs(pb)
        _cache[w.name] = (pb, A, B, np.linalg.solve(A, B))
    return _cache[w.name]


@pytest.mark.parametrize("make,opts,roots", CASES)
def test_wide_products(pf, make, opts, roots):
    w = make()
    pb, A, B, psi = oracle(w)
    s = pf.Solver(w, precision=pf.MIXED, **opts)
    plan = pf.pfmbem_plan(s.h)
    assert plan.nroot == roots and plan.super_p >= plan.p[0]
    rng = np.random.default_rng(7)
    x = rng.standard_normal(2 * s.E) + 1j * rng.standard_normal(2 * s.E)
    for v in (x, psi):
        v = np.ascontiguousarray(v)
        ref = A @ v
        y64 = np.zeros_like(v)
        y32 = np.zeros_like(v)
        s.matvec(v, y64, pf.FP64)
        s.matvec(v, y32, pf.MIXED)
        assert rel(y64, ref) < 1e-8, rel(y64, ref)
        assert rel(y32, ref) < 2e-6, rel(y32, ref)


@pytest.mark.parametrize("make,opts,roots", CASES[:2])
def test_wide_solution_coefficients_etc(pf, make, opts, roots):
    w = make()
    pb, A, B, psi_ref = oracle(w)
    s = pf.Solver(w, precision=pf.MIXED, **opts)
    psi = np.zeros(2 * s.E, dtype=np.complex128)
    info = s.solve(psi, tol=1e-10, maxit=2000)
    assert info.rel_residual <= 1e-10
    assert rel(psi, psi_ref) < 1e-6
    orders, R, T, energy = pf.pfmbem_coefficients(s.h, psi)
    ordr, Rr, Tr = bem.rayleigh(pb, psi_ref, np.asarray(orders))
    assert np.max(np.abs(np.asarray(R) - Rr)) < 1e-6 and np.max(np.abs(np.asarray(T) - Tr)) < 1e-6
    x1 = float(np.max(w.centres[:, 0]) + 0.25)          # the right edge of the last cell (a = 0.5)
    e_gpu = pf.pfmbem_etc(s.h, psi, x1, 256)
    e_ref = bem.etc(pb, psi_ref, npts=256, x1=x1)
    assert abs(e_gpu - e_ref) < 1e-6, (e_gpu, e_ref)
