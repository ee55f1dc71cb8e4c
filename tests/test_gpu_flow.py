"""The dataflow form of the single-launch product (per-box completion counters
instead of device-wide barriers) against the barrier form and the oracle.

* Same cached operators, both forms: FP64 products agree to rounding (1e-12);
  the FP32 forms differ in their near-field arithmetic (the dataflow form sums
  differences psi_j - psi_t of hi + lo densities and adds the row sums in FP64),
  so they agree to the FP32 tolerance of random vectors (2e-6).
* On the smooth incident-field density, the dataflow FP32 product matches the
  oracle rows to 2e-6: the differences remove the FP32 cancellation of the
  hypersingular same-fiber blocks.
* Products of both precisions interleaved, repeated and skipped by a converged
  cycle's flag keep their counters in step (each product's result unchanged).
* A device-side wait that runs out (a 1 us bound set through the options) ends
  the product with PFMBEM_ETIMEOUT, returned to the caller; the next products
  on that handle start afresh, and a handle with the default bound is unaffected.
"""
import os

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


def _flow_solver(pf, w, **kw):
    """The dataflow form is chosen at create when PFMBEM_FLOW=1 (off by default)."""
    os.environ["PFMBEM_FLOW"] = "1"
    try:
        return pf.Solver(w, **kw)
    finally:
        del os.environ["PFMBEM_FLOW"]


@pytest.mark.parametrize("make", [W.hexagon_8x8_n256, W.square_32x32_n128])
def test_dataflow_product_matches_barrier_product(pf, make):
    w = make()
    sf = _flow_solver(pf, w)
    sb = pf.Solver(w)
    for seed in (3, 4):
        x = W.density_vector(w.E, seed)
        for prec, tol in ((pf.FP64, 1e-12), (pf.MIXED, 2e-6)):
            yf = np.zeros_like(x)
            yb = np.zeros_like(x)
            sf.matvec(x, yf, prec)
            sb.matvec(x, yb, prec)
            assert rel(yf, yb) < tol, (seed, prec, rel(yf, yb))


def test_dataflow_fp32_on_smooth_density_matches_oracle_rows(pf):
    w = W.hexagon_8x8_n256()
    s = _flow_solver(pf, w)
    pb = bem.problem(w)
    rng = np.random.default_rng(11)
    rows_e = np.sort(rng.choice(w.E, size=6, replace=False))
    Mr = bem.operator_rows(pb, rows_e)
    idx = np.ravel(np.stack([2 * rows_e, 2 * rows_e + 1], axis=1))
    xs = bem.rhs(pb)
    ref = Mr @ xs
    y = np.zeros_like(xs)
    s.matvec(xs, y, pf.MIXED)
    assert rel(y[idx], ref) < 2e-6, rel(y[idx], ref)


def test_interleaved_and_skipped_products_keep_counters_in_step(pf):
    import torch
    w = W.hexagon_8x8_n256()
    s = _flow_solver(pf, w)
    x = W.density_vector(w.E, 9)
    ref = {}
    for prec in (pf.FP64, pf.MIXED):
        y = np.zeros_like(x)
        s.matvec(x, y, prec)
        ref[prec] = y
    xd = torch.from_numpy(x).cuda()
    yd = torch.zeros_like(xd)
    order = [pf.MIXED, pf.MIXED, pf.FP64, pf.MIXED, pf.FP64, pf.FP64, pf.MIXED]
    for prec in order:
        s.matvec(xd, yd, prec)
        torch.cuda.synchronize()
        assert rel(yd.cpu().numpy(), ref[prec]) < (1e-13 if prec == pf.FP64 else 1e-6)
    # a solve (whose converged cycles skip the products queued after them), then products again
    psi = np.zeros_like(x)
    info = s.solve(psi, tol=1e-8, maxit=500)
    assert info.rel_residual <= 1e-8
    for prec in (pf.FP64, pf.MIXED):
        y = np.zeros_like(x)
        s.matvec(x, y, prec)
        assert rel(y, ref[prec]) < (1e-13 if prec == pf.FP64 else 1e-6)


@pytest.mark.parametrize("form", ["barrier", "dataflow"])
def test_wait_that_runs_out_returns_etimeout(pf, form):
    """Every device-side wait of the product is bounded; a 1 us bound runs out."""
    w = W.hexagon_8x8_n256()
    make = _flow_solver if form == "dataflow" else (lambda p, ww, **kw: p.Solver(ww, **kw))
    s = make(pf, w, wait_us=1)
    x = W.density_vector(w.E, 2)
    y = np.zeros_like(x)
    for _ in range(2):                  # the second product starts from cleared wait state
        with pytest.raises(pf.PfmbemError) as e:
            s.matvec(x, y, pf.MIXED)
        assert e.value.status == 7
    psi = np.zeros_like(x)
    with pytest.raises(pf.PfmbemError) as e:
        s.solve(psi, tol=1e-6, maxit=50)
    assert e.value.status == 7
    s.close()
    ok = make(pf, w)
    y2 = np.zeros_like(x)
    ok.matvec(x, y2, pf.FP64)
    ref = pf.Solver(w, launch=1)        # per-stage kernels: no device-wide waits
    y3 = np.zeros_like(x)
    ref.matvec(x, y3, pf.FP64)
    assert rel(y2, y3) < 1e-12
