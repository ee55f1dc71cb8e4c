"""GPU (C-ABI) against the CPU oracle on the same seeded inputs.

Tolerances: FP64 matvec relative L2 error <= 1e-8 and solved densities <= 1e-6
relative (the plain-method targets); self-element integrals and the incident
right-hand side to rounding; lattice sums on the local expansion they generate
(coefficient j weighted by |J_j(k rho)|, rho = 0.75 H) to 1e-10.

Matvecs are checked on two kinds of density: seeded random vectors, whose
products are dominated by the near-field and same-fiber blocks, and smooth
physical densities (the incident right-hand side, the solution), whose products
also expose the far field's truncation.  The mixed (FP32) product is held to
2e-6 on both.  On smooth densities the hypersingular same-fiber operator sums
terms of size ~1/h that cancel to O(1); the product therefore sums the near
field in differences psi_j - psi_t of hi + lo densities (row sums in FP64) and
runs the same-fiber FFTs in FP64 (plain FP32 sums left ~5e-5 there).
"""
import math

import numpy as np
import pytest
from scipy import special as sp

from oracle import bem, lattice
from paper_1910_10863_gb300 import workloads as W
from tests.gpu_common import ensure_built, hexagon_4x4_ragged, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    ensure_built()
    from paper_1910_10863_gb300 import pfmbem
    return pfmbem


_cache = {}


def oracle_system(w):
    if w.name not in _cache:
        pb = bem.problem(w)
        _cache[w.name] = (pb, bem.operator_rows(pb), bem.rhs(pb))
    return _cache[w.name]


SMALL = [W.square_2x2_n64, hexagon_4x4_ragged]
MIXED_SMOOTH = 2e-6


@pytest.mark.parametrize("make", SMALL)
def test_self_terms(pf, make):
    w = make()
    s = pf.Solver(w)
    out = np.zeros(4 * s.E, dtype=np.complex128)
    pf.pfmbem_self_terms(s.h, out)
    el = bem.elements(w.nodes, w.nodes_per_fiber)
    Sk, Tk = bem.self_integrals(w.k, el.h)
    S1, T1 = bem.self_integrals(w.k1, el.h)
    got = out.reshape(-1, 4)
    for col, ref in enumerate((Sk, Tk, S1, T1)):
        assert np.max(np.abs(got[:, col] - ref) / np.abs(ref)) < 1e-12


@pytest.mark.parametrize("kH,theta,jmax,rho", [(2.0, math.radians(30), 24, 0.75), (5.0, 0.3, 24, 0.75),
                                                (20.0, math.radians(30), 24, 0.75),
                                                (20.0, math.radians(30), 108, 1.9),
                                                (5.0, 0.3, 64, 1.9)])
def test_lattice_sums(pf, kH, theta, jmax, rho):
    """jmax = 108 is the largest order the 32x32 block's root translation uses
    (2 p0 at kH = 20); on the circle rho = 1.9 H every order up to it carries
    weight, so each one is checked, not only the low ones."""
    w = W.square_2x2_n64()
    w.k = kH / w.H
    w.k1 = w.k * 1490 / 1450
    w.theta = theta
    s = pf.Solver(w, p=12, depth=2)
    S = np.zeros(2 * jmax + 1, dtype=np.complex128)
    pf.pfmbem_lattice_sums(s.h, jmax, S)
    js, ref = lattice.lattice_sums(w.k, w.k * w.H * math.sin(theta), w.H, jmax, rho=rho * w.H,
                                   npts=8192 if rho > 1 else None)
    wgt = np.abs(sp.jv(js, w.k * rho * w.H))
    err = np.max(np.abs(S - ref) * wgt) / np.max(np.abs(ref) * wgt)
    assert err < 1e-10, err


@pytest.mark.parametrize("make", SMALL)
def test_rhs(pf, make):
    w = make()
    s = pf.Solver(w)
    B = np.zeros(2 * s.E, dtype=np.complex128)
    s.rhs(B)
    _, _, Bo = oracle_system(w)
    assert rel(B, Bo) < 1e-13


@pytest.mark.parametrize("make", SMALL)
def test_matvec_fp64_matches_dense_oracle(pf, make):
    import torch
    w = make()
    s = pf.Solver(w)
    _, Mo, _ = oracle_system(w)
    for seed in (1, 2):
        x = W.density_vector(s.E, seed)
        y_ref = Mo @ x
        xd = torch.from_numpy(x).cuda()
        yd = torch.zeros_like(xd)
        s.matvec(xd, yd)
        torch.cuda.synchronize()
        assert rel(yd.cpu().numpy(), y_ref) < 1e-8
    # host buffers give the same result
    yh = np.zeros_like(x)
    s.matvec(x, yh)
    assert rel(yh, y_ref) < 1e-8
    # the physical density: the dense solution of the block
    pb, _, Bo = oracle_system(w)
    psi = np.linalg.solve(Mo, Bo)
    y = np.zeros_like(psi)
    s.matvec(psi, y)
    assert rel(y, Bo) < 1e-8
    s.matvec(psi, y, pf.MIXED)
    assert rel(y, Bo) < MIXED_SMOOTH


@pytest.mark.parametrize("make", SMALL)
def test_solve_fp64_matches_dense_lu(pf, make):
    w = make()
    s = pf.Solver(w)
    pb, Mo, Bo = oracle_system(w)
    psi_ref = np.linalg.solve(Mo, Bo)
    psi = np.zeros(2 * s.E, dtype=np.complex128)
    info = s.solve(psi, tol=1e-10, maxit=500)
    assert info.rel_residual <= 1e-10
    assert rel(psi, psi_ref) < 1e-6


def test_invalid_inputs_rejected(pf):
    w = W.square_2x2_n64()
    cw = w.nodes.copy()
    cw[:64] = cw[:64][::-1]          # first fiber clockwise
    with pytest.raises(pf.PfmbemError) as e:
        pf.pfmbem_create(w.M, w.nodes_per_fiber, cw, w.H, 0, w.k, w.k1, w.rho_ratio, w.theta)
    assert e.value.status == 2
    # exactly at a Wood anomaly: kH(1 + sin theta) = 2 pi
    th = math.asin(2 * math.pi / (w.k * w.H) - 1) if w.k * w.H > math.pi else None
    kH = 2 * math.pi / (1 + math.sin(math.radians(30)))
    with pytest.raises(pf.PfmbemError) as e:
        pf.pfmbem_create(w.M, w.nodes_per_fiber, w.nodes, w.H, 0, kH / w.H, kH / w.H, w.rho_ratio,
                         math.radians(30))
    assert e.value.status == 3
    del th


@pytest.mark.parametrize("make", SMALL)
@pytest.mark.parametrize("m2l_mode", [1, 2])
def test_matvec_mixed_matches_dense_oracle(pf, make, m2l_mode):
    w = make()
    s = pf.Solver(w, m2l_mode=m2l_mode)
    _, Mo, _ = oracle_system(w)
    x = W.density_vector(s.E, 4)
    y = np.zeros_like(x)
    s.matvec(x, y, pf.MIXED)
    assert rel(y, Mo @ x) < 2e-6


@pytest.mark.parametrize("make", SMALL)
def test_solve_mixed_refined_matches_dense_lu(pf, make):
    w = make()
    s = pf.Solver(w, precision=pf.MIXED)
    pb, Mo, Bo = oracle_system(w)
    psi_ref = np.linalg.solve(Mo, Bo)
    psi = np.zeros(2 * s.E, dtype=np.complex128)
    info = s.solve(psi, tol=1e-8, maxit=500)
    assert info.rel_residual <= 1e-8          # FP64 true residual after refinement
    assert info.restarts >= 1                 # at least one refinement step ran
    assert rel(psi, psi_ref) < 1e-6


def test_matvec_uncached_fp64(pf):
    w = hexagon_4x4_ragged()
    s = pf.Solver(w, near_mode=1)
    _, Mo, _ = oracle_system(w)
    x = W.density_vector(s.E, 5)
    y = np.zeros_like(x)
    s.matvec(x, y)
    assert rel(y, Mo @ x) < 1e-8


@pytest.mark.parametrize("make", SMALL)
def test_bragg_coefficients_and_field(pf, make):
    w = make()
    s = pf.Solver(w)
    pb, Mo, Bo = oracle_system(w)
    psi = np.linalg.solve(Mo, Bo)
    orders, R, T, energy = pf.pfmbem_coefficients(s.h, psi)
    o_ref, R_ref, T_ref = bem.rayleigh(pb, psi)
    assert list(orders) == list(o_ref)
    assert np.max(np.abs(R - R_ref)) < 1e-10 and np.max(np.abs(T - T_ref)) < 1e-10
    assert abs(energy - bem.energy(pb, o_ref, R_ref, T_ref)) < 1e-10
    # scattered field at points between the fibers and beside the block
    el = bem.elements(w.nodes, w.nodes_per_fiber)
    xmid = 0.5 * (el.a[:, 0].min() + el.a[:, 0].max())
    pts = np.array([[xmid, el.c[:, 1].min() - 0.02], [el.a[:, 0].max() + 0.05, 0.3],
                    [el.a[:, 0].min() - 0.05, 0.7], [xmid, el.c[:, 1].max() + 1.37]])
    u = np.zeros(len(pts), dtype=np.complex128)
    pf.pfmbem_field(s.h, psi, pts, u)
    u_ref = bem.potential(pb, psi, pts)
    assert np.max(np.abs(u - u_ref)) < 1e-8 * np.max(np.abs(u_ref))


def test_full_size_hexagon_rows(pf):
    """hexagon 8x8, 256 elements per fiber (16384 elements): sampled rows of the
    FP64 and the mixed matvec against rows of the dense oracle operator."""
    w = W.hexagon_8x8_n256()
    s = pf.Solver(w)
    x = W.density_vector(s.E, 6)
    y64 = np.zeros_like(x)
    y32 = np.zeros_like(x)
    s.matvec(x, y64, pf.FP64)
    s.matvec(x, y32, pf.MIXED)
    rng = np.random.default_rng(0)
    rows_e = np.sort(rng.choice(s.E, size=6, replace=False))
    rows_e[0] = 0                        # first element of the first fiber
    rows_e[-1] = s.E - 1                 # last element of the last fiber
    pb = bem.problem(w)
    Mr = bem.operator_rows(pb, rows_e)
    ref = Mr @ x
    idx = np.ravel(np.stack([2 * rows_e, 2 * rows_e + 1], axis=1))
    assert rel(y64[idx], ref) < 1e-8
    assert rel(y32[idx], ref) < 2e-6
    _smooth_rows(pf, s, pb, Mr, idx)


def _smooth_rows(pf, s, pb, Mr, idx):
    """The incident right-hand side as a smooth density on the same sampled rows."""
    xs = bem.rhs(pb)
    ref = Mr @ xs
    y64 = np.zeros_like(xs)
    y32 = np.zeros_like(xs)
    s.matvec(xs, y64, pf.FP64)
    s.matvec(xs, y32, pf.MIXED)
    assert rel(y64[idx], ref) < 1e-8
    assert rel(y32[idx], ref) < MIXED_SMOOTH


def test_tensor_core_m2l_matches_cuda_core_m2l(pf):
    """Mixed matvec with the tcgen05 BF16x3 M2L against the FP32 CUDA-core M2L and
    the FP64 matvec on the full-size hexagon block (the small blocks check both
    M2L engines against the dense oracle in test_matvec_mixed_matches_dense_oracle)."""
    w = W.hexagon_8x8_n256()
    st = pf.Solver(w, m2l_mode=2)      # tensor cores
    sc = pf.Solver(w, m2l_mode=1)      # CUDA cores
    x = W.density_vector(st.E, 8)
    yt = np.zeros_like(x)
    yc = np.zeros_like(x)
    y64 = np.zeros_like(x)
    st.matvec(x, yt, pf.MIXED)
    sc.matvec(x, yc, pf.MIXED)
    st.matvec(x, y64, pf.FP64)
    assert rel(yc, y64) < 2e-6
    assert rel(yt, y64) < 2e-6


def test_round_square_scatterers_full_fiber_blocks(pf):
    """Round-square scatterers (Sec. 4) are not regular polygons, so their
    same-fiber blocks are stored in full (the circles use the circulant form)."""
    w = W.round_square_block(2, 2, 1.0, 0.35, 40, 2.5, math.radians(20))
    pb = bem.problem(w)
    Mo = bem.operator_rows(pb)
    x = W.density_vector(w.E, 12)
    s = pf.Solver(w)
    assert s.plan().fiber_entries == 4 * (2 * 40) ** 2
    for prec, tol in ((pf.FP64, 1e-8), (pf.MIXED, 2e-6)):
        y = np.zeros_like(x)
        s.matvec(x, y, prec)
        assert rel(y, Mo @ x) < tol


def test_full_size_square_32x32_rows(pf):
    """square 32x32, 128 elements per fiber (131072 elements, kH = 20, level-
    dependent orders up to the root): sampled rows of the FP64 and mixed matvecs
    against rows of the dense oracle operator."""
    w = W.square_32x32_n128()
    s = pf.Solver(w)
    plan = s.plan()
    assert plan.p[0] > plan.p[plan.depth]          # orders grow toward the root at kH = 20
    x = W.density_vector(s.E, 7)
    y64 = np.zeros_like(x)
    y32 = np.zeros_like(x)
    s.matvec(x, y64, pf.FP64)
    s.matvec(x, y32, pf.MIXED)
    rng = np.random.default_rng(1)
    rows_e = np.sort(rng.choice(s.E, size=4, replace=False))
    pb = bem.problem(w)
    Mr = bem.operator_rows(pb, rows_e)
    ref = Mr @ x
    idx = np.ravel(np.stack([2 * rows_e, 2 * rows_e + 1], axis=1))
    assert rel(y64[idx], ref) < 1e-8
    assert rel(y32[idx], ref) < 2e-6
    _smooth_rows(pf, s, pb, Mr, idx)


@pytest.mark.parametrize("make", SMALL + [W.hexagon_8x8_n256])
def test_single_launch_matvec_matches_per_stage_kernels(pf, make):
    """The cooperative single-launch matvec (default) against the one-kernel-per-
    stage path on the same cached operators: FP64 to rounding, mixed to the
    FP32 reordering of the M2L sums."""
    w = make()
    sf = pf.Solver(w)
    ss = pf.Solver(w, launch=1)
    x = W.density_vector(sf.E, 13)
    for prec, tol in ((pf.FP64, 1e-12), (pf.MIXED, 1e-5)):
        yf = np.zeros_like(x)
        ys = np.zeros_like(x)
        sf.matvec(x, yf, prec)
        ss.matvec(x, ys, prec)
        assert rel(yf, ys) < tol


def _two_fibers_across_the_period():
    """Two small circles centred 0.03 above the bottom and 0.03 below the top of
    the period: the root box is [0, 1) in y, so each fiber straddles it and
    part of its elements are wrapped by one period (phase alpha^-m0)."""
    nodes = np.concatenate([W.circle_nodes(0.3, 0.03, 0.04, 48), W.circle_nodes(0.7, 0.97, 0.04, 40)])
    return W.Workload(name="wrapped_pair", H=1.0, lattice=0, k=3.0, k1=3.0 * 1490 / 1450, rho_ratio=1000 / 13600,
                      theta=0.4, nodes_per_fiber=np.array([48, 40], dtype=np.int32), nodes=nodes)


@pytest.mark.parametrize("make", [_two_fibers_across_the_period,
                                  lambda: W.single_fiber(0.2, 32, 4.0, 4.0 * 1490 / 1450, 1000 / 13600, 0.7,
                                                         centre=(0.5, 0.5))])
def test_wrapped_and_single_fiber_blocks(pf, make):
    """Degenerate and boundary cases of the tree: fibers cut by the root box
    (elements wrapped into it) and a block of one fiber; both matvec paths and
    both precisions against the dense oracle."""
    w = make()
    pb = bem.problem(w)
    Mo = bem.operator_rows(pb)
    x = W.density_vector(w.E, 21)
    for launch in (0, 1):
        s = pf.Solver(w, launch=launch)
        for prec, tol in ((pf.FP64, 1e-8), (pf.MIXED, 2e-6)):
            y = np.zeros_like(x)
            s.matvec(x, y, prec)
            assert rel(y, Mo @ x) < tol, (launch, prec)
        psi = np.zeros_like(x)
        info = s.solve(psi, tol=1e-9, maxit=400)
        assert info.rel_residual <= 1e-9
        assert rel(psi, np.linalg.solve(Mo, bem.rhs(pb))) < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("make", SMALL)
def test_block_jacobi_preconditioner_same_solution_fewer_iterations(pf, prec, make):
    """The right block-Jacobi preconditioner (inverse same-fiber blocks, by FFT for
    2^j elements and as a circulant row pair otherwise) changes the iteration
    count, not the solution: both solves match dense LU."""
    w = make()
    pb, Mo, Bo = oracle_system(w)
    psi_ref = np.linalg.solve(Mo, Bo)
    p = pf.FP64 if prec == "fp64" else pf.MIXED
    res = {}
    for pc in (0, 1):
        s = pf.Solver(w, precision=p, precond=pc)
        psi = np.zeros(2 * s.E, dtype=np.complex128)
        info = s.solve(psi, tol=1e-8, maxit=500)
        assert info.rel_residual <= 1e-8
        assert rel(psi, psi_ref) < 1e-6
        res[pc] = info.iters
    assert res[0] < res[1], res


def test_block_jacobi_full_size_hexagon(pf):
    w = W.hexagon_8x8_n256()
    its = {}
    for pc in (0, 1):
        s = pf.Solver(w, precision=pf.MIXED, precond=pc)
        psi = np.zeros(2 * s.E, dtype=np.complex128)
        info = s.solve(psi, tol=1e-6)
        assert info.rel_residual <= 1e-6
        its[pc] = (info.iters, psi)
    assert its[0][0] < its[1][0]
    assert rel(its[0][1], its[1][1]) < 2e-4          # two solutions at residual 1e-6
