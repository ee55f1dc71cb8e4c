"""The regular-triangle quadtree for hexagon lattices (Sec. 3.1, Fig. 5): every
fiber in the hexagonal cell of its lattice point, the cell split into six
triangles and each triangle into four, neighbours where cells or triangles
touch.  Against the dense CPU oracle, which has no tree: the FP64 product (with
cached element integrals, and with the integrals in every product) on random and
smooth densities at several depths, the solution, the Bragg coefficients and
ETC; on a larger hexagon block and on Table 3's hexagon rows against the square
tree; and the geometry the tree rejects."""
import math

import numpy as np
import pytest

from oracle import bem
from paper_1910_10863_gb300 import workloads as W
from tests.gpu_common import ensure_built, rel

pytestmark = pytest.mark.gpu


def hexagon(ncol, nrow, n, kH, theta_deg, seed, H=1.0):
    w = W.hexagon_block(ncol, nrow, H, n, kH, math.radians(theta_deg), seed,
                        name=f"tri_hexagon_{ncol}x{nrow}_n{n}_kH{kH:g}")
    lattice = dict(tree=1, **W.hexagon_block_lattice(H, nrow))
    return w, lattice


CASES = [
    # (workload args, extra options); near_mode 1: the element integrals in every product
    ((3, 2, 32, 3.0, 20.0, 5), {}),
    ((3, 2, 32, 3.0, 20.0, 5), {"depth": 2}),
    ((2, 3, 40, 4.5, 35.0, 6), {"depth": 3}),
    ((2, 3, 40, 4.5, 35.0, 6), {"depth": 3, "near_mode": 1}),
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


@pytest.mark.parametrize("args,opts", CASES)
def test_triangle_tree_product(pf, args, opts):
    w, lat = hexagon(*args)
    pb, A, B, psi = oracle(w)
    s = pf.Solver(w, **lat, **opts)
    plan = pf.pfmbem_plan(s.h)
    assert plan.nroot == w.M and plan.super_p >= plan.p[0] and plan.cached == 0
    if "depth" in opts:
        assert plan.depth == opts["depth"]
    assert plan.m2l_pairs > 0 or plan.depth == 1
    rng = np.random.default_rng(7)
    x = rng.standard_normal(2 * s.E) + 1j * rng.standard_normal(2 * s.E)
    for v in (x, psi):
        v = np.ascontiguousarray(v)
        ref = A @ v
        y = np.zeros_like(v)
        s.matvec(v, y, pf.FP64)
        assert rel(y, ref) < 1e-8, rel(y, ref)
    s.close()


@pytest.mark.parametrize("args,opts", CASES[1:])
def test_triangle_tree_solution_coefficients_etc(pf, args, opts):
    w, lat = hexagon(*args)
    pb, A, B, psi_ref = oracle(w)
    s = pf.Solver(w, **lat, **opts)
    psi = np.zeros(2 * s.E, dtype=np.complex128)
    info = s.solve(psi, tol=1e-10, maxit=2000)
    assert info.rel_residual <= 1e-10
    assert rel(psi, psi_ref) < 1e-6
    orders, R, T, energy = pf.pfmbem_coefficients(s.h, psi)
    ordr, Rr, Tr = bem.rayleigh(pb, psi_ref, np.asarray(orders))
    assert np.max(np.abs(np.asarray(R) - Rr)) < 1e-6 and np.max(np.abs(np.asarray(T) - Tr)) < 1e-6
    a = w.H / args[1]
    x1 = float(np.max(w.centres[:, 0]) + 0.5 * a)       # right of the last column of cells
    e_gpu = pf.pfmbem_etc(s.h, psi, x1, 256)
    e_ref = bem.etc(pb, psi_ref, npts=256, x1=x1)
    assert abs(e_gpu - e_ref) < 1e-6, (e_gpu, e_ref)
    s.close()


def test_triangle_tree_against_square_tree_on_a_larger_block(pf):
    # 4 x 4 cells, 96 elements each (1536 elements), triangle tree of depth 2:
    # both trees' FP64 solutions to 1e-11 agree to the FMM truncation of either
    w, lat = hexagon(4, 4, 96, 6.0, 25.0, 11)
    st = pf.Solver(w, depth=2, **lat)
    sq = pf.Solver(w)
    assert pf.pfmbem_plan(st.h).depth == 2
    p_t = np.zeros(2 * st.E, dtype=np.complex128)
    p_s = np.zeros(2 * sq.E, dtype=np.complex128)
    i_t = st.solve(p_t, tol=1e-11, maxit=3000)
    i_s = sq.solve(p_s, tol=1e-11, maxit=3000)
    assert i_t.rel_residual <= 1e-11 and i_s.rel_residual <= 1e-11
    assert rel(p_t, p_s) < 1e-7, rel(p_t, p_s)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(2 * st.E) + 1j * rng.standard_normal(2 * st.E)
    y_t = np.zeros_like(x)
    y_s = np.zeros_like(x)
    st.matvec(x, y_t, pf.FP64)
    sq.matvec(x, y_s, pf.FP64)
    assert rel(y_t, y_s) < 1e-8, rel(y_t, y_s)
    st.close()
    sq.close()


def test_triangle_tree_rejections(pf):
    w, lat = hexagon(3, 2, 32, 3.0, 20.0, 5)
    # no lattice spacing
    with pytest.raises(pf.PfmbemError) as e:
        pf.Solver(w, tree=1)
    assert e.value.status == 1
    # a lattice whose cells do not hold the fibers (origin moved by half a spacing)
    bad = dict(lat, tri_oy=lat["tri_oy"] + 0.5 * lat["tri_a"])
    with pytest.raises(pf.PfmbemError) as e:
        pf.Solver(w, **bad)
    assert e.value.status == 2
    # a period that is not a multiple of the spacing
    bad = dict(lat, tri_a=lat["tri_a"] * 1.1)
    with pytest.raises(pf.PfmbemError) as e:
        pf.Solver(w, **bad)
    assert e.value.status == 2
    # the batched solver takes square-tree handles only
    s = pf.Solver(w, **lat)
    psi = np.zeros(2 * s.E, dtype=np.complex128)
    st, _ = pf.pfmbem_solve_batch([s.h], [psi], 1e-6, 100)
    assert st == 1
    s.close()


@pytest.mark.parametrize("fill,ka,stop", [(0.35, 0.45, True), (0.35, 0.12, False), (0.50, 0.52, True),
                                          (0.50, 0.12, False)])
def test_triangle_tree_table3_hexagon_rows(pf, fill, ka, stop):
    """Table 3's circular scatterers in the hexagon lattice, solved on the tree the
    paper builds for that lattice: ETC on the block's right edge equals the square
    tree's to 1e-6, below 3 % inside the first stop band and above it below."""
    w = W.table3_block(ka, fill, "hexagon", "circular")
    x1 = 4 * 0.5 * 3 ** 0.5 / 2
    etc = []
    for opts in (dict(tree=1, **W.table3_hexagon_lattice()), {}):
        s = pf.Solver(w, **opts)
        psi = np.zeros(2 * s.E, dtype=np.complex128)
        info = s.solve(psi, tol=1e-9, maxit=3000)
        assert info.rel_residual <= 1e-9
        etc.append(pf.pfmbem_etc(s.h, psi, x1, 256))
        s.close()
    assert abs(etc[0] - etc[1]) < 1e-6, etc
    assert (etc[0] < 0.03) == stop, etc
