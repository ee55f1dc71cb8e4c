"""Pins of the dense oracle's quadrature and outputs (CPU only).

* Element integrals (``bem.pair_integrals``): every quadrature class against
  scipy's adaptive Gauss-Kronrod quadrature of the same kernels to 1e-13:
  adjacent elements, near elements (midpoint distance below 2h), same-fiber and
  other-fiber far elements, for the free-space kernel at k and k1 and for the
  quasi-periodic kernel, plus a pair across the period cell edge whose nearest
  image is m = -1 and the smooth image remainder on the self element.
* ETC (Sec. 4): with zero densities the field is the incident wave, so
  ETC = cos(theta) exactly; and ETC from the Rayleigh series equals ETC from
  du/dx1 of the spatial (Ewald) representation of eq. 7 at the same points.
* The periodic field of eq. 7: quasi-periodic, u(x + h) = alpha u(x), and equal
  to the Rayleigh (plane-wave) expansion on either side of the block.
* The quadtree rule (Sec. 3.1) and Table 1: the worst gamma, lambda, tau over
  the M2L pairs of the symmetric square tree are the printed L = 0 column; the
  asymmetric columns from the cell geometry of Theorems 1-2.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import bem, greens, tree
from paper_1910_10863_gb300 import workloads as W


@pytest.fixture(scope="module")
def c1():
    w = W.square_2x2_n64()
    return w, bem.problem(w)


def _adaptive(pb, ker, ti, sj, lo=0.0, hi=1.0):
    el = pb.el
    x, nx, ny = el.c[ti], el.nu[ti], el.nu[sj]
    a, b, h = el.a[sj], el.b[sj], el.h[sj]

    def f(s):
        y = a + (b - a) * s
        z1 = np.array([x[0] - y[0]])
        z2 = np.array([x[1] - y[1]])
        if ker.periodic:
            d = greens.qp_ewald(ker.kappa, ker.beta, ker.H, z1, z2)
        else:
            d = greens.free_space(ker.kappa, z1, z2)
        v = np.array([complex(q[0]) for q in greens.layer_kernels(d, (nx[0], nx[1]), (ny[0], ny[1]))]) * h
        return np.concatenate([v.real, v.imag])

    r, _ = integrate.quad_vec(f, lo, hi, epsabs=0, epsrel=1e-14, limit=2000)
    return r[:4] + 1j * r[4:]


def _pairs(pb):
    el = pb.el
    ti = 5
    d = np.hypot(el.c[:, 0] - el.c[ti, 0], el.c[:, 1] - el.c[ti, 1])
    near = [j for j in range(el.E) if abs(j - ti) > 1 and el.fiber[j] == el.fiber[ti] and d[j] < 2 * el.h[j]]
    assert near
    other = int(np.nonzero(el.fiber != el.fiber[ti])[0][0])
    return ti, {"adjacent": ti + 1, "near": near[0], "same-fiber far": ti + 20, "other fiber": other}


@pytest.mark.parametrize("which", ["k", "k1", "periodic"])
def test_pair_integrals_match_adaptive_quadrature(c1, which):
    _, pb = c1
    if which == "periodic":
        ker = bem.Kernel(pb.k, periodic=True, beta=pb.beta, H=pb.H)
    else:
        ker = bem.Kernel(pb.k if which == "k" else pb.k1, periodic=False)
    ti, pairs = _pairs(pb)
    for cls, sj in pairs.items():
        got = np.array(bem.pair_integrals(ker, pb.el, [ti], [sj]))[:, 0]
        ref = _adaptive(pb, ker, ti, sj)
        assert np.all(np.abs(got - ref) <= 1e-13 * np.abs(ref) + 1e-15), (cls, got, ref)


def test_pair_integrals_across_the_period_edge(c1):
    """Target at the bottom of the lower-left fiber (y ~ 0.1), source at the top of the
    upper-left fiber (y ~ 0.9): the nearest image of the source is m = -1."""
    _, pb = c1
    el = pb.el
    ker = bem.Kernel(pb.k, periodic=True, beta=pb.beta, H=pb.H)
    left_low = (np.abs(el.c[:, 0] - 0.25) < 0.2) & (el.c[:, 1] < 0.5)
    left_high = (np.abs(el.c[:, 0] - 0.25) < 0.2) & (el.c[:, 1] > 0.5)
    ti = int(np.nonzero(left_low)[0][np.argmin(el.c[left_low, 1])])
    sj = int(np.nonzero(left_high)[0][np.argmax(el.c[left_high, 1])])
    assert np.rint((el.c[ti, 1] - el.c[sj, 1]) / pb.H) == -1
    got = np.array(bem.pair_integrals(ker, el, [ti], [sj]))[:, 0]
    ref = _adaptive(pb, ker, ti, sj)
    assert np.all(np.abs(got - ref) <= 1e-13 * np.abs(ref) + 1e-15)


def test_self_element_image_remainder(c1):
    """Periodic minus free-space self integrals = the smooth image remainder
    G_qp - Phi over the element, against a 24-node Gauss rule (even, so no node sits
    at the collocation point) of the remainder evaluated directly."""
    _, pb = c1
    el = pb.el
    e = 10
    kq = bem.Kernel(pb.k, periodic=True, beta=pb.beta, H=pb.H)
    kf = bem.Kernel(pb.k, periodic=False)
    got = np.array(bem.pair_integrals(kq, el, [e], [e]))[:, 0] - np.array(bem.pair_integrals(kf, el, [e], [e]))[:, 0]
    u, w = np.polynomial.legendre.leggauss(24)
    s = 0.5 * u * el.h[e]
    z1 = -s * el.t[e, 0]
    z2 = -s * el.t[e, 1]
    g = greens.qp_ewald(pb.k, pb.beta, pb.H, z1, z2)
    f = greens.free_space(pb.k, z1, z2)
    rem = {key: g[key] - f[key] for key in g}
    nu = (np.full(24, el.nu[e, 0]), np.full(24, el.nu[e, 1]))
    k4 = greens.layer_kernels(rem, nu, nu)
    ref = np.array([np.sum(0.5 * w * el.h[e] * kk) for kk in k4])
    # S, D, K: the remainder is smooth, 1e-13; T: the direct remainder loses digits to
    # cancellation against 1/r^2 at the Gauss nodes nearest the midpoint
    assert np.all(np.abs(got[:3] - ref[:3]) <= 1e-13 * np.abs(ref[:3]) + 1e-15)
    assert abs(got[3] - ref[3]) <= 1e-9 * abs(ref[3])


def test_etc_of_the_incident_wave_is_cos_theta(c1):
    _, pb = c1
    psi = np.zeros(2 * pb.el.E, dtype=np.complex128)
    assert abs(bem.etc(pb, psi, npts=64, x1=1.0) - math.cos(pb.theta)) < 1e-14


@pytest.fixture(scope="module")
def c1_solution(c1):
    _, pb = c1
    return bem.solve(pb)


def test_etc_rayleigh_equals_spatial_field(c1, c1_solution):
    _, pb = c1
    psi = c1_solution
    npts = 48
    x2 = bem.etc_points(pb, npts)
    pts = np.stack([np.full(npts, 1.0), x2], axis=1)
    _, dus = bem.potential(pb, psi, pts, grad=True)
    d = np.array([math.cos(pb.theta), math.sin(pb.theta)])
    du_inc = 1j * pb.k * d[0] * np.exp(1j * pb.k * (pts @ d))
    spatial = float(np.mean(np.abs(du_inc + dus)) / pb.k)
    ray = bem.etc(pb, psi, nmax=60, npts=npts, x1=1.0)
    assert abs(ray - spatial) < 1e-10 * spatial


def test_periodic_field_is_quasi_periodic_and_matches_rayleigh_expansion(c1, c1_solution):
    _, pb = c1
    psi = c1_solution
    rng = np.random.default_rng(2)
    right = np.stack([rng.uniform(1.0, 1.3, 4), rng.uniform(-0.5, 1.5, 4)], axis=1)
    left = np.stack([rng.uniform(-0.3, 0.0, 4), rng.uniform(-0.5, 1.5, 4)], axis=1)
    alpha = np.exp(1j * pb.beta)
    u = bem.potential(pb, psi, np.concatenate([right, left]))
    u_up = bem.potential(pb, psi, np.concatenate([right, left]) + [0.0, pb.H])
    assert np.max(np.abs(u_up - alpha * u)) < 1e-12 * np.max(np.abs(u))
    orders = np.arange(-60, 61)
    o, R, T = bem.rayleigh(pb, psi, orders)
    ky = pb.k * math.sin(pb.theta) + 2 * math.pi * o / pb.H
    kx = np.sqrt((pb.k**2 - ky**2).astype(np.complex128))
    ur = np.array([np.sum((T - (o == 0)) * np.exp(1j * (kx * x[0] + ky * x[1]))) for x in right])
    ul = np.array([np.sum(R * np.exp(1j * (-kx * x[0] + ky * x[1]))) for x in left])
    assert np.max(np.abs(ur - u[:4])) < 1e-10 * np.max(np.abs(u))
    assert np.max(np.abs(ul - u[4:])) < 1e-10 * np.max(np.abs(u))


def test_table1_symmetric_square_tree_from_the_interaction_lists():
    """L = 0 column: the worst M2L pair of the tree rule (levels 3 and 4)."""
    for level in (3, 4):
        g, lam, tau = tree.symmetric_tree_factors(level)
        assert (round(g, 4), round(lam, 4), round(tau, 4)) == (0.4714, 0.6009, 0.6009)


@pytest.mark.parametrize("L,offset,size_c,gamma,lam", [
    (1, (2.5, 0.5), 2.0, 0.7071, 0.6374),
    (2, (3.5, 0.5), 4.0, 0.9428, 0.6640),
])
def test_table1_asymmetric_square_tree(L, offset, size_c, gamma, lam):
    """L > 0: the source cell is 2^L times the target cell; its nearest admissible
    position leaves one target side between them."""
    g, l = tree.gamma_lambda(offset, size_c)
    assert round(g, 4) == gamma
    assert round(l, 4) == lam
    assert round(max(g, l), 4) == max(gamma, lam)


def test_interaction_list_counts():
    """27 sources for an interior box (6 x 6 children of the parent's neighbourhood
    minus its own 3 x 3), fewer at the x edges, 27 at the y edges (images)."""
    assert len(tree.interaction_list(4, 7, 7)) == 27
    assert len(tree.interaction_list(4, 7, 0)) == 27
    assert len(tree.interaction_list(4, 0, 7)) == 18
    assert all(m in (-1, 0, 1) for _, _, m in tree.interaction_list(4, 5, 15))


def test_triangle_tree_geometry():
    """The regular-triangle tree of Sec. 3.1 (Fig. 5): each cell of side 2 holds
    exactly four cells of side 1 (its three corner children and the inverted
    middle one), which cover its area; the circumradius is s / sqrt(3)."""
    from collections import Counter
    cells = [(i, j, up) for i in range(-4, 4) for j in range(-4, 4) for up in (True, False)]
    kids = Counter(tree.triangle_parent(c) for c in cells)
    inner = [p for p in kids if all(-1 <= x <= 0 for x in p[:2])]
    assert inner and all(kids[p] == 4 for p in inner)
    v = tree.triangle_vertices(0, 0, True, 1.0)
    o = tree.triangle_centre(v)
    assert all(abs(math.hypot(p[0] - o[0], p[1] - o[1]) - 1 / math.sqrt(3)) < 1e-14 for p in v)
    assert tree.triangle_parent((0, 0, False)) == (0, 0, True)        # the middle child


def test_table1_triangular_tree():
    """Table 1, triangular tree columns.  L = 0: lambda 0.6663 is the worst of the
    interaction list (the opposite-orientation sources whose centres lie sqrt(7/3)
    sides away); gamma 0.4000 is that of the nearest same-orientation source of
    the list (centres sqrt(3) sides apart).  L = 1: a source one level up, touching
    the target's parent, and the parent's middle child as the target: gamma
    0.7559 and lambda 0.6863."""
    for D in [(0, 0, True), (0, 0, False)]:
        lst = tree.triangle_interaction_list(D)
        lam = max(tree.triangle_gamma_lambda(c, 1.0, D, 1.0)[1] for c in lst)
        assert round(lam, 4) == 0.6663
    assert (1, 1, True) in tree.triangle_interaction_list((0, 0, True))
    g, _ = tree.triangle_gamma_lambda((1, 1, True), 1.0, (0, 0, True), 1.0)
    assert round(g, 4) == 0.4000
    g, lam = tree.triangle_gamma_lambda((1, 0, True), 2.0, (0, 0, False), 1.0)
    assert (round(g, 4), round(lam, 4)) == (0.7559, 0.6863)
