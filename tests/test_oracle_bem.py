"""Pins for the oracle's constant-element BEM (CPU only).

* self-element integrals: the closed forms against adaptive quadrature of the
  defining integrals (log-weighted S; T as the limit of the normal derivative of
  the double-layer potential approached off the element) and the Laplace limit
  -2/(pi h) of the finite part;
* the whole formulation (eqs. 4-9) against the Mie series of an isolated fiber:
  the error falls at first order in h (ratio ~2 per doubling of N; constant-
  element collocation of the hypersingular T is first-order consistent);
* energy balance of the Bragg orders (lossless media) at the same rate;
* supercell invariance: two identical fibers stacked with period H equal one
  fiber with period H/2 and Bloch phase exp(i k (H/2) sin theta) -- an exact
  identity of the discrete systems;
* no contrast (k1 = k, rho = 1): no reflection up to discretisation error;
* the Mie series itself: the transmission conditions of eq. 2 on the circle.
"""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy import special as sp

from oracle import bem, mie
from paper_1910_10863_gb300 import workloads as W


def test_self_single_layer_matches_log_weighted_quadrature():
    kap, h = 7.3, 0.05
    S, _ = bem.self_integrals(kap, np.array([h]))
    a = h / 2
    # (i/4)H0 = (i/4)J0 - Y0/4, Y0 = (2/pi) J0 ln(x/2) + smooth
    re = 2 * integrate.quad(lambda s: -0.25 * sp.y0(kap * s), 0, a, epsabs=1e-16, epsrel=1e-13, limit=200)[0]
    im = 2 * integrate.quad(lambda s: 0.25 * sp.j0(kap * s), 0, a, epsabs=1e-16, epsrel=1e-13)[0]
    assert abs(S[0] - (re + 1j * im)) < 1e-12 * abs(S[0])


def test_self_hypersingular_is_limit_of_double_layer_normal_derivative():
    kap, h = 7.3, 0.05
    _, T = bem.self_integrals(kap, np.array([h]))
    a = h / 2

    def Tdelta(delta):
        # target x = (0, delta), element on the x-axis, normals (0, 1)
        def f(s, part):
            from oracle import greens
            d = greens.free_space(kap, np.array([-s]), np.array([delta]))
            _, _, _, t = greens.layer_kernels(d, (np.array([0.0]), np.array([1.0])), (np.array([0.0]), np.array([1.0])))
            return t[0].real if part == 0 else t[0].imag
        re = integrate.quad(f, -a, a, args=(0,), points=[0.0], epsabs=1e-14, epsrel=1e-13, limit=400)[0]
        im = integrate.quad(f, -a, a, args=(1,), points=[0.0], epsabs=1e-14, epsrel=1e-13, limit=400)[0]
        return re + 1j * im

    d1, d2 = 1e-5 * h, 0.5e-5 * h
    t1, t2 = Tdelta(d1), Tdelta(d2)
    assert abs(t2 - T[0]) < 1e-5 * abs(T[0])
    assert abs(t2 - T[0]) < abs(t1 - T[0])       # converging toward the closed form


def test_self_hypersingular_laplace_limit():
    h = 0.02
    _, T = bem.self_integrals(1e-7, np.array([h]))
    assert abs(T[0].real - (-2.0 / (math.pi * h))) < 1e-9 * (2.0 / (math.pi * h))


def test_mie_series_first_order_convergence():
    k, th, R = 3.0, 0.4, 0.5
    k1, rho = k * 1490 / 1450, 1000 / 13600
    pts = np.array([[1.2 * math.cos(t), 1.2 * math.sin(t)] for t in np.linspace(0, 2 * math.pi, 7, endpoint=False)])
    ref = mie.scattered(k, k1, rho, R, th, pts)
    errs = []
    for N in (32, 64, 128):
        pb = bem.problem(W.single_fiber(R, N, k, k1, rho, th), periodic=False)
        psi = bem.solve(pb)
        us = bem.potential(pb, psi, pts)
        errs.append(np.max(np.abs(us - ref)) / np.max(np.abs(ref)))
    assert errs[-1] < 0.02
    for e0, e1 in zip(errs[:-1], errs[1:]):
        assert 1.8 < e0 / e1 < 2.2


def test_energy_balance_converges():
    errs = []
    for N in (32, 64):
        pb = bem.problem(W.square_block(2, 2, 1.0, 0.3, N, 2.0, math.radians(30)))
        psi = bem.solve(pb)
        o, R, T = bem.rayleigh(pb, psi)
        errs.append(abs(1.0 - bem.energy(pb, o, R, T)))
    assert errs[1] < 2e-3
    assert 1.8 < errs[0] / errs[1] < 2.2


def test_supercell_invariance():
    H, kH, th, N, r = 1.0, 3.0, math.radians(20), 24, 0.12
    k = kH / H
    k1, rho = k * 1490 / 1450, 1000 / 13600
    one = W.single_fiber(r, N, k, k1, rho, th, centre=(0.3, 0.25), H=H / 2)
    two = W.Workload(name="two", H=H, lattice=0, k=k, k1=k1, rho_ratio=rho, theta=th,
                     nodes_per_fiber=np.array([N, N], dtype=np.int32),
                     nodes=np.concatenate([W.circle_nodes(0.3, 0.25, r, N), W.circle_nodes(0.3, 0.75, r, N)]))
    p1 = bem.problem(one)
    p2 = bem.problem(two)
    s1 = bem.solve(p1)
    s2 = bem.solve(p2)
    bloch = np.exp(1j * k * (H / 2) * math.sin(th))
    assert np.max(np.abs(s2[:2 * N] - s1)) < 1e-10 * np.max(np.abs(s1))
    assert np.max(np.abs(s2[2 * N:] - bloch * s1)) < 1e-10 * np.max(np.abs(s1))


def test_no_contrast_no_reflection():
    w = W.square_block(2, 2, 1.0, 0.3, 48, 2.0, math.radians(30))
    w.k1 = w.k
    w.rho_ratio = 1.0
    pb = bem.problem(w)
    psi = bem.solve(pb)
    o, R, T = bem.rayleigh(pb, psi)
    assert np.max(np.abs(R)) < 5e-3
    assert abs(abs(T[list(o).index(0)]) - 1.0) < 5e-3


def test_mie_series_satisfies_the_transmission_conditions():
    """u_inc + u^s = u_i and d/dr (u_inc + u^s) = rho d/dr u_i on r = R (eq. 2,
    rho = rho_matrix / rho_fiber), by central differences across the circle."""
    k, th, R = 3.0, 0.4, 0.5
    k1, rho = k * 1490 / 1450, 1000 / 13600
    ang = np.linspace(0, 2 * math.pi, 11, endpoint=False)

    def total(r):
        p = np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1)
        return np.exp(1j * k * (p @ np.array([math.cos(th), math.sin(th)]))) + mie.scattered(k, k1, rho, R, th, p)

    def inner(r):
        p = np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1)
        return mie.interior(k, k1, rho, R, th, p)

    assert np.max(np.abs(total(R) - inner(R))) < 1e-12
    e = 1e-5
    dout = (total(R + e) - total(R - e)) / (2 * e)
    din = (inner(R + e) - inner(R - e)) / (2 * e)
    assert np.max(np.abs(dout - rho * din)) < 1e-7 * np.max(np.abs(dout))


def test_mlp_oracle_gradient_matches_finite_differences():
    from oracle import mlp
    dims = [5, 7, 7, 3]
    rng = np.random.default_rng(3)
    _, n = mlp.layout(dims)
    p = rng.standard_normal(n) * 0.4
    X = rng.standard_normal((4, 5))
    T = rng.standard_normal((4, 3))
    _, g = mlp.loss_and_grad(p, dims, X, T)
    eps = 1e-6
    for i in rng.choice(n, size=25, replace=False):
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        fd = (mlp.loss_and_grad(pp, dims, X, T)[0] - mlp.loss_and_grad(pm, dims, X, T)[0]) / (2 * eps)
        assert abs(fd - g[i]) < 1e-7 * max(1.0, abs(g[i]))
