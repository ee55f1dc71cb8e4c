"""High-order Nystrom discretisation of the Kress transmission system on circles.

Test infrastructure (FP64 numpy/scipy), used only to pin the physics of the
formulation at tolerances the constant elements of ``bem`` cannot reach: the
Mie series of an isolated fiber, energy balance of the Bragg orders and the
no-contrast case.  It discretises the same equations (eq. 8, rows of eq. 9) and
hands its operators to ``bem.assemble``; outputs (Rayleigh coefficients, field)
come from ``bem`` through the node quadrature.

Each circle of radius R about c is parametrised x(t) = c + R (cos t, sin t) with
n equispaced nodes t_j = 2 pi j / n (n even), outward normal (cos t, sin t) and
ds = R dt.  The unknowns are the densities at the nodes, collocated at the
nodes.  Integrals over a circle use:

* the trapezoid rule (weight 2 pi R / n) for smooth kernels: other fibers, and
  the smooth remainder G_qp - Phi of the periodic kernel on the same fiber;
* Kress's product quadrature for the logarithmic kernels of S, D and K on their
  own circle: the kernel is split as M1(t, tau) ln(4 sin^2((t - tau)/2)) + M2(t, tau)
  with M1, M2 smooth, the log part integrated exactly against the trigonometric
  interpolant of M1 times the density (weights from ln(4 sin^2(s/2)) =
  -2 sum_{m>=1} cos(m s)/m) and M2 by the trapezoid rule;
* for the hypersingular T on its own circle, Maue's identity
  T phi = d/ds S (d phi/ds) + kappa^2 nu . S (nu phi), with the tangential
  derivatives taken by trigonometric differentiation at the nodes (the
  treatment of T in Kress, J. Comput. Appl. Math. 61 (1995), the paper's [4]).

On a circle the layer kernels are explicit: with s = t - tau and
r = 2 R |sin(s/2)|, the single-layer kernel is (i/4) H0(kappa r) R and both the
double-layer (d/dnu_y) and adjoint (d/dnu_x) kernels equal -(i kappa/8) r H1(kappa r),
since nu_y.(x - y) = -r^2/(2R) and nu_x.(x - y) = r^2/(2R).  Their log parts are
M1 = -(R/(4 pi)) J0(kappa r) and L1 = (kappa r/(8 pi)) J1(kappa r), and the
diagonal limits are M2(t,t) = R (i/4 - (ln(kappa R/2) + C)/(2 pi)) (C Euler's
constant) and L2(t,t) = -1/(4 pi).

The method converges spectrally for analytic boundaries and data.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
from scipy import special as sp

from . import bem, greens

EULER = 0.57721566490153286061


@dataclass
class Nodes:
    """Collocation nodes of all circles (duck-types the element arrays of ``bem``)."""
    c: np.ndarray       # [Q, 2] node positions (collocation points)
    nu: np.ndarray      # [Q, 2] outward normals
    w: np.ndarray       # [Q] trapezoid weights 2 pi R / n
    fiber: np.ndarray   # [Q] fiber index
    t: np.ndarray       # [Q] parameter angle
    R: np.ndarray       # [Q] radius of the node's circle
    centre: np.ndarray  # [M, 2]
    radius: np.ndarray  # [M]
    n: np.ndarray       # [M] nodes per circle

    @property
    def E(self):
        return len(self.w)


def nodes(centres, radii, n):
    centres = np.asarray(centres, dtype=np.float64).reshape(-1, 2)
    radii = np.asarray(radii, dtype=np.float64).ravel()
    ns = np.broadcast_to(np.asarray(n), radii.shape).astype(int)
    C, NU, Wt, F, T, RR = [], [], [], [], [], []
    for i, (cc, R, m) in enumerate(zip(centres, radii, ns)):
        if m % 2:
            raise ValueError("an even number of nodes per circle is required")
        t = 2 * math.pi * np.arange(m) / m
        nu = np.stack([np.cos(t), np.sin(t)], axis=1)
        C.append(cc[None, :] + R * nu)
        NU.append(nu)
        Wt.append(np.full(m, 2 * math.pi * R / m))
        F.append(np.full(m, i))
        T.append(t)
        RR.append(np.full(m, R))
    return Nodes(c=np.concatenate(C), nu=np.concatenate(NU), w=np.concatenate(Wt), fiber=np.concatenate(F),
                 t=np.concatenate(T), R=np.concatenate(RR), centre=centres, radius=radii, n=ns)


def problem(centres, radii, n, k, k1, rho, theta, H=1.0, eta=None, periodic=True) -> bem.Problem:
    return bem.Problem(el=nodes(centres, radii, n), k=k, k1=k1, rho=rho, theta=theta, H=H,
                       eta=k if eta is None else eta, periodic=periodic)


def log_weights(n):
    """W[i, j] = int_0^{2pi} ln(4 sin^2((t_i - tau)/2)) L_j(tau) dtau for the trigonometric
    Lagrange basis L_j of the n equispaced nodes (n even): the m-th Fourier mode of the
    log kernel is -2 pi/|m| (0 for m = 0), the Nyquist mode enters with half weight."""
    s = 2 * math.pi * (np.arange(n)[:, None] - np.arange(n)[None, :]) / n
    W = np.zeros((n, n))
    for m in range(1, n // 2):
        W -= (4 * math.pi / n) * np.cos(m * s) / m
    W -= (4 * math.pi / n**2) * np.cos((n // 2) * s)
    return W


def diff_matrix(n):
    """Derivative of the trigonometric interpolant at the n equispaced nodes (n even):
    Dt[i, j] = (1/2) (-1)^(i-j) cot((t_i - t_j)/2), zero diagonal."""
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    s = 2 * math.pi * (i - j) / n
    with np.errstate(divide="ignore", invalid="ignore"):
        Dt = 0.5 * (-1.0) ** (i - j) / np.tan(0.5 * s)
    Dt[i == j] = 0.0
    return Dt


def same_circle(kappa, R, n):
    """S, D, K, T of the free-space kernel Phi = (i/4) H0(kappa r) on one circle of radius
    R with n nodes, as n x n matrices acting on nodal densities (ds = R dt included)."""
    t = 2 * math.pi * np.arange(n) / n
    s = t[:, None] - t[None, :]
    off = ~np.eye(n, dtype=bool)
    r = 2 * R * np.abs(np.sin(0.5 * s))
    ln4 = np.zeros((n, n))
    ln4[off] = np.log(4 * np.sin(0.5 * s[off]) ** 2)
    W = log_weights(n)
    h = 2 * math.pi / n

    # single layer
    M1 = np.full((n, n), -R / (4 * math.pi), dtype=np.complex128)
    M1[off] = -R / (4 * math.pi) * sp.j0(kappa * r[off])
    M2 = np.empty((n, n), dtype=np.complex128)
    M2[off] = 0.25j * R * sp.hankel1(0, kappa * r[off]) - M1[off] * ln4[off]
    M2[~off] = R * (0.25j - (math.log(0.5 * kappa * R) + EULER) / (2 * math.pi))
    S = W * M1 + h * M2

    # double layer and its adjoint coincide on a circle
    L1 = np.zeros((n, n), dtype=np.complex128)
    L1[off] = kappa * r[off] / (8 * math.pi) * sp.j1(kappa * r[off])
    L2 = np.empty((n, n), dtype=np.complex128)
    L2[off] = -0.125j * kappa * r[off] * sp.hankel1(1, kappa * r[off]) - L1[off] * ln4[off]
    L2[~off] = -1.0 / (4 * math.pi)
    D = W * L1 + h * L2
    K = D.copy()

    # hypersingular operator by Maue's identity; d/ds = (1/R) d/dt
    Dt = diff_matrix(n)
    T = (Dt @ S @ Dt) / R**2 + kappa**2 * S * np.cos(s)
    return S, D, K, T


def _smooth_ops(d, nx, ny, w):
    S, D, K, T = greens.layer_kernels(d, (nx[:, 0][:, None], nx[:, 1][:, None]), (ny[:, 0][None, :], ny[:, 1][None, :]))
    return S * w, D * w, K * w, T * w


def operators(pb: bem.Problem):
    """The eight layer operators of eq. 8 at the nodes (see ``bem.assemble``)."""
    nd = pb.el
    Q = nd.E
    ops = {key: np.zeros((Q, Q), dtype=np.complex128) for key in ("S1", "D1", "K1", "T1", "S2", "D2", "K2", "T2")}
    starts = np.concatenate([[0], np.cumsum(nd.n)])
    x = nd.c
    z1 = x[:, 0][:, None] - x[:, 0][None, :]
    z2 = x[:, 1][:, None] - x[:, 1][None, :]
    w = nd.w[None, :]
    same = nd.fiber[:, None] == nd.fiber[None, :]

    # other fibers: the full kernel, trapezoid rule
    if pb.periodic:
        d = greens.qp_ewald(pb.k, pb.beta, pb.H, z1[~same], z2[~same])
    else:
        d = greens.free_space(pb.k, z1[~same], z2[~same])
    ii, jj = np.nonzero(~same)
    k4 = greens.layer_kernels(d, (nd.nu[ii, 0], nd.nu[ii, 1]), (nd.nu[jj, 0], nd.nu[jj, 1]))
    for key, val in zip(("S2", "D2", "K2", "T2"), k4):
        ops[key][ii, jj] = val * nd.w[jj]

    # own fiber: free-space kernel by the product rules, plus the periodic remainder
    R0 = greens.qp_remainder_at_origin(pb.k, pb.beta, pb.H) if pb.periodic else None
    for f in range(len(nd.n)):
        sl = slice(starts[f], starts[f + 1])
        R = float(nd.radius[f])
        for key, val in zip(("S2", "D2", "K2", "T2"), same_circle(pb.k, R, int(nd.n[f]))):
            ops[key][sl, sl] = val
        for key, val in zip(("S1", "D1", "K1", "T1"), same_circle(pb.k1, R, int(nd.n[f]))):
            ops[key][sl, sl] = val
        if pb.periodic:
            n = int(nd.n[f])
            a1 = z1[sl, sl]
            a2 = z2[sl, sl]
            off = ~np.eye(n, dtype=bool)
            rem = {key: np.empty((n, n), dtype=np.complex128) for key in ("g", "g1", "g2", "g11", "g12", "g22")}
            g = greens.qp_ewald(pb.k, pb.beta, pb.H, a1[off], a2[off])
            fs = greens.free_space(pb.k, a1[off], a2[off])
            for key in rem:
                rem[key][off] = g[key] - fs[key]
                rem[key][~off] = R0[key]
            for key, val in zip(("S2", "D2", "K2", "T2"), _smooth_ops(rem, nd.nu[sl], nd.nu[sl], nd.w[sl][None, :])):
                ops[key][sl, sl] += val
    del w
    return ops


def system(pb: bem.Problem):
    """(I - A) and B of eq. 9 at the nodes."""
    ops = operators(pb)
    return bem.assemble(pb, np.arange(pb.el.E), ops), bem.rhs(pb)


def solve(pb: bem.Problem):
    M, B = system(pb)
    return np.linalg.solve(M, B)
