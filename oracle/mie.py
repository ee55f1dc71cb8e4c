"""Mie series for one isolated circular fiber (test infrastructure; FP64).

Physics check of the transmission problem (Sec. 2, eqs. 1-2) without periodicity:
incident exp(i k x.d) on a circle of radius R centred at the origin, fiber
wavenumber k1, varrho = rho_matrix / rho_fiber.  With the Jacobi-Anger expansion
exp(i k r cos(t - theta)) = sum_n i^n J_n(k r) e^{i n (t - theta)}:

  u^s = sum_n a_n H_n(k r) e^{i n (t - theta)},   u_i = sum_n b_n J_n(k1 r) e^{i n (t - theta)},

and continuity of u and of (1/rho) du/dr at r = R (eq. 2, so varrho du_i/dr = du/dr)
gives per order n the 2x2 system solved below.
"""
from __future__ import annotations

import numpy as np
from scipy import special as sp


def coefficients(k, k1, rho, R, nmax):
    n = np.arange(-nmax, nmax + 1)
    J, Jp = sp.jv(n, k * R), sp.jvp(n, k * R)
    J1, J1p = sp.jv(n, k1 * R), sp.jvp(n, k1 * R)
    Hn, Hp = sp.hankel1(n, k * R), sp.h1vp(n, k * R)
    a = np.zeros(n.size, dtype=np.complex128)
    b = np.zeros(n.size, dtype=np.complex128)
    for q in range(n.size):
        # [ H_n(kR)        -J_n(k1R)         ] [a]   [ -i^n J_n(kR)     ]
        # [ k H_n'(kR)     -rho k1 J_n'(k1R) ] [b] = [ -i^n k J_n'(kR)  ]
        A = np.array([[Hn[q], -J1[q]], [k * Hp[q], -rho * k1 * J1p[q]]])
        rhs = -(1j ** n[q]) * np.array([J[q], k * Jp[q]])
        a[q], b[q] = np.linalg.solve(A, rhs)
    return n, a, b


def scattered(k, k1, rho, R, theta, pts, nmax=40):
    n, a, _ = coefficients(k, k1, rho, R, nmax)
    pts = np.asarray(pts)
    r = np.hypot(pts[:, 0], pts[:, 1])
    t = np.arctan2(pts[:, 1], pts[:, 0])
    return (a[None, :] * sp.hankel1(n[None, :], k * r[:, None]) * np.exp(1j * n[None, :] * (t[:, None] - theta))).sum(axis=1)


def interior(k, k1, rho, R, theta, pts, nmax=40):
    n, _, b = coefficients(k, k1, rho, R, nmax)
    pts = np.asarray(pts)
    r = np.hypot(pts[:, 0], pts[:, 1])
    t = np.arctan2(pts[:, 1], pts[:, 0])
    return (b[None, :] * sp.jv(n[None, :], k1 * r[:, None]) * np.exp(1j * n[None, :] * (t[:, None] - theta))).sum(axis=1)
