"""Oracle lattice sums (test infrastructure; FP64).

Sec. 3.3: the periodic translation at the root needs
    S_j = sum_{|m| >= 2} alpha^m H_j^(1)(k |m| H) e^{i j theta_{-m h}},
theta_{-m h} = -pi/2 for m > 0 and +pi/2 for m < 0, j in [-2p, 2p].  For real k the
series converges only conditionally (Sec. 2: O(1/sqrt(q))), so its plain
definition is evaluated here through the function it generates: by Graf's
theorem (eq. 10) the image field
    T(z) = G_qp(z) - sum_{|m| <= 1} alpha^m Phi(z - m h)
has the local expansion T(z) = (i/4) sum_l J_l(k|z|) e^{i l psi} S_{-l} about
z = 0, so the l-th Fourier coefficient of T on a circle of radius rho equals
(i/4) J_l(k rho) S_{-l}.  G_qp comes from the Ewald form in ``greens``.

``direct_sum`` is the definition itself, truncated, which converges
geometrically only in an absorbing medium (Im k > 0); it pins the above.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special as sp

from . import greens


def image_field_coeffs(k, beta, H, rho, lmax, npts=None):
    """c_l = (1/2pi) int T(rho e^{i psi}) e^{-i l psi} dpsi for l in [-lmax, lmax]."""
    if npts is None:
        npts = max(256, 4 * (2 * lmax + 1))
    psi = 2 * math.pi * np.arange(npts) / npts
    z1 = rho * np.cos(psi)
    z2 = rho * np.sin(psi)
    Tz = greens.qp_ewald(k, beta, H, z1, z2)["g"]
    alpha = np.exp(1j * beta)
    for m in (-1, 0, 1):
        Tz = Tz - alpha**m * greens.free_space(k, z1, z2 - m * H)["g"]
    c = np.fft.fft(Tz) / npts
    ls = np.arange(-lmax, lmax + 1)
    return ls, c[ls % npts]


def lattice_sums(k, beta, H, jmax, rho=None, npts=None):
    """S_j for j in [-jmax, jmax] from the Fourier coefficients of the image field.

    The nearest excluded images sit at distance 2H, so the coefficients decay
    like (rho / 2H)^|l|: a circle close to that limit (rho = 1.9 H with a few
    thousand points) keeps the high orders (|j| ~ 100) accurate."""
    if rho is None:
        rho = 0.75 * H
    ls, c = image_field_coeffs(k, beta, H, rho, jmax, npts)
    Jl = sp.jv(ls, k * rho)
    S_minus_l = 4.0 * c / (1j * Jl)
    # S_j with j = -l
    js = -ls
    order = np.argsort(js)
    return js[order], S_minus_l[order]


def direct_sum(k, beta, H, jmax, mmax):
    """Truncated definition sum_{2<=|m|<=mmax} alpha^m H_j(k|m|H) e^{i j theta_{-mh}}."""
    js = np.arange(-jmax, jmax + 1)
    alpha = np.exp(1j * beta)
    S = np.zeros(js.shape, dtype=np.complex128)
    for m in range(2, mmax + 1):
        hj = sp.hankel1(js, k * m * H)
        S += alpha**m * hj * np.exp(-0.5j * math.pi * js)      # image below: angle -pi/2
        S += alpha**(-m) * hj * np.exp(0.5j * math.pi * js)    # image above: angle +pi/2
    return js, S
