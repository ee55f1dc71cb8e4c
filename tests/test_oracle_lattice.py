"""Pins for the oracle's lattice sums (Sec. 3.3) on the CPU.

In an absorbing medium the defining image sum converges geometrically and is the
reference; for real k the Fourier coefficients of the image field must not depend
on the radius of the circle they are taken on.  Errors are measured on the local
expansion itself: coefficient j weighted by |J_j(k rho)|.
"""
import math

import numpy as np
from scipy import special as sp

from oracle import lattice


def _weighted(js, a, b, k, rho):
    w = np.abs(sp.jv(-js, k * rho))
    return float(np.max(np.abs(a - b) * w) / np.max(np.abs(b) * w))


def test_lattice_sums_match_direct_sum_in_absorbing_medium():
    H = 1.0
    k = 3.0 + 0.5j
    beta = k * H * math.sin(math.radians(30))
    js, S = lattice.lattice_sums(k, beta, H, 20)
    _, D = lattice.direct_sum(k, beta, H, 20, 600)
    assert _weighted(js, S, D, k, 0.75 * H) < 1e-12
    # low orders individually
    mid = np.abs(js) <= 6
    assert np.max(np.abs(S[mid] - D[mid]) / np.abs(D[mid])) < 1e-6


def test_lattice_sums_independent_of_circle_radius():
    H = 1.0
    for kH, theta in ((2.0, math.radians(30)), (5.0, 0.3)):
        k = kH / H
        beta = kH * math.sin(theta)
        js, a = lattice.lattice_sums(k, beta, H, 16, rho=0.6 * H)
        _, b = lattice.lattice_sums(k, beta, H, 16, rho=0.9 * H)
        assert _weighted(js, a, b, k, 0.6 * H) < 1e-11


def test_high_orders_match_direct_sum_in_absorbing_medium():
    """Orders up to 108 (twice the root order of the 32x32 block at kH = 20), each
    on its own: the circle at 1.9 H keeps every coefficient well above rounding."""
    H = 1.0
    k = 20.0 + 0.5j
    beta = k * H * math.sin(math.radians(30))
    js, S = lattice.lattice_sums(k, beta, H, 108, rho=1.9 * H, npts=8192)
    _, D = lattice.direct_sum(k, beta, H, 108, 300)
    assert np.max(np.abs(S - D) / np.abs(D)) < 1e-11


def test_high_orders_independent_of_circle_radius():
    H = 1.0
    k = 20.0
    beta = k * H * math.sin(math.radians(30))
    js, a = lattice.lattice_sums(k, beta, H, 108, rho=1.9 * H, npts=8192)
    _, b = lattice.lattice_sums(k, beta, H, 108, rho=1.75 * H, npts=8192)
    assert _weighted(js, a, b, k, 1.75 * H) < 1e-11
