"""Pins for the oracle's Green's functions (CPU only).

Each check compares two independent evaluations: finite differences of scipy's
Hankel function, the Ewald split against the spectral (Rayleigh) series, and the
Ewald split against the plain image sum in an absorbing medium (where the sum
converges geometrically), plus the quasi-periodicity G(z + h) = alpha G(z) of eq. 3.
"""
import math

import numpy as np
import pytest

from oracle import greens

KEYS = ("g", "g1", "g2", "g11", "g12", "g22")


def _rel(a, b):
    return max(float(np.max(np.abs(a[k] - b[k])) / np.max(np.abs(b[k]))) for k in KEYS)


def test_free_space_derivatives_match_finite_differences():
    kap = 3.7
    z1 = np.array([0.3, -0.11, 0.05])
    z2 = np.array([0.2, 0.41, -0.07])
    d = greens.free_space(kap, z1, z2)
    e = 1e-5
    fx = lambda a, b: greens.free_space(kap, a, b)
    p, m = fx(z1 + e, z2), fx(z1 - e, z2)
    assert np.allclose((p["g"] - m["g"]) / (2 * e), d["g1"], rtol=1e-7)
    assert np.allclose((p["g1"] - m["g1"]) / (2 * e), d["g11"], rtol=1e-7)
    assert np.allclose((p["g2"] - m["g2"]) / (2 * e), d["g12"], rtol=1e-7)
    p, m = fx(z1, z2 + e), fx(z1, z2 - e)
    assert np.allclose((p["g"] - m["g"]) / (2 * e), d["g2"], rtol=1e-7)
    assert np.allclose((p["g2"] - m["g2"]) / (2 * e), d["g22"], rtol=1e-7)
    # Helmholtz: g11 + g22 + k^2 g = 0 away from the source
    assert np.allclose(d["g11"] + d["g22"] + kap**2 * d["g"], 0, atol=1e-10)


@pytest.mark.parametrize("kH,theta", [(2.0, math.radians(30)), (5.0, 0.3), (20.0, math.radians(30)), (0.5, 1.2)])
def test_ewald_matches_spectral_series(kH, theta):
    H = 1.0
    k = kH / H
    beta = k * H * math.sin(theta)
    rng = np.random.default_rng(7)
    z1 = rng.uniform(0.05, 1.0, 64) * rng.choice([-1.0, 1.0], 64)
    z2 = rng.uniform(-1.3, 1.3, 64)
    assert _rel(greens.qp_ewald(k, beta, H, z1, z2), greens.qp_spectral(k, beta, H, z1, z2)) < 1e-12


def test_ewald_matches_direct_sum_in_absorbing_medium():
    H = 1.0
    k = 3.0 + 0.5j
    beta = k * H * math.sin(math.radians(30))
    z1 = np.array([0.01, 0.3, -0.2, 0.0, 0.7, 0.002])
    z2 = np.array([0.02, 0.9, -0.4, 0.3, 1.5, -0.001])
    assert _rel(greens.qp_ewald(k, beta, H, z1, z2), greens.qp_direct(k, beta, H, z1, z2, 400)) < 1e-12


def test_quasi_periodicity():
    H, k, theta = 1.0, 5.0, 0.3
    beta = k * H * math.sin(theta)
    z1 = np.array([0.1, -0.4, 0.33])
    z2 = np.array([0.2, 0.05, -0.31])
    a = greens.qp_ewald(k, beta, H, z1, z2 + H)
    b = greens.qp_ewald(k, beta, H, z1, z2)
    alpha = np.exp(1j * beta)
    for key in KEYS:
        assert np.allclose(a[key], alpha * b[key], rtol=1e-13, atol=1e-13)
