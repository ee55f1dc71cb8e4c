"""Oracle Green's functions (test infrastructure; FP64, numpy/scipy).

Free space (Sec. 2): Phi(x, y) = (i/4) H0^(1)(kappa |x - y|).
Quasi-periodic (Sec. 2, eqs. 7-8): G_qp(z) = sum_m alpha^m Phi(z - m h),
z = x - y, h = (0, H), alpha = exp(i beta), beta = k H sin(theta).

Every function returns the value and the first and second derivatives with
respect to z = x - y as a dict {g, g1, g2, g11, g12, g22}; the layer kernels
follow from them:
    S: g               D (d/dnu_y): -(g1 nu_y1 + g2 nu_y2)
    K (d/dnu_x): g1 nu_x1 + g2 nu_x2
    T (d2/dnu_x dnu_y): -(nu_x^T Hess(g) nu_y)

G_qp is evaluated by the Ewald split (C. M. Linton, J. Eng. Math. 33 (1998)):
a spectral part summed over the Bragg orders kappa_n = (beta + 2 pi n)/H with
complementary error functions, and a spatial part summed over images with
exponential integrals E_{j+1}.  The spectral (Rayleigh) series and the direct
image sum for an absorbing medium (complex k) are independent check forms.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special as sp

SQRT_PI = math.sqrt(math.pi)


def free_space(kappa, z1, z2):
    """(i/4) H0(kappa r) and its z-derivatives, r = |z| > 0."""
    z1 = np.asarray(z1, dtype=np.float64)
    z2 = np.asarray(z2, dtype=np.float64)
    r = np.hypot(z1, z2)
    x = kappa * r
    h0 = sp.hankel1(0, x)
    h1 = sp.hankel1(1, x)
    g = 0.25j * h0
    f = -0.25j * kappa * h1 / r                              # dg/dz_a = f z_a
    fp = -0.25j * kappa * (kappa * h0 / r - 2.0 * h1 / r**2)  # df/dr
    return dict(g=g, g1=f * z1, g2=f * z2,
                g11=fp * z1 * z1 / r + f, g12=fp * z1 * z2 / r, g22=fp * z2 * z2 / r + f)


def _gamma(kap, k):
    """gamma_n = sqrt(kappa_n^2 - k^2) on the outgoing branch (Re >= 0; -i sqrt(k^2-kappa^2)
    for real k and propagating orders)."""
    g = np.sqrt(kap * kap - k * k + 0j)
    flip = (np.real(g) == 0.0) & (np.imag(g) > 0.0)
    return np.where(flip, -g, g)


def ewald_parameter(k, H):
    return max(SQRT_PI, abs(k) * H / 3.0) / H


def qp_ewald(k, beta, H, z1, z2, E=None):
    """Quasi-periodic Green's function and derivatives by the Ewald split.

    k may be complex (absorbing medium); beta = k H sin(theta) is then complex too.
    Valid for any z not on the lattice {m h}."""
    z1 = np.atleast_1d(np.asarray(z1, dtype=np.float64))
    z2 = np.atleast_1d(np.asarray(z2, dtype=np.float64))
    if E is None:
        E = ewald_parameter(k, H)
    out = {key: np.zeros(z1.shape, dtype=np.complex128) for key in ("g", "g1", "g2", "g11", "g12", "g22")}

    # spectral part: (1/4H) sum_n e^{i kappa_n z2} [A+ + A-]/gamma_n
    kH = abs(k) * H
    ns = int(math.ceil(2.2 * E * H + kH / (2 * math.pi))) + 3
    nc = int(round(-np.real(beta) / (2 * math.pi)))
    w0 = np.exp(-z1 * z1 * E * E)
    for n in range(nc - ns, nc + ns + 1):
        kap = (beta + 2 * math.pi * n) / H
        gam = _gamma(kap, k)
        w = np.exp(-gam * gam / (4 * E * E)) * w0
        ep = sp.erfcx(gam / (2 * E) + z1 * E)
        em = sp.erfcx(gam / (2 * E) - z1 * E)
        P = w * (ep + em)
        Q = w * (ep - em)
        gg = (2 * E / SQRT_PI) * w
        ph = np.exp(1j * kap * z2) / (4 * H)
        out["g"] += ph * P / gam
        out["g1"] += ph * Q
        out["g2"] += ph * 1j * kap * P / gam
        out["g11"] += ph * (gam * P - 2 * gg)
        out["g12"] += ph * 1j * kap * Q
        out["g22"] += ph * (-kap * kap) * P / gam

    # spatial part: (1/4 pi) sum_m alpha^m sum_j c_j E_{j+1}(r_m^2 E^2)
    q = (k / (2 * E)) ** 2
    nj = 2
    term = 1.0
    while True:
        term *= abs(q) / nj
        nj += 1
        if term < 1e-19 and nj > 4:
            break
    c = np.array([q**j / math.factorial(j) for j in range(nj)], dtype=np.complex128)
    reach = 6.6 / E
    mlo = int(math.floor((z2.min() - reach) / H))
    mhi = int(math.ceil((z2.max() + reach) / H))
    alpha = np.exp(1j * beta)
    for m in range(mlo, mhi + 1):
        t2 = z2 - m * H
        rho = z1 * z1 + t2 * t2
        x = rho * E * E
        live = x < 50.0
        if not np.any(live):
            continue
        xl = x[live]
        # E_n(x) for n = -1 .. nj
        en = np.empty((nj + 2, xl.size))
        ex = np.exp(-xl)
        en[0] = ex * (xl + 1) / (xl * xl)     # E_{-1}
        en[1] = ex / xl                         # E_0
        for nn in range(1, nj + 1):
            en[nn + 1] = sp.expn(nn, xl)
        F = (c[:, None] * en[2:2 + nj]).sum(axis=0)              # sum c_j E_{j+1}
        F1 = -E * E * (c[:, None] * en[1:1 + nj]).sum(axis=0)     # dF/drho
        F2 = E**4 * (c[:, None] * en[0:nj]).sum(axis=0)           # d2F/drho2
        s = alpha**m / (4 * math.pi)
        a1 = z1[live]
        a2 = t2[live]
        out["g"][live] += s * F
        out["g1"][live] += s * 2 * F1 * a1
        out["g2"][live] += s * 2 * F1 * a2
        out["g11"][live] += s * (4 * F2 * a1 * a1 + 2 * F1)
        out["g12"][live] += s * (4 * F2 * a1 * a2)
        out["g22"][live] += s * (4 * F2 * a2 * a2 + 2 * F1)
    return out


def qp_spectral(k, beta, H, z1, z2, nmax=None):
    """Spectral (Rayleigh) series G_qp = (1/2H) sum_n e^{i kappa_n z2} e^{-gamma_n |z1|}/gamma_n,
    with derivatives; converges geometrically for |z1| > 0."""
    z1 = np.atleast_1d(np.asarray(z1, dtype=np.float64))
    z2 = np.atleast_1d(np.asarray(z2, dtype=np.float64))
    a = np.abs(z1)
    sgn = np.sign(z1)
    if nmax is None:
        amin = max(float(a.min()), 1e-3 * H)
        nmax = int(math.ceil(40.0 * H / (2 * math.pi * amin) + abs(k) * H / (2 * math.pi))) + 2
    out = {key: np.zeros(z1.shape, dtype=np.complex128) for key in ("g", "g1", "g2", "g11", "g12", "g22")}
    nc = int(round(-np.real(beta) / (2 * math.pi)))
    for n in range(nc - nmax, nc + nmax + 1):
        kap = (beta + 2 * math.pi * n) / H
        gam = _gamma(kap, k)
        t = np.exp(1j * kap * z2 - gam * a) / (2 * H * gam)
        out["g"] += t
        out["g1"] += -gam * sgn * t
        out["g2"] += 1j * kap * t
        out["g11"] += gam * gam * t
        out["g12"] += -gam * sgn * 1j * kap * t
        out["g22"] += -kap * kap * t
    return out


def qp_direct(k, beta, H, z1, z2, mmax):
    """Direct image sum sum_{|m|<=mmax} alpha^m Phi(z - m h); converges only for Im k > 0."""
    z1 = np.atleast_1d(np.asarray(z1, dtype=np.float64))
    z2 = np.atleast_1d(np.asarray(z2, dtype=np.float64))
    alpha = np.exp(1j * beta)
    out = {key: np.zeros(z1.shape, dtype=np.complex128) for key in ("g", "g1", "g2", "g11", "g12", "g22")}
    for m in range(-mmax, mmax + 1):
        f = free_space(k, z1, z2 - m * H)
        for key in out:
            out[key] += alpha**m * f[key]
    return out


def layer_kernels(d, nx, ny):
    """S, D, K, T kernels from value/derivative dict d; nx = normal at the target x,
    ny = normal at the source y (each a pair of arrays)."""
    S = d["g"]
    D = -(d["g1"] * ny[0] + d["g2"] * ny[1])
    K = d["g1"] * nx[0] + d["g2"] * nx[1]
    T = -(nx[0] * (d["g11"] * ny[0] + d["g12"] * ny[1]) + nx[1] * (d["g12"] * ny[0] + d["g22"] * ny[1]))
    return S, D, K, T


def qp_remainder_at_origin(k, beta, H, npts=256):
    """R = G_qp - Phi (all images m != 0) and its z-derivatives at z = 0.

    R is smooth in |z| < H and solves the Helmholtz equation there, so by Graf's
    theorem (eq. 10) it has the local expansion R(z) = (i/4) sum_l S'_{-l}
    J_l(k|z|) e^{i l psi} with S'_j = sum_{m != 0} alpha^m H_j(k|m|H) e^{i j theta_{-mh}}.
    The coefficients S'_l for |l| <= 2 come from the Fourier coefficients of R on a
    circle of radius rho < H (chosen away from the zeros of J_0, J_1, J_2), and the
    value, gradient and Hessian at 0 follow from J_0 = 1 - (kr)^2/4, J_{+-1} e^{+-i psi}
    = +-(k/2)(z1 +- i z2), J_{+-2} e^{+-2i psi} = (k^2/8)(z1 +- i z2)^2 to second order."""
    cands = H * np.linspace(0.25, 0.6, 15)
    score = [min(abs(sp.jv(l, k * r)) for l in (0, 1, 2)) for r in cands]
    rho = float(cands[int(np.argmax(score))])
    psi = 2 * math.pi * np.arange(npts) / npts
    z1 = rho * np.cos(psi)
    z2 = rho * np.sin(psi)
    Rz = qp_ewald(k, beta, H, z1, z2)["g"] - free_space(k, z1, z2)["g"]
    c = np.fft.fft(Rz) / npts
    # S'_{-l} = 4 c_l / (i J_l(k rho))
    Sp = {-l: 4.0 * c[l % npts] / (1j * sp.jv(l, k * rho)) for l in (-2, -1, 0, 1, 2)}
    q = 0.25j
    g = q * Sp[0]
    g1 = q * 0.5 * k * (Sp[-1] - Sp[1])
    g2 = q * 0.5j * k * (Sp[-1] + Sp[1])
    g11 = q * (-0.5 * k * k * Sp[0] + 0.25 * k * k * (Sp[-2] + Sp[2]))
    g22 = q * (-0.5 * k * k * Sp[0] - 0.25 * k * k * (Sp[-2] + Sp[2]))
    g12 = q * 0.25j * k * k * (Sp[-2] - Sp[2])
    return dict(g=g, g1=g1, g2=g2, g11=g11, g12=g12, g22=g22)
