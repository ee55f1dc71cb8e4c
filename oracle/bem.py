"""Oracle BEM: constant-element collocation of the Kress transmission system.

Test infrastructure; plain FP64 numpy/scipy; slow by design.

Discretisation (readings of Sec. 2 and Sec. 4, where the paper is silent):
each fiber boundary is the closed polygon through its counter-clockwise nodes;
element e is the chord from node j to node j+1 with midpoint c_e, length h_e and
outward normal nu_e (tangent turned clockwise).  Both densities (phi: double
layer, varphi: single layer, eq. 4) are constant per element and the equations
are collocated at the midpoints.  Matrix entries are the EXACT element integrals
of the kernels, so the discrete operator is:

  row 2e   : phi_e - (D1 phi)_e + i eta (S1 varphi)_e + (D2b phi)_e - i eta (S2b varphi)_e
  row 2e+1 : varphi_e + c2 [ (T2b phi)_e - i eta (K2b varphi)_e - rho ((T1 phi)_e - i eta (K1 varphi)_e) ]

with c2 = 2 / (i eta (1 + rho)) (eq. 9), the k1 operators coupling elements of the
same fiber only (eq. 5) and the barred operators using the quasi-periodic kernel
G_qp (eqs. 7-8).  Right-hand side (eq. 9): B_2e = -u_inc(c_e),
B_2e+1 = -c2 du_inc/dnu(c_e), u_inc = exp(i k x.d), d = (cos theta, sin theta).

Element integrals:
* self element: D = K = 0 (flat element); S and the finite-part T in closed form
  from the Struve-function integral of H0 (Abramowitz & Stegun 11.1.7-11.1.8):
      S_ee = (i/2)(1/kappa) int_0^{kappa a} H0(t) dt,
      T_ee = (i/2) kappa [ int_0^{kappa a} H0(t) dt - H1(kappa a) ],   a = h/2;
* other elements: the nearest image alpha^m Phi(x - y - m h) by composite
  Gauss-Legendre (4 panels x 16 nodes when the target is within 2h of the
  element midpoint, else 16 nodes), plus the smooth remainder
  G_qp - alpha^m Phi(. - m h) by 4- or 8-node Gauss-Legendre.

In free-space mode (``periodic=False``) the barred operators use Phi itself:
one isolated block of fibers, used for the Mie-series check.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np
from scipy import special as sp
from scipy import linalg as sla

from . import greens

_GL16 = np.polynomial.legendre.leggauss(16)
_GL8 = np.polynomial.legendre.leggauss(8)
_GL4 = np.polynomial.legendre.leggauss(4)


@dataclass
class Elements:
    a: np.ndarray      # [E,2] start node
    b: np.ndarray      # [E,2] end node
    c: np.ndarray      # [E,2] midpoint
    h: np.ndarray      # [E] length
    t: np.ndarray      # [E,2] unit tangent
    nu: np.ndarray     # [E,2] outward unit normal
    fiber: np.ndarray  # [E] fiber index

    @property
    def E(self):
        return len(self.h)


def elements(nodes, nodes_per_fiber) -> Elements:
    nodes = np.asarray(nodes, dtype=np.float64)
    A, B, F = [], [], []
    off = 0
    for i, n in enumerate(nodes_per_fiber):
        p = nodes[off:off + n]
        A.append(p)
        B.append(np.roll(p, -1, axis=0))
        F.append(np.full(n, i))
        off += n
    a = np.concatenate(A)
    b = np.concatenate(B)
    d = b - a
    h = np.hypot(d[:, 0], d[:, 1])
    t = d / h[:, None]
    nu = np.stack([t[:, 1], -t[:, 0]], axis=1)
    return Elements(a=a, b=b, c=0.5 * (a + b), h=h, t=t, nu=nu, fiber=np.concatenate(F))


def _int_h0(x):
    """int_0^x H0^(1)(t) dt for real x > 0 (A&S 11.1.7-11.1.8, Struve H0, H1)."""
    j0, j1, y0, y1 = sp.j0(x), sp.j1(x), sp.y0(x), sp.y1(x)
    s0, s1 = sp.struve(0, x), sp.struve(1, x)
    ij = x * j0 + 0.5 * math.pi * x * (j1 * s0 - j0 * s1)
    iy = x * y0 + 0.5 * math.pi * x * (y1 * s0 - y0 * s1)
    return ij + 1j * iy


def self_integrals(kappa, h):
    """(S_ee, T_ee) of (i/4)H0(kappa r) over a flat element of length h at its midpoint."""
    a = 0.5 * np.asarray(h, dtype=np.float64)
    ih = _int_h0(kappa * a)
    S = 0.5j / kappa * ih
    T = 0.5j * kappa * (ih - sp.hankel1(1, kappa * a))
    return S, T


class Kernel:
    """Either free space (periodic=False, wavenumber kappa) or quasi-periodic (k, beta, H)."""

    def __init__(self, kappa, periodic=False, beta=0.0, H=1.0):
        self.kappa = kappa
        self.periodic = periodic
        self.beta = beta
        self.H = H
        self.alpha = np.exp(1j * beta)


def _nthreads():
    return max(1, min(32, os.cpu_count() or 1))


def _parallel_map(fn, n, chunk):
    idx = [(s, min(n, s + chunk)) for s in range(0, n, chunk)]
    if len(idx) == 1:
        return [fn(*idx[0])]
    with ThreadPoolExecutor(_nthreads()) as ex:
        return list(ex.map(lambda se: fn(*se), idx))


def pair_integrals(ker: Kernel, el: Elements, ti, sj):
    """Element integrals int_{e_j} K(c_i, y) ds_y for pairs (ti[p], sj[p]).

    Returns S, D, K, T arrays (complex128) of the pair count."""
    ti = np.asarray(ti)
    sj = np.asarray(sj)
    n = len(ti)
    S = np.zeros(n, dtype=np.complex128)
    D = np.zeros_like(S)
    K = np.zeros_like(S)
    T = np.zeros_like(S)
    x = el.c[ti]
    nx = el.nu[ti]
    ny = el.nu[sj]
    hj = el.h[sj]
    tj = el.t[sj]
    cj = el.c[sj]
    H = ker.H

    # nearest image of the source element as seen from the target
    if ker.periodic:
        mstar = np.rint((x[:, 1] - cj[:, 1]) / H)
    else:
        mstar = np.zeros(n)
    shift = mstar * H
    ph = ker.alpha ** mstar
    rel = np.stack([x[:, 0] - cj[:, 0], x[:, 1] - cj[:, 1] - shift], axis=1)
    dist = np.hypot(rel[:, 0], rel[:, 1])
    selfp = (ti == sj)
    near = (~selfp) & (dist < 2.0 * hj)
    far = (~selfp) & (~near)

    def singular_part(mask, panels):
        idx = np.nonzero(mask)[0]
        if idx.size == 0:
            return
        u, w = _GL16
        # composite rule: panel p covers s in [-h/2 + p h/P, -h/2 + (p+1) h/P]
        P = panels
        su = ((np.arange(P)[:, None] + 0.5 * (u[None, :] + 1.0)) / P - 0.5).ravel()   # in [-1/2, 1/2]
        sw = (np.tile(w, P) / (2.0 * P))
        acc = [np.zeros(idx.size, dtype=np.complex128) for _ in range(4)]
        for q in range(su.size):
            s = su[q] * hj[idx]
            z1 = rel[idx, 0] - s * tj[idx, 0]
            z2 = rel[idx, 1] - s * tj[idx, 1]
            d = greens.free_space(ker.kappa, z1, z2)
            k4 = greens.layer_kernels(d, (nx[idx, 0], nx[idx, 1]), (ny[idx, 0], ny[idx, 1]))
            for r in range(4):
                acc[r] += sw[q] * hj[idx] * k4[r]
        for r, arr in enumerate((S, D, K, T)):
            arr[idx] += ph[idx] * acc[r]

    singular_part(far, 1)
    singular_part(near, 4)

    if np.any(selfp):
        idx = np.nonzero(selfp)[0]
        s0, t0 = self_integrals(ker.kappa, hj[idx])
        S[idx] += s0
        T[idx] += t0

    if ker.periodic:
        # smooth remainder R = G_qp - alpha^m* Phi(. - m* h) by low-order GL
        gl = _GL4 if float(np.max(hj)) < 0.02 * H else _GL8
        u, w = gl
        Z1 = (rel[:, 0][:, None] - 0.5 * u[None, :] * hj[:, None] * tj[:, 0][:, None])
        Z2 = (rel[:, 1][:, None] - 0.5 * u[None, :] * hj[:, None] * tj[:, 1][:, None])
        # back to the true displacement x - y (undo the nearest-image shift)
        Z2t = Z2 + shift[:, None]
        flat1 = Z1.ravel()
        flat2 = Z2t.ravel()
        near1 = Z1.ravel()
        near2 = Z2.ravel()
        phf = np.repeat(ph, u.size)

        def work(s, e):
            g = greens.qp_ewald(ker.kappa, ker.beta, H, flat1[s:e], flat2[s:e])
            f = greens.free_space(ker.kappa, near1[s:e], near2[s:e])
            return {key: g[key] - phf[s:e] * f[key] for key in g}

        parts = _parallel_map(work, flat1.size, 8192)
        R = {key: np.concatenate([p[key] for p in parts]).reshape(n, u.size) for key in parts[0]}
        nxr = (nx[:, 0][:, None], nx[:, 1][:, None])
        nyr = (ny[:, 0][:, None], ny[:, 1][:, None])
        k4 = greens.layer_kernels(R, nxr, nyr)
        wq = 0.5 * w[None, :] * hj[:, None]
        for r, arr in enumerate((S, D, K, T)):
            arr += (wq * k4[r]).sum(axis=1)
    return S, D, K, T


@dataclass
class Problem:
    el: Elements
    k: float
    k1: float
    rho: float
    theta: float
    H: float
    eta: float
    periodic: bool = True

    @property
    def beta(self):
        return self.k * self.H * math.sin(self.theta)

    @property
    def c2(self):
        return 2.0 / (1j * self.eta * (1.0 + self.rho))


def problem(w, eta=None, periodic=True) -> Problem:
    el = elements(w.nodes, w.nodes_per_fiber)
    return Problem(el=el, k=w.k, k1=w.k1, rho=w.rho_ratio, theta=w.theta, H=w.H,
                   eta=w.k if eta is None else eta, periodic=periodic)


def operator_rows(pb: Problem, rows_e=None):
    """Rows of (I - A) (eq. 9) for the target elements rows_e (default: all).

    Returns a complex128 array [2*len(rows_e), 2E]."""
    el = pb.el
    E = el.E
    if rows_e is None:
        rows_e = np.arange(E)
    rows_e = np.asarray(rows_e)
    R = len(rows_e)
    ti = np.repeat(rows_e, E)
    sj = np.tile(np.arange(E), R)
    kq = Kernel(pb.k, periodic=pb.periodic, beta=pb.beta, H=pb.H)
    S2, D2, K2, T2 = [a.reshape(R, E) for a in pair_integrals(kq, el, ti, sj)]
    # interior (k1) operators: same fiber only, free space
    same = el.fiber[ti] == el.fiber[sj]
    k1k = Kernel(pb.k1, periodic=False)
    S1 = np.zeros(R * E, dtype=np.complex128)
    D1 = np.zeros_like(S1)
    K1 = np.zeros_like(S1)
    T1 = np.zeros_like(S1)
    idx = np.nonzero(same)[0]
    s1, d1, kk1, t1 = pair_integrals(k1k, el, ti[idx], sj[idx])
    S1[idx], D1[idx], K1[idx], T1[idx] = s1, d1, kk1, t1
    S1, D1, K1, T1 = [a.reshape(R, E) for a in (S1, D1, K1, T1)]
    return assemble(pb, rows_e, dict(S1=S1, D1=D1, K1=K1, T1=T1, S2=S2, D2=D2, K2=K2, T2=T2))


def assemble(pb: Problem, rows_e, ops):
    """The rows of (I - A) of eq. 9 from the discrete layer operators.

    ops holds [R, E] arrays: S1, D1, K1, T1 (wavenumber k1, same fiber only, zero
    elsewhere) and S2, D2, K2, T2 (the barred quasi-periodic operators at k, or
    free-space ones when the problem is not periodic); entry [r, e] is the
    operator's weight of unknown e at collocation point rows_e[r].  Row 2r carries
    the first equation of eq. 8, row 2r+1 the second scaled by
    c2 = 2 / (i eta (1 + rho)), so that both have the identity on the diagonal."""
    E = pb.el.E
    R = len(rows_e)
    ie = 1j * pb.eta
    c2 = pb.c2
    M = np.zeros((2 * R, 2 * E), dtype=np.complex128)
    M[0::2, 0::2] = -ops["D1"] + ops["D2"]
    M[0::2, 1::2] = ie * ops["S1"] - ie * ops["S2"]
    M[1::2, 0::2] = c2 * (ops["T2"] - pb.rho * ops["T1"])
    M[1::2, 1::2] = c2 * (-ie * ops["K2"] + pb.rho * ie * ops["K1"])
    for r, e in enumerate(rows_e):
        M[2 * r, 2 * e] += 1.0
        M[2 * r + 1, 2 * e + 1] += 1.0
    return M


def rhs(pb: Problem):
    el = pb.el
    d = np.array([math.cos(pb.theta), math.sin(pb.theta)])
    x = el.c
    uinc = np.exp(1j * pb.k * (x @ d))
    dn = 1j * pb.k * (el.nu @ d) * uinc
    B = np.empty(2 * el.E, dtype=np.complex128)
    B[0::2] = -uinc
    B[1::2] = -pb.c2 * dn
    return B


def solve(pb: Problem, M=None, B=None):
    if M is None:
        M = operator_rows(pb)
    if B is None:
        B = rhs(pb)
    lu = sla.lu_factor(M)
    return sla.lu_solve(lu, B)


def quadrature(pb: Problem, nq=16):
    """Source points of the boundary integrals: points y [Q, 2], normals [Q, 2],
    weights [Q] and the unknown (element or node) each point carries.

    Constant elements: nq Gauss-Legendre nodes per element.  A discretisation
    whose unknowns are point values with their own weights (the Nystrom mode of
    ``nystrom``) brings them along as el.w."""
    el = pb.el
    if hasattr(el, "w"):
        return el.c, el.nu, el.w, np.arange(el.E)
    u, w = np.polynomial.legendre.leggauss(nq)
    s = 0.5 * u[None, :] * el.h[:, None]
    y = np.stack([(el.c[:, 0][:, None] + s * el.t[:, 0][:, None]).ravel(),
                  (el.c[:, 1][:, None] + s * el.t[:, 1][:, None]).ravel()], axis=1)
    nu = np.repeat(el.nu, nq, axis=0)
    wq = (0.5 * w[None, :] * el.h[:, None]).ravel()
    return y, nu, wq, np.repeat(np.arange(el.E), nq)


def potential(pb: Problem, psi, pts, interior_fiber=None, grad=False, nq=32):
    """Scattered field u^s (eq. 4/7) at points pts [P,2] outside all fibers, or the
    interior field u_i (eq. 5) of fiber ``interior_fiber`` at points inside it.

    With grad=True also returns du/dx1 at the points (the x1-derivative of the
    layer kernels: d/dx1 of Phi is g1, of its nu_y-derivative -(g11 nu1 + g12 nu2))."""
    el = pb.el
    pts = np.asarray(pts, dtype=np.float64)
    phi = psi[0::2]
    vphi = psi[1::2]
    y, nu, wq, idx = quadrature(pb, nq)
    if interior_fiber is None:
        ker = Kernel(pb.k, periodic=pb.periodic, beta=pb.beta, H=pb.H)
    else:
        ker = Kernel(pb.k1, periodic=False)
        keep = el.fiber[idx] == interior_fiber
        y, nu, wq, idx = y[keep], nu[keep], wq[keep], idx[keep]
    out = np.zeros(len(pts), dtype=np.complex128)
    dout = np.zeros(len(pts), dtype=np.complex128)
    for p, x in enumerate(pts):
        z1 = x[0] - y[:, 0]
        z2 = x[1] - y[:, 1]
        if ker.periodic:
            d = greens.qp_ewald(ker.kappa, ker.beta, pb.H, z1, z2)
        else:
            d = greens.free_space(ker.kappa, z1, z2)
        Dk = -(d["g1"] * nu[:, 0] + d["g2"] * nu[:, 1])
        out[p] = np.sum(wq * (Dk * phi[idx] - 1j * pb.eta * d["g"] * vphi[idx]))
        if grad:
            dD = -(d["g11"] * nu[:, 0] + d["g12"] * nu[:, 1])
            dout[p] = np.sum(wq * (dD * phi[idx] - 1j * pb.eta * d["g1"] * vphi[idx]))
    return (out, dout) if grad else out


def bragg_orders(pb: Problem):
    """Indices n of the propagating orders: |k sin(theta) + 2 pi n / H| < k."""
    ks = pb.k * math.sin(pb.theta)
    nlo = int(math.floor((-pb.k - ks) * pb.H / (2 * math.pi))) - 1
    nhi = int(math.ceil((pb.k - ks) * pb.H / (2 * math.pi))) + 1
    return np.array([n for n in range(nlo, nhi + 1) if abs(ks + 2 * math.pi * n / pb.H) < pb.k])


def rayleigh(pb: Problem, psi, orders=None):
    """Reflection R_n and transmission T_n of the Bragg orders n (plane-wave amplitudes of
    the total field left and right of the block), from the spectral form of G_qp:
    right of every source u^s = sum_n (T_n - delta_n0) e^{i(kx_n x1 + ky_n x2)}, left of
    them u^s = sum_n R_n e^{i(-kx_n x1 + ky_n x2)}, with ky_n = k sin(theta) + 2 pi n / H and
    kx_n = sqrt(k^2 - ky_n^2) (Im kx_n >= 0 for the evanescent orders)."""
    if orders is None:
        orders = bragg_orders(pb)
    phi = psi[0::2]
    vphi = psi[1::2]
    y, nu, wq, idx = quadrature(pb, 16)
    R = []
    T = []
    for n in orders:
        ky = pb.k * math.sin(pb.theta) + 2 * math.pi * n / pb.H
        kx = np.sqrt(complex(pb.k**2 - ky**2))
        pref = 1j / (2 * pb.H * kx)
        out = []
        for sgn in (+1, -1):
            e = np.exp(-1j * (sgn * kx * y[:, 0] + ky * y[:, 1]))
            dn = -1j * (sgn * kx * nu[:, 0] + ky * nu[:, 1]) * e
            out.append(pref * np.sum(wq * (dn * phi[idx] - 1j * pb.eta * e * vphi[idx])))
        T.append((1.0 if n == 0 else 0.0) + out[0])
        R.append(out[1])
    return np.asarray(orders), np.array(R), np.array(T)


def energy(pb: Problem, orders, R, T):
    """sum over propagating orders of (k_x,n / k_x,0)(|R_n|^2 + |T_n|^2); 1 for a lossless block."""
    k0 = pb.k * math.cos(pb.theta)
    tot = 0.0
    for n, r, t in zip(orders, R, T):
        ky = pb.k * math.sin(pb.theta) + 2 * math.pi * n / pb.H
        kx = math.sqrt(pb.k**2 - ky**2)
        tot += kx / k0 * (abs(r) ** 2 + abs(t) ** 2)
    return tot


def etc_points(pb: Problem, npts):
    """Midpoints x2 = H (j + 1/2) / npts of the ETC line integral over one period."""
    return pb.H * (np.arange(npts) + 0.5) / npts


def etc(pb: Problem, psi, nmax=20, npts=512, x1=None):
    """Energy transmission coefficient (Sec. 4): (1/kH) int_0^H |du/dx1(L, x2)| dx2 with
    L the right edge of the block (x1, default the right-most node) and u the total
    field, from the Rayleigh expansion to the right (orders -nmax..nmax), by the
    midpoint rule with npts points."""
    el = pb.el
    if x1 is None:
        L = float(np.max(el.b[:, 0])) if hasattr(el, "b") else float(np.max(el.c[:, 0]))
    else:
        L = float(x1)
    orders = np.arange(-nmax, nmax + 1)
    ordr, _, T = rayleigh(pb, psi, orders)
    x2 = etc_points(pb, npts)
    du = np.zeros(npts, dtype=np.complex128)
    for n, t in zip(ordr, T):
        ky = pb.k * math.sin(pb.theta) + 2 * math.pi * n / pb.H
        kx = np.sqrt(complex(pb.k**2 - ky**2))
        du += 1j * kx * t * np.exp(1j * (kx * L + ky * x2))
    return float(np.mean(np.abs(du)) * pb.H / (pb.k * pb.H))
