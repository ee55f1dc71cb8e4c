"""Seeded synthetic inputs: fiber boundary nodes and physical parameters.

This module only generates inputs (node coordinates of the fiber boundaries,
wavenumbers, density ratio, incidence angle).  It holds none of the method's
arithmetic, so both the CUDA path and the CPU oracle may use it.

The workloads follow the paper's liquid phononic-crystal experiments (Sec. 4):
water and mercury, circular fibers arranged in square or hexagon lattices inside
one fundamental block that repeats with period H along y (Sec. 2, eq. 3).
Nodes of each fiber are listed counter-clockwise so that the outward normal of
the chord from node j to node j+1 is the tangent turned clockwise.

Material constants: water c = 1490 m/s, rho = 1000 kg/m^3; mercury c = 1450 m/s,
rho = 13600 kg/m^3 (Sec. 4 prints c = 1500 for water; 1490 is used here).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_WATER, RHO_WATER = 1490.0, 1000.0
C_MERCURY, RHO_MERCURY = 1450.0, 13600.0


@dataclass
class Workload:
    name: str
    H: float                      # period along y (the paper's H)
    lattice: int                  # 0 = square, 1 = hexagon
    k: float                      # matrix wavenumber
    k1: float                     # fiber wavenumber
    rho_ratio: float              # varrho = rho_matrix / rho_fiber (eq. 6)
    theta: float                  # incidence angle (rad), d = (cos, sin)
    nodes_per_fiber: np.ndarray   # int32 [M]
    nodes: np.ndarray             # float64 [sum N][2], CCW per fiber
    centres: np.ndarray = field(default=None)   # float64 [M][2]
    radii: np.ndarray = field(default=None)     # float64 [M]

    @property
    def M(self) -> int:
        return int(len(self.nodes_per_fiber))

    @property
    def E(self) -> int:
        return int(self.nodes_per_fiber.sum())


def circle_nodes(cx: float, cy: float, r: float, n: int, phase: float = 0.0) -> np.ndarray:
    t = phase + 2.0 * np.pi * np.arange(n) / n
    return np.stack([cx + r * np.cos(t), cy + r * np.sin(t)], axis=1)


def _materials(kH: float, H: float, matrix: str = "water"):
    k = kH / H
    if matrix == "water":
        k1 = k * C_WATER / C_MERCURY
        rho = RHO_WATER / RHO_MERCURY
    else:
        k1 = k * C_MERCURY / C_WATER
        rho = RHO_MERCURY / RHO_WATER
    return k, k1, rho


def wood_distance(kH: float, theta: float) -> float:
    """Distance of kH(1 +- sin theta) from the nearest multiple of 2 pi (Sec. 2)."""
    s = math.sin(theta)
    d = math.inf
    for v in (kH * (1 + s), kH * (1 - s)):
        d = min(d, abs(v - 2 * math.pi * round(v / (2 * math.pi))))
    return d


def _from_fibers(name, H, lattice, kH, theta, centres, radii, npf, matrix="water"):
    k, k1, rho = _materials(kH, H, matrix)
    nodes = np.concatenate([circle_nodes(c[0], c[1], r, n) for c, r, n in zip(centres, radii, npf)])
    return Workload(name=name, H=H, lattice=lattice, k=k, k1=k1, rho_ratio=rho, theta=theta,
                    nodes_per_fiber=np.asarray(npf, dtype=np.int32), nodes=nodes,
                    centres=np.asarray(centres, dtype=np.float64), radii=np.asarray(radii, dtype=np.float64))


def square_block(nx: int, ny: int, H: float, r_frac: float, n: int, kH: float, theta: float,
                 name: str | None = None, matrix: str = "water") -> Workload:
    """nx columns by ny rows of equal circles, spacing a = H/ny, radius r_frac*a."""
    a = H / ny
    centres = [((ix + 0.5) * a, (iy + 0.5) * a) for ix in range(nx) for iy in range(ny)]
    radii = [r_frac * a] * len(centres)
    npf = [n] * len(centres)
    return _from_fibers(name or f"square_{nx}x{ny}_n{n}_kH{kH:g}", H, 0, kH, theta, centres, radii, npf, matrix)


def round_square_nodes(cx: float, cy: float, r: float, n: int) -> np.ndarray:
    """Nodes of the round-square scatterer of Sec. 4,
    (r (3 + 2 sin^2 t) cos t, r (3 + 2 cos^2 t) sin t), at n uniform parameter values."""
    t = 2.0 * np.pi * np.arange(n) / n
    return np.stack([cx + r * (3 + 2 * np.sin(t) ** 2) * np.cos(t), cy + r * (3 + 2 * np.cos(t) ** 2) * np.sin(t)],
                    axis=1)


def round_square_block(nx: int, ny: int, H: float, extent_frac: float, n: int, kH: float, theta: float,
                       name: str | None = None) -> Workload:
    """Square lattice of round-square scatterers whose half-extent 3r is extent_frac * a."""
    a = H / ny
    r = extent_frac * a / 3.0
    k, k1, rho = _materials(kH, H)
    centres = [((ix + 0.5) * a, (iy + 0.5) * a) for ix in range(nx) for iy in range(ny)]
    nodes = np.concatenate([round_square_nodes(c[0], c[1], r, n) for c in centres])
    return Workload(name=name or f"roundsquare_{nx}x{ny}_n{n}_kH{kH:g}", H=H, lattice=0, k=k, k1=k1, rho_ratio=rho,
                    theta=theta, nodes_per_fiber=np.full(len(centres), n, dtype=np.int32), nodes=nodes,
                    centres=np.asarray(centres), radii=np.full(len(centres), 3 * r))


def square_2x2_n64():
    """Square lattice, H = 1, 2x2 circles at 0.25/0.75, r = 0.15, 64 elements each, kH = 2, theta = 30 deg."""
    w = square_block(2, 2, 1.0, 0.3, 64, 2.0, math.radians(30.0), name="square_2x2_n64_kH2")
    return w


def hexagon_block(ncol: int, nrow: int, H: float, n: int, kH: float, theta: float, seed: int,
                  r_lo: float = 0.1, r_hi: float = 0.3, jitter: float = 0.05, gap: float = 0.05,
                  name: str | None = None, n_of_r=None) -> Workload:
    """Hexagon lattice: columns along y at spacing a = H/nrow, column pitch a*sqrt(3)/2,
    odd columns shifted by a/2.  Radii uniform in [r_lo, r_hi]*a, centres jittered
    uniformly in a disk of radius jitter*a; draws leaving a gap < gap*a between
    neighbours (including periodic images in y) are redrawn."""
    rng = np.random.default_rng(seed)
    a = H / nrow
    pitch = a * math.sqrt(3.0) / 2.0
    base = []
    for c in range(ncol):
        for j in range(nrow):
            base.append(((c + 0.5) * pitch, (j + 0.5 + 0.5 * (c % 2)) * a))
    base = np.array(base)
    M = len(base)
    radii = rng.uniform(r_lo, r_hi, size=M) * a
    centres = base.copy()
    for i in range(M):
        for _ in range(1000):
            rr = jitter * a * math.sqrt(rng.uniform())
            tt = rng.uniform(0, 2 * math.pi)
            cand = base[i] + rr * np.array([math.cos(tt), math.sin(tt)])
            ok = True
            for j in range(i):
                for m in (-1, 0, 1):
                    dx = cand[0] - centres[j][0]
                    dy = cand[1] - centres[j][1] - m * H
                    if math.hypot(dx, dy) - radii[i] - radii[j] < gap * a:
                        ok = False
            if cand[0] - radii[i] < 0 or ok is False:
                continue
            centres[i] = cand
            break
    if n_of_r is None:
        npf = [n] * M
    else:
        npf = [int(n_of_r(r / a)) for r in radii]
    return _from_fibers(name or f"hexagon_{ncol}x{nrow}_n{n}_kH{kH:g}", H, 1, kH, theta, centres, radii, npf)


def hexagon_block_lattice(H: float, nrow: int) -> dict:
    """The hexagonal lattice of hexagon_block (spacing a = H/nrow, one lattice vector
    along y, the point of column 0, row 0), as the triangle tree's options."""
    a = H / nrow
    return {"tri_a": a, "tri_ox": 0.5 * a * math.sqrt(3.0) / 2.0, "tri_oy": 0.5 * a}


def table3_hexagon_lattice() -> dict:
    """The hexagonal lattice of table3_block(lattice="hexagon") (a = 0.5, the point
    of column 0, row 0), as the triangle tree's options."""
    a = 0.5
    return {"tri_a": a, "tri_ox": 0.5 * a * math.sqrt(3.0) / 2.0, "tri_oy": 0.25 * a}


def hexagon_8x8_n256(seed: int = 1911) -> Workload:
    """Hexagon lattice, 8x8 = 64 fibers, radii in [0.1,0.3]*spacing with jitter, 256
    elements each (16384 elements, 32768 unknowns), kH = 5, theta uniform in
    [0, 90 deg) avoiding Wood anomalies by at least 1e-3."""
    rng = np.random.default_rng(seed)
    kH = 5.0
    while True:
        theta = rng.uniform(0.0, math.pi / 2)
        if wood_distance(kH, theta) > 1e-3:
            break
    return hexagon_block(8, 8, 1.0, 256, kH, theta, seed + 100, name="hexagon_8x8_n256_kH5")


def square_32x32_n128() -> Workload:
    """Square lattice, 32x32 = 1024 fibers of radius 0.2*spacing, 128 elements each
    (131072 elements, 262144 unknowns), kH = 20, theta = 30 deg."""
    return square_block(32, 32, 1.0, 0.2, 128, 20.0, math.radians(30.0), name="square_32x32_n128_kH20")


def batch_instances(count: int, seed: int = 1912):
    """Band-gap-sweep style instances: M = 16 fibers (4x4 square or hexagon), radii in
    [0.1,0.35]*spacing, elements per fiber 64..256 growing with radius, kH in
    [0.5, 8], theta in [0, 90 deg) away from Wood anomalies."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        while True:
            kH = rng.uniform(0.5, 8.0)
            theta = rng.uniform(0.0, math.pi / 2)
            if wood_distance(kH, theta) > 1e-3:
                break
        n_of_r = lambda rf: int(round(64 + 192 * (rf - 0.1) / 0.25))
        if i % 2 == 0:
            a = 0.25
            radii = rng.uniform(0.1, 0.35, size=16) * a
            centres = [((ix + 0.5) * a, (iy + 0.5) * a) for ix in range(4) for iy in range(4)]
            npf = [n_of_r(r / a) for r in radii]
            out.append(_from_fibers(f"batch{i}_square4x4", 1.0, 0, kH, theta, centres, radii, npf))
        else:
            out.append(hexagon_block(4, 4, 1.0, 0, kH, theta, int(rng.integers(1 << 30)), r_lo=0.1, r_hi=0.35,
                                     name=f"batch{i}_hexagon4x4", n_of_r=n_of_r))
    return out


def single_fiber(r: float, n: int, k: float, k1: float, rho_ratio: float, theta: float,
                 centre=(0.0, 0.0), H: float = 1.0) -> Workload:
    return Workload(name=f"single_r{r:g}_n{n}", H=H, lattice=0, k=k, k1=k1, rho_ratio=rho_ratio,
                    theta=theta, nodes_per_fiber=np.array([n], dtype=np.int32),
                    nodes=circle_nodes(centre[0], centre[1], r, n),
                    centres=np.array([centre], dtype=np.float64), radii=np.array([r]))


def density_vector(E: int, seed: int) -> np.ndarray:
    """Seeded complex128 test vector of 2E unknowns (phi_e, varphi_e interleaved)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(2 * E) + 1j * rng.standard_normal(2 * E)


def table3_square(ka2pi: float, f: float = 0.35, n: int = 256, c_water: float = 1500.0,
                  name: str | None = None) -> Workload:
    """The water/mercury crystal of Sec. 4 (Table 3, circular scatterers in a
    square lattice): water cylinders in a mercury matrix, lattice constant
    a = 0.5, M_H = 6 rows (period H = 3) by M_L = 4 columns, radius r = a sqrt(f/pi)
    for filling fraction f, n elements per circle, normal incidence d = (1, 0),
    normalised frequency ka/2pi.  k = omega / c_mercury and k1 = omega / c_water
    (Sec. 4 prints c_water = 1500 m/s, hence k = 1.0345 k1); varrho = 13600/1000."""
    a = 0.5
    H = 6 * a
    k = 2.0 * math.pi * ka2pi / a
    r = a * math.sqrt(f / math.pi)
    centres = [((ix + 0.5) * a, (iy + 0.5) * a) for ix in range(4) for iy in range(6)]
    nodes = np.concatenate([circle_nodes(c[0], c[1], r, n) for c in centres])
    return Workload(name=name or f"table3_square_f{f:g}_ka{ka2pi:g}", H=H, lattice=0, k=k,
                    k1=k * C_MERCURY / c_water, rho_ratio=RHO_MERCURY / RHO_WATER, theta=0.0,
                    nodes_per_fiber=np.full(len(centres), n, dtype=np.int32), nodes=nodes,
                    centres=np.asarray(centres), radii=np.full(len(centres), r))


def mercury_water_block(ka2pi: float, f: float = 0.35, ml: int = 4, n: int = 256, c_water: float = 1500.0,
                        rows: int = 12, name: str | None = None) -> Workload:
    """The mercury/water crystal of Sec. 4 (the last experiment): mercury cylinders in a
    water matrix, square lattice of constant a = 0.5, M_L = ml columns, circles of
    radius r = a sqrt(f / pi), n elements each, normal incidence, normalised frequency
    ka/2pi.  k = omega / c_water (matrix) and k1 = omega / c_mercury (fibers);
    varrho = rho_water / rho_mercury.  The crystal repeats along y with period 6a
    (M_H = 6); the fundamental block is taken two periods tall (12 rows, H = 6a), which
    describes the same crystal (at normal incidence the field is 6a-periodic, hence
    also 12a-periodic) and keeps the block's width ml a within H for ml <= 12 (Wood
    anomalies of the taller period: ka/2pi = n/12).  rows = 6 gives the one-period
    block, which for ml > 6 is wider than its period (a row of root squares)."""
    a = 0.5
    H = rows * a
    k = 2.0 * math.pi * ka2pi / a
    r = a * math.sqrt(f / math.pi)
    centres = [((ix + 0.5) * a, (iy + 0.5) * a) for ix in range(ml) for iy in range(rows)]
    nodes = np.concatenate([circle_nodes(c[0], c[1], r, n) for c in centres])
    return Workload(name=name or f"mercury_water_ml{ml}_rows{rows}_f{f:g}_ka{ka2pi:g}", H=H, lattice=0, k=k,
                    k1=k * c_water / C_MERCURY, rho_ratio=RHO_WATER / RHO_MERCURY, theta=0.0,
                    nodes_per_fiber=np.full(len(centres), n, dtype=np.int32), nodes=nodes,
                    centres=np.asarray(centres), radii=np.full(len(centres), r))


def round_square_area(r: float = 1.0) -> float:
    """Area enclosed by the round-square curve of Sec. 4 at scale r: 23 pi r^2 / 2 (Sec. 4)."""
    return 23.0 * math.pi * r * r / 2.0


def table3_block(ka2pi: float, f: float = 0.35, lattice: str = "square", scatterer: str = "circular",
                 n: int = 256, c_water: float = 1500.0, name: str | None = None) -> Workload:
    """The water/mercury crystals of Table 3 (Sec. 4): water scatterers in a mercury
    matrix, lattice constant a = 0.5 (nearest-neighbour spacing), M_H = 6 scatterers
    per column along y (period H = 3) and M_L = 4 columns, normal incidence.
    square: columns at x = (i + 1/2) a; hexagon: columns a sqrt(3)/2 apart, every
    other column shifted by a/2 along y.  The scatterer's area is f times the unit
    cell's (a^2, or a^2 sqrt(3)/2 for the hexagon lattice): a circle of radius r, or
    the round-square curve scaled to that area."""
    a = 0.5
    H = 6 * a
    k = 2.0 * math.pi * ka2pi / a
    if lattice == "square":
        cell = a * a
        centres = [((ix + 0.5) * a, (iy + 0.5) * a) for ix in range(4) for iy in range(6)]
    elif lattice == "hexagon":
        cell = a * a * math.sqrt(3.0) / 2.0
        dx = a * math.sqrt(3.0) / 2.0
        centres = [((ix + 0.5) * dx, (iy + 0.25 + 0.5 * (ix % 2)) * a) for ix in range(4) for iy in range(6)]
    else:
        raise ValueError(lattice)
    if scatterer == "circular":
        r = math.sqrt(f * cell / math.pi)
        nodes = np.concatenate([circle_nodes(c[0], c[1], r, n) for c in centres])
        radius = r
    elif scatterer == "roundsquare":
        r = math.sqrt(f * cell / round_square_area(1.0))
        nodes = np.concatenate([round_square_nodes(c[0], c[1], r, n) for c in centres])
        radius = 3.0 * r
    else:
        raise ValueError(scatterer)
    return Workload(name=name or f"table3_{scatterer}_{lattice}_f{f:g}_ka{ka2pi:g}", H=H,
                    lattice=0 if lattice == "square" else 1, k=k, k1=k * C_MERCURY / c_water,
                    rho_ratio=RHO_MERCURY / RHO_WATER, theta=0.0,
                    nodes_per_fiber=np.full(len(centres), n, dtype=np.int32), nodes=nodes,
                    centres=np.asarray(centres), radii=np.full(len(centres), radius))

