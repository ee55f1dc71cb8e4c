"""Oracle quadtree rules (test infrastructure): which boxes interact by M2L, and
the convergence factors of Sec. 3.2 (Theorems 1-2, Table 1), for the square tree
and for the regular-triangle tree of hexagon lattices (Sec. 3.1, Fig. 5; the GPU
path builds the square tree for both lattices).

Square tree over the root cell of side H (the y-period): level l has 2^l x 2^l
boxes of side H / 2^l, indexed (ix, iy).  Along y the block repeats, so a box
seen through the images m = -1, 0, 1 of the root (Sec. 3.1: adjacent basic
trees share a vertex and take part in the ordinary lists) is addressed by its
index in the root and its image m; along x nothing wraps.

M2L list of a target box (the classical rule, Sec. 3.1 "traditional way"):
the children of its parent's neighbours (the parent's own 3 x 3 neighbourhood,
images included) that are not neighbours of the target itself.
"""
from __future__ import annotations

import math


def interaction_list(level, ix, iy):
    """Sources (sx, sy, m) of the M2L list of box (ix, iy) at level >= 2, where
    (sx, sy) is the box inside the root and m its image (source centre shifted
    by m H along y)."""
    nl = 1 << level
    px, py = ix >> 1, iy >> 1
    out = []
    for qx in (px - 1, px, px + 1):
        if qx < 0 or qx >= nl // 2:
            continue
        for qy in (py - 1, py, py + 1):
            for cx in (0, 1):
                for cy in (0, 1):
                    sx, sy = 2 * qx + cx, 2 * qy + cy
                    if abs(ix - sx) <= 1 and abs(iy - sy) <= 1:
                        continue
                    out.append((sx, sy % nl, sy // nl))
    return out


def gamma_lambda(offset, size_c, size_d=1.0):
    """gamma (Theorem 1) and lambda (Theorem 2) for a target cell D of side size_d whose
    centre sits at `offset` from the centre O_C of a source cell C of side size_c
    (axis-aligned squares):

        gamma  = max_{y in C} |y - O_C| / min_{x in D} |x - O_C|,
        lambda = max_{x in D} |x - O_D| / |O_D - O_C| * exp(3 max_{y in C} |y - O_C| / (2 |O_D - O_C|)).
    """
    rC = size_c / math.sqrt(2.0)
    rD = size_d / math.sqrt(2.0)
    ox, oy = offset
    nx = max(abs(ox) - size_d / 2, 0.0)
    ny = max(abs(oy) - size_d / 2, 0.0)
    gamma = rC / math.hypot(nx, ny)
    R = math.hypot(ox, oy)
    lam = rD / R * math.exp(1.5 * rC / R)
    return gamma, lam


def symmetric_tree_factors(level=3):
    """(gamma, lambda, tau) of the symmetric square tree (source and target cells on
    one level, Table 1's L = 0): the worst case over every M2L pair of the level,
    in units of the box side."""
    nl = 1 << level
    g = lam = 0.0
    for ix in range(nl):
        for iy in range(nl):
            for sx, sy, m in interaction_list(level, ix, iy):
                off = (ix - sx, iy - (sy + m * nl))
                a, b = gamma_lambda(off, 1.0, 1.0)
                g, lam = max(g, a), max(lam, b)
    return g, lam, max(g, lam)


# ------------------------------------------------------------ regular-triangle tree
# Sec. 3.1 (Fig. 5): the hexagonal unit cell (level 0) splits into six equilateral
# triangles (level 1), each of which splits into four (level 2, ...); the cells of
# one level tile the plane as the regular triangular tiling.  Here a cell of side s
# is (i, j, up): the triangle with corner s (i e1 + j e2), e1 = (1, 0),
# e2 = (1/2, sqrt(3)/2), pointing up or down in its rhombus.  The cell's centre O is
# its centroid and its radius the circumradius s / sqrt(3).

_E1 = (1.0, 0.0)
_E2 = (0.5, math.sqrt(3.0) / 2.0)


def triangle_vertices(i, j, up, s=1.0):
    ox, oy = s * (i * _E1[0] + j * _E2[0]), s * (i * _E1[1] + j * _E2[1])
    a = (ox + s * _E1[0], oy + s * _E1[1])
    b = (ox + s * _E2[0], oy + s * _E2[1])
    if up:
        return [(ox, oy), a, b]
    return [a, (a[0] + s * _E2[0], a[1] + s * _E2[1]), b]


def triangle_centre(v):
    return (sum(p[0] for p in v) / 3.0, sum(p[1] for p in v) / 3.0)


def point_triangle_distance(p, v):
    """Distance from point p to the closed triangle v (0 inside)."""
    def cross(o, a, b):
        return (a[0] - o[0]) * (b[1] - o[1]) - (a[1] - o[1]) * (b[0] - o[0])
    d = [cross(v[k], v[(k + 1) % 3], p) for k in range(3)]
    if all(x >= -1e-12 for x in d) or all(x <= 1e-12 for x in d):
        return 0.0
    best = float("inf")
    for k in range(3):
        a, b = v[k], v[(k + 1) % 3]
        ex, ey = b[0] - a[0], b[1] - a[1]
        t = max(0.0, min(1.0, ((p[0] - a[0]) * ex + (p[1] - a[1]) * ey) / (ex * ex + ey * ey)))
        best = min(best, math.hypot(p[0] - a[0] - t * ex, p[1] - a[1] - t * ey))
    return best


def triangle_parent(cell, s=1.0):
    """The cell of side 2 s that contains the cell of side s."""
    cx, cy = triangle_centre(triangle_vertices(*cell, s))
    b = cy / (2 * s * _E2[1])
    a = cx / (2 * s) - b / 2
    i, j = math.floor(a), math.floor(b)
    return (i, j, (a - i) + (b - j) < 1.0)


def _touch(v, w):
    return min(min(point_triangle_distance(p, w) for p in v), min(point_triangle_distance(p, v) for p in w)) < 1e-9


def triangle_gamma_lambda(src, s_src, dst, s_dst):
    """gamma and lambda of Theorems 1-2 for source cell src (side s_src) and
    target cell dst (side s_dst), each (i, j, up): gamma = r_C / min_{x in D}
    |x - O_C|, lambda = r_D / |O_D - O_C| exp(3 r_C / (2 |O_D - O_C|)), r the
    circumradius."""
    vs, vd = triangle_vertices(*src, s_src), triangle_vertices(*dst, s_dst)
    oc, od = triangle_centre(vs), triangle_centre(vd)
    rc, rd = s_src / math.sqrt(3.0), s_dst / math.sqrt(3.0)
    R = math.hypot(od[0] - oc[0], od[1] - oc[1])
    dmin = point_triangle_distance(oc, vd)
    gamma = rc / dmin if dmin > 0 else float("inf")
    return gamma, (rd / R * math.exp(1.5 * rc / R) if R > 0 else float("inf"))


def triangle_interaction_list(dst, span=6):
    """Same-level sources (side 1) of target cell dst: the children of the cells
    that touch dst's parent (side 2), less the cells that touch dst (Sec. 3.1,
    'quite similar to that in the square tree')."""
    pd = triangle_vertices(*triangle_parent(dst), 2.0)
    vd = triangle_vertices(*dst, 1.0)
    out = []
    for i in range(-span, span + 1):
        for j in range(-span, span + 1):
            for up in (True, False):
                c = (i, j, up)
                if not _touch(triangle_vertices(*triangle_parent(c), 2.0), pd):
                    continue
                if _touch(triangle_vertices(*c, 1.0), vd):
                    continue
                out.append(c)
    return out
