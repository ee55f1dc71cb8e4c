"""Oracle quadtree rules (test infrastructure): which boxes interact by M2L, and
the convergence factors of Sec. 3.2 (Theorems 1-2, Table 1).

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
