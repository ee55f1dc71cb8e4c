"""The hexagonal lattices that the triangle tree is given for the synthetic
blocks: every fiber centre of the generator lies within its jitter of a point of
the stated lattice (spacing a, lattice vectors (0, a) and (a sqrt 3 / 2, a / 2)),
distinct fibers on distinct points, and the period a multiple of the spacing."""
import math

import numpy as np
import pytest

from paper_1910_10863_gb300 import workloads as W


def _nearest(p, lat):
    a, ox, oy = lat["tri_a"], lat["tri_ox"], lat["tri_oy"]
    e2 = (a * math.sqrt(3.0) / 2.0, a / 2.0)
    v = (p[0] - ox) / e2[0]
    u = (p[1] - oy - v * e2[1]) / a
    best = None
    for vv in range(math.floor(v) - 1, math.floor(v) + 3):
        for uu in range(math.floor(u) - 1, math.floor(u) + 3):
            q = (ox + vv * e2[0], oy + uu * a + vv * e2[1])
            d = math.hypot(p[0] - q[0], p[1] - q[1])
            if best is None or d < best[0]:
                best = (d, uu, vv)
    return best


@pytest.mark.parametrize("ncol,nrow", [(3, 2), (2, 3), (4, 4), (8, 8)])
def test_hexagon_block_lattice(ncol, nrow):
    H = 1.0
    w = W.hexagon_block(ncol, nrow, H, 16, 3.0, 0.3, 5)
    lat = W.hexagon_block_lattice(H, nrow)
    a = lat["tri_a"]
    assert abs(H / a - round(H / a)) < 1e-12 and round(H / a) >= 2
    seen = set()
    for p in w.centres:
        d, u, v = _nearest(p, lat)
        assert d <= 0.05 * a + 1e-12               # the generator's jitter
        key = (u % round(H / a), v)
        assert key not in seen
        seen.add(key)


@pytest.mark.parametrize("lattice", ["hexagon"])
def test_table3_hexagon_lattice(lattice):
    w = W.table3_block(0.45, 0.5, lattice, "circular")
    lat = W.table3_hexagon_lattice()
    assert abs(w.H / lat["tri_a"] - 6) < 1e-12
    for p in w.centres:
        assert _nearest(p, lat)[0] < 1e-12           # no jitter: on the lattice
    # every node within the hexagonal cell of its fiber's point (apothem a / 2)
    nodes = np.asarray(w.nodes).reshape(-1, 2)
    off = np.concatenate([[0], np.cumsum(w.nodes_per_fiber)])
    for i, p in enumerate(w.centres):
        q = nodes[off[i]:off[i + 1]] - p
        for ang in (math.pi / 6, math.pi / 2, 5 * math.pi / 6):
            assert np.max(np.abs(q[:, 0] * math.cos(ang) + q[:, 1] * math.sin(ang))) < 0.5 * lat["tri_a"]
