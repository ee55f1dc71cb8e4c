"""Shared helpers of the GPU parity tests (not collected as tests)."""
import math
import os

import numpy as np

from paper_1910_10863_gb300 import workloads as W


def ensure_built():
    from paper_1910_10863_gb300 import build, pfmbem
    if not os.path.exists(pfmbem.LIB_PATH):
        build.build()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def hexagon_4x4_ragged():
    """Hexagon block of 16 fibers whose radii (0.1..0.3 spacing) set 28..36 elements each;
    odd columns straddle the period cell, so elements wrap into the root box."""
    return W.hexagon_block(4, 4, 1.0, 0, 3.0, math.radians(17.0), seed=5,
                           n_of_r=lambda rf: 24 + int(round(40 * rf)), name="hexagon_4x4_ragged_kH3")
