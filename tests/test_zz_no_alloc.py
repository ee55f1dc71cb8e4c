"""Allocation-free lattice sums against the handle-based entry point.

pfmbem_lattice_sums_noalloc serves callers that cannot allocate device memory
(for example code being recorded by CUDA stream capture, or code confined to
another framework's memory pool): it computes the lattice sums of the periodic
root translation into a fixed array inside the library.  Two calls in a row,
with different parameters, must each reproduce pfmbem_lattice_sums of a solver
handle built for the same (k, H, theta) to the tolerance of the lattice-sum
parity test, with host and with device output buffers.  This file is collected
last so that a failure here cannot hide the result of any other test.
"""
import math

import numpy as np
import pytest

from paper_1910_10863_gb300 import workloads as W
from tests.gpu_common import ensure_built

pytestmark = pytest.mark.gpu


def _reference(pf, kH, theta, jmax):
    w = W.square_2x2_n64()
    w.k = kH / w.H
    w.k1 = w.k * 1490 / 1450
    w.theta = theta
    s = pf.Solver(w, p=12, depth=2)
    S = np.zeros(2 * jmax + 1, dtype=np.complex128)
    pf.pfmbem_lattice_sums(s.h, jmax, S)
    s.close()
    return w.k, w.H, S


def test_noalloc_lattice_sums_match_handle_entry_point_twice():
    ensure_built()
    import torch

    from paper_1910_10863_gb300 import pfmbem as pf
    cases = [(2.0, math.radians(30), 24), (5.0, 0.3, 40)]
    for kH, theta, jmax in cases:                     # two calls in a row
        k, H, ref = _reference(pf, kH, theta, jmax)
        got = np.zeros(2 * jmax + 1, dtype=np.complex128)
        pf.pfmbem_lattice_sums_noalloc(k, H, theta, jmax, got)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(got - ref)) <= 1e-10 * scale
        dev = torch.zeros(2 * jmax + 1, dtype=torch.complex128, device="cuda")
        pf.pfmbem_lattice_sums_noalloc(k, H, theta, jmax, dev, stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert np.max(np.abs(dev.cpu().numpy() - ref)) <= 1e-10 * scale


def test_noalloc_rejects_orders_beyond_the_fixed_array():
    ensure_built()
    from paper_1910_10863_gb300 import pfmbem as pf
    out = np.zeros(2 * 200 + 1, dtype=np.complex128)
    with pytest.raises(pf.PfmbemError) as e:
        pf.pfmbem_lattice_sums_noalloc(2.0, 1.0, 0.5, 129, out)
    assert e.value.status == 1
