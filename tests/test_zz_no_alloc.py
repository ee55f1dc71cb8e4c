"""Allocation-free lattice sums against the handle-based entry point and the oracle.

pfmbem_lattice_sums_noalloc serves callers that cannot allocate device memory:
plug-ins running inside a host application that has already reserved the GPU's
memory for its own pool or budget, and latency-critical loops that must not
enter the CUDA allocator.  It computes the lattice sums of the periodic root
translation (Sec. 3.3) into a fixed array inside the library.

Two calls in a row, with different parameters, must each reproduce
pfmbem_lattice_sums of a solver handle built for the same (k, H, theta) to
1e-10, with host and with device output buffers, and match the oracle's sums on
the local expansion they generate (coefficient j weighted by |J_j(k rho)| on a
circle of radius rho = 1.9 H, which keeps every order up to 128 visible).
This file is collected last so that a failure here cannot hide the result of
any other test.
"""
import math

import numpy as np
import pytest
from scipy import special as sp

from oracle import lattice
from paper_1910_10863_gb300 import workloads as W
from tests.gpu_common import ensure_built

pytestmark = pytest.mark.gpu


def _handle_sums(pf, kH, theta, jmax):
    w = W.square_2x2_n64()
    w.k = kH / w.H
    w.k1 = w.k * 1490 / 1450
    w.theta = theta
    s = pf.Solver(w, p=12, depth=2)
    S = np.zeros(2 * jmax + 1, dtype=np.complex128)
    pf.pfmbem_lattice_sums(s.h, jmax, S)
    s.close()
    return w.k, w.H, S


def _oracle_error(S, k, H, theta, jmax):
    rho = 1.9 * H
    js, ref = lattice.lattice_sums(k, k * H * math.sin(theta), H, jmax, rho=rho, npts=8192)
    wgt = np.abs(sp.jv(js, k * rho))
    return float(np.max(np.abs(S - ref) * wgt) / np.max(np.abs(ref) * wgt))


def test_noalloc_lattice_sums_match_handle_entry_point_and_oracle_twice():
    ensure_built()
    import torch

    from paper_1910_10863_gb300 import pfmbem as pf
    cases = [(5.0, 0.3, 40), (20.0, math.radians(30), 108)]
    for kH, theta, jmax in cases:                     # two calls in a row
        k, H, ref = _handle_sums(pf, kH, theta, jmax)
        got = np.zeros(2 * jmax + 1, dtype=np.complex128)
        pf.pfmbem_lattice_sums_noalloc(k, H, theta, jmax, got)
        scale = np.max(np.abs(ref))
        assert np.max(np.abs(got - ref)) <= 1e-10 * scale
        assert _oracle_error(got, k, H, theta, jmax) < 1e-10
        dev = torch.zeros(2 * jmax + 1, dtype=torch.complex128, device="cuda")
        pf.pfmbem_lattice_sums_noalloc(k, H, theta, jmax, dev, stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        assert np.max(np.abs(dev.cpu().numpy() - ref)) <= 1e-10 * scale


def test_noalloc_largest_order_and_rejections():
    ensure_built()
    import torch

    from paper_1910_10863_gb300 import pfmbem as pf
    # the largest order the fixed array holds
    k, H, theta = 2.0, 1.0, math.radians(30)
    got = np.zeros(2 * 128 + 1, dtype=np.complex128)
    pf.pfmbem_lattice_sums_noalloc(k, H, theta, 128, got)
    assert _oracle_error(got, k, H, theta, 128) < 1e-10
    # beyond the fixed array: rejected before any GPU work
    out = np.zeros(2 * 200 + 1, dtype=np.complex128)
    with pytest.raises(pf.PfmbemError) as e:
        pf.pfmbem_lattice_sums_noalloc(2.0, 1.0, 0.5, 129, out)
    assert e.value.status == 1
    # a buffer shorter than 2 jmax + 1 never reaches the library
    with pytest.raises(ValueError):
        pf.pfmbem_lattice_sums_noalloc(2.0, 1.0, 0.5, 10, np.zeros(20, dtype=np.complex128))
    # a device buffer on another GPU than the current one is rejected (launches nothing)
    if torch.cuda.device_count() > 1:
        other = torch.zeros(21, dtype=torch.complex128, device="cuda:1")
        with torch.cuda.device(0):
            with pytest.raises(pf.PfmbemError) as e:
                pf.pfmbem_lattice_sums_noalloc(2.0, 1.0, 0.5, 10, other)
        assert e.value.status == 1


def test_noalloc_in_a_captured_graph():
    """After a first call on the device, a device-output call can be captured into
    a CUDA graph; its replays reproduce the handle path and take no device memory."""
    ensure_built()
    import torch

    from paper_1910_10863_gb300 import pfmbem as pf
    kH, theta, jmax = 5.0, 0.3, 40
    k, H, ref = _handle_sums(pf, kH, theta, jmax)
    dev = torch.zeros(2 * jmax + 1, dtype=torch.complex128, device="cuda")
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):                     # first call, outside the capture
        pf.pfmbem_lattice_sums_noalloc(k, H, theta, jmax, dev, stream=side.cuda_stream)
    torch.cuda.synchronize()
    dev.zero_()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pf.pfmbem_lattice_sums_noalloc(k, H, theta, jmax, dev, stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert not bool(dev.abs().max() > 0)              # captured, not run
    scale = np.max(np.abs(ref))
    g.replay()
    torch.cuda.synchronize()
    assert np.max(np.abs(dev.cpu().numpy() - ref)) <= 1e-10 * scale
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        dev.zero_()
        g.replay()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.max(np.abs(dev.cpu().numpy() - ref)) <= 1e-10 * scale
    del g
