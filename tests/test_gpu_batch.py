"""Batched solve of a band-gap sweep: every instance solved inside one
persistent launch (groups of blocks taking instances longest first), against
dense LU of the oracle, with uneven element counts, mixed-precision and FP64
handles in the same batch, and the host-driven lockstep as a second path."""
import math
import os

import numpy as np
import pytest

from oracle import bem
from paper_1910_10863_gb300 import workloads as W
from tests.gpu_common import ensure_built, rel

pytestmark = pytest.mark.gpu


def _sweep_blocks(count=16):
    """Square and hexagon blocks of 4 or 9 fibers whose radii set 14..60
    elements per fiber, frequencies kH in [0.6, 7.5] and angles in [0, 80) deg
    (seeded; Wood anomalies resampled)."""
    rng = np.random.default_rng(20)
    ws = []
    while len(ws) < count:
        i = len(ws)
        kH = float(rng.uniform(0.6, 7.5))
        th = float(rng.uniform(0.0, 80.0))
        s = math.sin(math.radians(th))
        if min(abs(v - 2 * math.pi * round(v / (2 * math.pi))) for v in (kH * (1 + s), kH * (1 - s))) < 1e-2:
            continue
        nf = 2 if i % 2 == 0 else 3
        n_of_r = (lambda lo, hi: (lambda rf: lo + int(round(hi * rf))))(14 + 2 * (i % 5), 20 + 2 * i)
        if i % 2 == 0:
            ws.append(W.hexagon_block(nf, nf, 1.0, 0, kH, math.radians(th), seed=100 + i, n_of_r=n_of_r,
                                      name=f"hex{i}"))
        else:
            ws.append(W.hexagon_block(nf, nf, 1.0, 0, kH, math.radians(th), seed=200 + i, n_of_r=n_of_r,
                                      name=f"hexb{i}"))
    return ws


@pytest.fixture(scope="module")
def sweep():
    ensure_built()
    ws = _sweep_blocks()
    refs = []
    for w in ws:
        pb = bem.problem(w)
        refs.append(np.linalg.solve(bem.operator_rows(pb), bem.rhs(pb)))
    return ws, refs


def _solve(ws, precisions, tol, streams=True):
    import torch

    from paper_1910_10863_gb300 import pfmbem as pf
    sts = [torch.cuda.Stream() for _ in ws] if streams else [None] * len(ws)
    solvers = [pf.Solver(w, precision=p, stream=(s.cuda_stream if s is not None else None))
               for w, p, s in zip(ws, precisions, sts)]
    psis = [np.zeros(2 * s.E, dtype=np.complex128) for s in solvers]
    st, infos = pf.pfmbem_solve_batch([s.h for s in solvers], psis, tol=tol, maxit=2000)
    return st, infos, psis, solvers


def test_batch_solve_matches_dense_lu(sweep):
    """16 uneven instances (64..450 elements), three of them FP64 handles, in one
    persistent launch: every instance reaches the tolerance and its densities
    agree with the oracle's dense LU solution."""
    from paper_1910_10863_gb300 import pfmbem as pf
    ws, refs = sweep
    E = [sum(w.nodes_per_fiber) for w in ws]
    assert len(ws) >= 16 and max(E) > 3 * min(E)
    precisions = [pf.FP64 if i % 5 == 2 else pf.MIXED for i in range(len(ws))]
    st, infos, psis, _ = _solve(ws, precisions, 1e-9)
    assert st == 0
    for w, psi, info, ref in zip(ws, psis, infos, refs):
        assert info.status == 0 and info.rel_residual <= 1e-9, w.name
        assert rel(psi, ref) < 1e-6, w.name


def test_batch_matches_single_solves_and_lockstep(sweep):
    """The persistent launch and the host-driven lockstep give the same
    solutions as one pfmbem_solve per instance (to the solve tolerance)."""
    import subprocess
    import sys
    from paper_1910_10863_gb300 import pfmbem as pf
    ws, refs = sweep
    ws = ws[:8]
    st, infos, psis, solvers = _solve(ws, [pf.MIXED] * len(ws), 1e-10, streams=False)
    assert st == 0
    for s, psi in zip(solvers, psis):
        one = np.zeros_like(psi)
        s.solve(one, tol=1e-10, maxit=2000)
        assert rel(psi, one) < 1e-7
    # the lockstep path (PFMBEM_BATCH_LOCKSTEP is read once per process: a child)
    code = (
        "import numpy as np, json, sys\n"
        "sys.path.insert(0, %r)\n"
        "from tests.test_gpu_batch import _sweep_blocks, _solve\n"
        "from paper_1910_10863_gb300 import pfmbem as pf\n"
        "ws = _sweep_blocks()[:8]\n"
        "st, infos, psis, _ = _solve(ws, [pf.MIXED] * len(ws), 1e-10, streams=False)\n"
        "np.save(sys.argv[1], np.concatenate(psis))\n"
        "print(st)\n" % os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import tempfile
    with tempfile.TemporaryDirectory() as td:
        out = os.path.join(td, "lock.npy")
        env = dict(os.environ, PFMBEM_BATCH_LOCKSTEP="1")
        r = subprocess.run([sys.executable, "-c", code, out], env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        assert r.stdout.strip().splitlines()[-1] == "0"
        lock = np.load(out)
    assert rel(np.concatenate(psis), lock) < 1e-7


def test_batch_wait_that_runs_out_returns_etimeout(pf=None):
    """Every group barrier of the persistent launch is bounded by
    options.wait_us; with 1 us a wait runs out, the launch ends early and the
    batch returns PFMBEM_ETIMEOUT for its instances (no trap, no unbounded wait).
    A following batch with the default bound solves."""
    ensure_built()
    from paper_1910_10863_gb300 import pfmbem as pf
    ws = _sweep_blocks(4)
    solvers = [pf.Solver(w, precision=pf.MIXED, wait_us=1) for w in ws]
    psis = [np.zeros(2 * s.E, dtype=np.complex128) for s in solvers]
    st, infos = pf.pfmbem_solve_batch([s.h for s in solvers], psis, tol=1e-8, maxit=500)
    assert st == 7                                # PFMBEM_ETIMEOUT
    assert all(i.status == 7 for i in infos)
    solvers = [pf.Solver(w, precision=pf.MIXED) for w in ws]
    psis = [np.zeros(2 * s.E, dtype=np.complex128) for s in solvers]
    st, infos = pf.pfmbem_solve_batch([s.h for s in solvers], psis, tol=1e-8, maxit=500)
    assert st == 0 and all(i.rel_residual <= 1e-8 for i in infos)


def test_batch_with_initial_guesses_matches_dense_lu(sweep):
    """use_guess: every block starts from a perturbed copy of its dense-LU solution
    (scaled by the residual-minimising gamma on the device); one of them from
    large random noise, which the scaling reduces to almost nothing.  All reach
    the tolerance and the oracle's solution."""
    import torch
    from paper_1910_10863_gb300 import pfmbem as pf
    ws, refs = sweep
    ws, refs = ws[:6], refs[:6]
    rng = np.random.default_rng(4)
    solvers = [pf.Solver(w, precision=pf.FP64 if i == 3 else pf.MIXED) for i, w in enumerate(ws)]
    guesses = []
    for i, ref in enumerate(refs):
        noise = rng.standard_normal(ref.shape) + 1j * rng.standard_normal(ref.shape)
        g = 0.7 * ref + 1e-2 * np.linalg.norm(ref) / math.sqrt(ref.size) * noise
        if i == 5:
            g = 1e3 * noise                      # no better than a zero start
        guesses.append(torch.from_numpy(np.ascontiguousarray(g)).cuda())
    st, infos = pf.pfmbem_solve_batch([s.h for s in solvers], guesses, tol=1e-9, maxit=2000, use_guess=True)
    assert st == 0
    for g, ref, info in zip(guesses, refs, infos):
        assert info.rel_residual <= 1e-9
        assert rel(g.cpu().numpy(), ref) < 1e-6
