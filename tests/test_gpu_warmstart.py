"""Learned warm start: network gradients against the FP64 oracle, the Fourier
feature/target/decode kernels, and what the trained network gains over zero-start
GMRES on held-out blocks (M = 16 fibers, band-gap-sweep style)."""
import math

import numpy as np
import pytest

from oracle import mlp as omlp
from paper_1910_10863_gb300 import workloads as W
from tests.gpu_common import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pf():
    ensure_built()
    from paper_1910_10863_gb300 import pfmbem
    return pfmbem


def test_mlp_loss_and_gradient_match_fp64_oracle(pf):
    dims = [50, 256, 256, 256, 1088]
    net = pf.MLP(50, 256, 3, 1088, seed=7)
    rng = np.random.default_rng(0)
    X = rng.standard_normal((16, 50)).astype(np.float32)
    T = rng.standard_normal((16, 1088)).astype(np.float32) * 0.1
    loss, g = net.train(X, T, lr=0.0, want_grad=True)
    p = net.get_params().astype(np.float64)
    lo, go = omlp.loss_and_grad(p, dims, X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - lo) < 1e-5 * abs(lo)
    assert np.linalg.norm(g - go) < 1e-4 * np.linalg.norm(go)
    Y = net.forward(X)
    Yo, _, _ = omlp.forward(p, dims, X)
    assert np.max(np.abs(Y - Yo)) < 1e-4 * np.max(np.abs(Yo))


def test_adam_steps_reduce_the_loss(pf):
    net = pf.MLP(8, 32, 2, 4, seed=1)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((64, 8)).astype(np.float32)
    T = np.tanh(X[:, :4]).astype(np.float32)
    first = net.train(X, T)
    for _ in range(200):
        net.train(X, T, lr=3e-3)
    assert net.train(X, T) < 0.2 * first


def test_warm_targets_and_decode_are_inverse_on_band_limited_densities(pf):
    w = W.batch_instances(2, seed=5)[0]
    s = pf.Solver(w)
    rng = np.random.default_rng(2)
    nm = 8
    coef = (rng.standard_normal((w.M, 2, 2 * nm + 1)) + 1j * rng.standard_normal((w.M, 2, 2 * nm + 1))) * 0.5
    y = np.stack([coef.real, coef.imag], axis=-1).astype(np.float32).ravel()
    psi = np.zeros(2 * s.E, dtype=np.complex128)
    pf.pfmbem_warm_decode(s.h, y, psi, nm)
    t = pf.pfmbem_warm_targets(s.h, psi, w.M, nm)
    assert np.max(np.abs(t - y)) < 1e-5 * np.max(np.abs(y))
    x = pf.pfmbem_warm_features(s.h, w.M)
    assert x.shape == (50,) and abs(x[0] - w.k * w.H / 8) < 1e-6 and abs(x[1] - w.theta / (math.pi / 2)) < 1e-6
    # per-fiber rows: own radius, the nearest neighbour first, periodic images along y
    xl = pf.pfmbem_warm_features_local(s.h, w.M, 15)
    assert xl.shape == (w.M, 50)
    c, r = w.centres, w.radii
    for i in range(w.M):
        assert abs(xl[i, 2] - 4 * r[i] / w.H) < 1e-5
        d = []
        for j in range(w.M):
            if j != i:
                dy = c[j, 1] - c[i, 1]
                dy -= w.H * round(dy / w.H)
                d.append(math.hypot(c[j, 0] - c[i, 0], dy))
        nb = xl[i, 5:].reshape(15, 3)
        dist = np.hypot(nb[:, 0], nb[:, 1]) * w.H / 4
        assert np.all(np.diff(dist) >= -1e-6) and abs(dist[0] - min(d)) < 1e-5


def test_trained_network_reduces_gmres_iterations_on_held_out_blocks(pf):
    from paper_1910_10863_gb300 import warmstart as ws
    train = W.batch_instances(320, seed=101)
    test = W.batch_instances(24, seed=202)
    X, T, _, _ = ws.generate(train)
    net, hist = ws.train(X, T, epochs=150, batch=64, lr=2e-3, seed=3)
    assert hist[-1] < 0.5 * hist[0]
    rows = ws.evaluate(net, test)
    iz, iw, res0 = rows[:, 0], rows[:, 1], rows[:, 2]
    assert np.all(rows[:, 3] <= 1e-6) and np.all(rows[:, 4] <= 1e-6)     # both solves converge
    assert np.median(res0) < 1.0                                         # the guess beats a zero start
    assert iw.mean() < iz.mean()


def test_batched_warm_start_on_held_out_blocks(pf):
    """The whole pipeline in one batch: features of every held-out block, one
    forward pass, decode, one persistent solve with the guesses; fewer iterations
    than the batched zero start, the same solutions, both converged, and the
    warm-started solutions' residual judged by the oracle on sampled rows."""
    from paper_1910_10863_gb300 import warmstart as ws
    train = W.batch_instances(320, seed=101)
    test = W.batch_instances(24, seed=202)
    X, T, _, _ = ws.generate_batched(train)
    net, hist = ws.train(X, T, epochs=150, batch=64, lr=2e-3, seed=3)
    r = ws.evaluate_batched(net, test, fp64_sample=4, keep=2)
    assert r["status_zero"] == 0 and r["status_warm"] == 0
    assert r["max_rel_residual_warm"] <= 1e-6 and r["max_rel_residual_fp64"] <= 1e-6
    assert r["mean_iters_warm"] < r["mean_iters_zero"]
    assert r["max_rel_diff_warm_vs_zero"] < 1e-4
    # judged by the oracle: its residual of two warm-started solutions on sampled
    # element rows (exact element integrals, Ewald G_qp), at the solve tolerance
    from oracle import bem
    rng = np.random.default_rng(9)
    for w, psi in zip(test[:2], r["solutions"]):
        pb = bem.problem(w)
        sel = np.sort(rng.choice(w.E, size=6, replace=False))
        rows = bem.operator_rows(pb, sel)
        eq = np.stack([2 * sel, 2 * sel + 1], axis=1).ravel()
        B = bem.rhs(pb)[eq]
        assert np.linalg.norm(B - rows @ psi) / np.linalg.norm(B) < 5e-6
