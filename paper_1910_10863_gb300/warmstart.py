"""Learned GMRES warm start: data, training and evaluation drivers.

The network maps the block's parameters (pfmbem_warm_features: kH, theta and
every fiber's centre and radius) to the Fourier modes n = -8..8 of both
densities on every fiber (pfmbem_warm_targets, divided by the incident phase at
the fiber centre).  Training data are solutions produced by the solver itself;
forward, backward and Adam run in the library's kernels (pfmbem_mlp_*).  A
prediction is decoded (pfmbem_warm_decode) and passed to pfmbem_solve as the
initial guess; the solver falls back to a zero start when the guess's FP64
residual is not below ||B||.
"""
from __future__ import annotations

import numpy as np

from . import pfmbem as pf

NMODES = 8


def solve_instance(w, guess=None, tol=1e-6, maxit=2000, precision=pf.MIXED):
    """Solve one block; returns (psi, info, solver)."""
    s = pf.Solver(w, precision=precision)
    psi = np.zeros(2 * s.E, dtype=np.complex128)
    if guess is not None:
        psi[:] = guess
    info = s.solve(psi, tol=tol, maxit=maxit, use_guess=guess is not None, check=False)
    return psi, info, s


def generate(instances, tol=1e-6):
    """Features X [n][2+3M], targets T [n][M*2*17*2] and zero-start iteration counts."""
    X, T, iters = [], [], []
    for w in instances:
        psi, info, s = solve_instance(w, tol=tol)
        X.append(pf.pfmbem_warm_features(s.h, w.M))
        T.append(pf.pfmbem_warm_targets(s.h, psi, w.M, NMODES))
        iters.append(info.iters)
        s.close()
    return np.array(X, dtype=np.float32), np.array(T, dtype=np.float32), np.array(iters)


def train(X, T, hidden=256, layers=3, epochs=200, batch=256, lr=1e-3, seed=1913, log_every=0):
    """Adam on the mean-squared error; returns the network and the loss history."""
    net = pf.MLP(X.shape[1], hidden, layers, T.shape[1], seed=seed)
    rng = np.random.default_rng(seed)
    hist = []
    n = X.shape[0]
    for ep in range(epochs):
        perm = rng.permutation(n)
        tot = 0.0
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            tot += net.train(X[idx], T[idx], lr=lr) * len(idx)
        hist.append(tot / n)
        if log_every and ep % log_every == 0:
            print(f"epoch {ep} loss {hist[-1]:.4e}", flush=True)
    return net, hist


def main():
    """Train on --train band-gap-sweep blocks (M = 16) and report the gain on
    --test held-out blocks drawn from a disjoint seed; one JSON line."""
    import argparse
    import json
    import time

    from . import workloads as W
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=8192)
    ap.add_argument("--test", type=int, default=1024)
    ap.add_argument("--epochs", type=int, default=100)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--tol", type=float, default=1e-6)
    a = ap.parse_args()
    t0 = time.perf_counter()
    X, T, _ = generate(W.batch_instances(a.train, seed=1912), tol=a.tol)
    t1 = time.perf_counter()
    net, hist = train(X, T, epochs=a.epochs, batch=a.batch, lr=a.lr)
    t2 = time.perf_counter()
    rows = evaluate(net, W.batch_instances(a.test, seed=1915), tol=a.tol)
    t3 = time.perf_counter()
    iz, iw, r0 = rows[:, 0], rows[:, 1], rows[:, 2]
    print(json.dumps({
        "train_blocks": a.train, "test_blocks": a.test, "epochs": a.epochs, "final_loss": hist[-1],
        "first_loss": hist[0], "mean_iters_zero_start": float(iz.mean()), "mean_iters_warm_start": float(iw.mean()),
        "median_warm_start_residual": float(np.median(r0)), "fraction_guess_kept": float(np.mean(r0 < 1.0)),
        "mean_solve_ms_zero": float(rows[:, 5].mean()), "mean_solve_ms_warm": float(rows[:, 6].mean()),
        "all_converged": bool(np.all(rows[:, 3] <= a.tol) and np.all(rows[:, 4] <= a.tol)),
        "seconds": {"data": t1 - t0, "train": t2 - t1, "evaluate": t3 - t2}}), flush=True)


def evaluate(net, instances, tol=1e-6):
    """Per instance: zero-start and warm-start GMRES iterations and the FP64
    relative residual of the warm start itself."""
    rows = []
    for w in instances:
        s = pf.Solver(w, precision=pf.MIXED)
        x = pf.pfmbem_warm_features(s.h, w.M)
        y = net.forward(x[None, :])[0]
        psi0 = np.zeros(2 * s.E, dtype=np.complex128)
        pf.pfmbem_warm_decode(s.h, y, psi0, NMODES)
        B = np.zeros_like(psi0)
        s.rhs(B)
        r0 = np.zeros_like(psi0)
        s.matvec(psi0, r0, pf.FP64)
        res0 = float(np.linalg.norm(B - r0) / np.linalg.norm(B))
        psi = np.zeros_like(psi0)
        iz = s.solve(psi, tol=tol, check=False)
        psi_w = psi0.copy()
        iw = s.solve(psi_w, tol=tol, use_guess=True, check=False)
        rows.append((iz.iters, iw.iters, res0, iz.rel_residual, iw.rel_residual, iz.ms, iw.ms))
        s.close()
    return np.array(rows)


if __name__ == "__main__":
    main()
