"""Learned GMRES warm start: data, training and evaluation drivers.

Two models share the drivers below.  "global" (default): the network maps the
block's parameters (pfmbem_warm_features: kH, theta and every fiber's centre and
radius) to the Fourier modes n = -8..8 of both densities on every fiber
(pfmbem_warm_targets: angles measured from the incidence direction,
coefficients divided by the incident phase at the fiber centre).  "local": the
network maps one fiber's row of pfmbem_warm_features_local (kH, theta, its
radius, its distances to the block's edges and the relative positions and radii
of its 15 nearest neighbours) to that fiber's modes; the same weights serve
every fiber, so a block of M fibers gives M training rows.  Training data are solutions produced by the solver itself; forward,
backward and Adam run in the library's kernels (pfmbem_mlp_*).  A prediction is
decoded (pfmbem_warm_decode) and passed to pfmbem_solve as the initial guess,
which scales it by the residual-minimising factor and falls back to a zero start
when even the scaled guess's FP64 residual is not below ||B||.
"""
from __future__ import annotations

import numpy as np

from . import pfmbem as pf

NMODES = 8
NEIGHBOURS = 15
NOUT = 2 * (2 * NMODES + 1) * 2          # per fiber: 2 densities x 17 complex modes
MODEL = "global"


def solve_instance(w, guess=None, tol=1e-6, maxit=2000, precision=pf.MIXED):
    """Solve one block; returns (psi, info, solver)."""
    s = pf.Solver(w, precision=precision)
    psi = np.zeros(2 * s.E, dtype=np.complex128)
    if guess is not None:
        psi[:] = guess
    info = s.solve(psi, tol=tol, maxit=maxit, use_guess=guess is not None, check=False)
    return psi, info, s


def features(s, M, model=None):
    """Network input rows of one block: one row (global) or one row per fiber (local)."""
    if (model or MODEL) == "local":
        return pf.pfmbem_warm_features_local(s.h, M, NEIGHBOURS)
    return pf.pfmbem_warm_features(s.h, M)[None, :]


def targets(s, psi, M, model=None):
    t = pf.pfmbem_warm_targets(s.h, psi, M, NMODES)
    return t.reshape(M, NOUT) if (model or MODEL) == "local" else t.reshape(1, -1)


def generate(instances, tol=1e-6, model=None):
    """Rows of features X and targets T (one per block, or one per fiber for the
    local model), the block index of every row and the zero-start iterations."""
    X, T, inst, iters = [], [], [], []
    for q, w in enumerate(instances):
        psi, info, s = solve_instance(w, tol=tol)
        x = features(s, w.M, model)
        X.append(x)
        T.append(targets(s, psi, w.M, model))
        inst.append(np.full(x.shape[0], q))
        iters.append(info.iters)
        s.close()
    return (np.concatenate(X).astype(np.float32), np.concatenate(T).astype(np.float32), np.concatenate(inst),
            np.array(iters))


def _create_all(instances, precision=pf.MIXED, threads=16):
    """Handles of many blocks, created on a pool of host threads."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(threads) as ex:
        return list(ex.map(lambda w: pf.Solver(w, precision=precision), instances))


def generate_batched(instances, tol=1e-6, model=None, chunk=256):
    """As generate, with the blocks solved in persistent batched launches of
    chunk blocks (the training data of a sweep come at the batched rate)."""
    import torch
    X, T, inst, iters = [], [], [], []
    for c0 in range(0, len(instances), chunk):
        part = instances[c0:c0 + chunk]
        sols = _create_all(part)
        psis = [torch.zeros(2 * s.E, dtype=torch.complex128, device="cuda") for s in sols]
        st, infos = pf.pfmbem_solve_batch([s.h for s in sols], psis, tol=tol)
        for q, (w, s, psi, info) in enumerate(zip(part, sols, psis, infos)):
            p = psi.cpu().numpy()
            x = features(s, w.M, model)
            X.append(x)
            T.append(targets(s, p, w.M, model))
            inst.append(np.full(x.shape[0], c0 + q))
            iters.append(info.iters)
            s.close()
    return (np.concatenate(X).astype(np.float32), np.concatenate(T).astype(np.float32), np.concatenate(inst),
            np.array(iters))


def evaluate_batched(net, instances, tol=1e-6, model=None, fp64_sample=32, keep=0):
    """The whole warm-start pipeline on many held-out blocks at once: features of
    every block, one forward pass of the network over all of them, decode, and one
    persistent batched solve with the guesses; against the same blocks solved in
    one batch from zero, and against plain FP64 GMRES (one pfmbem_solve after
    another, FP64 handles, on the first fp64_sample blocks).  Times in seconds,
    handles created beforehand (outside every timed region).  keep > 0 adds the
    first keep warm-started solutions (host arrays) under "solutions"."""
    import time

    import torch
    tc = time.perf_counter()
    sols = _create_all(instances)
    n = len(sols)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - tc
    # zero start (after one untimed batch: first-launch costs stay out of the timing)
    psz = [torch.zeros(2 * s.E, dtype=torch.complex128, device="cuda") for s in sols]
    pf.pfmbem_solve_batch([s.h for s in sols], psz, tol=tol)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st0, iz = pf.pfmbem_solve_batch([s.h for s in sols], psz, tol=tol)
    t_zero = time.perf_counter() - t0
    # warm start: features, network, decode and solve, all timed
    psw = [torch.zeros(2 * s.E, dtype=torch.complex128, device="cuda") for s in sols]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Xf = np.concatenate([features(s, w.M, model) for s, w in zip(sols, instances)]).astype(np.float32)
    Y = net.forward(Xf)
    rows_per = Y.shape[0] // n
    for q, (s, psi) in enumerate(zip(sols, psw)):
        pf.pfmbem_warm_decode(s.h, Y[q * rows_per:(q + 1) * rows_per].ravel(), psi.data_ptr(), NMODES)
    st1, iw = pf.pfmbem_solve_batch([s.h for s in sols], psw, tol=tol, use_guess=True)
    t_warm = time.perf_counter() - t0
    # plain FP64 GMRES, one block after another
    sample = instances[:fp64_sample]
    s64 = _create_all(sample, precision=pf.FP64)
    psf = [torch.zeros(2 * s.E, dtype=torch.complex128, device="cuda") for s in s64]
    s64[0].solve(psf[0].data_ptr(), tol=tol, check=False)           # untimed first solve
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    i64 = [s.solve(p.data_ptr(), tol=tol, check=False) for s, p in zip(s64, psf)]
    torch.cuda.synchronize()
    t_fp64 = time.perf_counter() - t0
    diff = max(float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) for a, b in zip(psw, psz))
    out = {
        "blocks": n, "status_zero": st0, "status_warm": st1,
        "batched_zero_start_solves_per_s": n / t_zero,
        "batched_warm_start_solves_per_s": n / t_warm,
        "plain_fp64_solves_per_s": len(sample) / t_fp64, "plain_fp64_sample": len(sample),
        "mean_iters_zero": float(np.mean([i.iters for i in iz])), "mean_iters_warm": float(np.mean([i.iters for i in iw])),
        "mean_iters_fp64": float(np.mean([i.iters for i in i64])),
        "max_rel_residual_warm": float(max(i.rel_residual for i in iw)),
        "max_rel_residual_fp64": float(max(i.rel_residual for i in i64)),
        "max_rel_diff_warm_vs_zero": diff, "create_seconds": t_create}
    if keep > 0:
        out["solutions"] = [p.cpu().numpy() for p in psw[:keep]]
    tc = time.perf_counter()
    for s in sols + s64:
        s.close()
    out["destroy_seconds"] = time.perf_counter() - tc
    return out


def train(X, T, hidden=256, layers=3, epochs=200, batch=256, lr=1e-3, seed=1913, log_every=0, lr_final=0.05,
          X_val=None, T_val=None):
    """Adam on the mean-squared error with a cosine learning-rate decay from lr
    to lr * lr_final; returns the network and the loss history (and, with a
    validation set, its loss after every epoch as the attribute net.val_hist)."""
    net = pf.MLP(X.shape[1], hidden, layers, T.shape[1], seed=seed)
    rng = np.random.default_rng(seed)
    hist, val = [], []
    n = X.shape[0]
    for ep in range(epochs):
        a = lr * (lr_final + (1 - lr_final) * 0.5 * (1 + np.cos(np.pi * ep / max(epochs, 1))))
        perm = rng.permutation(n)
        tot = 0.0
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            tot += net.train(X[idx], T[idx], lr=a) * len(idx)
        hist.append(tot / n)
        if X_val is not None:
            val.append(net.train(X_val, T_val))
        if log_every and ep % log_every == 0:
            print(f"epoch {ep} loss {hist[-1]:.4e}" + (f" val {val[-1]:.4e}" if val else ""), flush=True)
    net.val_hist = val
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
    ap.add_argument("--model", default="global", choices=["global", "local"])
    ap.add_argument("--epochs", type=int, default=0, help="0: 1000 (global) or 300 (local)")
    ap.add_argument("--batch", type=int, default=0, help="0: 256 (global) or 512 (local)")
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--batched", action="store_true",
                    help="training data from batched solves; evaluation as one batched warm-started solve of all "
                         "held-out blocks against a batched zero start and plain FP64 GMRES")
    a = ap.parse_args()
    a.epochs = a.epochs or (1000 if a.model == "global" else 300)
    a.batch = a.batch or (256 if a.model == "global" else 512)
    t0 = time.perf_counter()
    gen = generate_batched if a.batched else generate
    X, T, inst, _ = gen(W.batch_instances(a.train, seed=1912), tol=a.tol, model=a.model)
    nv = max(1, a.train // 16)               # validation split: the first blocks' rows
    val = inst < nv
    t1 = time.perf_counter()
    net, hist = train(X[~val], T[~val], epochs=a.epochs, batch=a.batch, lr=a.lr, X_val=X[val], T_val=T[val])
    t2 = time.perf_counter()
    if a.batched:
        r = evaluate_batched(net, W.batch_instances(a.test, seed=1915), tol=a.tol, model=a.model)
        r.update({"model": a.model, "train_blocks": a.train - nv, "epochs": a.epochs, "final_loss": hist[-1],
                  "final_validation_loss": net.val_hist[-1],
                  "seconds": {"data": t1 - t0, "train": t2 - t1, "evaluate": time.perf_counter() - t2}})
        print(json.dumps(r), flush=True)
        return
    rows = evaluate(net, W.batch_instances(a.test, seed=1915), tol=a.tol, model=a.model)
    t3 = time.perf_counter()
    iz, iw, r0 = rows[:, 0], rows[:, 1], rows[:, 2]
    print(json.dumps({
        "model": a.model, "train_blocks": a.train - nv, "validation_blocks": nv, "test_blocks": a.test,
        "epochs": a.epochs,
        "train_rows": int((~val).sum()), "inputs": int(X.shape[1]), "outputs": int(T.shape[1]),
        "first_loss": hist[0], "final_loss": hist[-1], "final_validation_loss": net.val_hist[-1],
        "mean_iters_zero_start": float(iz.mean()), "mean_iters_warm_start": float(iw.mean()),
        "median_warm_start_residual": float(np.median(r0)),
        "median_projection_residual": float(np.median(rows[:, 7])),
        "fraction_guess_kept": float(np.mean(r0 < 1.0)),
        "mean_solve_ms_zero": float(rows[:, 5].mean()), "mean_solve_ms_warm": float(rows[:, 6].mean()),
        "mean_total_ms_warm": float(rows[:, 8].mean()),
        "all_converged": bool(np.all(rows[:, 3] <= a.tol) and np.all(rows[:, 4] <= a.tol)),
        "seconds": {"data": t1 - t0, "train": t2 - t1, "evaluate": t3 - t2}}), flush=True)


def _residual(s, B, psi):
    r = np.zeros_like(psi)
    s.matvec(psi, r, pf.FP64)
    return float(np.linalg.norm(B - r) / np.linalg.norm(B))


def evaluate(net, instances, tol=1e-6, model=None):
    """Per instance: zero-start and warm-start GMRES iterations (columns 0, 1),
    the FP64 relative residual of the decoded prediction (2), the final
    residuals (3, 4), the solve times in ms (5, 6), the residual of the exact
    solution's own 17-mode projection (7, the best any prediction in this
    representation can do) and the warm start's total time including the
    features, the network and the decode (8)."""
    import time
    rows = []
    for w in instances:
        s = pf.Solver(w, precision=pf.MIXED)
        B = np.zeros(2 * s.E, dtype=np.complex128)
        s.rhs(B)
        psi = np.zeros_like(B)
        iz = s.solve(psi, tol=tol, check=False)
        proj = np.zeros_like(B)
        pf.pfmbem_warm_decode(s.h, pf.pfmbem_warm_targets(s.h, psi, w.M, NMODES), proj, NMODES)
        t0 = time.perf_counter()
        y = net.forward(features(s, w.M, model))
        psi0 = np.zeros_like(B)
        pf.pfmbem_warm_decode(s.h, y.ravel(), psi0, NMODES)
        psi_w = psi0.copy()
        iw = s.solve(psi_w, tol=tol, use_guess=True, check=False)
        t1 = time.perf_counter()
        rows.append((iz.iters, iw.iters, _residual(s, B, psi0), iz.rel_residual, iw.rel_residual, iz.ms, iw.ms,
                     _residual(s, B, proj), 1e3 * (t1 - t0)))
        s.close()
    return np.array(rows)


if __name__ == "__main__":
    main()
