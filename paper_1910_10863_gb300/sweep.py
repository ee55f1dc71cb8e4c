"""Band-gap sweep: many (kH, theta) blocks with uneven element counts solved
together by pfmbem_solve_batch (one persistent launch: refined mixed-precision
GMRES, each instance solved by a group of blocks, longest first; plans chosen by
the autotuner; the handles created on a pool of host threads), against solving
the same blocks one at a time.  Prints one JSON line.

    python -m paper_1910_10863_gb300.sweep --count 512
"""
from __future__ import annotations

import argparse
import json
import os
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import autotune, pfmbem as pf, workloads as W


def run(count=512, chunk=128, tol=1e-6, sequential_sample=32, tune_path=None):
    import torch
    inst = W.batch_instances(count, seed=1912)
    tuner = autotune.Autotuner(tune_path or os.path.join(os.path.dirname(__file__), "_build", "autotune.json"))
    t0 = time.perf_counter()
    opts = [tuner.options(w) for w in inst]
    tuner.save()
    t_tune = time.perf_counter() - t0
    streams = [torch.cuda.Stream() for _ in range(chunk)]
    pool = ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1)))
    results = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t_create = 0.0
    t_solve = 0.0
    for c0 in range(0, count, chunk):
        part = inst[c0:c0 + chunk]
        tc = time.perf_counter()
        # the handles are independent: their host set-up runs on a pool of host
        # threads (the library releases the interpreter lock in every call)
        def make(i, w=None, o=None):
            w, o = part[i], opts[c0 + i]
            return pf.pfmbem_create(w.M, w.nodes_per_fiber, w.nodes, w.H, w.lattice, w.k, w.k1, w.rho_ratio,
                                    w.theta, o, streams[i].cuda_stream)
        hs = list(pool.map(make, range(len(part))))
        torch.cuda.synchronize()
        t_create += time.perf_counter() - tc
        psis = [torch.zeros(2 * w.E, dtype=torch.complex128, device="cuda") for w in part]
        ts = time.perf_counter()
        st, infos = pf.pfmbem_solve_batch(hs, psis, tol=tol)
        t_solve += time.perf_counter() - ts
        for h, w, psi, info in zip(hs, part, psis, infos):
            orders, R, T, energy = pf.pfmbem_coefficients(h, psi)
            results.append((info.iters, info.restarts, info.rel_residual, info.status, energy, w.E))
            pf.pfmbem_destroy(h)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    pool.shutdown()
    # one at a time, same plans, same stream
    t0 = time.perf_counter()
    seq = []
    for w, o in list(zip(inst, opts))[:sequential_sample]:
        s = pf.Solver(w, opt=o)
        psi = torch.zeros(2 * w.E, dtype=torch.complex128, device="cuda")
        info = s.solve(psi, tol=tol, check=False)
        pf.pfmbem_coefficients(s.h, psi)
        seq.append(info.iters)
        s.close()
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    r = np.array(results)
    return {
        "instances": count, "elements_min": int(r[:, 5].min()), "elements_max": int(r[:, 5].max()),
        "batched_solves_per_s": count / t_batch, "sequential_solves_per_s": sequential_sample / t_seq,
        "batched_seconds": t_batch, "create_seconds": t_create, "solve_seconds": t_solve,
        "batch_solve_only_per_s": count / t_solve, "tune_seconds": t_tune,
        "all_converged": bool(np.all(r[:, 2] <= tol)), "max_rel_residual": float(r[:, 2].max()),
        "mean_iters": float(r[:, 0].mean()), "mean_refinements": float(r[:, 1].mean()),
        "chunk": chunk, "tol": tol, "autotune_classes": len(tuner.table)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=512)
    ap.add_argument("--chunk", type=int, default=128)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--sequential-sample", type=int, default=32)
    a = ap.parse_args()
    print(json.dumps(run(a.count, a.chunk, a.tol, a.sequential_sample)), flush=True)


if __name__ == "__main__":
    main()
