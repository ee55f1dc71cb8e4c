"""Run the products of one workload a few times, for a profiler to capture.

    python -m paper_1910_10863_gb300.profile_products --workload hexagon_8x8_n256 --reps 3
    python -m paper_1910_10863_gb300.profile_products --sweep 32

The first form creates the block's handle and runs --reps pairs of products
(FP32 mixed, then FP64) on a device vector; the second solves a chunk of
band-gap-sweep instances in one persistent batched launch.  Prints one JSON
line with the device time of each (CUDA events; not a benchmark number under a
profiler).
"""
from __future__ import annotations

import argparse
import json

from . import pfmbem as pf
from . import workloads as W


def products(workload: str, reps: int) -> dict:
    import torch
    w = getattr(W, workload)()
    s = pf.Solver(w, precision=pf.MIXED)
    n = 2 * s.E
    x = torch.randn(n, dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    out = {"workload": w.name, "elements": int(w.E)}
    for prec, name in ((pf.MIXED, "fp32_ms"), (pf.FP64, "fp64_ms")):
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            pf.pfmbem_matvec(s.h, x.data_ptr(), y.data_ptr(), prec)
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        out[name] = times
    s.close()
    return out


def sweep(count: int) -> dict:
    import time

    import torch
    inst = W.batch_instances(count, seed=1912)
    sols = [pf.Solver(w, precision=pf.MIXED) for w in inst]
    psis = [torch.zeros(2 * w.E, dtype=torch.complex128, device="cuda") for w in inst]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, infos = pf.pfmbem_solve_batch([s.h for s in sols], psis, tol=1e-6)
    t1 = time.perf_counter()
    return {"instances": count, "status": st, "seconds": t1 - t0,
            "max_rel_residual": max(i.rel_residual for i in infos), "iters": sum(i.iters for i in infos)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="hexagon_8x8_n256", choices=["hexagon_8x8_n256", "square_32x32_n128",
                                                                       "square_2x2_n64"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--sweep", type=int, default=0, help="solve this many sweep instances in one batched launch")
    a = ap.parse_args()
    print(json.dumps(sweep(a.sweep) if a.sweep > 0 else products(a.workload, a.reps)), flush=True)


if __name__ == "__main__":
    main()
