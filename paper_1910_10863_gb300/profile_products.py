"""Run the products of one workload a few times, for a profiler to capture.

    python -m paper_1910_10863_gb300.profile_products --workload hexagon_8x8_n256 --reps 3
    python -m paper_1910_10863_gb300.profile_products --sweep 32
    python -m paper_1910_10863_gb300.profile_products --trees

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


def trees(reps: int, solve: bool = True, only: str | None = None) -> dict:
    """The square and the regular-triangle tree on the 8x8 hexagon block: the FP64
    product with cached element integrals (the square tree's per-stage form and
    the triangle tree's) and with the integrals in every product, its difference
    from the square tree's single-launch FP64 product, and each form's FP64 solve
    to 1e-6.  only: one of the forms' names."""
    import time

    import torch
    w = W.hexagon_8x8_n256()
    lat = dict(tree=1, leaf_max=16, **W.hexagon_block_lattice(w.H, 8))
    n = 2 * w.E
    x = torch.randn(n, dtype=torch.complex128, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    ref = torch.zeros_like(x)
    single = pf.Solver(w)
    pf.pfmbem_matvec(single.h, x.data_ptr(), ref.data_ptr(), pf.FP64)
    torch.cuda.synchronize()
    out = {"workload": w.name, "elements": int(w.E)}
    forms = (("square_cached", {"launch": 1}), ("square_onthefly", {"near_mode": 1}),
             ("triangle_cached", lat), ("triangle_onthefly", dict(lat, near_mode=1)))
    for name, opts in forms:
        if only is not None and name != only:
            continue
        t0 = time.perf_counter()
        s = pf.Solver(w, **opts)
        torch.cuda.synchronize()
        create_s = time.perf_counter() - t0
        pl = s.plan()
        y = torch.zeros_like(x)
        pf.pfmbem_matvec(s.h, x.data_ptr(), y.data_ptr(), pf.FP64)     # first product: lazy tables
        times = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            pf.pfmbem_matvec(s.h, x.data_ptr(), y.data_ptr(), pf.FP64)
            b.record()
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
        r = {"create_s": create_s, "depth": pl.depth, "p": list(pl.p)[:pl.depth + 1], "m2l_pairs": pl.m2l_pairs,
             "near_pairs": pl.near_pairs, "near_quad": pl.near_quad, "fp64_ms": times,
             "rel_diff_vs_single_launch": float(torch.linalg.vector_norm(y - ref) / torch.linalg.vector_norm(ref))}
        if name.startswith("triangle"):
            r["cells"] = pl.nroot
            r["super_p"] = pl.super_p
        if solve:
            psi = torch.zeros_like(x)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = s.solve(psi, tol=1e-6, maxit=2000)
            torch.cuda.synchronize()
            r["solve_s"] = time.perf_counter() - t0
            r["solve_iters"] = info.iters
            r["solve_rel_residual"] = info.rel_residual
        out[name] = r
        s.close()
    single.close()
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
    ap.add_argument("--trees", action="store_true",
                    help="square against regular-triangle tree on the 8x8 hexagon block (FP64 products and solves)")
    ap.add_argument("--only", choices=["square_cached", "square_onthefly", "triangle_cached", "triangle_onthefly"],
                    help="with --trees: one form")
    ap.add_argument("--no-solve", action="store_true", help="with --trees: products only")
    a = ap.parse_args()
    if a.trees:
        print(json.dumps(trees(a.reps, solve=not a.no_solve, only=a.only)), flush=True)
        return
    print(json.dumps(sweep(a.sweep) if a.sweep > 0 else products(a.workload, a.reps)), flush=True)


if __name__ == "__main__":
    main()
