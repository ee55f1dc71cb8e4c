"""Autotuner for the plan's tile shapes.

The leaf occupancy (how many elements a leaf box may hold, which sets the
quadtree depth and so the balance between the cached near-field blocks and the
M2L translations) is chosen per instance class by timing candidate plans on a
representative block:

    cost = create + solve,

the measured time of creating the plan and running one refined mixed-precision
solve of the block's own right-hand side to the sweep's tolerance.  Timing the
whole solve, not the product alone, charges each plan for its GMRES driver as
well (the single-launch product runs its Arnoldi steps on the device, the
per-stage path drives them from the host).  Results are cached in a JSON
file keyed by (elements rounded to a power of two, kH rounded to an integer).
"""
from __future__ import annotations

import json
import math
import os
import time


from . import pfmbem as pf

# The M2L engine is left to the library's own rule (tensor cores from 1024 boxes
# a level up, which no instance of a sweep reaches): forcing the tensor-core form
# on small blocks puts one 512-thread block per SM under every product, which
# keeps concurrent instances of a batch from sharing the GPU.
CANDIDATES = [dict(leaf_max=lm) for lm in (32, 64, 128)]


def instance_key(w) -> str:
    return f"E{1 << int(math.ceil(math.log2(max(w.E, 1))))}_kH{int(round(w.k * w.H))}"


def measure(w, cand, reps=3, stream=None, tol=1e-6):
    """Seconds of create and of one refined mixed-precision solve (the fastest
    of reps, after one untimed solve) for one candidate plan."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = pf.Solver(w, precision=pf.MIXED, stream=stream, **cand)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    psi = torch.zeros(2 * w.E, dtype=torch.complex128, device="cuda")
    try:
        s.solve(psi, tol=tol, check=False)
        t_solve = math.inf
        for _ in range(reps):
            psi.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            s.solve(psi, tol=tol, check=False)
            torch.cuda.synchronize()
            t_solve = min(t_solve, time.perf_counter() - t0)
    finally:
        s.close()
    return t_create, t_solve


class Autotuner:
    def __init__(self, path=None):
        self.path = path or os.path.join(os.path.expanduser("~"), ".cache", "pfmbem_autotune.json")
        self.table = {}
        if os.path.exists(self.path):
            try:
                with open(self.path) as f:
                    self.table = json.load(f)
            except (OSError, ValueError):
                self.table = {}

    def save(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        with open(self.path, "w") as f:
            json.dump(self.table, f, indent=1)

    def tune(self, w, candidates=CANDIDATES):
        key = instance_key(w)
        results = []
        for cand in candidates:
            try:
                tc, ts = measure(w, cand)
            except pf.PfmbemError:
                continue
            results.append((tc + ts, cand, tc, ts))
        results.sort(key=lambda r: r[0])
        best = results[0]
        self.table[key] = {"options": best[1], "cost_s": best[0],
                           "tried": [{"options": r[1], "cost_s": r[0], "create_s": r[2], "solve_s": r[3]}
                                     for r in results]}
        return best[1]

    def options(self, w, tune_missing=True):
        """Options for block w (tuned on first sight of its class)."""
        key = instance_key(w)
        if key not in self.table and tune_missing:
            self.tune(w)
        cand = self.table.get(key, {}).get("options", {})
        o = pf.Options()
        o.precision = pf.MIXED
        for k, v in cand.items():
            setattr(o, k, v)
        return o
