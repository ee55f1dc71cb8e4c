"""Autotuner for the plan's tile shapes.

The leaf occupancy (how many elements a leaf box may hold, which sets the
quadtree depth and so the balance between the cached near-field blocks and the
M2L translations) and the M2L engine (CUDA cores or tcgen05 tensor cores) are
chosen per instance class by timing candidate plans on a representative block:

    cost = create + ITERS_MIXED * matvec(mixed) + ITERS_FP64 * matvec(FP64),

the time of one refined mixed-precision solve with typical iteration counts.
Results are cached in a JSON file keyed by (elements rounded to a power of two,
kH rounded to an integer).
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from . import pfmbem as pf

ITERS_MIXED = 20
ITERS_FP64 = 3
CANDIDATES = [dict(leaf_max=lm, m2l_mode=mm) for lm in (32, 64, 128) for mm in (1, 2)]


def instance_key(w) -> str:
    return f"E{1 << int(math.ceil(math.log2(max(w.E, 1))))}_kH{int(round(w.k * w.H))}"


def measure(w, cand, reps=5, stream=None):
    """Seconds of create, mixed matvec and FP64 matvec for one candidate plan."""
    import torch
    x = torch.from_numpy(np.random.default_rng(0).standard_normal(2 * w.E)
                         + 1j * np.random.default_rng(1).standard_normal(2 * w.E)).cuda()
    y = torch.zeros_like(x)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = pf.Solver(w, precision=pf.MIXED, stream=stream, **cand)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    out = {}
    for name, prec in (("mixed", pf.MIXED), ("fp64", pf.FP64)):
        s.matvec(x, y, prec)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            s.matvec(x, y, prec)
        torch.cuda.synchronize()
        out[name] = (time.perf_counter() - t0) / reps
    s.close()
    return t_create, out["mixed"], out["fp64"]


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
                tc, tm, t64 = measure(w, cand)
            except pf.PfmbemError:
                continue
            results.append((tc + ITERS_MIXED * tm + ITERS_FP64 * t64, cand, tc, tm, t64))
        results.sort(key=lambda r: r[0])
        best = results[0]
        self.table[key] = {"options": best[1], "cost_s": best[0],
                           "tried": [{"options": r[1], "cost_s": r[0], "create_s": r[2], "matvec_mixed_s": r[3],
                                      "matvec_fp64_s": r[4]} for r in results]}
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
