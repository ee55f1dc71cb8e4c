"""Band-gap sweep of Sec. 4: energy transmission coefficient against frequency.

For the water/mercury square-lattice crystal of Table 3 (workloads.table3_square)
this script solves one block per normalised frequency ka/2pi (mixed precision,
FP64 residual 1e-6), evaluates ETC on the block's right edge x1 = 4a with
pfmbem_etc, and reports the frequency intervals where ETC < 3 %, the stop-band
criterion of Sec. 4.  Frequencies within 1e-3 of a Wood anomaly (ka/2pi = n/6 at
normal incidence) are skipped.  One JSON line per filling fraction.

    python -m paper_1910_10863_gb300.bandgap --fill 0.35 0.5
    python -m paper_1910_10863_gb300.bandgap --mercury-water 4 10 --fill 0.35 --fmin 0.3 --fmax 1.0

The second form sweeps the mercury/water crystal of the last experiment of Sec. 4
for M_L = 4 and 10 columns.
"""
from __future__ import annotations

import json
import math

import numpy as np

from . import pfmbem as pf
from . import workloads as W


def etc_curve(freqs, f=0.35, n=256, tol=1e-6, npts=256):
    out = []
    for ka in freqs:
        w = W.table3_square(float(ka), f=f, n=n)
        if W.wood_distance(w.k * w.H, w.theta) < 1e-3:
            continue
        s = pf.Solver(w, precision=pf.MIXED)
        psi = np.zeros(2 * s.E, dtype=np.complex128)
        info = s.solve(psi, tol=tol, check=False)
        etc = pf.pfmbem_etc(s.h, psi, 4 * 0.5, npts)
        out.append((float(ka), etc, info.iters, info.rel_residual))
        s.close()
    return out


def mercury_water_curve(freqs, ml=4, f=0.35, n=256, tol=1e-6, npts=256):
    """ETC on the right edge x1 = ml a of the mercury/water crystal (mercury
    cylinders in water, workloads.mercury_water_block) at each normalised
    frequency, skipping the Wood anomalies of its 12a-tall block (n/12)."""
    out = []
    for ka in freqs:
        w = W.mercury_water_block(float(ka), f=f, ml=ml, n=n)
        if W.wood_distance(w.k * w.H, w.theta) < 1e-3:
            continue
        s = pf.Solver(w, precision=pf.MIXED)
        psi = np.zeros(2 * s.E, dtype=np.complex128)
        info = s.solve(psi, tol=tol, check=False)
        etc = pf.pfmbem_etc(s.h, psi, ml * 0.5, npts)
        out.append((float(ka), etc, info.iters, info.rel_residual))
        s.close()
    return out


def gaps(curve, level=0.03):
    """Maximal runs of consecutive sweep points with ETC below level, as
    [first, last] frequency pairs."""
    res, cur = [], None
    for ka, e, _, _ in curve:
        if e < level:
            cur = [ka, ka] if cur is None else [cur[0], ka]
        elif cur is not None:
            res.append(cur)
            cur = None
    if cur is not None:
        res.append(cur)
    return res


def main():
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--fmin", type=float, default=0.05)
    ap.add_argument("--fmax", type=float, default=1.4)
    ap.add_argument("--step", type=float, default=0.01)
    ap.add_argument("--fill", type=float, nargs="*", default=[0.35, 0.5])
    ap.add_argument("--mercury-water", type=int, nargs="*", default=None, metavar="ML",
                    help="the mercury/water crystal instead, for these column counts M_L")
    a = ap.parse_args()
    freqs = np.round(np.arange(a.fmin, a.fmax + 1e-9, a.step), 6)
    if a.mercury_water:
        for ml in a.mercury_water:
            c = mercury_water_curve(freqs, ml=ml, f=a.fill[0])
            print(json.dumps({"crystal": "mercury/water", "ml": ml, "filling": a.fill[0],
                              "gaps_etc_below_3pct": gaps(c), "points": len(c),
                              "max_rel_residual": max(t[3] for t in c),
                              "curve": [[round(k, 4), round(e, 5), it] for k, e, it, _ in c]}), flush=True)
        return
    for f in a.fill:
        c = etc_curve(freqs, f=f)
        worst = max(c, key=lambda t: t[3])
        print(json.dumps({"filling": f, "gaps_etc_below_3pct": gaps(c), "points": len(c),
                          "max_rel_residual": worst[3], "max_rel_residual_at": worst[0],
                          "unconverged": [round(k, 4) for k, _, _, r in c if r > 1e-6],
                          "curve": [[round(k, 4), round(e, 5), it] for k, e, it, _ in c]}), flush=True)


if __name__ == "__main__":
    main()
