"""The single-launch product on few blocks: the batched launch runs each
instance's products on a group of 8..32 blocks, where the item forms of the
stages change (box items instead of coefficient items near the top of the
tree, no folded top levels, the generic box forms where the staged ones do not
fit).  Both products on grids capped at 8, 16, 24 and 32 blocks agree with the
full grid's, for sweep-sized blocks (16 fibers, 2400..2800 elements; the third
runs its level-1 L2L in the generic form on 16 blocks or fewer)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from tests.gpu_common import ensure_built

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, %r)
from paper_1910_10863_gb300 import pfmbem as pf, workloads as W
out = {}
sweep = W.batch_instances(13, seed=1912)
for w in (sweep[0], sweep[1], sweep[12]):
    s = pf.Solver(w, precision=pf.MIXED)
    rng = np.random.default_rng(3)
    n = 2 * s.E
    B = np.zeros(n, dtype=np.complex128)
    s.rhs(B)
    xs = {"random": rng.standard_normal(n) + 1j * rng.standard_normal(n), "rhs": B}
    res = {}
    for name, x in xs.items():
        x = np.ascontiguousarray(x, dtype=np.complex128)
        y64 = np.zeros_like(x)
        y32 = np.zeros_like(x)
        pf.pfmbem_matvec(s.h, x, y64, pf.FP64)
        pf.pfmbem_matvec(s.h, x, y32, pf.MIXED)
        res[name] = [y64.real.tolist(), y64.imag.tolist(), y32.real.tolist(), y32.imag.tolist()]
    out[w.name] = res
    s.close()
json.dump(out, open(sys.argv[1], "w"))
"""


def _run(tmp_path, grid):
    path = os.path.join(str(tmp_path), f"g{grid}.json")
    env = dict(os.environ)
    if grid:
        env["PFMBEM_FUSED_GRID"] = str(grid)
    r = subprocess.run([sys.executable, "-c", CHILD % ROOT, path], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    d = json.load(open(path))
    out = {}
    for wn, res in d.items():
        for xn, (a, b, c, e) in res.items():
            out[(wn, xn)] = (np.array(a) + 1j * np.array(b), np.array(c) + 1j * np.array(e))
    return out


def test_products_on_small_grids_match_full_grid(tmp_path):
    ensure_built()
    full = _run(tmp_path, 0)
    errs = {}
    for grid in (8, 16, 24, 32):
        got = _run(tmp_path, grid)
        for key, (y64, y32) in got.items():
            r64, r32 = full[key]
            e64 = float(np.linalg.norm(y64 - r64) / np.linalg.norm(r64))
            e32 = float(np.linalg.norm(y32 - r64) / np.linalg.norm(r64))
            errs[(grid,) + key] = (e64, e32)
    full_e32 = {key: float(np.linalg.norm(v[1] - v[0]) / np.linalg.norm(v[0])) for key, v in full.items()}
    print(json.dumps({"full_grid_e32": {str(k): v for k, v in full_e32.items()},
                      "small": {str(k): v for k, v in errs.items()}}))
    for k, (e64, e32) in errs.items():
        assert e64 < 1e-10, (k, e64)
        assert e32 < 4 * full_e32[k[1:]] + 1e-7, (k, e32, full_e32[k[1:]])
