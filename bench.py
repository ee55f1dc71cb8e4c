#!/usr/bin/env python
"""Throughput of the periodic FM-BEM solver on GB300.

One step = the whole hot path for one synthetic fundamental block: pfmbem_create
(geometry, periodic quadtree, self-element integrals, lattice sums, translation
tables), pfmbem_solve (FMM matrix-vector products inside GMRES to a relative
FP64 residual of 1e-6) and pfmbem_coefficients (Bragg orders), then destroy.
Workload: hexagon lattice, 8x8 = 64 fibers, 256 elements each (16384 elements,
32768 unknowns), kH = 5, water matrix / mercury fibers.

value = solves/s of the whole job (all ranks; each rank solves its own block:
weak scaling, no collective on the data path).  The JSON line also carries the
FMM matvec rate (Munknowns/s), the roofline of the dominant kernel, the CPU
oracle baseline, the end-to-end rate with host buffers and the SM clocks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GMRES solves/s and FMM matvec Munknowns/s at 1e-6 residual vs plain FP64, 1 GB300"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="own", choices=["own", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="steps of the plain FP64 comparator arm (default: --steps)")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--matvec-reps", type=int, default=20)
    ap.add_argument("--workload", default="hexagon_8x8_n256", choices=sorted(WORKLOADS))
    ap.add_argument("--launch", type=int, default=0, choices=[0, 1],
                    help="cached matvec: 0 = one cooperative launch per product, 1 = one kernel per stage")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the large-block (32x32 square, 131072 elements) and sweep-chunk (128 band-gap "
                         "instances) keys")
    ap.add_argument("--stage-times", action="store_true",
                    help="diagnostic: print the stage durations of the single-launch matvec (4 FP64 and 4 mixed "
                         "products of the workload, %%globaltimer read by block 0 after every device-wide "
                         "barrier) on stderr, then exit; no bench line")
    return ap.parse_args()


def stage_times(args):
    os.environ["PFMBEM_STAGE_TIMES"] = "1"      # read by the library at its first product
    import torch
    from paper_1910_10863_gb300 import pfmbem as pf
    from paper_1910_10863_gb300 import workloads as W
    if not os.path.exists(pf.LIB_PATH):
        from paper_1910_10863_gb300 import build
        build.build()
    w = workload(args.workload)
    x = torch.from_numpy(W.density_vector(w.E, 3)).cuda()
    s = pf.Solver(w)
    pl = s.plan()
    print(w.name, "depth", pl.depth, "p", list(pl.p)[:pl.depth + 1], file=sys.stderr, flush=True)
    for prec in (pf.FP64, pf.MIXED):
        y = torch.zeros_like(x)
        for _ in range(4):
            s.matvec(x, y, prec)
    torch.cuda.synchronize()
    s.close()


# hexagon 8x8 (16384 elements, kH = 5) is the headline block; the 32x32 square
# lattice (131072 elements, kH = 20) is the large-block case.
WORKLOADS = {"hexagon_8x8_n256": "hexagon_8x8_n256", "square_32x32_n128": "square_32x32_n128"}


def workload(name="hexagon_8x8_n256"):
    from paper_1910_10863_gb300 import workloads as W
    return getattr(W, WORKLOADS[name])()


# ------------------------------------------------------------------ clocks
CLOCK_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
# bits of NVML's clocks-event-reason mask (nvmlClocksEventReason* in nvml.h)
_NVML_REASON_BITS = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20,
                     "hw_thermal_slowdown": 0x40}


def summarize_clocks(rows, t0, t1, source):
    """Median SM clock, maximum clock and active slowdown reasons of the samples
    taken between t0 and t1 (host time, seconds).  rows: (time, sm MHz, max MHz,
    set of active reasons).  With no sample inside the window the nearest one on
    either side stands in, and in_window says so."""
    keep = [r for r in rows if t0 <= r[0] <= t1]
    if not keep and rows:
        before = [r for r in rows if r[0] < t0]
        after = [r for r in rows if r[0] > t1]
        keep = ([before[-1]] if before else []) + ([after[0]] if after else [])
    sm = [r[1] for r in keep]
    mx = [r[2] for r in keep]
    reasons = sorted({nm for r in keep for nm in r[3]})
    return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "samples": len(sm), "in_window": bool(keep) and all(t0 <= r[0] <= t1 for r in keep),
            "reasons": reasons, "source": source}


class _Nvml:
    """Read-only NVML queries through ctypes: SM clock, its maximum and the
    clocks-event-reason mask of one device.  Raises OSError when the library or
    the device is missing."""

    def __init__(self, index, pci=None):
        import ctypes
        self.c = ctypes
        lib = None
        for name in ("libnvidia-ml.so.1", "libnvidia-ml.so"):
            try:
                lib = ctypes.CDLL(name)
                break
            except OSError:
                continue
        if lib is None:
            raise OSError("libnvidia-ml not found")
        self.lib = lib
        if lib.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.dev = ctypes.c_void_p()
        # the CUDA device's PCI address names it whatever the visible-device list
        if (pci is None or lib.nvmlDeviceGetHandleByPciBusId_v2(pci.encode(), ctypes.byref(self.dev)) != 0) and \
                lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(index), ctypes.byref(self.dev)) != 0:
            raise OSError("no NVML device %d" % index)
        try:
            self.reason_fn = lib.nvmlDeviceGetCurrentClocksEventReasons
        except AttributeError:
            self.reason_fn = lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self.max_sm = self._clock(lib.nvmlDeviceGetMaxClockInfo)
        if self.max_sm is None:
            raise OSError("nvmlDeviceGetMaxClockInfo failed")

    def _clock(self, fn):
        v = self.c.c_uint()
        return float(v.value) if fn(self.dev, self.c.c_int(1), self.c.byref(v)) == 0 else None  # 1 = SM

    def sample(self):
        sm = self._clock(self.lib.nvmlDeviceGetClockInfo)
        m = self.c.c_ulonglong()
        mask = m.value if self.reason_fn(self.dev, self.c.byref(m)) == 0 else 0
        act = {nm for nm, bit in _NVML_REASON_BITS.items() if mask & bit}
        return sm, self.max_sm, act

    def close(self):
        self.lib.nvmlShutdown()


def pci_address(torch, dev):
    """domain:bus:device.function of a CUDA device, as NVML spells it, or None."""
    pr = torch.cuda.get_device_properties(dev)
    try:
        return "%08X:%02X:%02X.0" % (pr.pci_domain_id, pr.pci_bus_id, pr.pci_device_id)
    except AttributeError:
        return None


class Clocks:
    """SM clocks and slowdown reasons sampled during the timed region.

    A host thread reads NVML every 2 ms from start() to stop(), so a timed
    region of a few tens of milliseconds still holds samples; the samples are
    kept for the window between mark_start() and mark_stop().  Where NVML cannot
    be loaded, nvidia-smi samples every 50 ms instead."""

    def __init__(self, index, pci=None):
        self.index = index
        self.pci = pci
        self.proc = None
        self.path = None
        self.nvml = None
        self.thread = None
        self.rows = []
        self.t0 = self.t1 = None

    def start(self):
        import threading
        try:
            self.nvml = _Nvml(self.index, self.pci)
        except (OSError, AttributeError):
            self.nvml = None
        if self.nvml is not None:
            self.halt = threading.Event()

            def run():
                while not self.halt.is_set():
                    sm, mx, act = self.nvml.sample()
                    if sm is not None:
                        self.rows.append((time.time(), sm, mx, act))
                    time.sleep(0.002)
            self.thread = threading.Thread(target=run, daemon=True)
            self.thread.start()
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def wait_first(self, timeout=10.0):
        t = time.time()
        while time.time() - t < timeout:
            if self.thread is not None:
                if self.rows or not self.thread.is_alive():
                    return
            elif self.proc is None or os.path.getsize(self.path) > 0 or self.proc.poll() is not None:
                return
            time.sleep(0.02)

    def mark_start(self):
        self.t0 = time.time()

    def mark_stop(self):
        self.t1 = time.time()

    def stop(self):
        import datetime
        t0, t1 = self.t0 or 0.0, self.t1 or 1e300
        if self.thread is not None:
            self.halt.set()
            self.thread.join(timeout=5)
            self.nvml.close()
            return summarize_clocks(self.rows, t0, t1, "NVML, 2 ms")
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                act = {nm for nm, v in zip(CLOCK_REASONS, f[6:10]) if v.lower().startswith("active")}
                rows.append((ts, float(f[2]), float(f[3]), act))
            except ValueError:
                continue
        os.unlink(self.path)
        return summarize_clocks(rows, t0, t1, "nvidia-smi, 50 ms")


# ------------------------------------------------------------------ CPU oracle sample
def oracle_sample(w, rows=8, lu_n=2048, seed=0, keep=False):
    """Time the oracle on a bounded sample and extrapolate one dense solve of the block.

    Sample: assembly of `rows` element rows (2 equations each) of the dense operator
    (eq. 9) with the Ewald-summed kernel, plus an LU factorisation of a random
    complex matrix of size lu_n; the full solve is extrapolated as
    (E / rows) * t_rows + (2E / lu_n)^3 * t_lu.  keep=True also returns the
    assembled rows (element indices, operator rows, right-hand side rows)."""
    from scipy import linalg as sla

    from oracle import bem
    pb = bem.problem(w)
    rng = np.random.default_rng(seed)
    sel = np.sort(rng.choice(w.E, size=rows, replace=False))
    t0 = time.perf_counter()
    Mr = bem.operator_rows(pb, sel)
    t_rows = time.perf_counter() - t0
    A = rng.standard_normal((lu_n, lu_n)) + 1j * rng.standard_normal((lu_n, lu_n))
    t0 = time.perf_counter()
    sla.lu_factor(A, overwrite_a=True, check_finite=False)
    t_lu = time.perf_counter() - t0
    n = 2 * w.E
    t_full = (w.E / rows) * t_rows + (n / lu_n) ** 3 * t_lu
    sample = (f"assembly of {rows} of {w.E} element rows ({t_rows:.2f} s) + LU of a {lu_n}^2 complex matrix "
              f"({t_lu:.2f} s), extrapolated to one dense solve of {n} unknowns ({t_full:.0f} s)")
    if keep:
        B = bem.rhs(pb)
        eq = np.stack([2 * sel, 2 * sel + 1], axis=1).ravel()
        return 1.0 / t_full, sample, t_rows + t_lu, (sel, Mr, B[eq])
    return 1.0 / t_full, sample, t_rows + t_lu


def cpu_cores():
    return max(1, min(32, os.cpu_count() or 1))


# ------------------------------------------------------------------ reference arm
def run_reference(args, rank, world):
    if rank != 0:
        return
    w = workload(args.workload)
    vals = []
    sample = ""
    for _ in range(args.warmup):
        oracle_sample(w, rows=2, lu_n=512)
    t_all = 0.0
    for _ in range(args.steps):
        v, sample, t = oracle_sample(w, rows=4, lu_n=1536)
        vals.append(v)
        t_all += t
    value = float(np.mean(vals))
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name, "elements": w.E, "unknowns": 2 * w.E, "tol": args.tol,
                       "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ own arm
def aggregate_ranks(ms, world, dist=None, device="cpu"):
    """Replicas: every rank solves its own block (weak scaling, no collective on
    the data path).  The job's time per step is the slowest rank's (max over
    ranks of each entry of ms), and its rate the solves of all ranks per second:
    world * 1000 / ms.  Returns (max times, whole-job rates)."""
    import torch
    if dist is not None:
        t = torch.tensor([float(v) for v in ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = [float(v) for v in t]
    return list(ms), [world * 1000.0 / v for v in ms]


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.stage_times:
        stage_times(args)
        return
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1910_10863_gb300 import pfmbem as pf

    if not os.path.exists(pf.LIB_PATH):
        from paper_1910_10863_gb300 import build
        build.build()
    prec = pf.FP64 if args.precision == "fp64" else pf.MIXED
    w = workload(args.workload)
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    npf_d = torch.from_numpy(np.ascontiguousarray(w.nodes_per_fiber, dtype=np.int32)).cuda()
    nodes_d = torch.from_numpy(np.ascontiguousarray(w.nodes)).cuda()
    npf_h = torch.from_numpy(np.ascontiguousarray(w.nodes_per_fiber, dtype=np.int32)).pin_memory()
    nodes_h = torch.from_numpy(np.ascontiguousarray(w.nodes)).pin_memory()
    n = 2 * w.E
    psi_d = torch.zeros(n, dtype=torch.complex128, device="cuda")
    psi_h = torch.zeros(n, dtype=torch.complex128).pin_memory()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    opt = pf.Options()
    opt.precision = prec
    opt.launch = args.launch
    maxit = 2000
    prof_acc = {"ms": np.zeros(32), "launches": np.zeros(32, dtype=np.int64)}
    stats = {}

    opt_prof = pf.Options()
    opt_prof.precision = prec
    opt_prof.launch = args.launch
    opt_prof.profile = 1        # kernel timing from inside pfmbem_create on

    def step(host=False, profile=False, o=None):
        npf, nodes, psi = (npf_h, nodes_h, psi_h) if host else (npf_d, nodes_d, psi_d)
        oo = o or (opt_prof if profile else opt)
        h = pf.pfmbem_create(w.M, npf, nodes, w.H, w.lattice, w.k, w.k1, w.rho_ratio, w.theta, oo, sptr)
        try:
            info = pf.pfmbem_solve(h, None, psi, False, args.tol, maxit, check=False)
            if info.status != 0:
                stats["failed_status"] = pf.STATUS.get(info.status, info.status)
            orders, R, T, energy = pf.pfmbem_coefficients(h, psi)
            if profile:
                p = pf.pfmbem_profile_read(h)
                prof_acc["ms"] += np.array(p.ms)
                prof_acc["launches"] += np.array(p.launches)
            stats.update(iters=info.iters, restarts=info.restarts, rel_residual=info.rel_residual,
                         energy=energy, norders=len(orders))
            if "plan" not in stats:
                stats["plan"] = pf.pfmbem_plan(h)
        finally:
            pf.pfmbem_destroy(h)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(host, profile, steps=None, o=None):
        steps = steps or args.steps
        tot = 0.0
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(host=host, profile=profile, o=o)
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / steps

    clocks = Clocks(local, pci_address(torch, local))
    clocks.start()
    for _ in range(args.warmup):
        step()
    clocks.wait_first()
    barrier()
    clocks.mark_start()
    ms_step = timed(host=False, profile=False)
    clocks.mark_stop()
    clk = clocks.stop()
    main_stats = dict(stats)
    barrier()
    ms_e2e = timed(host=True, profile=False)
    barrier()
    # create time of a warm, unprofiled step (outside the timed region)
    stats.pop("plan", None)
    step()
    main_stats["plan"] = stats["plan"]
    barrier()
    # per-phase CUDA-event times and launch counts, from separate profiled steps
    # (the events around every launch would otherwise slow the timed steps)
    prof_steps = max(1, min(2, args.steps))
    timed(host=False, profile=True, steps=prof_steps)
    prof_iters = stats["iters"]          # FP32 products that ran in each profiled (mixed) step
    barrier()
    # plain FP64 FMM-GMRES comparator on the same block and tolerance
    o64 = pf.Options()
    o64.precision = pf.FP64
    o64.launch = args.launch
    step(o=o64)
    ms_fp64 = timed(host=False, profile=False, steps=args.fp64_steps or args.steps, o=o64)
    fp64_stats = dict(stats)
    stats.clear()
    stats.update(main_stats)
    barrier()
    (ms_step, ms_e2e), (value, e2e_value) = aggregate_ranks([ms_step, ms_e2e], world, dist, "cuda")

    # FMM matvec rate (FP64 and mixed) on one handle
    h = pf.pfmbem_create(w.M, npf_d, nodes_d, w.H, w.lattice, w.k, w.k1, w.rho_ratio, w.theta, opt, sptr)
    x = torch.from_numpy(pf_density(w)).cuda()
    y = torch.zeros_like(x)
    mv = {}
    for name, pr in (("fp64", pf.FP64), ("mixed", pf.MIXED)):
        for _ in range(3):
            pf.pfmbem_matvec(h, x, y, pr)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.matvec_reps):
            pf.pfmbem_matvec(h, x, y, pr)
        e1.record(stream)
        e1.synchronize()
        mv[name] = n / (e0.elapsed_time(e1) / args.matvec_reps * 1e-3) / 1e6
    pf.pfmbem_destroy(h)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    # accuracy of the benched solve (outside the timed region): the mixed solution at
    # the bench tolerance against an FP64 solve of the same block at 1e-10
    acc = solution_accuracy(pf, torch, w, opt, npf_d, nodes_d, sptr, args.tol, maxit)
    plan = stats["plan"]
    launches = int(round(prof_acc["launches"].sum() / prof_steps * args.steps))
    names = pf.PHASES
    ms_ph = prof_acc["ms"]
    fp64_peak = pf.pfmbem_probe_peak(0)
    fp32_peak = pf.pfmbem_probe_peak(1)
    roof = roofline(names, ms_ph, prof_acc["launches"], prof_steps, plan, fp64_peak, fp32_peak, w.E,
                    tensor_m2l=(opt.m2l_mode == 2), workload=w.name,
                    real_f32_products=prof_iters if prec == pf.MIXED else None)
    roof_p2p = roofline_p2p(ms_ph, prof_acc["launches"], prof_steps, plan, fp64_peak)
    ms_ph = ms_ph / prof_steps

    cpu = None
    if not args.no_cpu_baseline:
        v, sample, _, rows = oracle_sample(w, keep=True)
        cpu = {"value": v, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle", "sample": sample}
        # the oracle's residual of the benched solution on the rows it just assembled
        sel, Mr, Br = rows
        r = Br - Mr @ acc.pop("psi")
        acc["oracle_row_residual"] = {"rows": int(len(sel)), "rel": float(np.linalg.norm(r) / np.linalg.norm(Br)),
                                      "def": "||B_r - A_r psi|| / ||B_r|| over the sampled element rows, A_r and "
                                             "B_r assembled by the CPU oracle (exact element integrals, Ewald "
                                             "G_qp), psi the GPU mixed solution"}
    acc.pop("psi", None)
    extra = {}
    if not args.no_extra and world == 1:
        extra["large_block"] = large_block(pf, torch, args, stream, flush)
        extra["triangle_tree"] = triangle_tree(pf, torch, args, stream, flush, fp32_peak)
        extra["sweep_chunk"] = sweep_chunk(args)
        extra["warm_start_sweep"] = warm_start_sweep(args)
    h2d = int(npf_h.numel() * 4 + nodes_h.numel() * 8)
    d2h = int(psi_h.numel() * 16 + stats["norders"] * 2 * 16)
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": ("f64" if args.precision == "fp64" else
                      "f32/bf16x3+f64" if (opt.m2l_mode == 2 or plan.tc_levels) else "f32+f64"),
            "data": "synthetic",
            "config": {"workload": w.name, "elements": w.E, "unknowns": n, "fibers": w.M, "kH": w.k * w.H,
                       "tol": args.tol, "precision": args.precision, "depth": plan.depth,
                       "p": list(plan.p)[:plan.depth + 1],
                       "l2": "flushed between steps (256 MiB write); per-step working set is L2-resident by design",
                       "parallelism": f"replicas x{world}",
                       "matvec_launch": "one cooperative kernel" if args.launch == 0 else "one kernel per stage"},
            "matvec_munknowns_per_s": mv,
            "plain_fp64": {"solves_per_s": world * 1000.0 / ms_fp64, "ms_per_step": ms_fp64,
                           "iters": fp64_stats["iters"], "rel_residual": fp64_stats["rel_residual"],
                           "speedup_of_value": (world * 1000.0 / ms_step) / (world * 1000.0 / ms_fp64)},
            "solve": {"iters": stats["iters"], "restarts": stats["restarts"],
                      "rel_residual": stats["rel_residual"], "energy_sum": stats["energy"],
                      "setup_ms": plan.setup_ms},
            "phase_ms_per_step": {names[i]: float(ms_ph[i]) for i in range(len(names)) if names[i] and ms_ph[i] > 0},
            "roofline": roof,
            "roofline_p2p": roof_p2p,
            "err_vs_oracle": acc,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "clocks": clk,
            "gpu_launches": launches}
    line.update(extra)
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def solution_accuracy(pf, torch, w, opt, npf_d, nodes_d, sptr, tol, maxit):
    """Mixed solve at the bench tolerance against an FP64 solve at 1e-10 of the same
    block: relative L2 difference of the densities and the largest difference of the
    Bragg coefficients R_n, T_n."""
    o64 = pf.Options()
    o64.precision = pf.FP64
    out = {}
    sols = []
    for o, t in ((opt, tol), (o64, 1e-10)):
        psi = torch.zeros(2 * w.E, dtype=torch.complex128, device="cuda")
        h = pf.pfmbem_create(w.M, npf_d, nodes_d, w.H, w.lattice, w.k, w.k1, w.rho_ratio, w.theta, o, sptr)
        try:
            info = pf.pfmbem_solve(h, None, psi, False, t, maxit, check=False)
            orders, R, T, _ = pf.pfmbem_coefficients(h, psi)
        finally:
            pf.pfmbem_destroy(h)
        sols.append((psi.cpu().numpy(), R, T, info.rel_residual))
    (p1, R1, T1, r1), (p2, R2, T2, r2) = sols
    out["vs_fp64_tol1e-10"] = {"density_rel_l2": float(np.linalg.norm(p1 - p2) / np.linalg.norm(p2)),
                               "bragg_max_abs": float(max(np.max(np.abs(R1 - R2)), np.max(np.abs(T1 - T2)))),
                               "fp64_rel_residual": r2}
    out["psi"] = p1
    return out


def large_block(pf, torch, args, stream, flush, steps=5):
    """The 32x32 square block (131072 elements, kH = 20): create + mixed solve to the
    bench tolerance + Bragg coefficients, device buffers, L2 flushed between steps,
    against the plain FP64 solve of the same block."""
    from paper_1910_10863_gb300 import workloads as W
    w = W.square_32x32_n128()
    npf = torch.from_numpy(np.ascontiguousarray(w.nodes_per_fiber, dtype=np.int32)).cuda()
    nodes = torch.from_numpy(np.ascontiguousarray(w.nodes)).cuda()
    psi = torch.zeros(2 * w.E, dtype=torch.complex128, device="cuda")
    res = {}
    for name, prec in (("mixed", pf.MIXED), ("fp64", pf.FP64)):
        o = pf.Options()
        o.precision = prec
        info = None

        def one():
            nonlocal info
            h = pf.pfmbem_create(w.M, npf, nodes, w.H, w.lattice, w.k, w.k1, w.rho_ratio, w.theta, o,
                                 stream.cuda_stream)
            try:
                info = pf.pfmbem_solve(h, None, psi, False, args.tol, 2000, check=False)
                pf.pfmbem_coefficients(h, psi)
            finally:
                pf.pfmbem_destroy(h)
        one()
        tot = 0.0
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            one()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        res[name] = {"solves_per_s": 1000.0 * steps / tot, "iters": info.iters, "rel_residual": info.rel_residual}
    return {"workload": w.name, "elements": w.E, "unknowns": 2 * w.E, "steps": steps, **res,
            "speedup_mixed_over_fp64": res["mixed"]["solves_per_s"] / res["fp64"]["solves_per_s"]}


def triangle_tree(pf, torch, args, stream, flush, fp32_peak, steps=5, products=5):
    """The paper's regular-triangle tree (Sec. 3.1, Fig. 5) on the 8x8 hexagon block:
    create + FP64 solve to the bench tolerance + Bragg coefficients per step (device
    buffers, L2 flushed between steps), and the roofline of its dominant kernel, the
    M2L by offset groups in double-float arithmetic (phase "m2l" of the library's
    profile over a few products) on the FP32 pipes: flops = sum over levels of pairs
    x P^2 x 60 (four double-float multiply-adds of 15 FP32 flops per complex
    multiply-add)."""
    from paper_1910_10863_gb300 import workloads as W
    w = W.hexagon_8x8_n256()
    npf = torch.from_numpy(np.ascontiguousarray(w.nodes_per_fiber, dtype=np.int32)).cuda()
    nodes = torch.from_numpy(np.ascontiguousarray(w.nodes)).cuda()
    psi = torch.zeros(2 * w.E, dtype=torch.complex128, device="cuda")
    o = pf.Options()
    o.tree = 1
    o.leaf_max = 16
    for key, val in W.hexagon_block_lattice(w.H, 8).items():
        setattr(o, key, val)
    info = None

    def one():
        nonlocal info
        h = pf.pfmbem_create(w.M, npf, nodes, w.H, w.lattice, w.k, w.k1, w.rho_ratio, w.theta, o, stream.cuda_stream)
        try:
            info = pf.pfmbem_solve(h, None, psi, False, args.tol, 2000, check=False)
            pf.pfmbem_coefficients(h, psi)
        finally:
            pf.pfmbem_destroy(h)
    one()
    tot = 0.0
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        one()
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
    # products under the library's profile
    h = pf.pfmbem_create(w.M, npf, nodes, w.H, w.lattice, w.k, w.k1, w.rho_ratio, w.theta, o, stream.cuda_stream)
    try:
        plan = pf.pfmbem_plan(h)
        x = torch.ones(2 * w.E, dtype=torch.complex128, device="cuda")
        y = torch.zeros_like(x)
        pf.pfmbem_matvec(h, x.data_ptr(), y.data_ptr(), pf.FP64)
        torch.cuda.synchronize()
        pf.pfmbem_profile(h, True, True)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(products):
            pf.pfmbem_matvec(h, x.data_ptr(), y.data_ptr(), pf.FP64)
        e1.record(stream)
        e1.synchronize()
        prod_ms = e0.elapsed_time(e1) / products
        prof = pf.pfmbem_profile_read(h)
        m2l_ms = prof.ms[pf.PHASES.index("m2l")] / products
    finally:
        pf.pfmbem_destroy(h)
    flops = sum(plan.m2l_pairs_level[l] * (2 * plan.p[l] + 1) ** 2 * 60 for l in range(1, plan.depth + 1))
    ach = flops / (m2l_ms * 1e-3) / 1e12
    return {"workload": w.name, "tree": "regular triangles (64 hexagonal cells)", "elements": w.E, "steps": steps,
            "depth": plan.depth, "p": list(plan.p)[:plan.depth + 1], "precision": "fp64",
            "solves_per_s": 1000.0 * steps / tot, "iters": info.iters, "rel_residual": info.rel_residual,
            "product_ms": prod_ms,
            "roofline": {"kernel": "tri_m2l_dd_kernel (triangle tree, double-float M2L)", "bound": "alu",
                         "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                         "ms_per_product": m2l_ms, "flops_per_product": flops,
                         "peak_source": "FP32 FMA-chain probe (pfmbem_probe_peak)"}}


def sweep_chunk(args, count=128):
    """One chunk of the band-gap sweep: 128 instances of 16 fibers with 64-256
    elements each (kH in [0.5, 8]), plans from the autotuner, solved together by
    pfmbem_solve_batch (one persistent launch), wall time from the first create
    to the last coefficient; the batch call alone is timed too.  The first run
    tunes and warms up, the second is reported."""
    from paper_1910_10863_gb300 import sweep
    sweep.run(count=count, chunk=count, tol=args.tol, sequential_sample=2)
    r = sweep.run(count=count, chunk=count, tol=args.tol, sequential_sample=16)
    return {"instances": count, "batched_solves_per_s": r["batched_solves_per_s"],
            "batch_solve_only_per_s": r["batch_solve_only_per_s"], "create_seconds": r["create_seconds"],
            "sequential_solves_per_s": r["sequential_solves_per_s"], "all_converged": r["all_converged"],
            "max_rel_residual": r["max_rel_residual"], "mean_iters": r["mean_iters"],
            "elements": [r["elements_min"], r["elements_max"]], "tune_seconds": r["tune_seconds"],
            "launch": "one persistent cooperative launch for the whole chunk (groups of blocks per instance)"}


def warm_start_sweep(args, train=2048, test=512, epochs=300):
    """The learned warm start inside the batched sweep: the network (50 -> 3 x 256
    GELU -> 1088, trained on the GPU by the library's kernels on `train` sweep
    blocks solved in batched launches) predicts every held-out block's densities;
    features, one forward pass, decode and one persistent batched solve with the
    guesses are timed together, against the same blocks in one zero-start batch and
    against plain FP64 GMRES (pfmbem_solve one block after another).  A reduced
    form of the 8192 / 1024 training and held-out sets, to keep the bench short."""
    import time

    from paper_1910_10863_gb300 import warmstart as ws
    from paper_1910_10863_gb300 import workloads as W
    t0 = time.perf_counter()
    X, T, inst, _ = ws.generate_batched(W.batch_instances(train, seed=1912), tol=args.tol)
    net, hist = ws.train(X, T, epochs=epochs, batch=256, lr=1e-3)
    t1 = time.perf_counter()
    r = ws.evaluate_batched(net, W.batch_instances(test, seed=1915), tol=args.tol)
    r.update({"train_blocks": train, "epochs": epochs, "final_train_loss": hist[-1], "train_seconds": t1 - t0,
              "speedup_warm_batched_over_plain_fp64": r["batched_warm_start_solves_per_s"] / r["plain_fp64_solves_per_s"],
              "speedup_warm_over_zero_batched": r["batched_warm_start_solves_per_s"]
              / r["batched_zero_start_solves_per_s"]})
    return r


def pf_density(w):
    from paper_1910_10863_gb300 import workloads as W
    return W.density_vector(w.E, 11)


# Algorithmic work per unit.  Element-integral (P2P) evaluation: one unit = one
# kernel evaluation (target collocation point x Gauss node of a source element),
# 255 FP64 flops (2 per DFMA + DADD + DMUL, counted by ncu on the near-field and
# same-fiber cache-build kernels of the hexagon 8x8 block, series Hankel
# evaluation).  Cached applies: bytes of the resident operator plus the vectors
# they read and write.
FLOPS_PER_EVAL_FP64 = 255.0


def roofline_p2p(ms_ph, la_ph, steps, plan, fp64_peak):
    """Near-field and same-fiber element integrals (the P2P kernel evaluations, once per
    create): FP64 flops per evaluation x evaluations over the measured build time."""
    i = 10                                         # phase "p2p_cache_build"
    if not plan.cached or ms_ph[i] <= 0:
        return None
    units = plan.near_quad + plan.fiber_quad
    ms = ms_ph[i] / steps
    ach = units * FLOPS_PER_EVAL_FP64 / (ms * 1e-3) / 1e12
    return {"kernel": "p2p_cache_build (near_build, near_direct, fiber_build)", "bound": "alu",
            "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
            "ms_per_step": ms, "launches_per_step": la_ph[i] / steps, "units_per_step": int(units),
            "unit_def": "kernel evaluation (target x Gauss node x wavenumber), 255 FP64 flops",
            "peak_source": "FP64 FMA-chain probe (pfmbem_probe_peak)"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "MEASURED_PEAKS.json hbm_gbs (measured copy)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained"]), "MEASURED_PEAKS.json bf16_tflops_sustained (kernel inside a step)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback 1.7 PFLOP/s sustained"


# DRAM bytes (read + write) per launch of the single-launch matvec, from one
# ncu capture of the hexagon 8x8 block (profiles/matvec_fused_hexagon_8x8_n256.md;
# the mean of two launches each, cold caches).
# Valid only while the kernel source is the captured one: keyed by the sha256
# of matvec_fused.cu, else the line reports traffic null.
NCU_TRAFFIC = {
    "sha256": "23eb53664e42911a13ee1b18ed8c2ecfe8050027d6bce7bc24961810cd622839",
    ("hexagon_8x8_n256_kH5", "matvec_fused"): 189195648,
    ("hexagon_8x8_n256_kH5", "matvec_fused_f32"): 91566464,
}


def captured_traffic(workload, kernel):
    import hashlib
    src = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_1910_10863_gb300", "csrc", "matvec_fused.cu")
    try:
        with open(src, "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != NCU_TRAFFIC["sha256"]:
                return None
    except OSError:
        return None
    return NCU_TRAFFIC.get((workload, kernel))


def roofline(names, ms_ph, la_ph, steps, plan, fp64_peak, fp32_peak, E, tensor_m2l=False, workload="",
             real_f32_products=None):
    dom = int(np.argmax(ms_ph))
    name = names[dom]
    ms_step = ms_ph[dom] / steps
    launches = la_ph[dom] / steps
    per_launch = ms_step / max(launches, 1e-9)
    f32 = name.endswith("_f32")
    csz = 8 if f32 else 16
    hbm, hbm_src = measured_peaks()
    out = {"kernel": name, "ms_per_launch": per_launch, "launches_per_step": launches}
    if name == "matvec_fused_f32" and real_f32_products:
        # products queued after convergence return at once: divide the phase time by
        # the products that ran (the solve's inner iterations), not by the launches
        per_launch = ms_step / real_f32_products
        out.update(ms_per_launch=per_launch, products_per_step=real_f32_products,
                   note="phase time / products that ran; launches queued after convergence return at once")
    if name == "p2p_cache_build":
        units = plan.near_quad + plan.fiber_quad
        ach = units * FLOPS_PER_EVAL_FP64 / (ms_step * 1e-3) / 1e12
        out.update(bound="alu", achieved=ach, peak=fp64_peak, unit="TFLOP/s", frac=ach / fp64_peak, traffic=None,
                   peak_source="FP64 FMA-chain probe (pfmbem_probe_peak)", units_per_launch=int(units / 2),
                   unit_def="kernel evaluation, 255 FP64 flops")
    elif name.startswith("matvec_fused"):
        # the single-launch matvec streams the cached operators once per product:
        # near-field blocks, fiber row pairs / blocks, P2M and L2P coefficients,
        # plus x and y (FP64) and the sorted densities and potentials (written
        # and read back)
        PD = 2 * plan.p[plan.depth] + 1
        nbytes = ((plan.near_blocks * 4 + plan.fiber_entries + 2 * 2 * E * PD) * csz
                  + 2 * 2 * E * 16 + 2 * 2 * 2 * E * csz)
        ach = nbytes / (per_launch * 1e-3) / 1e9
        out.update(bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm,
                   traffic=captured_traffic(workload, name), peak_source=hbm_src, bytes_per_launch=int(nbytes))
    elif name.startswith("near_p2p") and plan.cached:
        nbytes = plan.near_blocks * 4 * csz + 2 * E * csz * 3
        ach = nbytes / (per_launch * 1e-3) / 1e9
        out.update(bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm, traffic=None,
                   peak_source=hbm_src, bytes_per_launch=int(nbytes))
    elif name.startswith("fiber_p2p_combine") and plan.cached:
        nbytes = plan.fiber_entries * csz + 2 * E * (16 + 16 + csz)
        ach = nbytes / (per_launch * 1e-3) / 1e9
        out.update(bound="hbm", achieved=ach, peak=hbm, unit="GB/s", frac=ach / hbm, traffic=None,
                   peak_source=hbm_src, bytes_per_launch=int(nbytes))
    elif name.startswith("m2l_l2l"):
        # algorithmic flops of one matvec's M2L: 8 (2p+1)^2 per translation; the
        # number of matvecs in the step is the launch count of the gather phase
        P = 2 * plan.p[plan.depth] + 1
        matvecs = la_ph[16 if f32 else 0] / steps
        flops = 8.0 * P * P * plan.m2l_pairs * matvecs
        ach = flops / (ms_step * 1e-3) / 1e12
        if f32 and tensor_m2l:
            peak, src = bf16_peak()
            out.update(bound="tensor", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak, traffic=None,
                       peak_source=src, note="algorithmic complex-M2L flops; the tensor cores issue 6 BF16 "
                                             "products of the real-embedded, padded operator")
        else:
            peak = fp32_peak if f32 else fp64_peak
            out.update(bound="alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak, traffic=None,
                       peak_source="FMA-chain probe (pfmbem_probe_peak)")
    else:
        out.update(bound="alu", achieved=None, peak=None, unit=None, frac=None, traffic=None)
    return out


if __name__ == "__main__":
    main()
