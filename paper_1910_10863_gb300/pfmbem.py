"""ctypes binding of the pfmbem C ABI (include/pfmbem.h).

Argument marshalling only: every computation runs in libpfmbem.so.  Buffers may
be torch tensors (CPU or CUDA), numpy arrays, or raw integer addresses; complex
vectors are complex128 (interleaved re/im doubles).  Loading fails loudly when
the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpfmbem.so")

FP64, MIXED = 0, 1
STATUS = {0: "OK", 1: "EINVAL", 2: "EGEOM", 3: "EWOOD", 4: "ENOMEM", 5: "ECUDA", 6: "ENOCONV", 7: "ETIMEOUT",
          8: "ENUMERIC"}


class Options(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("p_min", ctypes.c_int), ("eta", ctypes.c_double),
                ("leaf_max", ctypes.c_int), ("depth", ctypes.c_int), ("gmres_m", ctypes.c_int),
                ("precision", ctypes.c_int), ("near_mode", ctypes.c_int), ("m2l_mode", ctypes.c_int),
                ("profile", ctypes.c_int), ("launch", ctypes.c_int), ("precond", ctypes.c_int),
                ("wait_us", ctypes.c_int), ("p_min_mixed", ctypes.c_int), ("batch_group", ctypes.c_int),
                ("tree", ctypes.c_int), ("tri_a", ctypes.c_double), ("tri_ox", ctypes.c_double),
                ("tri_oy", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("restarts", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("ms", ctypes.c_double), ("status", ctypes.c_int)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("E", ctypes.c_int), ("M", ctypes.c_int), ("depth", ctypes.c_int), ("p", ctypes.c_int * 16),
                ("nleaf_nonempty", ctypes.c_int), ("m2l_pairs", ctypes.c_int64), ("near_pairs", ctypes.c_int64),
                ("near_quad", ctypes.c_int64), ("fiber_pairs", ctypes.c_int64), ("fiber_quad", ctypes.c_int64),
                ("p2m_nodes", ctypes.c_int), ("lattice_q", ctypes.c_int), ("root_x0", ctypes.c_double),
                ("root_y0", ctypes.c_double), ("setup_ms", ctypes.c_double), ("near_blocks", ctypes.c_int64),
                ("fiber_entries", ctypes.c_int64), ("cached", ctypes.c_int), ("tc_levels", ctypes.c_int),
                ("p32", ctypes.c_int * 16), ("m2l_pairs_level", ctypes.c_int64 * 16), ("nroot", ctypes.c_int),
                ("super_p", ctypes.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libpfmbem.so is not built ({LIB_PATH}); run paper_1910_10863_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        sigs = {
            "pfmbem_create": ([i, vp, vp, d, i, d, d, d, d, vp, vp, vp], i),
            "pfmbem_destroy": ([vp], None),
            "pfmbem_last_error": ([vp], ctypes.c_char_p),
            "pfmbem_plan": ([vp, vp], i),
            "pfmbem_rhs": ([vp, vp], i),
            "pfmbem_matvec": ([vp, vp, vp, i], i),
            "pfmbem_solve": ([vp, vp, vp, i, d, i, vp], i),
            "pfmbem_field": ([vp, vp, i, vp, vp], i),
            "pfmbem_coefficients": ([vp, vp, i, vp, vp, vp, vp, vp], i),
            "pfmbem_lattice_sums": ([vp, i, vp], i),
            "pfmbem_self_terms": ([vp, vp], i),
            "pfmbem_profile": ([vp, i, i], i),
            "pfmbem_profile_read": ([vp, vp], i),
            "pfmbem_probe_peak": ([i, vp], i),
            "pfmbem_lattice_sums_noalloc": ([d, d, d, i, vp, vp], i),
            "pfmbem_mlp_create": ([i, i, i, i, ctypes.c_uint64, vp, vp], i),
            "pfmbem_mlp_destroy": ([vp], None),
            "pfmbem_mlp_params": ([vp, vp, vp, vp], i),
            "pfmbem_mlp_forward": ([vp, i, vp, vp], i),
            "pfmbem_mlp_train": ([vp, i, vp, vp, ctypes.c_float, vp, vp], i),
            "pfmbem_field_dx1": ([vp, vp, i, vp, vp, vp], i),
            "pfmbem_etc": ([vp, vp, d, i, vp], i),
            "pfmbem_warm_features": ([vp, vp], i),
            "pfmbem_warm_features_local": ([vp, i, vp], i),
            "pfmbem_warm_targets": ([vp, i, vp, vp], i),
            "pfmbem_warm_decode": ([vp, i, vp, vp], i),
            "pfmbem_solve_batch": ([i, vp, vp, i, d, i, vp], i),
        }
        for name, (args, res) in sigs.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def addr(buf) -> int | None:
    """Address of a torch tensor, numpy array or integer (None passes NULL)."""
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    if hasattr(buf, "data_ptr"):
        return buf.data_ptr()
    if isinstance(buf, np.ndarray):
        return buf.ctypes.data
    raise TypeError(f"unsupported buffer type {type(buf)}")


class PfmbemError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _check(h, st):
    if st != 0:
        msg = lib().pfmbem_last_error(h).decode() if h else ""
        raise PfmbemError(st, msg)


def pfmbem_create(M, nodes_per_fiber, nodes_xy, H, lattice, k, k1, rho_ratio, theta, opt=None, stream=None):
    """Returns an opaque handle (int).  nodes_per_fiber int32[M], nodes_xy float64[sum N, 2]."""
    h = ctypes.c_void_p()
    st = lib().pfmbem_create(int(M), addr(nodes_per_fiber), addr(nodes_xy), float(H), int(lattice), float(k),
                             float(k1), float(rho_ratio), float(theta),
                             ctypes.byref(opt) if opt is not None else None, stream, ctypes.byref(h))
    if st != 0:
        msg = lib().pfmbem_last_error(h).decode() if h.value else ""
        if h.value:
            lib().pfmbem_destroy(h)
        raise PfmbemError(st, msg)
    return h.value


def pfmbem_destroy(h):
    lib().pfmbem_destroy(h)


def pfmbem_plan(h) -> PlanInfo:
    info = PlanInfo()
    _check(h, lib().pfmbem_plan(h, ctypes.byref(info)))
    return info


def pfmbem_rhs(h, B):
    _check(h, lib().pfmbem_rhs(h, addr(B)))


def pfmbem_matvec(h, x, y, precision=FP64):
    _check(h, lib().pfmbem_matvec(h, addr(x), addr(y), int(precision)))


def pfmbem_solve(h, B, psi, use_guess=False, tol=1e-8, maxit=1000, check=True) -> Info:
    info = Info()
    st = lib().pfmbem_solve(h, addr(B), addr(psi), int(bool(use_guess)), float(tol), int(maxit), ctypes.byref(info))
    if check:
        _check(h, st)
    return info


def pfmbem_solve_batch(handles, psis, tol=1e-6, maxit=2000, use_guess=False):
    """Solve of many handles in one persistent launch (host-driven lockstep when a
    handle cannot run in it); psis are complex128 buffers (host or device), read
    as initial guesses with use_guess."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*handles)
    ps = (ctypes.c_void_p * n)(*[addr(p) for p in psis])
    infos = (Info * n)()
    st = lib().pfmbem_solve_batch(n, hs, ps, int(bool(use_guess)), float(tol), int(maxit), infos)
    return st, list(infos)


def pfmbem_lattice_sums(h, jmax, S):
    _check(h, lib().pfmbem_lattice_sums(h, int(jmax), addr(S)))


def pfmbem_lattice_sums_noalloc(k, H, theta, jmax, S, stream=None):
    """Lattice sums without a handle or any device allocation (see include/pfmbem.h).

    S must be a contiguous complex128 torch tensor or numpy array with at least
    2 jmax + 1 entries: the library writes that many values unconditionally."""
    if isinstance(S, np.ndarray):
        ok = S.dtype == np.complex128 and S.flags.c_contiguous and S.size >= 2 * int(jmax) + 1
    elif hasattr(S, "data_ptr"):
        import torch
        ok = S.dtype == torch.complex128 and S.is_contiguous() and S.numel() >= 2 * int(jmax) + 1
    else:
        ok = False
    if not ok:
        raise ValueError("S must be a contiguous complex128 buffer of at least 2*jmax+1 entries")
    st = lib().pfmbem_lattice_sums_noalloc(float(k), float(H), float(theta), int(jmax), stream, addr(S))
    if st != 0:
        raise PfmbemError(st, "pfmbem_lattice_sums_noalloc failed")


def pfmbem_self_terms(h, out):
    _check(h, lib().pfmbem_self_terms(h, addr(out)))


def pfmbem_field(h, psi, pts, u):
    _check(h, lib().pfmbem_field(h, addr(psi), int(len(pts)), addr(pts), addr(u)))


def pfmbem_coefficients(h, psi, max_orders=64):
    n = ctypes.c_int(0)
    orders = np.zeros(max_orders, dtype=np.int32)
    R = np.zeros(max_orders, dtype=np.complex128)
    T = np.zeros(max_orders, dtype=np.complex128)
    en = ctypes.c_double(0)
    _check(h, lib().pfmbem_coefficients(h, addr(psi), max_orders, ctypes.byref(n), addr(orders), addr(R), addr(T),
                                        ctypes.byref(en)))
    c = n.value
    return orders[:c], R[:c], T[:c], en.value


PHASES = ["gather", "p2m", "m2m", "m2l_l2l", "l2p", "near_p2p", "fiber_p2p_combine", "gmres_blas", "setup",
          "outputs", "p2p_cache_build", "matvec_fused", "m2l", "", "", "",
          "gather_f32", "p2m_f32", "m2m_f32", "m2l_l2l_f32", "l2p_f32", "near_p2p_f32", "fiber_p2p_combine_f32",
          "", "", "", "", "matvec_fused_f32", "", "", "", ""]


class ProfileInfo(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 32), ("launches", ctypes.c_int64 * 32), ("total_launches", ctypes.c_int64)]


def pfmbem_profile(h, enable_timing=True, reset=True):
    _check(h, lib().pfmbem_profile(h, int(bool(enable_timing)), int(bool(reset))))


def pfmbem_profile_read(h) -> ProfileInfo:
    p = ProfileInfo()
    _check(h, lib().pfmbem_profile_read(h, ctypes.byref(p)))
    return p


def pfmbem_probe_peak(dtype) -> float:
    t = ctypes.c_double(0)
    st = lib().pfmbem_probe_peak(int(dtype), ctypes.byref(t))
    if st != 0:
        raise PfmbemError(st, "probe failed")
    return t.value


def _st(st, what):
    if st != 0:
        raise PfmbemError(st, what)


class MLP:
    """The warm-start network (pfmbem_mlp_*): FP32, GELU hidden layers."""

    def __init__(self, n_in, hidden, layers, n_out, seed=0, stream=None):
        h = ctypes.c_void_p()
        _st(lib().pfmbem_mlp_create(int(n_in), int(hidden), int(layers), int(n_out), int(seed), stream,
                                    ctypes.byref(h)), "pfmbem_mlp_create")
        self.h = h.value
        self.n_in, self.n_out = n_in, n_out

    def close(self):
        if self.h:
            lib().pfmbem_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def nparams(self):
        n = ctypes.c_int64(0)
        _st(lib().pfmbem_mlp_params(self.h, ctypes.byref(n), None, None), "pfmbem_mlp_params")
        return n.value

    def get_params(self):
        p = np.zeros(self.nparams(), dtype=np.float32)
        n = ctypes.c_int64(0)
        _st(lib().pfmbem_mlp_params(self.h, ctypes.byref(n), addr(p), None), "pfmbem_mlp_params")
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        n = ctypes.c_int64(0)
        _st(lib().pfmbem_mlp_params(self.h, ctypes.byref(n), None, addr(p)), "pfmbem_mlp_params")

    def forward(self, X, Y=None):
        X = np.ascontiguousarray(X, dtype=np.float32) if isinstance(X, np.ndarray) else X
        B = X.shape[0]
        if Y is None:
            Y = np.zeros((B, self.n_out), dtype=np.float32)
        _st(lib().pfmbem_mlp_forward(self.h, B, addr(X), addr(Y)), "pfmbem_mlp_forward")
        return Y

    def train(self, X, T, lr=0.0, want_grad=False):
        """MSE loss (and gradient); lr > 0 takes one Adam step."""
        X = np.ascontiguousarray(X, dtype=np.float32) if isinstance(X, np.ndarray) else X
        T = np.ascontiguousarray(T, dtype=np.float32) if isinstance(T, np.ndarray) else T
        loss = ctypes.c_float(0)
        g = np.zeros(self.nparams(), dtype=np.float32) if want_grad else None
        _st(lib().pfmbem_mlp_train(self.h, X.shape[0], addr(X), addr(T), float(lr), ctypes.byref(loss), addr(g)),
            "pfmbem_mlp_train")
        return (loss.value, g) if want_grad else loss.value


def pfmbem_field_dx1(h, psi, pts, u=None, dudx1=None):
    """Scattered field and its x1-derivative at pts [n][2] (outputs complex [n])."""
    pts = np.ascontiguousarray(pts, dtype=np.float64) if isinstance(pts, np.ndarray) else pts
    n = len(pts)
    _check(h, lib().pfmbem_field_dx1(h, addr(psi), n, addr(pts), addr(u), addr(dudx1)))
    return u, dudx1


def pfmbem_etc(h, psi, x1, npts=256):
    v = ctypes.c_double(0)
    _check(h, lib().pfmbem_etc(h, addr(psi), float(x1), int(npts), ctypes.byref(v)))
    return v.value


def pfmbem_warm_features(h, M):
    x = np.zeros(2 + 3 * M, dtype=np.float32)
    _check(h, lib().pfmbem_warm_features(h, addr(x)))
    return x


def pfmbem_warm_features_local(h, M, K=15):
    x = np.zeros((M, 5 + 3 * K), dtype=np.float32)
    _check(h, lib().pfmbem_warm_features_local(h, int(K), addr(x)))
    return x


def pfmbem_warm_targets(h, psi, M, nmodes=8):
    t = np.zeros(M * 2 * (2 * nmodes + 1) * 2, dtype=np.float32)
    _check(h, lib().pfmbem_warm_targets(h, int(nmodes), addr(psi), addr(t)))
    return t


def pfmbem_warm_decode(h, y, psi0, nmodes=8):
    y = np.ascontiguousarray(y, dtype=np.float32) if isinstance(y, np.ndarray) else y
    _check(h, lib().pfmbem_warm_decode(h, int(nmodes), addr(y), addr(psi0)))


class Solver:
    """Owns one pfmbem handle for a workload (see workloads.Workload)."""

    def __init__(self, w, opt: Options | None = None, stream=None, **kw):
        if opt is None:
            opt = Options()
        for key, val in kw.items():
            setattr(opt, key, val)
        self.w = w
        self._npf = np.ascontiguousarray(w.nodes_per_fiber, dtype=np.int32)
        self._nodes = np.ascontiguousarray(w.nodes, dtype=np.float64)
        self.h = pfmbem_create(w.M, self._npf, self._nodes, w.H, w.lattice, w.k, w.k1, w.rho_ratio, w.theta,
                               opt, stream)
        self.E = int(self._npf.sum())

    def close(self):
        if self.h:
            pfmbem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plan(self):
        return pfmbem_plan(self.h)

    def matvec(self, x, y, precision=FP64):
        pfmbem_matvec(self.h, x, y, precision)

    def rhs(self, B):
        pfmbem_rhs(self.h, B)

    def solve(self, psi, B=None, tol=1e-8, maxit=1000, use_guess=False, check=True):
        return pfmbem_solve(self.h, B, psi, use_guess, tol, maxit, check)
