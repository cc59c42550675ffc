"""ORACLE — test infrastructure only.

A plain FP64 CPU implementation of the D-iteration hot path (oracle.c), written from the paper
("Revisiting the D-iteration method: runtime comparison", Sections 2.3-2.5). Only the tests,
`__graft_entry__.smoke()` and the benchmark's CPU-baseline leg may import it. It shares no code
with the CUDA library in `paper_1204_6255_gb300`, and the library never imports it.

Parity status of each function (what pins it lives in tests/test_oracle_*.py):
  build, zero_in, zero_in_naive  pinned: brute force on tiny graphs, hand cases, naive == peeling
  di (DI-CYC, DI-SOP)            pinned: dense direct solve, closed forms, exact rational golden
                                 fixtures, mass invariant, identity X = H + (I-P)^-1 F
  di_refresh (DI-SOP, r taken    pinned: equals di bit for bit when r is taken once per cycle,
    every r_every ids)           dense direct solve, identity X = H + (I-P)^-1 F, a hand case
                                 where the refreshed r admits a node the cycle's r would not
  pi                             pinned: dense direct solve, closed forms
  pi_paper                       pinned: equals X / ||X||_1 for uniform B (derived invariant)
  residual                       pinned: zero at the dense solution, equals the remaining fluid
                                 of a partial D-iteration
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_oracle.so")
_lock = threading.Lock()
_libs: dict = {}

CYC = 0
SOP = 1


class DiInfo(ctypes.Structure):
    _fields_ = [
        ("cycles", ctypes.c_int64),
        ("visits", ctypes.c_int64),
        ("pushed_edges", ctypes.c_int64),
        ("fallback_cycles", ctypes.c_int64),
        ("e", ctypes.c_double),
        ("residual", ctypes.c_double),
        ("paper_error", ctypes.c_double),
        ("e_visits", ctypes.c_int64),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PiInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int64), ("residual", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def build_lib(force: bool = False, src: str = _SRC, out: str = _LIB) -> str:
    """Compile oracle.c (or another copy of it: the planted-mistake test compiles mutated
    copies) with gcc into a shared object."""
    with _lock:
        if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
            tmp = out + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-o", tmp, src, "-lm"])
            os.replace(tmp, out)
    return out


def _load():
    if "lib" in _libs:
        return _libs["lib"]
    # DI_ORACLE_LIB points the whole pin suite at a mutated copy of the oracle (planted-mistake
    # test only); normally the library is built from oracle.c.
    override = os.environ.get("DI_ORACLE_LIB")
    lib = ctypes.CDLL(override if override else build_lib())
    vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
    lib.or_build.restype = i64
    lib.or_build.argtypes = [i64, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.or_zero_in.restype = i64
    lib.or_zero_in.argtypes = [i64, vp, vp, vp, vp, vp, vp]
    lib.or_zero_in_naive.restype = i64
    lib.or_zero_in_naive.argtypes = [i64, vp, vp, vp, vp, vp]
    lib.or_di.restype = ctypes.c_int
    lib.or_di.argtypes = [i64, i64, vp, vp, vp, vp, dbl, dbl, ctypes.c_int, i64, vp, vp,
                          ctypes.POINTER(DiInfo)]
    lib.or_di_refresh.restype = ctypes.c_int
    lib.or_di_refresh.argtypes = [i64, i64, vp, vp, vp, vp, dbl, dbl, i64, i64, vp, vp, ctypes.POINTER(DiInfo)]
    lib.or_di_e.restype = ctypes.c_int
    lib.or_di_e.argtypes = [i64, i64, vp, vp, vp, vp, vp, ctypes.c_int32, vp, dbl, dbl, ctypes.c_int, i64, vp, vp,
                            ctypes.POINTER(DiInfo)]
    lib.or_di_from.restype = ctypes.c_int
    lib.or_di_from.argtypes = [i64, i64, vp, vp, vp, vp, vp, dbl, dbl, ctypes.c_int, i64, vp, vp, ctypes.POINTER(DiInfo)]
    lib.or_pi.restype = ctypes.c_int
    lib.or_pi.argtypes = [i64, vp, vp, vp, vp, dbl, dbl, i64, vp, ctypes.POINTER(PiInfo)]
    lib.or_pi_push.restype = ctypes.c_int
    lib.or_pi_push.argtypes = [i64, vp, vp, vp, dbl, dbl, i64, vp, ctypes.POINTER(PiInfo)]
    lib.or_pi_paper.restype = ctypes.c_int
    lib.or_pi_paper.argtypes = [i64, vp, vp, vp, dbl, dbl, i64, vp, ctypes.POINTER(PiInfo)]
    lib.or_residual.restype = dbl
    lib.or_residual.argtypes = [i64, vp, vp, vp, vp, dbl, vp, vp]
    _libs["lib"] = lib
    return lib


def _c(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


class Graph:
    """Iterators of the oracle: out-CSR (columns of P), in-CSR (rows of P), degrees, loops."""

    def __init__(self, n, rp_out, col_out, rp_in, col_in, outdeg, indeg, loop, stats):
        self.n = int(n)
        self.rp_out, self.col_out = rp_out, col_out
        self.rp_in, self.col_in = rp_in, col_in
        self.outdeg, self.indeg, self.loop = outdeg, indeg, loop
        self.L, self.D, self.O, self.max_in, self.max_out = (int(x) for x in stats)


def build(n: int, src, dst) -> Graph:
    """Iterator build (Section 2.1 "Init", Section 2.4). Raises ValueError on an id outside [0, n)."""
    lib = _load()
    src, ps = _c(src, np.int32)
    dst, pd = _c(dst, np.int32)
    m = len(src)
    rp_out = np.zeros(n + 1, np.int64)
    rp_in = np.zeros(n + 1, np.int64)
    col_out = np.zeros(max(m, 1), np.int32)
    col_in = np.zeros(max(m, 1), np.int32)
    outdeg = np.zeros(n, np.int32)
    indeg = np.zeros(n, np.int32)
    loop = np.zeros(n, np.uint8)
    stats = np.zeros(5, np.int64)
    L = lib.or_build(n, m, ps, pd, rp_out.ctypes.data, col_out.ctypes.data, rp_in.ctypes.data,
                     col_in.ctypes.data, outdeg.ctypes.data, indeg.ctypes.data, loop.ctypes.data,
                     stats.ctypes.data)
    if L < 0:
        raise ValueError(f"edge {-L - 1} has an id outside [0, {n})")
    return Graph(n, rp_out, col_out[:L].copy(), rp_in, col_in[:L].copy(), outdeg, indeg, loop, stats)


def zero_in(g: Graph):
    """E by peeling. Returns (e_mask uint8[n], level int32[n], |E|, n_levels)."""
    lib = _load()
    e_mask = np.zeros(g.n, np.uint8)
    level = np.zeros(g.n, np.int32)
    nl = ctypes.c_int32(0)
    cnt = lib.or_zero_in(g.n, g.rp_out.ctypes.data, g.col_out.ctypes.data, g.indeg.ctypes.data,
                         e_mask.ctypes.data, level.ctypes.data, ctypes.byref(nl))
    return e_mask, level, int(cnt), int(nl.value)


def zero_in_naive(g: Graph):
    """E by its definition iterated to the least fixpoint. Same return as zero_in."""
    lib = _load()
    e_mask = np.zeros(g.n, np.uint8)
    level = np.zeros(g.n, np.int32)
    nl = ctypes.c_int32(0)
    cnt = lib.or_zero_in_naive(g.n, g.rp_in.ctypes.data, g.col_in.ctypes.data,
                               e_mask.ctypes.data, level.ctypes.data, ctypes.byref(nl))
    return e_mask, level, int(cnt), int(nl.value)


def di(g: Graph, B, d: float, tol: float, schedule: int = SOP, max_cycles: int = 100_000):
    """Sequential D-iteration (Section 2.5), at most max_cycles cycles (< 0: no cap).
    Returns (H, F, info dict, converged)."""
    lib = _load()
    B, pb = _c(B, np.float64)
    H = np.zeros(g.n, np.float64)
    F = np.zeros(g.n, np.float64)
    info = DiInfo()
    rc = lib.or_di(g.n, g.L, g.rp_out.ctypes.data, g.col_out.ctypes.data, g.loop.ctypes.data, pb,
                   d, tol, schedule, max_cycles, H.ctypes.data, F.ctypes.data, ctypes.byref(info))
    return H, F, info.as_dict(), rc == 0


def di_refresh(g: Graph, B, d: float, tol: float, r_every: int, max_cycles: int = 100_000):
    """DI-SOP with r = ||F||_1 taken again every r_every node ids within a cycle (r_every <= 0
    or >= N: the plain DI-SOP of di). Returns (H, F, info dict, converged)."""
    lib = _load()
    B, pb = _c(B, np.float64)
    H = np.zeros(g.n, np.float64)
    F = np.zeros(g.n, np.float64)
    info = DiInfo()
    rc = lib.or_di_refresh(g.n, g.L, g.rp_out.ctypes.data, g.col_out.ctypes.data, g.loop.ctypes.data, pb,
                           d, tol, int(r_every), max_cycles, H.ctypes.data, F.ctypes.data, ctypes.byref(info))
    return H, F, info.as_dict(), rc == 0


def di_e(g: Graph, B, d: float, tol: float, schedule: int = SOP, max_cycles: int = 100_000):
    """D-iteration after the E-level pre-diffusion (every node of E visited once in level order,
    Section 2.4). Returns (H, F, info dict, converged); info["e_visits"] counts the pre-pass."""
    lib = _load()
    B, pb = _c(B, np.float64)
    e_mask, level, _, n_levels = zero_in(g)
    H = np.zeros(g.n, np.float64)
    F = np.zeros(g.n, np.float64)
    info = DiInfo()
    rc = lib.or_di_e(g.n, g.L, g.rp_out.ctypes.data, g.col_out.ctypes.data, g.loop.ctypes.data,
                     e_mask.ctypes.data, level.ctypes.data, n_levels, pb, d, tol, schedule, max_cycles,
                     H.ctypes.data, F.ctypes.data, ctypes.byref(info))
    return H, F, info.as_dict(), rc == 0


def di_from(g: Graph, H0, F0, d: float, tol: float, schedule: int = SOP, max_cycles: int = 100_000):
    """D-iteration from the state (H0, F0) instead of (0, B). Returns (H, F, info dict, converged)."""
    lib = _load()
    H0, p_h = _c(H0, np.float64)
    F0, p_f = _c(F0, np.float64)
    H = np.zeros(g.n, np.float64)
    F = np.zeros(g.n, np.float64)
    info = DiInfo()
    rc = lib.or_di_from(g.n, g.L, g.rp_out.ctypes.data, g.col_out.ctypes.data, g.loop.ctypes.data, p_h, p_f, d,
                        tol, schedule, max_cycles, H.ctypes.data, F.ctypes.data, ctypes.byref(info))
    return H, F, info.as_dict(), rc == 0


def pi(g: Graph, B, d: float, tol: float, max_iters: int = 100000):
    """Jacobi power iteration on X = P.X + B from X_0 = 0. Returns (X, info dict, converged)."""
    lib = _load()
    B, pb = _c(B, np.float64)
    X = np.zeros(g.n, np.float64)
    info = PiInfo()
    rc = lib.or_pi(g.n, g.rp_in.ctypes.data, g.col_in.ctypes.data, g.outdeg.ctypes.data, pb, d, tol,
                   max_iters, X.ctypes.data, ctypes.byref(info))
    return X, info.as_dict(), rc == 0


def pi_push(g: Graph, B, d: float, tol: float, max_iters: int = 100000):
    """Power iteration per column (PI'): the Jacobi iteration formed by scattering over the
    out-links. Returns (X, info dict, converged)."""
    lib = _load()
    B, pb = _c(B, np.float64)
    X = np.zeros(g.n, np.float64)
    info = PiInfo()
    rc = lib.or_pi_push(g.n, g.rp_out.ctypes.data, g.col_out.ctypes.data, pb, d, tol, max_iters, X.ctypes.data,
                        ctypes.byref(info))
    return X, info.as_dict(), rc == 0


def pi_paper(g: Graph, d: float, tol: float, max_iters: int = 100000):
    """The paper's normalised PageRank power iteration. Returns (x, info dict, converged)."""
    lib = _load()
    x = np.zeros(g.n, np.float64)
    info = PiInfo()
    rc = lib.or_pi_paper(g.n, g.rp_in.ctypes.data, g.col_in.ctypes.data, g.outdeg.ctypes.data, d, tol,
                         max_iters, x.ctypes.data, ctypes.byref(info))
    return x, info.as_dict(), rc == 0


def residual(g: Graph, B, d: float, H):
    """F* = B + P.H - H. Returns (F*, ||F*||_1)."""
    lib = _load()
    B, pb = _c(B, np.float64)
    H, ph = _c(H, np.float64)
    Fs = np.zeros(g.n, np.float64)
    norm = lib.or_residual(g.n, g.rp_in.ctypes.data, g.col_in.ctypes.data, g.outdeg.ctypes.data, pb, d,
                           ph, Fs.ctypes.data)
    return Fs, float(norm)


def uniform_B(n: int, d: float) -> np.ndarray:
    """PageRank right-hand side of the paper: B_i = (1 - d) / N (Section 2.5 DI-CYC init)."""
    return np.full(n, (1.0 - d) / n, dtype=np.float64)


def ppr_B(n: int, seeds, d: float) -> np.ndarray:
    """Personalised right-hand side: mass (1 - d) spread evenly over the seed nodes."""
    B = np.zeros(n, dtype=np.float64)
    seeds = np.asarray(seeds)
    B[seeds] = (1.0 - d) / len(seeds)
    return B
