"""GB300 (sm_103a) D-iteration: Python binding of the C ABI in include/di.h.

The functions here carry the C names and only marshal arguments: every step of the graph build
and of the solves runs in the CUDA library `_lib/libdi_gb300.so` (built from `csrc/` by
`build()`). Arrays may be numpy arrays (host) or torch tensors (host or CUDA); pointers go to the
library as they are, and CUDA work is ordered on torch's current stream when a CUDA tensor is
involved. There is no CPU fallback: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import LIB as _LIB_PATH, build as _build

__all__ = [
    "build", "load", "DiError", "Graph",
    "DI_CYC", "DI_SOP", "DI_FLUID_F32", "DI_FLUID_F64",
    "di_graph_create", "di_graph_destroy", "di_graph_stats_get", "di_graph_export",
    "di_solve", "di_solve_ex", "di_solve_resume", "di_power_iter", "di_power_iter_ex", "di_power_iter_push", "di_solve_batch", "di_ppr_batch", "di_residual_noalloc",
    "di_server_create", "di_server_submit", "di_server_wait", "di_server_destroy", "Server",
    "di_csr_validate", "di_graph_validate", "di_last_error", "di_version",
    "DI_WS_SOLVE", "DI_WS_BATCH", "di_workspace_size", "di_graph_set_workspace", "di_device_bytes_held",
    "di_autotune",
]

DI_CYC, DI_SOP = 0, 1
DI_WS_SOLVE, DI_WS_BATCH = 0, 1
NOALLOC_MAX_NODES = 1 << 20   # largest n di_residual_noalloc's static scratch holds
DI_FLUID_F32, DI_FLUID_F64 = 0, 1
STATUS = {0: "DI_OK", 1: "DI_ERR_INVALID_ARG", 2: "DI_ERR_OUT_OF_RANGE_ID", 3: "DI_ERR_OOM", 4: "DI_ERR_CUDA",
          5: "DI_ERR_NOT_CONVERGED", 6: "DI_ERR_BUSY", 7: "DI_ERR_TIMEOUT", 8: "DI_ERR_CORRUPT"}
ARRAYS = {  # di_array id -> (numpy dtype, length kind)
    "rowptr_out": (0, np.int64, "n+1"), "col_out": (1, np.int32, "L"), "rowptr_in": (2, np.int64, "n+1"),
    "col_in": (3, np.int32, "L"), "out_deg": (4, np.int32, "n"), "in_deg": (5, np.int32, "n"),
    "loop": (6, np.uint8, "n"), "e_mask": (7, np.uint8, "n"), "e_level": (8, np.int32, "n"),
}


class DiError(RuntimeError):
    """A non-zero di_status. `info` holds the call's report when it has one (a solve that hit its
    sweep cap still reports its state, and its outputs hold the current history)."""

    def __init__(self, status: int, message: str, info: dict | None = None):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message
        self.info = info


class GraphStats(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("L", ctypes.c_int64), ("D", ctypes.c_int64), ("E", ctypes.c_int64),
                ("O", ctypes.c_int64), ("max_in", ctypes.c_int32), ("max_out", ctypes.c_int32),
                ("e_levels", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("fluid", ctypes.c_int32), ("max_sweeps", ctypes.c_int32),
                ("refine", ctypes.c_int32), ("host_loop", ctypes.c_int32), ("rhs_tile", ctypes.c_int32),
                ("profile", ctypes.c_int32), ("e_prediffuse", ctypes.c_int32), ("r_refresh", ctypes.c_int32),
                ("exact_r", ctypes.c_int32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("d", ctypes.c_double), ("slots", ctypes.c_int32), ("sweeps_per_step", ctypes.c_int32),
                ("max_request_sweeps", ctypes.c_int32), ("tile_min_queue", ctypes.c_int32),
                ("mem_budget", ctypes.c_int64)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("sweeps", ctypes.c_int32), ("graph", ctypes.c_int32),
                ("slot", ctypes.c_int32), ("residual_l1", ctypes.c_double), ("queue_ms", ctypes.c_double),
                ("service_ms", ctypes.c_double), ("total_ms", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(ctypes.Structure):
    _fields_ = [("push_row", ctypes.c_int32), ("heavy_cut", ctypes.c_int32), ("heavy_chunk", ctypes.c_int32),
                ("rhs_tile", ctypes.c_int32), ("batch_heavy_cut", ctypes.c_int32),
                ("batch_heavy_chunk", ctypes.c_int32), ("single_probe_ms", ctypes.c_double),
                ("batch_rate", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class SolveInfo(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int32), ("refine_rounds", ctypes.c_int32), ("pushed_edges", ctypes.c_int64),
                ("visited_nodes", ctypes.c_int64), ("residual_l1", ctypes.c_double),
                ("dangling_mass_e", ctypes.c_double), ("paper_error", ctypes.c_double), ("ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("frontier_entries", ctypes.c_int64),
                ("select_ms", ctypes.c_double), ("push_ms", ctypes.c_double), ("reduce_ms", ctypes.c_double),
                ("refine_ms", ctypes.c_double), ("select_launches", ctypes.c_int32),
                ("push_launches", ctypes.c_int32), ("reduce_launches", ctypes.c_int32),
                ("refine_launches", ctypes.c_int32), ("rhs_tile", ctypes.c_int32), ("e_visits", ctypes.c_int32),
                ("column_links", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def build(force: bool = False) -> str:
    """Compile the CUDA library in-tree (nvcc, sm_103a)."""
    return _build(force=force)


def load(path: str | None = None):
    """Load the CUDA library (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _LIB_PATH
    if not os.path.exists(path):
        raise OSError(f"CUDA library {path} is missing: run paper_1204_6255_gb300.build() first")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    st = ctypes.c_int
    lib.di_graph_create.restype = st
    lib.di_graph_create.argtypes = [i32, vp, vp, i64, vp, ctypes.POINTER(vp)]
    lib.di_graph_destroy.restype = None
    lib.di_graph_destroy.argtypes = [vp]
    lib.di_graph_stats_get.restype = st
    lib.di_graph_stats_get.argtypes = [vp, ctypes.POINTER(GraphStats)]
    lib.di_graph_export.restype = st
    lib.di_graph_export.argtypes = [vp, i32, vp, i64, vp]
    lib.di_solve.restype = st
    lib.di_solve.argtypes = [vp, vp, dbl, dbl, i32, i32, vp, vp, ctypes.POINTER(SolveInfo), vp]
    lib.di_solve_ex.restype = st
    lib.di_solve_ex.argtypes = [vp, vp, dbl, dbl, ctypes.POINTER(SolveOpts), vp, vp, ctypes.POINTER(SolveInfo), vp]
    lib.di_power_iter.restype = st
    lib.di_power_iter.argtypes = [vp, vp, dbl, dbl, i32, vp, vp, ctypes.POINTER(SolveInfo), vp]
    lib.di_power_iter_ex.restype = st
    lib.di_power_iter_ex.argtypes = [vp, vp, dbl, dbl, ctypes.POINTER(SolveOpts), vp, vp, ctypes.POINTER(SolveInfo), vp]
    lib.di_solve_resume.restype = st
    lib.di_solve_resume.argtypes = [vp, vp, vp, vp, dbl, dbl, ctypes.POINTER(SolveOpts), vp, vp, vp,
                                    ctypes.POINTER(SolveInfo), vp]
    lib.di_csr_validate.restype = st
    lib.di_csr_validate.argtypes = [i32, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.di_graph_validate.restype = st
    lib.di_graph_validate.argtypes = [vp]
    lib.di_power_iter_push.restype = st
    lib.di_power_iter_push.argtypes = [vp, vp, dbl, dbl, i32, i32, vp, vp, ctypes.POINTER(SolveInfo), vp]
    lib.di_solve_batch.restype = st
    lib.di_solve_batch.argtypes = [vp, i32, vp, dbl, vp, ctypes.POINTER(SolveOpts), vp, vp, ctypes.POINTER(SolveInfo), vp]
    lib.di_ppr_batch.restype = st
    lib.di_ppr_batch.argtypes = [vp, i32, vp, vp, dbl, vp, ctypes.POINTER(SolveOpts), vp, vp,
                                 ctypes.POINTER(SolveInfo), vp]
    lib.di_server_create.restype = st
    lib.di_server_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]
    lib.di_server_submit.restype = st
    lib.di_server_submit.argtypes = [vp, i32, vp, i32, dbl, ctypes.POINTER(ctypes.c_int64)]
    lib.di_server_wait.restype = st
    lib.di_server_wait.argtypes = [vp, ctypes.c_int64, vp, ctypes.POINTER(RequestInfo), i32]
    lib.di_server_destroy.restype = None
    lib.di_server_destroy.argtypes = [vp]
    lib.di_residual_noalloc.restype = st
    lib.di_residual_noalloc.argtypes = [i32, vp, vp, vp, vp, dbl, vp, vp, vp, vp]
    lib.di_workspace_size.restype = st
    lib.di_workspace_size.argtypes = [vp, i32, i32, ctypes.POINTER(ctypes.c_int64)]
    lib.di_graph_set_workspace.restype = st
    lib.di_graph_set_workspace.argtypes = [vp, i32, vp, i64]
    lib.di_autotune.restype = st
    lib.di_autotune.argtypes = [vp, dbl, i32, ctypes.POINTER(Tuning), vp]
    lib.di_device_bytes_held.restype = i64
    lib.di_device_bytes_held.argtypes = []
    lib.di_last_error.restype = ctypes.c_char_p
    lib.di_last_error.argtypes = []
    lib.di_version.restype = ctypes.c_char_p
    lib.di_version.argtypes = []
    _lib = lib
    return lib


# ------------------------------------------------------------------------------------------
# marshalling helpers
# ------------------------------------------------------------------------------------------
def _is_torch(x) -> bool:
    return hasattr(x, "data_ptr") and hasattr(x, "is_cuda")


def _ptr(x, dtype):
    """Raw pointer of a contiguous numpy array or torch tensor of the given numpy dtype."""
    if x is None:
        return None
    if _is_torch(x):
        import torch
        tmap = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64, np.uint8: torch.uint8}
        if x.dtype != tmap[np.dtype(dtype).type] or not x.is_contiguous():
            raise TypeError(f"expected a contiguous {np.dtype(dtype)} tensor, got {x.dtype}")
        return x.data_ptr()
    if not isinstance(x, np.ndarray) or x.dtype != np.dtype(dtype) or not x.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a contiguous numpy {np.dtype(dtype)} array")
    return x.ctypes.data


def _stream(*arrays):
    for a in arrays:
        if _is_torch(a) and a.is_cuda:
            import torch
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


def _numel(x) -> int:
    return int(x.numel()) if _is_torch(x) else int(np.asarray(x).size)


def _need(n: int, **arrays):
    """Raises DiError (invalid argument) when an array given is shorter than its required
    length; the library takes lengths from the graph, not from the arrays."""
    for name, x in arrays.items():
        if x is not None and _numel(x) < n:
            raise DiError(1, f"{name} has {_numel(x)} entries; this call needs {n}")


def _check(status: int, info=None):
    if status != 0:
        raise DiError(status, load().di_last_error().decode(), info.as_dict() if info is not None else None)


def _like(x, n: int, dtype):
    if _is_torch(x):
        import torch
        return torch.empty(n, dtype=torch.float64, device=x.device)
    return np.empty(n, dtype=dtype)


# ------------------------------------------------------------------------------------------
# C ABI, same names
# ------------------------------------------------------------------------------------------
class Graph:
    """Owning wrapper of a di_graph handle."""

    def __init__(self, handle: int, n: int):
        self.handle = handle
        self.n = n
        self._stats = None
        self.workspaces = {}   # kind -> the caller's buffer while attached (kept alive here)

    @property
    def stats(self) -> dict:
        if self._stats is None:
            self._stats = di_graph_stats_get(self)
        return self._stats

    def close(self):
        if self.handle:
            load().di_graph_destroy(self.handle)
            self.handle = None
            self.workspaces = {}

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def di_graph_create(n_nodes: int, src, dst) -> Graph:
    lib = load()
    h = ctypes.c_void_p()
    m = int(src.shape[0])
    if int(dst.shape[0]) != m:
        raise ValueError("src and dst differ in length")
    _check(lib.di_graph_create(int(n_nodes), _ptr(src, np.int32), _ptr(dst, np.int32), m, _stream(src, dst),
                               ctypes.byref(h)))
    return Graph(h.value, int(n_nodes))


def di_graph_destroy(g: Graph):
    g.close()


def di_workspace_size(g: Graph, kind: int, param: int = 0) -> int:
    """Bytes of device scratch the solves of `kind` (DI_WS_SOLVE with param = fluid, DI_WS_BATCH
    with param = widest tile) need on this graph."""
    b = ctypes.c_int64()
    _check(load().di_workspace_size(g.handle, int(kind), int(param), ctypes.byref(b)))
    return b.value


def di_graph_set_workspace(g: Graph, kind: int, workspace=None):
    """Attach a caller-owned device buffer (a CUDA tensor, e.g. torch.empty(bytes, dtype=uint8,
    device='cuda')) as the scratch of the solves of `kind`, or detach it (None). The graph keeps a
    reference to the tensor while it is attached."""
    if workspace is None:
        _check(load().di_graph_set_workspace(g.handle, int(kind), None, 0))
        g.workspaces.pop(int(kind), None)
        return
    if not (_is_torch(workspace) and workspace.is_cuda and workspace.is_contiguous()):
        raise DiError(1, "the workspace must be a contiguous CUDA tensor")
    nbytes = workspace.numel() * workspace.element_size()
    _check(load().di_graph_set_workspace(g.handle, int(kind), workspace.data_ptr(), int(nbytes)))
    g.workspaces[int(kind)] = workspace


def di_autotune(g: Graph, d: float = 0.85, what: int = 3, set_split=None) -> dict:
    """Tune the push split on this graph (bit 0: single right-hand side, bit 1: batched; 0 only
    reports). set_split=(row, heavy_cut, heavy_chunk) sets the single right-hand-side split
    without probing. Returns the values in use."""
    t = Tuning()
    if set_split is not None:
        t.push_row, t.heavy_cut, t.heavy_chunk = (int(x) for x in set_split)
        what |= 4
    _check(load().di_autotune(g.handle, float(d), int(what), ctypes.byref(t), None))
    return t.as_dict()


def di_device_bytes_held() -> int:
    """Device bytes the library holds from its own allocations (all graphs of the process)."""
    return int(load().di_device_bytes_held())


def di_graph_stats_get(g: Graph) -> dict:
    s = GraphStats()
    _check(load().di_graph_stats_get(g.handle, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in s._fields_ if k != "reserved"}


def di_graph_export(g: Graph, which: str, out=None):
    """Copy an internal array ("rowptr_out", "col_out", "rowptr_in", "col_in", "out_deg", "in_deg",
    "loop", "e_mask", "e_level") into `out` (numpy or torch), or a new numpy array."""
    code, dtype, kind = ARRAYS[which]
    st = g.stats
    length = {"n+1": g.n + 1, "L": st["L"], "n": g.n}[kind]
    if out is None:
        out = np.empty(length, dtype=dtype)
    nbytes = out.numel() * out.element_size() if _is_torch(out) else out.nbytes
    _check(load().di_graph_export(g.handle, code, _ptr(out, dtype), nbytes, _stream(out)))
    return out


def di_solve(g: Graph, B, d: float, tol: float, schedule: int = DI_SOP, max_sweeps: int = 0, X_out=None):
    """D-iteration with default options (FP32 fluid + FP64 refinement). Returns (X, info)."""
    X = X_out if X_out is not None else _like(B, g.n, np.float64)
    _need(g.n, B=B, X_out=X)
    info = SolveInfo()
    res = ctypes.c_double()
    _check(load().di_solve(g.handle, _ptr(B, np.float64), float(d), float(tol), int(schedule), int(max_sweeps),
                           _ptr(X, np.float64), ctypes.byref(res), ctypes.byref(info), _stream(B, X)), info)
    return X, info.as_dict()


def di_solve_ex(g: Graph, B, d: float, tol: float, schedule: int = DI_SOP, fluid: int = DI_FLUID_F32,
                max_sweeps: int = 0, refine: int = 0, host_loop: int = 0, profile: int = 0, e_prediffuse: int = 0,
                r_refresh: int = 0, exact_r: int = 0, X_out=None):
    """D-iteration with explicit options. Returns (X, info)."""
    X = X_out if X_out is not None else _like(B, g.n, np.float64)
    _need(g.n, B=B, X_out=X)
    o = SolveOpts(int(schedule), int(fluid), int(max_sweeps), int(refine), int(host_loop), 0, int(profile),
                  int(e_prediffuse), int(r_refresh), int(exact_r))
    info = SolveInfo()
    res = ctypes.c_double()
    _check(load().di_solve_ex(g.handle, _ptr(B, np.float64), float(d), float(tol), ctypes.byref(o),
                              _ptr(X, np.float64), ctypes.byref(res), ctypes.byref(info), _stream(B, X)), info)
    return X, info.as_dict()


def di_solve_resume(g: Graph, B, H0, d: float, tol: float, F0=None, F_out=None, schedule: int = DI_SOP,
                    fluid: int = DI_FLUID_F32, max_sweeps: int = 0, refine: int = 0, host_loop: int = 0,
                    profile: int = 0, e_prediffuse: int = 0, X_out=None):
    """D-iteration from the state (H0, F0) (F0 None: the exact residual of H0, a warm start).
    Returns (X, info); the final fluid goes to F_out when given."""
    X = X_out if X_out is not None else _like(B, g.n, np.float64)
    _need(g.n, B=B, H0=H0, F0=F0, F_out=F_out, X_out=X)
    o = SolveOpts(int(schedule), int(fluid), int(max_sweeps), int(refine), int(host_loop), 0, int(profile),
                  int(e_prediffuse))
    info = SolveInfo()
    res = ctypes.c_double()
    _check(load().di_solve_resume(g.handle, _ptr(B, np.float64), _ptr(H0, np.float64), _ptr(F0, np.float64),
                                  float(d), float(tol), ctypes.byref(o), _ptr(X, np.float64), _ptr(F_out, np.float64),
                                  ctypes.byref(res), ctypes.byref(info), _stream(B, X)), info)
    return X, info.as_dict()


def di_power_iter(g: Graph, B, d: float, tol: float, max_iters: int = 0, X_out=None):
    """Jacobi power iteration on X = P.X + B. Returns (X, info)."""
    X = X_out if X_out is not None else _like(B, g.n, np.float64)
    _need(g.n, B=B, X_out=X)
    info = SolveInfo()
    res = ctypes.c_double()
    _check(load().di_power_iter(g.handle, _ptr(B, np.float64), float(d), float(tol), int(max_iters),
                                _ptr(X, np.float64), ctypes.byref(res), ctypes.byref(info), _stream(B, X)), info)
    return X, info.as_dict()


def di_power_iter_ex(g: Graph, B, d: float, tol: float, fluid: int = DI_FLUID_F32, max_iters: int = 0,
                     refine: int = 0, profile: int = 0, X_out=None):
    """Power iteration with options: fluid DI_FLUID_F32 (FP32 increments, exact certification) or
    DI_FLUID_F64 (FP64 throughout). Returns (X, info)."""
    X = X_out if X_out is not None else _like(B, g.n, np.float64)
    _need(g.n, B=B, X_out=X)
    o = SolveOpts(0, int(fluid), int(max_iters), int(refine), 0, 0, int(profile), 0, 0, 0)
    info = SolveInfo()
    res = ctypes.c_double()
    _check(load().di_power_iter_ex(g.handle, _ptr(B, np.float64), float(d), float(tol), ctypes.byref(o),
                                   _ptr(X, np.float64), ctypes.byref(res), ctypes.byref(info), _stream(B, X)), info)
    return X, info.as_dict()


def di_power_iter_push(g: Graph, B, d: float, tol: float, max_iters: int = 0, fluid: int = DI_FLUID_F32,
                       X_out=None):
    """Power iteration per column (PI', a push over the out-links): the Jacobi iteration on
    X = P.X + B with the same stopping rule as di_power_iter. Returns (X, info)."""
    X = X_out if X_out is not None else _like(B, g.n, np.float64)
    _need(g.n, B=B, X_out=X)
    info = SolveInfo()
    res = ctypes.c_double()
    _check(load().di_power_iter_push(g.handle, _ptr(B, np.float64), float(d), float(tol), int(max_iters), int(fluid),
                                _ptr(X, np.float64), ctypes.byref(res), ctypes.byref(info), _stream(B, X)), info)
    return X, info.as_dict()


def _tol_array(tol, k, like):
    if np.isscalar(tol):
        return np.full(k, float(tol), dtype=np.float64)
    return tol


def di_solve_batch(g: Graph, B, d: float, tol, schedule: int = DI_SOP, max_sweeps: int = 0, rhs_tile: int = 0,
                   refine: int = 0, X_out=None, res_out=None):
    """k right-hand sides at once; B has shape (k, n) (row r is the right-hand side of column r).
    tol is a scalar or k values. Returns (X (k, n), residuals (k,), info)."""
    k = int(B.shape[0])
    tol = _tol_array(tol, k, B)
    X = X_out if X_out is not None else (_like(B, k * g.n, np.float64).reshape(k, g.n))
    res = res_out if res_out is not None else np.empty(k, dtype=np.float64)
    _need(k * g.n, B=B, X_out=X)
    _need(k, tol=tol, res_out=res)
    o = SolveOpts(int(schedule), DI_FLUID_F32, int(max_sweeps), int(refine), 0, int(rhs_tile), 0, 0)
    info = SolveInfo()
    _check(load().di_solve_batch(g.handle, k, _ptr(B, np.float64), float(d), _ptr(tol, np.float64), ctypes.byref(o),
                                 _ptr(X, np.float64), _ptr(res, np.float64), ctypes.byref(info), _stream(B, X)),
           info)
    return X, res, info.as_dict()


def di_ppr_batch(g: Graph, seed_offsets, seeds, d: float, tol, schedule: int = DI_SOP, max_sweeps: int = 0,
                 rhs_tile: int = 0, refine: int = 0, host_loop: int = 0, profile: int = 0, X_out=None, res_out=None):
    """Personalised PageRank for k seed sets (seed_offsets int64[k+1], seeds int32): column r has
    B_r = (1-d)/|S_r| on its seeds. Returns (X (k, n), residuals (k,), info)."""
    k = int(seed_offsets.shape[0]) - 1
    tol = _tol_array(tol, k, seeds)
    X = X_out if X_out is not None else (_like(seeds, k * g.n, np.float64).reshape(k, g.n))
    res = res_out if res_out is not None else np.empty(k, dtype=np.float64)
    _need(k * g.n, X_out=X)
    _need(k, tol=tol, res_out=res)
    o = SolveOpts(int(schedule), DI_FLUID_F32, int(max_sweeps), int(refine), int(host_loop), int(rhs_tile),
                  int(profile), 0)
    info = SolveInfo()
    _check(load().di_ppr_batch(g.handle, k, _ptr(seed_offsets, np.int64), _ptr(seeds, np.int32), float(d),
                               _ptr(tol, np.float64), ctypes.byref(o), _ptr(X, np.float64), _ptr(res, np.float64),
                               ctypes.byref(info), _stream(seeds, X)), info)
    return X, res, info.as_dict()


def di_residual_noalloc(n: int, rp_in, col_in, out_deg, B, d: float, H, norm_out, Fstar_out=None):
    """Exact residual F* = B + P.H - H and ||F*||_1 (into the one-element CUDA tensor norm_out)
    with no allocation: every argument is a CUDA tensor the caller owns, all on one device.
    Only enqueues work on that device's current torch stream. The lengths are checked here,
    since the C call trusts n: rp_in n+1 entries, out_deg, B, H and Fstar_out at least n,
    norm_out at least one."""
    import torch
    n = int(n)
    args = {"rp_in": rp_in, "col_in": col_in, "out_deg": out_deg, "B": B, "H": H, "norm_out": norm_out}
    if Fstar_out is not None:
        args["Fstar_out"] = Fstar_out
    for name, t in args.items():
        if not (_is_torch(t) and t.is_cuda):
            raise DiError(1, f"{name} must be a CUDA tensor")
    dev = H.device
    for name, t in args.items():
        if t.device != dev:
            raise DiError(1, f"{name} is on {t.device}, H on {dev}: every tensor must be on one device")
    if 1 <= n <= NOALLOC_MAX_NODES:   # other n: the library rejects it with its own message
        need = {"rp_in": n + 1, "out_deg": n, "B": n, "H": n, "norm_out": 1, "Fstar_out": n}
        for name, want in need.items():
            if name in args and (args[name].numel() < want or (name == "rp_in" and args[name].numel() != want)):
                raise DiError(1, f"{name} has {args[name].numel()} entries; n = {n} needs "
                                 f"{'exactly' if name == 'rp_in' else 'at least'} {want}")
    with torch.cuda.device(dev):
        _check(load().di_residual_noalloc(n, _ptr(rp_in, np.int64), _ptr(col_in, np.int32), _ptr(out_deg, np.int32),
                                          _ptr(B, np.float64), float(d), _ptr(H, np.float64),
                                          _ptr(Fstar_out, np.float64), _ptr(norm_out, np.float64), _stream(H)))
    return norm_out


class Server:
    """Owning wrapper of a di_server handle (keeps its graphs alive)."""

    def __init__(self, handle: int, graphs):
        self.handle = handle
        self.graphs = list(graphs)

    def close(self):
        if self.handle:
            load().di_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def di_server_create(graphs, d: float = 0.85, slots: int = 0, sweeps_per_step: int = 0, max_request_sweeps: int = 0,
                     mem_budget: int = 0, tile_min_queue: int = 0) -> Server:
    lib = load()
    arr = (ctypes.c_void_p * len(graphs))(*[g.handle for g in graphs])
    o = ServerOpts(float(d), int(slots), int(sweeps_per_step), int(max_request_sweeps), int(tile_min_queue),
                   int(mem_budget))
    h = ctypes.c_void_p()
    _check(lib.di_server_create(arr, len(graphs), ctypes.byref(o), ctypes.byref(h)))
    return Server(h.value, graphs)


def di_server_submit(srv: Server, graph: int, seeds, tol: float) -> int:
    seeds = np.ascontiguousarray(seeds, dtype=np.int32)
    rid = ctypes.c_int64()
    _check(load().di_server_submit(srv.handle, int(graph), seeds.ctypes.data, int(seeds.shape[0]), float(tol),
                                   ctypes.byref(rid)))
    return rid.value


def di_server_wait(srv: Server, request_id: int, X_out=None, timeout_ms: int = 60000):
    """Waits for a request; returns (X or None, info). Raises DiError (status 7) on timeout."""
    info = RequestInfo()
    st = load().di_server_wait(srv.handle, int(request_id), _ptr(X_out, np.float64), ctypes.byref(info),
                               int(timeout_ms))
    if st != 0:
        raise DiError(st, load().di_last_error().decode(), info.as_dict())
    return X_out, info.as_dict()


def di_server_destroy(srv: Server):
    srv.close()


def di_csr_validate(n: int, L: int, rp_out, col_out, rp_in, col_in, out_deg=None, in_deg=None, loop=None,
                    e_mask=None, e_level=None):
    """Checks graph arrays (host numpy, as di_graph_export returns them) against the build's
    invariants; raises DiError (status 8) naming the first inconsistency."""
    _check(load().di_csr_validate(int(n), int(L), _ptr(rp_out, np.int64), _ptr(col_out, np.int32),
                                  _ptr(rp_in, np.int64), _ptr(col_in, np.int32), _ptr(out_deg, np.int32),
                                  _ptr(in_deg, np.int32), _ptr(loop, np.uint8), _ptr(e_mask, np.uint8),
                                  _ptr(e_level, np.int32)))


def di_graph_validate(g: Graph):
    """Checks every array of a built graph (copied to the host); raises DiError on an inconsistency."""
    _check(load().di_graph_validate(g.handle))


def di_last_error() -> str:
    return load().di_last_error().decode()


def di_version() -> str:
    return load().di_version().decode()
