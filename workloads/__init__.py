"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

The graphs stand in for the paper's web graphs (Section 2.6 Table 1, Section 2.8 Table 8), which
are not available: power-law out-degree, power-law in-degree by static preferential attachment,
host locality, dangling nodes, loop nodes and zero-in-degree chains. This module holds no
D-iteration arithmetic: it only draws edge lists and personalised seed sets from a counter-based
SplitMix64 stream (see gen.c for the recipe), so both sides of a parity test can use it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, asdict, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "_gen.so")
_lock = threading.Lock()
_lib = None

BASE_SEED = 12046255


class _GenParams(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int64),
        ("p_dangling", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("cap", ctypes.c_int32),
        ("mean_out", ctypes.c_double),
        ("p_local", ctypes.c_double),
        ("window", ctypes.c_int32),
        ("chain_frac", ctypes.c_double),
        ("chain_min", ctypes.c_int32),
        ("chain_max", ctypes.c_int32),
        ("p_loop", ctypes.c_double),
        ("seed", ctypes.c_uint64),
    ]


def build(force: bool = False) -> str:
    """Compile gen.c into a shared object next to it (gcc, OpenMP)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.gen_graph_count.restype = ctypes.c_int64
        lib.gen_graph_count.argtypes = [ctypes.POINTER(_GenParams), ctypes.c_void_p]
        lib.gen_graph_fill.restype = ctypes.c_int64
        lib.gen_graph_fill.argtypes = [ctypes.POINTER(_GenParams), ctypes.c_void_p, ctypes.c_void_p]
        lib.gen_seed_sets.restype = ctypes.c_int64
        lib.gen_seed_sets.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                      ctypes.c_void_p, ctypes.c_void_p]
        lib.gen_u64.restype = None
        lib.gen_u64.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
        lib.gen_draw.restype = None
        lib.gen_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
        _lib = lib
    return _lib


@dataclass(frozen=True)
class GraphSpec:
    """Shape of one synthetic graph (see gen.c for how each field is used)."""
    n: int
    p_dangling: float = 0.2
    alpha: float = 2.1
    cap: int = 5000
    mean_out: float = 0.0          # mean out-degree of non-dangling nodes; 0: Zipf from 1
    p_local: float = 0.0
    window: int = 1000
    chain_frac: float = 0.0
    chain_min: int = 2
    chain_max: int = 10
    p_loop: float = 0.1
    seed: int = BASE_SEED
    transpose: bool = False        # reverse every link (the graph of P transposed)

    def with_seed(self, seed: int) -> "GraphSpec":
        return replace(self, seed=seed)

    def as_dict(self) -> dict:
        return asdict(self)


# The workloads. Seeds are BASE_SEED + index of the untransposed workload.
WORKLOADS = {
    # plain DI-CYC + DI-SOP + PI in FP64 on a 10k-node preferential-attachment graph
    "pa_n10k": dict(spec=GraphSpec(n=10_000, p_dangling=0.15, cap=500, mean_out=0.0, p_local=0.0,
                                   chain_frac=0.0, seed=BASE_SEED + 0),
                    d=0.85, tol=1e-10, fluid="f64"),
    # single solve, 1M nodes, ~8M links, 70% local links, 20% dangling, ~10% chain nodes
    "web_n1m": dict(spec=GraphSpec(n=1_000_000, p_dangling=0.2, cap=5000, mean_out=10.0, p_local=0.7,
                                   chain_frac=0.1, seed=BASE_SEED + 1),
                    d=0.85, tol=1e-8, fluid="f32"),
    # single solve, 10M nodes, ~150M links after dedupe (150.5M), same generator, d in {0.85, 0.95}
    "web_n10m": dict(spec=GraphSpec(n=10_000_000, p_dangling=0.2, cap=5000, mean_out=20.0, p_local=0.7,
                                    chain_frac=0.1, seed=BASE_SEED + 2),
                     d=0.85, tol=1e-8, fluid="f32"),
    # batched personalised PageRank: 2M nodes, ~30M links after dedupe (30.0M), 256 seed sets of
    # 1..1000 nodes
    "ppr_n2m_k256": dict(spec=GraphSpec(n=2_000_000, p_dangling=0.2, cap=5000, mean_out=20.0, p_local=0.7,
                                        chain_frac=0.1, seed=BASE_SEED + 3),
                         d=0.85, tol=1e-6, fluid="f32", k=256, max_seeds=1000),
    # the 1M- and 10M-node graphs with every link reversed (P transposed): the heavy-tailed
    # in-degrees become out-degrees, and the dangling nodes become zero-in-degree nodes of E
    "web_n1m_t": dict(spec=GraphSpec(n=1_000_000, p_dangling=0.2, cap=5000, mean_out=10.0, p_local=0.7,
                                     chain_frac=0.1, seed=BASE_SEED + 1, transpose=True),
                      d=0.85, tol=1e-8, fluid="f32"),
    "web_n10m_t": dict(spec=GraphSpec(n=10_000_000, p_dangling=0.2, cap=5000, mean_out=20.0, p_local=0.7,
                                      chain_frac=0.1, seed=BASE_SEED + 2, transpose=True),
                       d=0.85, tol=1e-8, fluid="f32"),
    # a web-like graph where E dominates (E/N about 0.87, 22 levels; the paper's Dataset 2 has
    # E/N = 0.91): 87% of the nodes sit on zero-in-degree chains of 20 that feed a small core
    "web_n10m_e": dict(spec=GraphSpec(n=10_000_000, p_dangling=0.02, cap=5000, mean_out=20.0, p_local=0.7,
                                      chain_frac=0.87, chain_min=20, chain_max=20, seed=BASE_SEED + 5),
                       d=0.85, tol=1e-8, fluid="f32"),
    # serving: four resident graphs
    "serve_4g": dict(specs=[GraphSpec(n=n, p_dangling=0.2, cap=5000, mean_out=20.0, p_local=0.7,
                                      chain_frac=0.1, seed=BASE_SEED + 4 + 1000 * i)
                            for i, n in enumerate((100_000, 500_000, 2_000_000, 5_000_000))],
                     d=0.85, tols=(1e-4, 1e-6, 1e-8), max_seeds=1000),
}


def generate(spec: GraphSpec):
    """Return (n, src, dst) int32 edge arrays for `spec` (duplicates kept)."""
    lib = _load()
    p = _GenParams(spec.n, spec.p_dangling, spec.alpha, spec.cap, spec.mean_out, spec.p_local,
                   spec.window, spec.chain_frac, spec.chain_min, spec.chain_max, spec.p_loop,
                   spec.seed & 0xFFFFFFFFFFFFFFFF)
    deg = np.empty(spec.n, dtype=np.int32)
    total = lib.gen_graph_count(ctypes.byref(p), deg.ctypes.data)
    if total < 0:
        raise MemoryError("generator failed")
    src = np.empty(total, dtype=np.int32)
    dst = np.empty(total, dtype=np.int32)
    got = lib.gen_graph_fill(ctypes.byref(p), src.ctypes.data, dst.ctypes.data)
    if got != total:
        raise RuntimeError(f"generator wrote {got} of {total} links")
    if spec.transpose:
        return spec.n, dst, src
    return spec.n, src, dst


def seed_sets(n: int, k: int, max_size: int, seed: int):
    """k personalised seed sets: sizes log-uniform in [1, max_size], members uniform without
    replacement. Returns (offsets[k+1] int64, seeds int32)."""
    lib = _load()
    sizes = np.empty(k, dtype=np.int32)
    seeds = np.empty(int(k) * int(min(max_size, n)), dtype=np.int32)
    total = lib.gen_seed_sets(n, k, max_size, seed & 0xFFFFFFFFFFFFFFFF, sizes.ctypes.data, seeds.ctypes.data)
    offsets = np.zeros(k + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    return offsets, seeds[:total].copy()


def u64(seed: int, purpose: int, count: int) -> np.ndarray:
    """Seeded uniform 64-bit integers (for shuffles and random small inputs in tests)."""
    lib = _load()
    out = np.empty(count, dtype=np.uint64)
    lib.gen_u64(seed & 0xFFFFFFFFFFFFFFFF, purpose, count, out.ctypes.data)
    return out


def draw(key: int, first: int, count: int) -> np.ndarray:
    """Raw outputs first .. first + count - 1 of the SplitMix64 stream whose state starts at
    `key` (the generator's counter-based draw)."""
    lib = _load()
    out = np.empty(count, dtype=np.uint64)
    lib.gen_draw(key & 0xFFFFFFFFFFFFFFFF, first & 0xFFFFFFFFFFFFFFFF, count, out.ctypes.data)
    return out


def uniform(seed: int, purpose: int, count: int) -> np.ndarray:
    """Seeded uniform doubles in [0, 1)."""
    return (u64(seed, purpose, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def small_random_graph(n: int, m: int, seed: int, p_loop: float = 0.2, p_dangling: float = 0.2):
    """Tiny random directed graph for brute-force tests: m candidate links, a fraction of nodes
    forced dangling, some self-loops, duplicates kept. Returns (n, src, dst)."""
    r = u64(seed, 1, 3 * m + n)
    src = (r[:m] % np.uint64(n)).astype(np.int32)
    dst = (r[m:2 * m] % np.uint64(n)).astype(np.int32)
    dang = (uniform(seed, 2, n) < p_dangling)
    keep = ~dang[src]
    src, dst = src[keep], dst[keep]
    loops = np.nonzero((uniform(seed, 3, n) < p_loop) & ~dang)[0].astype(np.int32)
    src = np.concatenate([src, loops])
    dst = np.concatenate([dst, loops])
    perm = np.argsort(u64(seed, 4, len(src)), kind="stable")
    return n, src[perm].copy(), dst[perm].copy()
