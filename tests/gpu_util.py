"""Helpers shared by the GPU parity tests (imported by test modules; holds no test itself)."""
import numpy as np

import oracle
import paper_1204_6255_gb300 as di

ARRAYS = ["rowptr_out", "col_out", "rowptr_in", "col_in", "out_deg", "in_deg", "loop", "e_mask", "e_level"]

_built = False


def lib():
    """Build (once per process) and load the CUDA library; fails loudly without it."""
    global _built
    if not _built:
        di.build()
        _built = True
    return di.load()


def rel_l1(x, ref) -> float:
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.abs(x - ref).sum() / np.abs(ref).sum())


def to_host(x):
    if hasattr(x, "cpu"):
        return x.cpu().numpy()
    return np.asarray(x)


def assert_build_matches_oracle(g, og, check_e=True):
    """Every exported build array of the GPU graph `g` equals the oracle's, bit for bit."""
    ref = {
        "rowptr_out": og.rp_out, "col_out": og.col_out, "rowptr_in": og.rp_in, "col_in": og.col_in,
        "out_deg": og.outdeg, "in_deg": og.indeg, "loop": og.loop,
    }
    st = g.stats
    assert st["n_nodes"] == og.n and st["L"] == og.L and st["D"] == og.D and st["O"] == og.O
    assert st["max_in"] == og.max_in and st["max_out"] == og.max_out
    for name, want in ref.items():
        got = di.di_graph_export(g, name)
        assert got.dtype == want.dtype, name
        assert np.array_equal(got, want), f"{name} differs from the oracle"
    if check_e:
        e_mask, level, count, n_levels = oracle.zero_in(og)
        assert np.array_equal(di.di_graph_export(g, "e_mask"), e_mask)
        assert np.array_equal(di.di_graph_export(g, "e_level"), level)
        assert st["E"] == count and st["e_levels"] == n_levels
