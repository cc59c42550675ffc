"""The FP32 solve's refinement rounds and its output copy, through the C ABI.

A refined FP32 solve refines first halfway (log scale) between ||B||_1 and tol, then at the
end; the last refinement leaves H unchanged, so X may be copied out beside it (device or pinned
host memory) or after it (pageable memory). Whatever memory X_out is, the returned X must be the
final history: its exact residual, recomputed by the oracle, is the residual the solve reports.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_1204_6255_gb300 as di
import workloads
from gpu_util import lib, rel_l1, to_host

pytestmark = pytest.mark.gpu
D = 0.85


def _graph(n, seed):
    lib()
    spec = workloads.GraphSpec(n=n, p_dangling=0.2, cap=500, mean_out=8.0, p_local=0.7, chain_frac=0.1, seed=seed)
    n, src, dst = workloads.generate(spec)
    return n, di.di_graph_create(n, src, dst), oracle.build(n, src, dst)


def _x_out(kind, n):
    if kind == "pageable":
        return np.empty(n)
    if kind == "pinned":
        return torch.empty(n, dtype=torch.float64).pin_memory()
    return torch.empty(n, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("kind", ["pageable", "pinned", "device"])
@pytest.mark.parametrize("schedule", [di.DI_SOP, di.DI_CYC])
def test_returned_X_is_the_final_history(kind, schedule):
    n, g, og = _graph(120000, 6400)
    B = oracle.uniform_B(n, D)
    ref, _, _, ok = oracle.di(og, B, D, 1e-15, oracle.SOP)
    assert ok
    tol = 1e-9
    X, info = di.di_solve_ex(g, B, D, tol, schedule=schedule, X_out=_x_out(kind, n))
    Xh = to_host(X)
    # halfway and final refinement: the first stop is far above tol
    assert info["refine_rounds"] >= 2
    assert info["residual_l1"] <= tol
    assert rel_l1(Xh, ref) <= 1e-6
    # the reported residual is the exact residual of exactly this X (the two sums differ by the
    # double-float rounding of P.H, a small fraction of tol; an X from before the last sweeps
    # would have the residual of the halfway point, four orders of magnitude larger)
    _, r = oracle.residual(og, B, D, Xh)
    assert abs(r - info["residual_l1"]) <= 1e-2 * info["residual_l1"]


def test_fp32_refinement_rounds_and_work():
    """An FP32 solve from (0, B) takes exactly two refinements (halfway and final), and its
    rounding costs at most a few percent more pushed links than the FP64 fluid, which has no
    rounding to clear."""
    n, g, og = _graph(120000, 6401)
    B = oracle.uniform_B(n, D)
    tol = 1e-9
    _, f32 = di.di_solve_ex(g, B, D, tol, fluid=di.DI_FLUID_F32)
    _, f64 = di.di_solve_ex(g, B, D, tol, fluid=di.DI_FLUID_F64)
    assert f32["residual_l1"] <= tol and f64["residual_l1"] <= tol
    assert f32["refine_rounds"] == 2
    assert f32["pushed_edges"] <= 1.10 * f64["pushed_edges"]
