"""DI-SOP with r refreshed within a sweep (opts r_refresh: a sweep selects in parts of the node
range with r taken again before each), and with r summed exactly after every sweep (exact_r):
the fixed point is the oracle's, in FP32 and FP64 fluid, host- and graph-driven. Also the
reported diagnostics (Section 2.5 DI-CYC's error normalisation): paper_error is
residual / (1 - d - d e), and e, the dangling mass, is within ||F||_1 / (1 - d) of the sum of the
exact solution over the dangling nodes."""
import numpy as np
import pytest

import oracle
import paper_1204_6255_gb300 as di
import workloads
from gpu_util import lib, rel_l1

pytestmark = pytest.mark.gpu
D = 0.85


def _graph(n, seed):
    lib()
    spec = workloads.GraphSpec(n=n, p_dangling=0.2, cap=800, mean_out=9.0, p_local=0.7, chain_frac=0.1,
                               seed=workloads.BASE_SEED + seed)
    n, src, dst = workloads.generate(spec)
    return n, di.di_graph_create(n, src, dst), oracle.build(n, src, dst)


@pytest.mark.parametrize("parts", [2, 3, 7])
@pytest.mark.parametrize("fluid,host_loop", [(di.DI_FLUID_F32, 0), (di.DI_FLUID_F64, 0), (di.DI_FLUID_F32, 1)])
def test_refreshed_r_reaches_the_oracle_fixed_point(parts, fluid, host_loop):
    n, g, og = _graph(30_000, 6100)
    B = workloads.uniform(6101, 1, n) * (1 - D) / n
    ref, _, _, ok = oracle.di(og, B, D, 1e-15, oracle.SOP)
    assert ok
    tol = 1e-11 if fluid == di.DI_FLUID_F32 else 1e-13
    X, info = di.di_solve_ex(g, B, D, tol, schedule=di.DI_SOP, fluid=fluid, host_loop=host_loop, r_refresh=parts)
    assert rel_l1(X, ref) <= (1e-6 if fluid == di.DI_FLUID_F32 else 1e-10)
    assert info["residual_l1"] <= tol
    # every part of a sweep launches select, push and reduce
    base = di.di_solve_ex(g, B, D, tol, schedule=di.DI_SOP, fluid=fluid, host_loop=host_loop)[1]
    assert info["sweeps"] >= 1 and base["sweeps"] >= 1


def test_refreshed_r_matches_the_oracle_variant_on_a_tiny_case():
    # the hand case of the oracle's pins: with a fresh r before node 2, a sweep in two parts
    # visits nodes 2 and 3 in the sweep where the cycle's r admits node 0 only
    n = 4
    src = np.array([1, 2, 3], np.int32)
    dst = np.array([2, 3, 2], np.int32)
    lib()
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    B = np.array([0.9, 0.0, 0.05, 0.05])
    X, info = di.di_solve_ex(g, B, D, 1e-14, schedule=di.DI_SOP, fluid=di.DI_FLUID_F64, r_refresh=2)
    ref, _, _, _ = oracle.di_refresh(og, B, D, 1e-16, 2)
    assert rel_l1(X, ref) <= 1e-12


def test_exact_r_and_tracked_r_reach_the_same_fixed_point():
    n, g, og = _graph(60_000, 6200)
    B = oracle.uniform_B(n, D)
    ref, _, _, ok = oracle.di(og, B, D, 1e-15, oracle.SOP)
    assert ok
    for exact in (0, 1):
        X, info = di.di_solve_ex(g, B, D, 1e-10, schedule=di.DI_SOP, exact_r=exact)
        assert rel_l1(X, ref) <= 1e-6 and info["residual_l1"] <= 1e-10


@pytest.mark.parametrize("schedule,fluid", [(di.DI_SOP, di.DI_FLUID_F32), (di.DI_CYC, di.DI_FLUID_F32),
                                            (di.DI_SOP, di.DI_FLUID_F64)])
def test_reported_diagnostics(schedule, fluid):
    n, g, og = _graph(40_000, 6300)
    B = oracle.uniform_B(n, D)     # ||B||_1 = 1 - d, the paper's normalisation
    ref, _, _, ok = oracle.di(og, B, D, 1e-15, oracle.SOP)
    assert ok
    tol = 1e-9
    X, info = di.di_solve_ex(g, B, D, tol, schedule=schedule, fluid=fluid)
    r, e = info["residual_l1"], info["dangling_mass_e"]
    assert info["paper_error"] == pytest.approx(r / (1 - D - D * e), rel=1e-12)
    dangling = og.outdeg == 0
    # e sums the history over D, and H is within ||F||_1 / (1 - d) of X (identity H + (I-P)^-1 F)
    # (e adds the FP32 transits in FP32 partial sums, so it matches to FP32 accuracy)
    assert abs(e - X[dangling].sum()) <= 1e-6 * X[dangling].sum() + 1e-15
    assert abs(e - ref[dangling].sum()) <= r / (1 - D) + 1e-6 * ref[dangling].sum()
    # with ||B||_1 = 1 - d, ||X||_1 = (1 - d - d sum_D X) / (1 - d), so the paper's error
    # bounds the relative L1 error of H up to the residual's own contribution
    assert rel_l1(X, ref) <= info["paper_error"] * 1.01 + 1e-12
    assert info["visited_nodes"] > 0 and info["pushed_edges"] >= info["frontier_entries"]
