"""D-iteration from a given state (di_solve_resume) against the oracle, through the C ABI.

The visit keeps X = H + (I - P)^-1 F for any state, so a run stopped after k sweeps resumes
from (X_out, F_out), and the exact residual of an approximate solution H0 turns it into a warm
start for a new B (the fluid may then be negative). Expected values come from the oracle's
di / di_from, which are pinned against dense solves.
"""
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
    spec = workloads.GraphSpec(n=n, p_dangling=0.2, cap=500, mean_out=8.0, p_local=0.7, chain_frac=0.1, seed=seed)
    n, src, dst = workloads.generate(spec)
    return n, di.di_graph_create(n, src, dst), oracle.build(n, src, dst)


@pytest.mark.parametrize("fluid", [di.DI_FLUID_F64, di.DI_FLUID_F32])
@pytest.mark.parametrize("schedule", [di.DI_SOP, di.DI_CYC])
def test_checkpoint_resumes_the_run(fluid, schedule):
    n, g, og = _graph(50000, 6100)
    B = oracle.uniform_B(n, D)
    ref, _, _, ok = oracle.di(og, B, D, 1e-15, oracle.SOP)
    assert ok
    tol = 1e-13 if fluid == di.DI_FLUID_F64 else 1e-9
    _, full = di.di_solve_ex(g, B, D, tol, schedule=schedule, fluid=fluid)
    k = max(1, full["sweeps"] // 3)
    H, F = np.empty(n), np.empty(n)
    with pytest.raises(di.DiError) as e:                     # stopped after k sweeps
        di.di_solve_resume(g, B, np.zeros(n), D, tol, F0=B, F_out=F, schedule=schedule, fluid=fluid,
                           max_sweeps=k, X_out=H)
    assert e.value.status == 5
    # the checkpoint is a state of this problem: H + (I - P)^-1 F = X
    assert np.abs(F).sum() > tol
    X, info = di.di_solve_resume(g, B, H, D, tol, F0=F, schedule=schedule, fluid=fluid)
    assert info["residual_l1"] <= tol
    assert rel_l1(X, ref) <= (1e-10 if fluid == di.DI_FLUID_F64 else 1e-6)
    assert info["sweeps"] <= full["sweeps"]                  # the resumed part is not a restart


@pytest.mark.parametrize("schedule", [di.DI_SOP, di.DI_CYC])
def test_warm_start_for_a_new_right_hand_side(schedule):
    n, g, og = _graph(60000, 6200)
    off, seeds = workloads.seed_sets(n, 2, 400, seed=6201)
    B1 = oracle.ppr_B(n, seeds[off[0]:off[1]], D)
    B2 = B1 + oracle.ppr_B(n, seeds[off[1]:off[2]], D) * 0.05  # a few more seeds, same graph
    B2[seeds[0]] *= 0.8                                          # and one seed weighs less
    tol = 1e-10
    X1, _ = di.di_solve_ex(g, B1, D, 1e-12, schedule=schedule)
    ref2, _, _, ok = oracle.di(og, B2, D, 1e-14, oracle.SOP)
    assert ok
    _, cold = di.di_solve_ex(g, B2, D, tol, schedule=schedule)
    Fw = np.empty(n)
    X2, warm = di.di_solve_resume(g, B2, X1, D, tol, schedule=schedule, F_out=Fw)
    assert warm["residual_l1"] <= tol
    assert rel_l1(X2, ref2) <= 1e-6
    assert warm["pushed_edges"] < cold["pushed_edges"]
    # the oracle from the same warm state agrees (its fluid is signed: H0 overshoots at seeds[0])
    P_res = oracle.residual(og, B2, D, X1)[0]
    assert P_res.min() < 0.0
    Ho, _, _, ok = oracle.di_from(og, X1, P_res, D, 1e-14, oracle.SOP)
    assert ok and rel_l1(Ho, ref2) <= 1e-10


def test_resume_errors():
    n, g, og = _graph(3000, 6300)
    B = oracle.uniform_B(n, D)
    with pytest.raises(di.DiError) as e:
        di.di_solve_resume(g, B, None, D, 1e-8)
    assert e.value.status == 1
    bad = np.zeros(n)
    bad[5] = np.nan
    with pytest.raises(di.DiError) as e:
        di.di_solve_resume(g, B, np.zeros(n), D, 1e-8, F0=bad)
    assert e.value.status == 1
    with pytest.raises(di.DiError) as e:
        di.di_solve_resume(g, B, bad, D, 1e-8)
    assert e.value.status == 1
    X, info = di.di_solve_resume(g, B, np.zeros(n), D, 1e-8)   # the graph still works
    assert info["residual_l1"] <= 1e-8
