"""Power iteration per column (di_power_iter_push, PI' of Section 2.5) against the oracle.

PI' is the Jacobi iteration on X = P.X + B formed over the columns of P (a push over l_out). It
has PI's stopping rule, and the paper's tables give the two equal iteration counts. The GPU
pushes the increments X_(k+1) - X_k with a self-link as a plain link, so after k sweeps it holds
the k-th iterate. Expected values come from the oracle's or_pi_push and or_pi, which are pinned
to each other iterate by iterate and to dense solves.
"""
import numpy as np
import pytest

import oracle
import paper_1204_6255_gb300 as di
import workloads
from gpu_util import lib, rel_l1

pytestmark = pytest.mark.gpu
D = 0.85


def _graph(n, seed, p_loop=0.3):
    lib()
    spec = workloads.GraphSpec(n=n, p_dangling=0.15, cap=400, mean_out=7.0, p_local=0.6, chain_frac=0.1,
                               p_loop=p_loop, seed=seed)
    n, src, dst = workloads.generate(spec)
    return n, di.di_graph_create(n, src, dst), oracle.build(n, src, dst)


@pytest.mark.parametrize("fluid", [di.DI_FLUID_F64, di.DI_FLUID_F32])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_converged_pi_push_matches_oracle(fluid, seed):
    n, g, og = _graph(40000, 5100 + seed)
    assert og.O > 0
    B = workloads.uniform(5200 + seed, 1, n) * (1 - D) / n
    tol = 1e-10 * B.sum()
    Xr, ir, ok = oracle.pi(og, B, D, tol)
    Xc, ic, ok2 = oracle.pi_push(og, B, D, tol)
    assert ok and ok2
    X, info = di.di_power_iter_push(g, B, D, tol, fluid=fluid)
    assert info["residual_l1"] <= tol
    if fluid == di.DI_FLUID_F64:
        # the same iteration: PI's iterate and iteration count (up to the last step's rounding)
        assert rel_l1(X, Xr) <= 1e-10 and rel_l1(X, Xc) <= 1e-10
        assert abs(info["sweeps"] - ir["iterations"]) <= 1
    else:
        # FP32 increments: the exact-residual continuation may add iterations, never remove any
        assert rel_l1(X, Xr) <= 1e-6 and rel_l1(X, Xc) <= 1e-6
        assert info["sweeps"] >= ir["iterations"] - 1


@pytest.mark.parametrize("fluid", [di.DI_FLUID_F64, di.DI_FLUID_F32])
@pytest.mark.parametrize("k", [1, 2, 5, 12])
def test_k_iterations_give_the_kth_iterate(fluid, k):
    n, g, og = _graph(20000, 5300)
    B = workloads.uniform(5301, 1, n) * (1 - D) / n
    Xk, _, _ = oracle.pi_push(og, B, D, 0.0, max_iters=k)
    X = np.empty(n)
    with pytest.raises(di.DiError) as e:         # tol 1e-300 is not reached in k iterations
        di.di_power_iter_push(g, B, D, 1e-300, max_iters=k, fluid=fluid, X_out=X)
    assert e.value.status == 5 and e.value.info["sweeps"] == k
    assert rel_l1(X, Xk) <= (1e-12 if fluid == di.DI_FLUID_F64 else 1e-6)


def test_pi_push_on_the_1m_node_workload():
    lib()
    cfg = workloads.WORKLOADS["web_n1m"]
    n, src, dst = workloads.generate(cfg["spec"])
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    B = np.full(n, (1 - cfg["d"]) / n)
    ref, _, ok = oracle.pi(og, B, cfg["d"], 1e-13)
    assert ok
    X, info = di.di_power_iter_push(g, B, cfg["d"], cfg["tol"])
    assert info["residual_l1"] <= cfg["tol"]
    assert rel_l1(X, ref) <= 1e-6
    X64, info64 = di.di_power_iter_push(g, B, cfg["d"], cfg["tol"], fluid=di.DI_FLUID_F64)
    assert rel_l1(X64, ref) <= 1e-6
    Xp, pinfo = di.di_power_iter(g, B, cfg["d"], cfg["tol"])
    assert abs(info64["sweeps"] - pinfo["sweeps"]) <= 1
