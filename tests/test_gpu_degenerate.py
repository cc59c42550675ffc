"""Degenerate inputs through every solve entry point of the C ABI.

  * no links at all: every node is dangling and in E, P = 0, so X = B exactly;
  * B = 0: X = 0 with residual 0 (nothing to diffuse);
  * a ragged node count (not a multiple of any tile, chunk or segment size).
"""
import numpy as np
import pytest

import oracle
import paper_1204_6255_gb300 as di
import workloads
from gpu_util import lib, rel_l1

pytestmark = pytest.mark.gpu
D = 0.85


def _no_links(n):
    lib()
    e = np.zeros(0, np.int32)
    return di.di_graph_create(n, e, e)


@pytest.mark.parametrize("n", [1, 7, 5003])
def test_no_links_gives_X_equal_B(n):
    g = _no_links(n)
    st = g.stats
    assert st["L"] == 0 and st["D"] == n and st["E"] == n and st["e_levels"] == (1 if n else 0)
    B = workloads.uniform(7000 + n, 1, n) + 0.1
    for sched in (di.DI_CYC, di.DI_SOP):
        for fluid in (di.DI_FLUID_F32, di.DI_FLUID_F64):
            for e in (0, 1):
                X, info = di.di_solve_ex(g, B, D, 1e-12, schedule=sched, fluid=fluid, e_prediffuse=e)
                assert rel_l1(X, B) <= (1e-7 if fluid == di.DI_FLUID_F32 else 1e-15)
                assert info["residual_l1"] <= 1e-12
    X, info = di.di_power_iter(g, B, D, 1e-12)
    assert rel_l1(X, B) <= 1e-12
    for fluid in (di.DI_FLUID_F32, di.DI_FLUID_F64):
        X, info = di.di_power_iter_push(g, B, D, 1e-12, fluid=fluid)
        assert rel_l1(X, B) <= 1e-7
    X, res, info = di.di_solve_batch(g, np.stack([B, 2 * B]), D, 1e-12)
    assert rel_l1(X[0], B) <= 1e-7 and rel_l1(X[1], 2 * B) <= 1e-7
    X, info = di.di_solve_resume(g, B, np.zeros(n), D, 1e-12)
    assert rel_l1(X, B) <= 1e-7


def test_zero_right_hand_side():
    lib()
    n, src, dst = workloads.small_random_graph(4099, 20000, seed=7100)
    g = di.di_graph_create(n, src, dst)
    B = np.zeros(n)
    for sched in (di.DI_CYC, di.DI_SOP):
        for fluid in (di.DI_FLUID_F32, di.DI_FLUID_F64):
            X, info = di.di_solve_ex(g, B, D, 1e-12, schedule=sched, fluid=fluid)
            assert np.all(X == 0.0) and info["residual_l1"] == 0.0 and info["sweeps"] == 0
    X, info = di.di_power_iter(g, B, D, 1e-12)
    assert np.all(X == 0.0)
    X, info = di.di_power_iter_push(g, B, D, 1e-12)
    assert np.all(X == 0.0) and info["sweeps"] == 0
    X, res, info = di.di_solve_batch(g, np.zeros((3, n)), D, 1e-12)
    assert np.all(X == 0.0) and np.all(res == 0.0)


@pytest.mark.parametrize("n", [2047, 2049, 4097, 10007])
def test_ragged_node_counts(n):
    lib()
    n, src, dst = workloads.small_random_graph(n, 5 * n, seed=7200 + n)
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    B = oracle.uniform_B(n, D)
    ref, _, _, ok = oracle.di(og, B, D, 1e-15, oracle.SOP)
    assert ok
    X, info = di.di_solve_ex(g, B, D, 1e-11, schedule=di.DI_SOP)
    assert rel_l1(X, ref) <= 1e-6
    X, info = di.di_power_iter_push(g, B, D, 1e-11)
    assert rel_l1(X, ref) <= 1e-6
    X, res, info = di.di_ppr_batch(g, np.array([0, 1, 3], np.int64), np.array([0, n - 1, n // 2], np.int32), D,
                                   1e-10)
    for r, sd in enumerate(([0], [n - 1, n // 2])):
        pr, _, _, ok = oracle.di(og, oracle.ppr_B(n, np.array(sd), D), D, 1e-15, oracle.SOP)
        assert ok and rel_l1(X[r], pr) <= 1e-6


def test_fp32_transit_widened_exactly():
    """With no links each node's history is its own B after one visit: the FP32 transit is
    widened to FP64 exactly, for normal and subnormal FP32 values alike."""
    vals = np.array([1.5, 0.15625, 2.0 ** 100, 2.0 ** -126, 2.0 ** -127, 2.0 ** -140, 2.0 ** -149,
                     3 * 2.0 ** -149, (2 - 2.0 ** -23) * 2.0 ** -100, 0.0], np.float64)
    B = vals.astype(np.float32).astype(np.float64)   # every value exact in FP32
    assert np.array_equal(B, vals)
    g = _no_links(B.size)
    for sched in (di.DI_CYC, di.DI_SOP):
        for e in (0, 1):
            X, info = di.di_solve_ex(g, B, D, 1e-300, schedule=sched, fluid=di.DI_FLUID_F32, e_prediffuse=e)
            assert np.array_equal(X, B), (sched, e, X, B)
