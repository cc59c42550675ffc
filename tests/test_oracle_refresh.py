"""Pins for the oracle's DI-SOP with r refreshed within a cycle (oracle.di_refresh): r = ||F||_1
taken again every r_every node ids, instead of once per cycle (Section 2.3 takes r_n' once per
cycle; refreshing it is the threshold variant the GPU measures as sub-sweeps).

Expected values come from elsewhere than oracle.c: the plain DI-SOP (itself pinned), numpy's
dense solve, the mass law and the identity X = H + (I - P)^-1 F, and one cycle worked by hand.
"""
import numpy as np
import pytest

import oracle
import workloads
from test_oracle_solve import dense_I_minus_P, graph_from, rel_l1


@pytest.mark.parametrize("seed", range(6))
def test_once_per_cycle_is_plain_di_sop_bit_for_bit(seed):
    n = [20, 60, 150][seed % 3]
    n, src, dst = workloads.small_random_graph(n, 4 * n, seed=5100 + seed)
    g = oracle.build(n, src, dst)
    B = workloads.uniform(seed, 21, n) / n
    for cycles in (1, 3, 50):
        H0, F0, i0, _ = oracle.di(g, B, 0.85, 1e-14, oracle.SOP, max_cycles=cycles)
        for r_every in (0, n, 10 * n):
            H1, F1, i1, _ = oracle.di_refresh(g, B, 0.85, 1e-14, r_every, max_cycles=cycles)
            assert np.array_equal(H0, H1) and np.array_equal(F0, F1)
            assert i0["visits"] == i1["visits"] and i0["cycles"] == i1["cycles"]


@pytest.mark.parametrize("seed", range(8))
def test_fixed_point_matches_dense_solve(seed):
    n = [10, 40, 120, 200][seed % 4]
    d = [0.85, 0.95][seed % 2]
    n, src, dst = workloads.small_random_graph(n, 3 * n, seed=5200 + seed)
    g = oracle.build(n, src, dst)
    B = workloads.uniform(seed, 22, n) * (1 - d) / n
    X = np.linalg.solve(dense_I_minus_P(n, src, dst, d), B)
    for r_every in (1, 3, max(1, n // 2)):
        H, F, info, ok = oracle.di_refresh(g, B, d, 1e-15, r_every)
        assert ok
        assert rel_l1(H, X) < 1e-12, r_every


@pytest.mark.parametrize("seed", range(3))
def test_mass_and_identity_after_every_cycle(seed):
    n, d = 90, 0.85
    n, src, dst = workloads.small_random_graph(n, 3 * n, seed=5300 + seed)
    g = oracle.build(n, src, dst)
    B = workloads.uniform(seed, 23, n) / n
    A = dense_I_minus_P(n, src, dst, d)
    X = np.linalg.solve(A, B)
    dangling = g.outdeg == 0
    for k in range(6):
        H, F, info, _ = oracle.di_refresh(g, B, d, 0.0, 7, max_cycles=k)
        mass = F.sum() + (1 - d) * H[~dangling].sum() + H[dangling].sum()
        assert mass == pytest.approx(B.sum(), rel=1e-13)
        assert np.allclose(H + np.linalg.solve(A, F), X, rtol=1e-12, atol=1e-17)


def test_refreshed_r_admits_a_node_the_cycle_r_would_not():
    # links 1->2, 2->3, 3->2 (L = 3); node 0 dangling. F = B = (0.9, 0, 0.05, 0.05), r = 1.
    # Plain cycle: threshold (1/3) * out; only node 0 (dangling, threshold 0) is visited.
    # With r taken again before node 2 (r_every = 2): r = 0.1, threshold 0.1/3 < 0.05, so node 2
    # is visited (H_2 = 0.05, F_3 = 0.05 + 0.85 * 0.05 = 0.0925), then node 3 under the same r
    # (H_3 = 0.0925, F_2 = 0.85 * 0.0925 = 0.078625).
    g, _, _ = graph_from(4, [(1, 2), (2, 3), (3, 2)])
    B = np.array([0.9, 0.0, 0.05, 0.05])
    H, F, info, _ = oracle.di(g, B, 0.85, 0.0, oracle.SOP, max_cycles=1)
    assert info["visits"] == 1
    assert np.allclose(H, [0.9, 0, 0, 0], rtol=0, atol=1e-16) and np.allclose(F, [0, 0, 0.05, 0.05], atol=1e-16)
    H, F, info, _ = oracle.di_refresh(g, B, 0.85, 0.0, 2, max_cycles=1)
    assert info["visits"] == 3
    assert np.allclose(H, [0.9, 0.0, 0.05, 0.0925], rtol=1e-15, atol=0)
    assert np.allclose(F, [0.0, 0.0, 0.078625, 0.0], rtol=1e-15, atol=0)
