"""Pins for the oracle's D-iteration from a given state (or_di_from).

The visit step keeps X = H + (I - P)^-1 F for any state (H, F) (Section 2.5 DI-CYC body, by
linearity), so a run from (H0, F0) converges to H0 + (I - P)^-1 F0. Expected values come from a
dense solve with P built in the test from the links, not from oracle.c:
  * from an arbitrary state, signed fluid included, the limit is H0 + (I - P)^-1 F0;
  * a warm start from B1's solution with F0 = B2 + P.H0 - H0 reaches B2's solution;
  * resuming a capped run from its (H, F) reproduces the uninterrupted run exactly.
"""
import numpy as np
import pytest

import oracle
import workloads

from test_oracle_solve import dense_I_minus_P, rel_l1


def _graph(n, seed):
    spec = workloads.GraphSpec(n=n, p_dangling=0.15, cap=30, mean_out=5.0, p_local=0.6, window=12,
                               chain_frac=0.1, p_loop=0.2, seed=seed)
    n, src, dst = workloads.generate(spec)
    return n, src, dst, oracle.build(n, src, dst)


@pytest.mark.parametrize("schedule", [oracle.CYC, oracle.SOP])
@pytest.mark.parametrize("seed", range(4))
def test_limit_from_any_state(schedule, seed):
    n, src, dst, g = _graph([40, 90, 160, 200][seed], 1300 + seed)
    d = 0.85
    H0 = workloads.uniform(1310 + seed, 1, n)
    F0 = workloads.uniform(1320 + seed, 1, n) - 0.4          # signed fluid
    H, F, info, ok = oracle.di_from(g, H0, F0, d, 1e-13 * np.abs(F0).sum(), schedule)
    assert ok
    A = dense_I_minus_P(n, src, dst, d)
    X = H0 + np.linalg.solve(A, F0)
    assert np.abs(H - X).sum() <= 1e-11 * np.abs(X).sum()


@pytest.mark.parametrize("seed", range(4))
def test_warm_start_reaches_the_new_solution(seed):
    n, src, dst, g = _graph([60, 120, 180, 200][seed], 1400 + seed)
    d = 0.85
    A = dense_I_minus_P(n, src, dst, d)
    P = np.eye(n) - A
    B1 = workloads.uniform(1410 + seed, 1, n)
    B2 = B1.copy()
    B2[: n // 3] *= 1.5                                     # the right-hand side changes
    H0 = np.linalg.solve(A, B1)
    F0 = B2 + P @ H0 - H0
    H, F, info, ok = oracle.di_from(g, H0, F0, d, 1e-13 * B2.sum(), oracle.SOP)
    assert ok
    assert rel_l1(H, np.linalg.solve(A, B2)) <= 1e-11
    cold = oracle.di(g, B2, d, 1e-13 * B2.sum(), oracle.SOP)[2]
    assert info["pushed_edges"] < cold["pushed_edges"]     # the warm start has less left to do


@pytest.mark.parametrize("schedule", [oracle.CYC, oracle.SOP])
@pytest.mark.parametrize("k", [1, 3, 8])
def test_resuming_a_checkpoint_continues_the_run(schedule, k):
    n, src, dst, g = _graph(150, 1500 + k)
    d = 0.85
    B = workloads.uniform(1510 + k, 1, n)
    tol = 1e-12 * B.sum()
    Hk, Fk, ik, _ = oracle.di(g, B, d, tol, schedule, max_cycles=k)
    assert ik["cycles"] == k
    H, F, info, ok = oracle.di_from(g, Hk, Fk, d, tol, schedule)
    Hr, Fr, ir, ok2 = oracle.di(g, B, d, tol, schedule)
    assert ok and ok2
    assert info["cycles"] + k == ir["cycles"]
    assert np.array_equal(H, Hr) and np.array_equal(F, Fr)
