"""Pins for the oracle's E-level pre-diffusion (or_di_e).

E is the recursively zero-in-degree set (Section 2.4), whose nodes converge exactly in finitely
many steps. Every in-neighbour of a node of E lies in E at a lower level, so visiting E once in
level order leaves every node of E with its exact value and no fluid ever reaches E again. The
expected values here come from a dense direct solve of (I - P) X = B (numpy, P built in the
test from the links), not from oracle.c:
  * on a DAG every node is in E, so the pre-pass alone is the exact solution with F = 0 exactly;
  * with no cycle after the pre-pass, H on E is the exact X on E and F on E is zero;
  * the converged result equals the plain D-iteration's and the dense solve's.
"""
import numpy as np
import pytest

import oracle
import workloads

from test_oracle_solve import dense_I_minus_P, rel_l1


def random_dag(n, m, seed):
    """Links only from lower to higher ids (no self-loops): a DAG, so E is every node."""
    u = workloads.u64(seed, 1, 2 * m)
    a = (u[:m] % np.uint64(n)).astype(np.int64)
    b = (u[m:] % np.uint64(n)).astype(np.int64)
    keep = a != b
    src = np.minimum(a, b)[keep].astype(np.int32)
    dst = np.maximum(a, b)[keep].astype(np.int32)
    return src, dst


@pytest.mark.parametrize("seed", range(6))
def test_dag_is_solved_by_the_prepass_alone(seed):
    n = [5, 40, 150, 300, 77, 200][seed]
    d = [0.85, 0.95, 0.5, 0.99, 0.85, 0.7][seed]
    src, dst = random_dag(n, 4 * n, seed=900 + seed)
    g = oracle.build(n, src, dst)
    e_mask, level, cnt, nl = oracle.zero_in(g)
    assert cnt == n
    B = workloads.uniform(950 + seed, 1, n) + 0.01
    H, F, info, ok = oracle.di_e(g, B, d, 1e-300)
    assert ok and info["cycles"] == 0 and info["e_visits"] == n
    assert np.all(F == 0.0)
    X = np.linalg.solve(dense_I_minus_P(n, src, dst, d), B)
    assert rel_l1(H, X) <= 1e-12


@pytest.mark.parametrize("seed", range(8))
def test_prepass_gives_exact_values_on_E(seed):
    n = [30, 80, 150, 200][seed % 4]
    d = [0.85, 0.95][seed % 2]
    # the web-like generator: chains (nodes of E), dangling nodes, loops, local and hub links
    spec = workloads.GraphSpec(n=n, p_dangling=0.2, cap=20, mean_out=4.0, p_local=0.7, window=10,
                               chain_frac=0.3, seed=960 + seed)
    n, src, dst = workloads.generate(spec)
    g = oracle.build(n, src, dst)
    e_mask, level, cnt, nl = oracle.zero_in(g)
    assert cnt > 0
    B = workloads.uniform(970 + seed, 1, n) + 0.01
    H, F, info, _ = oracle.di_e(g, B, d, 1e-300, max_cycles=0)
    assert info["e_visits"] == cnt and info["cycles"] == 0
    E = e_mask.astype(bool)
    X = np.linalg.solve(dense_I_minus_P(n, src, dst, d), B)
    assert np.all(F[E] == 0.0)
    assert np.abs(H[E] - X[E]).sum() <= 1e-12 * np.abs(X[E]).sum()
    # nodes outside E have not been visited: no history yet
    assert np.all(H[~E] == 0.0)


@pytest.mark.parametrize("schedule", [oracle.CYC, oracle.SOP])
@pytest.mark.parametrize("seed", range(4))
def test_converged_result_equals_plain_di_and_dense(schedule, seed):
    n = [60, 120, 200, 180][seed]
    spec = workloads.GraphSpec(n=n, p_dangling=0.15, cap=30, mean_out=5.0, p_local=0.6, window=15,
                               chain_frac=0.2, seed=980 + seed)
    n, src, dst = workloads.generate(spec)
    g = oracle.build(n, src, dst)
    d = 0.85
    B = workloads.uniform(990 + seed, 1, n) + 0.001
    He, Fe, ie, ok1 = oracle.di_e(g, B, d, 1e-14 * B.sum(), schedule)
    Hp, Fp, ip, ok2 = oracle.di(g, B, d, 1e-14 * B.sum(), schedule)
    assert ok1 and ok2
    X = np.linalg.solve(dense_I_minus_P(n, src, dst, d), B)
    assert rel_l1(He, X) <= 1e-12 and rel_l1(Hp, X) <= 1e-12
    # after the pre-pass no node of E is visited again: its value is already exact
    E = oracle.zero_in(g)[0].astype(bool)
    assert np.abs(He[E] - X[E]).sum() <= 1e-12 * max(np.abs(X[E]).sum(), 1e-300)
    assert ie["e_visits"] == int(E.sum())
