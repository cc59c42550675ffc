"""Pins for the oracle's D-iteration (DI-CYC, DI-SOP), power iteration and residual.

None of these checks calls oracle.c to produce its expected value:
  * dense direct solve of (I - P) X = B with numpy.linalg.solve, P built here from the links;
  * closed forms on cycles, stars, chains and loop nodes, derived by hand from X = P.X + B;
  * exact rational golden fixtures (tests/golden, written by oracle/exact.py);
  * invariants derived from the diffusion step (Section 2.5 DI-CYC): mass conservation and
    X = H + (I - P)^-1 F after any number of cycles; finite convergence on E (Section 2.4);
  * the paper's normalised PI equals X / ||X||_1 for uniform B.
"""
import json
import glob
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def dense_I_minus_P(n, src, dst, d):
    links = sorted(set(zip(np.asarray(src).tolist(), np.asarray(dst).tolist())))
    out = np.zeros(n)
    for s, _ in links:
        out[s] += 1
    A = np.eye(n)
    for s, t in links:
        A[t, s] -= d / out[s]
    return A


def rel_l1(x, ref):
    return float(np.abs(x - ref).sum() / np.abs(ref).sum())


def graph_from(n, edges):
    src = np.array([s for s, _ in edges], np.int32)
    dst = np.array([t for _, t in edges], np.int32)
    return oracle.build(n, src, dst), src, dst


def all_solvers(g, B, d, tol=1e-15):
    H1, F1, i1, ok1 = oracle.di(g, B, d, tol, oracle.CYC)
    H2, F2, i2, ok2 = oracle.di(g, B, d, tol, oracle.SOP)
    X3, i3, ok3 = oracle.pi(g, B, d, tol)
    assert ok1 and ok2 and ok3
    return {"cyc": H1, "sop": H2, "pi": X3}


# ---------------------------------------------------------------- dense direct solve (P1)

@pytest.mark.parametrize("seed", range(16))
def test_fixed_point_matches_dense_solve(seed):
    n = [3, 8, 25, 60, 120, 200][seed % 6]
    d = [0.85, 0.95, 0.5, 0.99][seed % 4]
    n, src, dst = workloads.small_random_graph(n, 3 * n, seed=3000 + seed)
    g = oracle.build(n, src, dst)
    u = workloads.uniform(seed, 9, n)
    B = np.where(u < 0.3, 0.0, u) * (1 - d) / n        # non-uniform, some zeros
    X = np.linalg.solve(dense_I_minus_P(n, src, dst, d), B)
    for name, x in all_solvers(g, B, d, tol=1e-14 * B.sum()).items():
        assert rel_l1(x, X) < 1e-11, name


# ---------------------------------------------------------------- closed forms (P2)

D = 0.85


def test_closed_form_cycle_nonuniform():
    n = 7
    g, _, _ = graph_from(n, [(i, (i + 1) % n) for i in range(n)])
    B = np.arange(1, n + 1, dtype=np.float64) / 100
    # X_i = sum_k d^k B_{i-k} / (1 - d^n)
    X = np.array([sum(D ** k * B[(i - k) % n] for k in range(n)) / (1 - D ** n) for i in range(n)])
    for name, x in all_solvers(g, B, D).items():
        assert np.allclose(x, X, rtol=1e-12, atol=0), name


def test_closed_form_star_out():
    n = 6   # centre 0 -> leaves 1..5, leaves dangling
    g, _, _ = graph_from(n, [(0, k) for k in range(1, n)])
    b = 0.01
    B = np.full(n, b)
    X = np.array([b] + [b + D * b / (n - 1)] * (n - 1))
    for name, x in all_solvers(g, B, D).items():
        assert np.allclose(x, X, rtol=1e-13), name


def test_closed_form_star_in():
    n = 6   # leaves 1..5 -> centre 0
    g, _, _ = graph_from(n, [(k, 0) for k in range(1, n)])
    b = 0.01
    B = np.full(n, b)
    X = np.array([b * (1 + D * (n - 1))] + [b] * (n - 1))
    for name, x in all_solvers(g, B, D).items():
        assert np.allclose(x, X, rtol=1e-13), name


def test_closed_form_star_bidirectional():
    m = 5
    n = m + 1
    g, _, _ = graph_from(n, [(0, k) for k in range(1, n)] + [(k, 0) for k in range(1, n)])
    b = 0.01
    B = np.full(n, b)
    xc = b * (1 + D * m) / (1 - D * D)
    X = np.array([xc] + [b + D * xc / m] * m)
    for name, x in all_solvers(g, B, D).items():
        assert np.allclose(x, X, rtol=1e-12), name


def test_closed_form_loop_nodes():
    # 0: loop only -> b/(1-d), reached by ONE visit; 1: loop + link to 2 -> b/(1-d/2)
    g, _, _ = graph_from(3, [(0, 0), (1, 1), (1, 2)])
    b = 0.05
    B = np.full(3, b)
    x1 = b / (1 - D / 2)
    X = np.array([b / (1 - D), x1, b + D / 2 * x1])
    for name, x in all_solvers(g, B, D).items():
        assert np.allclose(x, X, rtol=1e-13), name
    H, F, info, ok = oracle.di(g, B, D, 1e-300, oracle.CYC)
    assert ok and info["cycles"] == 1 and F.sum() == 0.0   # finite: 0 -> 1 -> 2 in id order
    assert H[0] == pytest.approx(b / (1 - D), rel=1e-15)


def test_closed_form_chain_and_finite_convergence():
    n = 12
    g, _, _ = graph_from(n, [(i, i + 1) for i in range(n - 1)])
    b = 0.01
    B = np.full(n, b)
    X = np.array([b * sum(D ** j for j in range(k + 1)) for k in range(n)])
    for name, x in all_solvers(g, B, D).items():
        assert np.allclose(x, X, rtol=1e-13), name
    # ascending chain: one DI-CYC cycle empties the fluid exactly (E converges in finite steps)
    H, F, info, ok = oracle.di(g, B, D, 0.0, oracle.CYC)
    assert info["cycles"] == 1 and np.all(F == 0.0)
    assert np.allclose(H, X, rtol=1e-14)


# ---------------------------------------------------------------- golden fixtures (exact)

@pytest.mark.parametrize("path", sorted(glob.glob(os.path.join(GOLDEN, "*.json"))))
def test_golden_exact(path):
    case = json.load(open(path))
    n = case["n"]
    g, _, _ = graph_from(n, case["edges"])
    d = float(Fraction(case["d"]))
    B = np.array([float(Fraction(b)) for b in case["B"]])
    X = np.array([float(Fraction(x)) for x in case["X"]])
    for name, x in all_solvers(g, B, d, tol=1e-16).items():
        assert rel_l1(x, X) < 1e-13, (case["name"], name)


# ---------------------------------------------------------------- invariants (P3, P4, P5)

@pytest.mark.parametrize("schedule", [oracle.CYC, oracle.SOP])
@pytest.mark.parametrize("seed", range(4))
def test_mass_and_identity_after_every_cycle(schedule, seed):
    n = 80
    d = 0.85
    n, src, dst = workloads.small_random_graph(n, 3 * n, seed=4000 + seed)
    g = oracle.build(n, src, dst)
    B = workloads.uniform(seed, 11, n) / n
    A = dense_I_minus_P(n, src, dst, d)
    X = np.linalg.solve(A, B)
    dangling = g.outdeg == 0
    for k in range(0, 6):
        H, F, info, _ = oracle.di(g, B, d, 0.0, schedule, max_cycles=k)
        # mass: ||B||_1 = ||F||_1 + (1-d) sum_{not D} H + sum_D H
        mass = F.sum() + (1 - d) * H[~dangling].sum() + H[dangling].sum()
        assert mass == pytest.approx(B.sum(), rel=1e-13)
        assert info["e"] == pytest.approx(H[dangling].sum(), rel=1e-12, abs=1e-300)
        # identity: X = H + (I - P)^-1 F, hence H <= X and ||X - H|| <= ||F|| / (1 - d)
        assert np.allclose(H + np.linalg.solve(A, F), X, rtol=1e-12, atol=1e-17)
        assert np.all(H <= X * (1 + 1e-12))
        assert np.abs(X - H).sum() <= F.sum() / (1 - d) * (1 + 1e-12)
        # the residual of H is exactly the remaining fluid
        Fs, norm = oracle.residual(g, B, d, H)
        assert np.allclose(Fs, F, rtol=1e-9, atol=1e-15 * B.sum())


def test_paper_error_normalisation():
    # with ||B||_1 = 1 - d, ||X||_1 = (1 - d - d * sum_D X) / (1 - d)  (derived from the mass law)
    spec = workloads.WORKLOADS["pa_n10k"]["spec"]
    n, src, dst = workloads.generate(spec)
    g = oracle.build(n, src, dst)
    d = 0.85
    B = oracle.uniform_B(n, d)
    H, F, info, ok = oracle.di(g, B, d, 1e-13, oracle.SOP)
    assert ok
    e = H[g.outdeg == 0].sum()
    assert H.sum() == pytest.approx((1 - d - d * e) / (1 - d), rel=1e-10)
    assert info["paper_error"] == pytest.approx(info["residual"] / (1 - d - d * info["e"]))


# ---------------------------------------------------------------- DI-SOP specifics

def test_sop_threshold_tie_falls_back_to_cyc():
    # all links leave node 0, and only node 0 holds fluid: F_0 = r = r * out_0 / L, so no node
    # passes F_i > r * out_i / L and the cycle must run as DI-CYC
    n = 4
    g, _, _ = graph_from(n, [(0, 1), (0, 2), (0, 3)])
    B = np.array([0.1, 0.0, 0.0, 0.0])
    H, F, info, ok = oracle.di(g, B, D, 1e-14, oracle.SOP)
    assert ok and info["fallback_cycles"] >= 1
    assert np.allclose(H, [0.1, D * 0.1 / 3, D * 0.1 / 3, D * 0.1 / 3], rtol=1e-14)


def test_sop_selects_by_fluid_per_link():
    # cycle 0 of DI-SOP on a graph where node 0 holds little fluid per link: it is skipped
    n = 5
    g, _, _ = graph_from(n, [(0, 1), (0, 2), (0, 3), (0, 4), (1, 0), (2, 0), (3, 0), (4, 0)])
    B = np.array([0.04, 0.03, 0.03, 0.0, 0.0])
    # r = 0.1, L = 8: thresholds 0.05 for node 0 (4 links), 0.0125 for the others
    H, F, info, ok = oracle.di(g, B, D, 0.0, oracle.SOP, max_cycles=1)
    assert H[0] == 0.0 and H[1] > 0 and H[2] > 0 and info["visits"] == 2
    # node 0 received d*0.03 twice, and was not visited in that cycle
    assert F[0] == pytest.approx(0.04 + 2 * D * 0.03)


def test_iteration_counts_follow_paper_trend():
    # Tables 2-7: DI-SOP needs fewer equivalent iterations (pushed links / L) than DI-CYC, which
    # needs fewer than PI. Qualitative only: the graphs differ from the paper's.
    spec = workloads.WORKLOADS["pa_n10k"]["spec"]
    n, src, dst = workloads.generate(spec)
    g = oracle.build(n, src, dst)
    d = 0.85
    B = oracle.uniform_B(n, d)
    tol = 1.0 / n * (1 - d)
    _, _, icyc, _ = oracle.di(g, B, d, tol, oracle.CYC)
    _, _, isop, _ = oracle.di(g, B, d, tol, oracle.SOP)
    _, ipi, _ = oracle.pi(g, B, d, tol)
    cyc = icyc["pushed_edges"] / g.L
    sop = isop["pushed_edges"] / g.L
    assert sop < cyc < ipi["iterations"]


# ---------------------------------------------------------------- PI

def test_pi_paper_mode_is_normalised_solution():
    spec = workloads.WORKLOADS["pa_n10k"]["spec"]
    n, src, dst = workloads.generate(spec)
    g = oracle.build(n, src, dst)
    d = 0.85
    x, info, ok = oracle.pi_paper(g, d, 1e-13)
    X, _, ok2 = oracle.pi(g, oracle.uniform_B(n, d), d, 1e-15)
    assert ok and ok2
    assert x.sum() == pytest.approx(1.0, rel=1e-12)
    assert rel_l1(x, X / X.sum()) < 1e-10


def test_pi_iteration_count_geometric():
    # on a cycle with uniform B, X_k = b (1 + d + ... + d^(k-1)): ||X_k - X_{k-1}|| = n b d^(k-1)
    n = 10
    g, _, _ = graph_from(n, [(i, (i + 1) % n) for i in range(n)])
    b = 0.015
    B = np.full(n, b)
    tol = 1e-9
    X, info, ok = oracle.pi(g, B, D, tol)
    k = info["iterations"]
    assert ok
    assert n * b * D ** (k - 1) <= tol < n * b * D ** (k - 2)
    assert info["residual"] == pytest.approx(n * b * D ** (k - 1), rel=1e-9)


# ---------------------------------------------------------------- PI' (power iteration per column)

@pytest.mark.parametrize("seed", range(6))
def test_pi_push_iterates_equal_pull_iterates_and_dense(seed):
    # the column form scatters d X_i / out_i over l_out; the row form gathers it over l_in; both
    # are the same Jacobi iterate of X = P.X + B (Section 2.5 PI and PI'), here checked iterate by
    # iterate, and their fixed point is the dense solve's
    n = [20, 60, 150, 200, 90, 120][seed]
    d = [0.85, 0.95, 0.5, 0.85, 0.99, 0.7][seed]
    spec = workloads.GraphSpec(n=n, p_dangling=0.15, cap=25, mean_out=4.0, p_local=0.5, window=10,
                               chain_frac=0.1, p_loop=0.3, seed=1100 + seed)
    n, src, dst = workloads.generate(spec)
    g = oracle.build(n, src, dst)
    assert g.O > 0                              # self-links take part as plain entries of P
    B = workloads.uniform(1200 + seed, 1, n) + 0.01
    for k in (1, 2, 3, 7):
        Xr, _, _ = oracle.pi(g, B, d, 0.0, max_iters=k)
        Xc, ic, _ = oracle.pi_push(g, B, d, 0.0, max_iters=k)
        assert ic["iterations"] == k
        assert np.abs(Xc - Xr).sum() <= 1e-13 * np.abs(Xr).sum()
    Xc, ic, ok = oracle.pi_push(g, B, d, 1e-13 * B.sum())
    Xr, ir, ok2 = oracle.pi(g, B, d, 1e-13 * B.sum())
    assert ok and ok2 and abs(ic["iterations"] - ir["iterations"]) <= 1
    X = np.linalg.solve(dense_I_minus_P(n, src, dst, d), B)
    assert rel_l1(Xc, X) <= 1e-11
