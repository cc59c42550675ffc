"""GPU D-iteration (DI-CYC, DI-SOP) and power iteration against the oracle and closed forms,
through the C ABI. The parallel sweep diffuses selected nodes concurrently, so only the fixed
point X is compared, never the trajectory: ||X_gpu - X_ref||_1 / ||X_ref||_1 <= 1e-6 with the
fluid in FP32 (1e-10 with FP64 fluid)."""
import numpy as np
import pytest

import oracle
import paper_1204_6255_gb300 as di
import workloads
from gpu_util import lib, rel_l1, to_host

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-6
TOL_F64 = 1e-10
D = 0.85


def gpu_graph(n, edges_or_src, dst=None):
    lib()
    if dst is None:
        src = np.array([s for s, _ in edges_or_src], np.int32)
        dst = np.array([t for _, t in edges_or_src], np.int32)
    else:
        src = edges_or_src
    return di.di_graph_create(n, src, dst), oracle.build(n, src, dst)


def oracle_X(og, B, d):
    H, F, info, ok = oracle.di(og, B, d, 1e-15 * max(B.sum(), 1e-300), oracle.SOP)
    assert ok
    return H


MODES = [
    dict(schedule=di.DI_SOP, fluid=di.DI_FLUID_F64, host_loop=0),
    dict(schedule=di.DI_CYC, fluid=di.DI_FLUID_F64, host_loop=0),
    dict(schedule=di.DI_SOP, fluid=di.DI_FLUID_F32, host_loop=0),
    dict(schedule=di.DI_CYC, fluid=di.DI_FLUID_F32, host_loop=0),
    dict(schedule=di.DI_SOP, fluid=di.DI_FLUID_F32, host_loop=1),
    dict(schedule=di.DI_CYC, fluid=di.DI_FLUID_F64, host_loop=1),
]


def solve(g, B, d, mode, tol=None):
    tol = tol if tol is not None else (1e-13 if mode["fluid"] == di.DI_FLUID_F64 else 1e-10) * B.sum()
    return di.di_solve_ex(g, B, d, tol, **mode)


def bound(mode):
    return TOL_F64 if mode["fluid"] == di.DI_FLUID_F64 else TOL_F32


@pytest.mark.parametrize("mode", MODES, ids=lambda m: f"s{m['schedule']}f{m['fluid']}h{m['host_loop']}")
@pytest.mark.parametrize("n,m,seed", [(1, 1, 1), (5, 12, 2), (33, 100, 3), (200, 700, 4), (3000, 9000, 5),
                                      (20000, 90000, 6)])
def test_random_graphs_match_oracle(mode, n, m, seed):
    n, src, dst = workloads.small_random_graph(n, m, seed=seed)
    g, og = gpu_graph(n, src, dst)
    u = workloads.uniform(seed, 21, n)
    B = np.where(u < 0.2, 0.0, u) * (1 - D) / n
    if B.sum() == 0:
        B[:] = (1 - D) / n
    X, info = solve(g, B, D, mode)
    assert rel_l1(X, oracle_X(og, B, D)) <= bound(mode)
    assert info["residual_l1"] <= (1e-13 if mode["fluid"] else 1e-10) * B.sum()


@pytest.mark.parametrize("mode", MODES[:4], ids=lambda m: f"s{m['schedule']}f{m['fluid']}")
def test_closed_form_cycle_and_stars(mode):
    n = 9
    g, _ = gpu_graph(n, [(i, (i + 1) % n) for i in range(n)])
    B = np.arange(1, n + 1, dtype=np.float64) / 100
    X = np.array([sum(D ** k * B[(i - k) % n] for k in range(n)) / (1 - D ** n) for i in range(n)])
    assert rel_l1(solve(g, B, D, mode)[0], X) <= bound(mode)
    m = 6   # bidirectional star
    g, _ = gpu_graph(m + 1, [(0, k) for k in range(1, m + 1)] + [(k, 0) for k in range(1, m + 1)])
    b = 0.01
    xc = b * (1 + D * m) / (1 - D * D)
    X = np.array([xc] + [b + D * xc / m] * m)
    assert rel_l1(solve(g, np.full(m + 1, b), D, mode)[0], X) <= bound(mode)


@pytest.mark.parametrize("fluid", [di.DI_FLUID_F32, di.DI_FLUID_F64])
def test_loop_nodes_closed_form(fluid):
    g, _ = gpu_graph(3, [(0, 0), (1, 1), (1, 2)])
    b = 0.05
    x1 = b / (1 - D / 2)
    X = np.array([b / (1 - D), x1, b + D / 2 * x1])
    got, info = di.di_solve_ex(g, np.full(3, b), D, 1e-14, schedule=di.DI_CYC, fluid=fluid)
    assert rel_l1(got, X) <= (TOL_F64 if fluid else TOL_F32)


def test_chain_converges_exactly_in_level_count_sweeps():
    # E (Section 2.4) converges in finite steps: on a chain the fluid leaves the graph through
    # the dangling end, so DI-CYC empties F exactly after at most (levels) sweeps
    n = 50
    g, og = gpu_graph(n, [(i, i + 1) for i in range(n - 1)])
    B = np.full(n, 0.01)
    X, info = di.di_solve_ex(g, B, D, 1e-300, schedule=di.DI_CYC, fluid=di.DI_FLUID_F64, refine=-1)
    assert info["residual_l1"] == 0.0
    assert info["sweeps"] <= g.stats["e_levels"]
    Xc = np.array([0.01 * sum(D ** j for j in range(k + 1)) for k in range(n)])
    assert rel_l1(X, Xc) <= 1e-13


@pytest.mark.parametrize("fluid", [di.DI_FLUID_F32, di.DI_FLUID_F64])
def test_sop_tie_falls_back_to_cyc(fluid):
    # all fluid on node 0, which owns every link: F_0 = r * out_0 / L, so DI-SOP selects nothing
    g, _ = gpu_graph(4, [(0, 1), (0, 2), (0, 3)])
    B = np.array([0.1, 0.0, 0.0, 0.0])
    X, info = di.di_solve_ex(g, B, D, 1e-15, schedule=di.DI_SOP, fluid=fluid)
    want = np.array([0.1, D * 0.1 / 3, D * 0.1 / 3, D * 0.1 / 3])
    assert rel_l1(X, want) <= (TOL_F64 if fluid else TOL_F32)
    assert info["sweeps"] >= 2   # one empty DI-SOP sweep, then a DI-CYC sweep


def test_heavy_nodes_push_and_pull():
    # hub 0 <-> 20000 leaves: out- and in-degree above both split thresholds
    n = 20001
    src = np.concatenate([np.zeros(n - 1, np.int32), np.arange(1, n, dtype=np.int32)])
    dst = np.concatenate([np.arange(1, n, dtype=np.int32), np.zeros(n - 1, np.int32)])
    g, og = gpu_graph(n, src, dst)
    B = oracle.uniform_B(n, D)
    ref = oracle_X(og, B, D)
    for mode in MODES[:4]:
        assert rel_l1(solve(g, B, D, mode)[0], ref) <= bound(mode)
    X, info = di.di_power_iter(g, B, D, 1e-14)
    assert rel_l1(X, ref) <= 1e-10


@pytest.mark.parametrize("fluid", [di.DI_FLUID_F32, di.DI_FLUID_F64], ids=["f32inc", "f64"])
@pytest.mark.parametrize("n,m,seed", [(1, 1, 11), (40, 100, 12), (5000, 20000, 13), (30000, 120000, 14)])
def test_power_iteration_matches_oracle(n, m, seed, fluid):
    n, src, dst = workloads.small_random_graph(n, m, seed=seed)
    g, og = gpu_graph(n, src, dst)
    B = workloads.uniform(seed, 22, n) * (1 - D) / n
    X, info = di.di_power_iter_ex(g, B, D, 1e-14, fluid=fluid)
    Xo, oinfo, ok = oracle.pi(og, B, D, 1e-14)
    assert ok and rel_l1(X, Xo) <= 1e-12
    # Jacobi from X_0 = 0: the same iterates up to rounding, so the same count (+-1 when the
    # residual lands next to tol)
    assert abs(info["sweeps"] - oinfo["iterations"]) <= 1
    assert info["residual_l1"] <= 1e-14


def test_power_iteration_residual_is_the_exact_next_increment():
    # the FP32-increment path reports ||B + P.X - X||_1 of the X it returns (the oracle's residual
    # of that X), which is PI's ||X_(k+1) - X_k||_1 taken exactly
    n, src, dst = workloads.small_random_graph(20000, 90000, seed=15)
    g, og = gpu_graph(n, src, dst)
    B = workloads.uniform(15, 22, n) * (1 - D) / n
    for tol in (1e-6, 1e-9, 1e-12):
        X, info = di.di_power_iter(g, B, D, tol)
        _, norm = oracle.residual(og, B, D, X)
        assert info["residual_l1"] <= tol
        assert abs(norm - info["residual_l1"]) <= 1e-6 * norm + 1e-15
    # without the exact certification the residual is the last FP32 increment's norm
    X, info = di.di_power_iter_ex(g, B, D, 1e-9, refine=-1)
    Xo, _, _ = oracle.pi(og, B, D, 1e-14)
    assert info["refine_rounds"] == 0 and rel_l1(X, Xo) <= 1e-6


def test_history_never_exceeds_solution_and_error_bound():
    n, src, dst = workloads.small_random_graph(3000, 12000, seed=31)
    g, og = gpu_graph(n, src, dst)
    B = oracle.uniform_B(n, D)
    ref = oracle_X(og, B, D)
    for tol in (1e-4, 1e-6):
        H, info = di.di_solve_ex(g, B, D, tol, schedule=di.DI_SOP, fluid=di.DI_FLUID_F64)
        r = info["residual_l1"]
        assert r <= tol
        assert np.all(H <= ref * (1 + 1e-12) + 1e-18)                  # X = H + (I-P)^-1 F, F >= 0
        assert np.abs(ref - H).sum() <= r / (1 - D) * (1 + 1e-9) + 1e-12 * ref.sum()


def test_device_tensors_in_and_out():
    import torch
    n, src, dst = workloads.small_random_graph(2000, 8000, seed=41)
    g, og = gpu_graph(n, src, dst)
    B = oracle.uniform_B(n, D)
    Bt = torch.from_numpy(B).cuda()
    Xt = torch.empty(n, dtype=torch.float64, device="cuda")
    X, info = di.di_solve(g, Bt, D, 1e-10 * B.sum(), di.DI_SOP, 0, X_out=Xt)
    assert X is Xt
    assert rel_l1(to_host(Xt), oracle_X(og, B, D)) <= TOL_F32


def test_errors_are_status_codes():
    lib()
    g, og = gpu_graph(4, [(0, 1), (1, 2), (2, 0), (3, 3)])
    B = np.full(4, 0.01)
    for bad_B in (np.array([0.01, -1e-3, 0.0, 0.0]), np.array([0.01, np.nan, 0, 0]), np.array([np.inf, 0, 0, 0.0])):
        with pytest.raises(di.DiError) as e:
            di.di_solve(g, bad_B, D, 1e-10)
        assert e.value.status == 1
    for d_bad in (1.0, -0.1):
        with pytest.raises(di.DiError) as e:
            di.di_solve(g, B, d_bad, 1e-10)
        assert e.value.status == 1
    with pytest.raises(di.DiError) as e:
        di.di_solve(g, B, D, 0.0)
    assert e.value.status == 1
    X = np.zeros(4)
    with pytest.raises(di.DiError) as e:
        di.di_solve_ex(g, B, D, 1e-14, schedule=di.DI_CYC, max_sweeps=2, refine=-1, X_out=X)
    assert e.value.status == 5 and X.sum() > 0       # the current history is still returned
    # the graph is usable after every error
    Xok, info = di.di_solve(g, B, D, 1e-12)
    assert info["residual_l1"] <= 1e-12
