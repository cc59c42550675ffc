"""Batched (multi-RHS) D-iteration and personalised PageRank against the oracle, through the C ABI.

Every column of a batch is an independent problem X_r = P.X_r + B_r; the oracle solves each one
alone. Columns share only the frontier (a node is visited when any column selects it), which
changes trajectories but not fixed points, so each column must match its solo oracle solve and
its solo GPU solve within ||X - X_ref||_1 / ||X_ref||_1 <= 1e-6, whatever its batch-mates are.
"""
import numpy as np
import pytest

import oracle
import paper_1204_6255_gb300 as di
import workloads
from gpu_util import lib, rel_l1, to_host

pytestmark = pytest.mark.gpu
D = 0.85
TOL_X = 1e-6


def _graph(n, m, seed):
    lib()
    n, src, dst = workloads.small_random_graph(n, m, seed=seed)
    return n, di.di_graph_create(n, src, dst), oracle.build(n, src, dst)


def _oracle_X(og, B, d=D):
    H, _, _, ok = oracle.di(og, B, d, 1e-15 * B.sum(), oracle.SOP)
    assert ok
    return H


@pytest.mark.parametrize("tile", [4, 8, 16, 32, 0])
@pytest.mark.parametrize("k", [1, 5, 37])
def test_dense_batch_matches_oracle(tile, k):
    n, g, og = _graph(3000, 12000, seed=51)
    u = workloads.uniform(52, 1, k * n).reshape(k, n)
    B = np.where(u < 0.5, 0.0, u) * (1 - D) / n
    tol = np.linspace(1e-9, 1e-11, k) * B.sum(axis=1)
    X, res, info = di.di_solve_batch(g, B, D, tol, rhs_tile=tile)
    assert info["rhs_tile"] in (4, 8, 16, 32) and (tile == 0 or info["rhs_tile"] == tile)
    assert np.all(res <= tol)
    for r in range(k):
        assert rel_l1(X[r], _oracle_X(og, B[r])) <= TOL_X, r


@pytest.mark.parametrize("tile", [8, 32])
def test_ppr_batch_matches_oracle_and_solo(tile):
    n, g, og = _graph(20000, 90000, seed=61)
    off, seeds = workloads.seed_sets(n, 20, 300, seed=62)
    tol = 1e-10
    X, res, info = di.di_ppr_batch(g, off, seeds, D, tol, rhs_tile=tile)
    assert np.all(res <= tol)
    for r in range(20):
        B = oracle.ppr_B(n, seeds[off[r]:off[r + 1]], D)
        ref = _oracle_X(og, B)
        assert rel_l1(X[r], ref) <= TOL_X, r
        solo, _ = di.di_solve(g, B, D, tol)
        assert rel_l1(X[r], solo) <= TOL_X, r


def test_column_result_independent_of_batch_mates():
    # the same request alone, beside one other, and inside a full tile of different requests
    n, g, og = _graph(5000, 25000, seed=71)
    off, seeds = workloads.seed_sets(n, 32, 500, seed=72)
    tol = 1e-10
    X_all, _, _ = di.di_ppr_batch(g, off, seeds, D, tol, rhs_tile=32)
    X_two, _, _ = di.di_ppr_batch(g, off[:3] - off[0], seeds[off[0]:off[2]], D, tol, rhs_tile=32)
    X_one, _, _ = di.di_ppr_batch(g, off[:2], seeds[:off[1]], D, tol, rhs_tile=32)
    ref = _oracle_X(og, oracle.ppr_B(n, seeds[:off[1]], D))
    for X in (X_all[0], X_two[0], X_one[0]):
        assert rel_l1(X, ref) <= TOL_X


def test_mixed_tolerances_retire_per_column():
    n, g, og = _graph(4000, 16000, seed=81)
    off, seeds = workloads.seed_sets(n, 12, 200, seed=82)
    tol = np.array([1e-4, 1e-6, 1e-8, 1e-10] * 3)
    X, res, info = di.di_ppr_batch(g, off, seeds, D, tol, rhs_tile=16)
    assert np.all(res <= tol)
    for r in range(12):
        ref = _oracle_X(og, oracle.ppr_B(n, seeds[off[r]:off[r + 1]], D))
        # the error of a column is bounded by its own tolerance: ||X - H|| <= res / (1 - d)
        assert np.abs(ref - X[r]).sum() <= res[r] / (1 - D) * (1 + 1e-6) + 1e-12


def test_batch_device_buffers_and_errors():
    import torch
    n, g, og = _graph(2000, 8000, seed=91)
    off, seeds = workloads.seed_sets(n, 6, 50, seed=92)
    Xt = torch.empty((6, n), dtype=torch.float64, device="cuda")
    X, res, info = di.di_ppr_batch(g, torch.from_numpy(off).cuda(), torch.from_numpy(seeds).cuda(), D, 1e-10,
                                   X_out=Xt)
    ref = _oracle_X(og, oracle.ppr_B(n, seeds[off[0]:off[1]], D))
    assert rel_l1(to_host(Xt)[0], ref) <= TOL_X
    bad = seeds.copy()
    bad[3] = n
    with pytest.raises(di.DiError) as e:
        di.di_ppr_batch(g, off, bad, D, 1e-10)
    assert e.value.status == 2
    empty = off.copy()
    empty[2] = empty[1]
    with pytest.raises(di.DiError) as e:
        di.di_ppr_batch(g, empty, seeds, D, 1e-10)
    assert e.value.status == 1
    with pytest.raises(di.DiError) as e:
        di.di_solve_batch(g, -np.ones((2, n)), D, 1e-10)
    assert e.value.status == 1
    # the graph still works
    X, res, info = di.di_ppr_batch(g, off, seeds, D, 1e-10)
    assert np.all(res <= 1e-10)


def test_ppr_workload_sample():
    # the batched PPR workload shape (N=2M, ~30M links, seed sets of 1..1000 nodes), sampled:
    # 64 columns, 4 of them checked against the oracle
    cfg = workloads.WORKLOADS["ppr_n2m_k256"]
    n, src, dst = workloads.generate(cfg["spec"])
    lib()
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    off, seeds = workloads.seed_sets(n, 64, cfg["max_seeds"], seed=cfg["spec"].seed)
    X, res, info = di.di_ppr_batch(g, off, seeds, cfg["d"], cfg["tol"], max_sweeps=20000)
    assert np.all(res <= cfg["tol"])
    for r in (0, 17, 40, 63):
        B = oracle.ppr_B(n, seeds[off[r]:off[r + 1]], cfg["d"])
        H, _, _, ok = oracle.di(og, B, cfg["d"], 1e-10, oracle.SOP)
        assert ok
        # tol 1e-6 on ||F||_1 bounds the error by 1e-6 / (1 - d) in L1
        assert np.abs(H - X[r]).sum() <= cfg["tol"] / (1 - cfg["d"]) + 1e-10


def test_first_batch_call_with_explicit_tile_and_host_loop():
    # a fresh graph whose first batched call names its tile width (no autotuning beforehand)
    n, g, og = _graph(1500, 6000, seed=101)
    off, seeds = workloads.seed_sets(n, 5, 40, seed=102)
    X1, res1, _ = di.di_ppr_batch(g, off, seeds, D, 1e-10, rhs_tile=8, host_loop=1)
    X2, res2, _ = di.di_ppr_batch(g, off, seeds, D, 1e-10, rhs_tile=8)
    for r in range(5):
        ref = _oracle_X(og, oracle.ppr_B(n, seeds[off[r]:off[r + 1]], D))
        assert rel_l1(X1[r], ref) <= TOL_X and rel_l1(X2[r], ref) <= TOL_X


@pytest.mark.parametrize("tile", [8, 32])
def test_batch_with_nodes_of_many_out_links(tile):
    # two nodes with more out-links than one warp should walk (pushed in chunks over all warps)
    lib()
    n, src, dst = workloads.small_random_graph(20000, 80000, seed=111)
    fan = workloads.u64(112, 1, 14000) % np.uint64(n)
    hub_src = np.concatenate([np.full(9000, 5, np.int32), np.full(5000, 17, np.int32)])
    src = np.concatenate([src, hub_src])
    dst = np.concatenate([dst, fan.astype(np.int32)])
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    assert int(og.outdeg[5]) > 4096 and int(og.outdeg[17]) > 4096
    off = np.array([0, 1, 3, 6], np.int64)
    seeds = np.array([5, 17, 900, 5, 17, 3000], np.int32)
    X, res, info = di.di_ppr_batch(g, off, seeds, D, 1e-10, rhs_tile=tile)
    assert np.all(res <= 1e-10)
    for r in range(3):
        ref = _oracle_X(og, oracle.ppr_B(n, seeds[off[r]:off[r + 1]], D))
        assert rel_l1(X[r], ref) <= TOL_X, r


def test_profiled_batch_times_its_kernels_and_counts_link_columns():
    """opts.profile on a batched solve drives the sweeps from the host and times each select,
    push and reduce; the results equal the oracle's as in graph mode, and the push's
    link-column updates lie between the frontier's links (one column) and T times them."""
    n, g, og = _graph(20000, 90000, seed=61)
    off, seeds = workloads.seed_sets(n, 12, 300, seed=63)
    tol = 1e-10
    X, res, info = di.di_ppr_batch(g, off, seeds, D, tol, rhs_tile=8, profile=1)
    assert np.all(res <= tol)
    for r in range(12):
        ref = _oracle_X(og, oracle.ppr_B(n, seeds[off[r]:off[r + 1]], D))
        assert rel_l1(X[r], ref) <= TOL_X, r
    assert info["push_launches"] > 0 and info["push_ms"] > 0.0
    assert info["select_launches"] == info["push_launches"] == info["reduce_launches"]
    assert 0 < info["column_links"] <= 8 * info["pushed_edges"]
    _, _, plain = di.di_ppr_batch(g, off, seeds, D, tol, rhs_tile=8)
    assert plain["push_launches"] == 0 and plain["column_links"] > 0
