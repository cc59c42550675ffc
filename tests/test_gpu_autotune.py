"""The push autotuner (di_autotune): it picks the single right-hand-side split (row cut-off,
heavy cut-off, chunk length) and the batched tile width and split from the candidate sets, and
solves with the tuned values reach the oracle's fixed point, single and batched. A graph with a
node of very high out-degree (a reversed star) makes the heavy cut-off matter."""
import numpy as np
import pytest

import oracle
import paper_1204_6255_gb300 as di
import workloads
from gpu_util import lib, rel_l1

pytestmark = pytest.mark.gpu
D = 0.85


def test_tuned_split_solves_match_oracle():
    lib()
    spec = workloads.GraphSpec(n=80_000, p_dangling=0.2, cap=6000, mean_out=12.0, p_local=0.7, chain_frac=0.1,
                               seed=workloads.BASE_SEED + 8100, transpose=True)
    n, src, dst = workloads.generate(spec)
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    before = di.di_autotune(g, D, what=0)
    assert (before["push_row"], before["heavy_cut"], before["heavy_chunk"]) == (64, 4096, 1024)
    t = di.di_autotune(g, D, what=3)
    assert t["push_row"] in (32, 64, 128, 256)
    assert t["heavy_cut"] in (1024, 2048, 4096, 8192) and t["batch_heavy_cut"] in (1024, 2048, 4096, 8192)
    assert t["heavy_chunk"] in (256, 512, 1024, 2048) and t["heavy_chunk"] <= t["heavy_cut"]
    assert t["rhs_tile"] in (4, 8, 16, 32) and t["single_probe_ms"] > 0 and t["batch_rate"] > 0
    B = oracle.uniform_B(n, D)
    ref, _, _, ok = oracle.di(og, B, D, 1e-15, oracle.SOP)
    assert ok
    for sched in (di.DI_SOP, di.DI_CYC):
        X, info = di.di_solve(g, B, D, 1e-10, sched)
        assert rel_l1(X, ref) <= 1e-6
    X, info = di.di_solve_ex(g, B, D, 1e-12, schedule=di.DI_SOP, fluid=di.DI_FLUID_F64)
    assert rel_l1(X, ref) <= 1e-10
    off, seeds = workloads.seed_sets(n, 9, 300, seed=8101)
    Xb, res, binfo = di.di_ppr_batch(g, off, seeds, D, 1e-8)
    assert binfo["rhs_tile"] == t["rhs_tile"]
    for r in (0, 4, 8):
        xr, _, _, _ = oracle.di(og, oracle.ppr_B(n, seeds[off[r]:off[r + 1]], D), D, 1e-15, oracle.SOP)
        assert rel_l1(Xb[r], xr) <= 1e-6


def test_tuning_on_a_star_with_both_directions():
    # node 0 links to every other node (out-degree n - 1, far above any cut-off) and every leaf
    # links back: the default split and the tuned one give the oracle's fixed point
    n = 30001
    src = np.concatenate([np.zeros(n - 1, np.int32), np.arange(1, n, dtype=np.int32)])
    dst = np.concatenate([np.arange(1, n, dtype=np.int32), np.zeros(n - 1, np.int32)])
    lib()
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    B = oracle.uniform_B(n, D)
    ref, _, _, ok = oracle.di(og, B, D, 1e-15, oracle.SOP)
    X, info = di.di_solve(g, B, D, 1e-11, di.DI_SOP)
    assert rel_l1(X, ref) <= 1e-6
    t = di.di_autotune(g, D, what=1)
    X, info = di.di_solve(g, B, D, 1e-11, di.DI_SOP)
    assert rel_l1(X, ref) <= 1e-6
