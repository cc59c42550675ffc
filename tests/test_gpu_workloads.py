"""Parity on the full-size synthetic workloads, in the launch configuration the benchmark times.

  pa_n10k : N=10k preferential-attachment graph, FP64 fluid, tol 1e-10: DI-CYC, DI-SOP and PI
            against the oracle's fixed point.
  web_n1m : N=1M web-like graph, FP32 fluid + FP64 refinement, tol 1e-8: DI-SOP, DI-CYC and PI.
  web_n1m_t: the same graph with every link reversed (P transposed: hubs become heavy pushers,
            dangling nodes become zero-in-degree nodes): build, DI-SOP with and without the E
            pre-diffusion, DI-CYC and PI.
  web_n10m_t, web_n10m_e, serve_4g: the bench legs' graphs at full size (transposed: DI-SOP and
            PI'; E-dominated: the pre-diffused DI-SOP; serving: one request per graph and
            tolerance), each against the oracle.
  web_n10m: N=10M, ~150M links: bit-exact graph build; DI-SOP at d=0.85 against the oracle's
            DI-SOP fixed point; d=0.95 certified by the oracle's exact residual of the GPU
            history (||X - H||_1 <= ||B + P.H - H||_1 / (1 - d), a bound that holds at any size).
"""
import numpy as np
import pytest

import oracle
import paper_1204_6255_gb300 as di
import workloads
from gpu_util import assert_build_matches_oracle, lib, rel_l1

pytestmark = pytest.mark.gpu
TOL_X = 1e-6


def _setup(name):
    cfg = workloads.WORKLOADS[name]
    n, src, dst = workloads.generate(cfg["spec"])
    lib()
    return cfg, n, src, dst, di.di_graph_create(n, src, dst), oracle.build(n, src, dst)


def test_pa_n10k_fp64():
    cfg, n, src, dst, g, og = _setup("pa_n10k")
    d, tol = cfg["d"], cfg["tol"]
    B = oracle.uniform_B(n, d)
    ref, _, _, ok = oracle.di(og, B, d, 1e-16, oracle.SOP)
    assert ok
    for sched in (di.DI_CYC, di.DI_SOP):
        X, info = di.di_solve_ex(g, B, d, tol, schedule=sched, fluid=di.DI_FLUID_F64)
        assert rel_l1(X, ref) <= TOL_X and info["residual_l1"] <= tol
    X, info = di.di_power_iter(g, B, d, tol)
    assert rel_l1(X, ref) <= TOL_X


def test_web_n1m_fp32_fluid():
    cfg, n, src, dst, g, og = _setup("web_n1m")
    assert_build_matches_oracle(g, og)
    d, tol = cfg["d"], cfg["tol"]
    B = oracle.uniform_B(n, d)
    ref, _, oinfo, ok = oracle.di(og, B, d, 1e-13, oracle.SOP)
    assert ok
    for sched in (di.DI_SOP, di.DI_CYC):
        X, info = di.di_solve_ex(g, B, d, tol, schedule=sched, fluid=di.DI_FLUID_F32)
        assert info["residual_l1"] <= tol
        assert rel_l1(X, ref) <= TOL_X
    X, info = di.di_power_iter(g, B, d, tol)
    assert rel_l1(X, ref) <= TOL_X


def test_web_n1m_transposed():
    cfg, n, src, dst, g, og = _setup("web_n1m_t")
    assert_build_matches_oracle(g, og)
    assert g.stats["max_out"] > 4096          # rows pushed by the heavy-node path
    d, tol = cfg["d"], cfg["tol"]
    B = oracle.uniform_B(n, d)
    ref, _, _, ok = oracle.di(og, B, d, 1e-13, oracle.SOP)
    assert ok
    for kw in (dict(schedule=di.DI_SOP), dict(schedule=di.DI_SOP, e_prediffuse=1), dict(schedule=di.DI_CYC)):
        X, info = di.di_solve_ex(g, B, d, tol, fluid=di.DI_FLUID_F32, **kw)
        assert info["residual_l1"] <= tol
        assert rel_l1(X, ref) <= TOL_X
    X, info = di.di_power_iter(g, B, d, tol)
    assert rel_l1(X, ref) <= TOL_X


def test_web_n10m_full_size():
    cfg, n, src, dst, g, og = _setup("web_n10m")
    assert_build_matches_oracle(g, og)
    di.di_graph_validate(g)
    tol = cfg["tol"]
    d = 0.85
    B = oracle.uniform_B(n, d)
    X, info = di.di_solve_ex(g, B, d, tol, schedule=di.DI_SOP, fluid=di.DI_FLUID_F32, max_sweeps=20000)
    assert info["residual_l1"] <= tol
    ref, _, _, ok = oracle.di(og, B, d, 1e-11, oracle.SOP)
    assert ok and rel_l1(X, ref) <= TOL_X
    # d = 0.95: certify with the oracle's exact residual of the GPU history
    d = 0.95
    B = oracle.uniform_B(n, d)
    X, info = di.di_solve_ex(g, B, d, tol, schedule=di.DI_SOP, fluid=di.DI_FLUID_F32, max_sweeps=20000)
    _, res = oracle.residual(og, B, d, X)
    assert res <= 1.01 * tol
    assert res / (1 - d) <= TOL_X * np.abs(X).sum()


def test_web_n10m_transposed_full_size():
    # the transposed benchmark graph at full size, as the transposed bench leg runs it
    cfg, n, src, dst, g, og = _setup("web_n10m_t")
    di.di_graph_validate(g)
    d, tol = cfg["d"], cfg["tol"]
    B = oracle.uniform_B(n, d)
    ref, _, _, ok = oracle.di(og, B, d, 1e-11, oracle.SOP)
    assert ok
    X, info = di.di_solve_ex(g, B, d, tol, schedule=di.DI_SOP, max_sweeps=20000)
    assert info["residual_l1"] <= tol and rel_l1(X, ref) <= TOL_X
    X, info = di.di_power_iter_push(g, B, d, tol, max_iters=20000)
    assert info["residual_l1"] <= tol and rel_l1(X, ref) <= TOL_X


def test_web_n10m_e_full_size():
    # the E-dominated graph at full size: the pre-diffused solve against the oracle's
    cfg, n, src, dst, g, og = _setup("web_n10m_e")
    di.di_graph_validate(g)
    d, tol = cfg["d"], cfg["tol"]
    B = oracle.uniform_B(n, d)
    ref, _, oinfo, ok = oracle.di_e(og, B, d, 1e-11, oracle.SOP)
    assert ok and oinfo["e_visits"] == g.stats["E"]
    X, info = di.di_solve_ex(g, B, d, tol, schedule=di.DI_SOP, e_prediffuse=1, max_sweeps=20000)
    assert info["residual_l1"] <= tol and rel_l1(X, ref) <= TOL_X


def test_serving_workload_graphs_full_size():
    # the four resident graphs of the serving leg at full size; one request per graph and
    # tolerance, each against the oracle's solution within its tolerance's error bound
    cfg = workloads.WORKLOADS["serve_4g"]
    d = cfg["d"]
    lib()
    built = []
    for spec in cfg["specs"]:
        n, src, dst = workloads.generate(spec)
        built.append((di.di_graph_create(n, src, dst), oracle.build(n, src, dst)))
    srv = di.di_server_create([g for g, _ in built], d=d, slots=16)
    reqs = []
    for gi, (g, og) in enumerate(built):
        for t, tol in enumerate(cfg["tols"]):
            off, seeds = workloads.seed_sets(g.n, 1, cfg["max_seeds"], seed=9000 + 10 * gi + t)
            reqs.append((gi, seeds, tol, di.di_server_submit(srv, gi, seeds, tol)))
    for gi, seeds, tol, rid in reqs:
        g, og = built[gi]
        X = np.empty(g.n)
        _, info = di.di_server_wait(srv, rid, X_out=X, timeout_ms=600000)
        assert info["status"] == 0 and info["residual_l1"] <= tol
        ref, _, _, ok = oracle.di(og, oracle.ppr_B(g.n, seeds, d), d, 1e-12, oracle.SOP)
        assert ok
        assert np.abs(ref - X).sum() <= tol / (1 - d) * (1 + 1e-6) + 1e-11
    srv.close()
