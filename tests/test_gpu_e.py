"""E-level pre-diffusion (di_solve_ex with e_prediffuse = 1) against the oracle, through the C ABI.

E, the recursively zero-in-degree set, converges in finitely many steps (Section 2.4): visiting
it once in level order leaves every node of E with its exact value, and no fluid reaches E
afterwards. On a DAG every node is in E, so the pre-pass alone solves the system. Expected
values come from the oracle's or_di_e and or_di, which are pinned against dense solves.
"""
import numpy as np
import pytest

import oracle
import paper_1204_6255_gb300 as di
import workloads
from gpu_util import lib, rel_l1

pytestmark = pytest.mark.gpu
D = 0.85


def _dag(n, m, seed):
    u = workloads.u64(seed, 1, 2 * m)
    a = (u[:m] % np.uint64(n)).astype(np.int64)
    b = (u[m:] % np.uint64(n)).astype(np.int64)
    keep = a != b
    return np.minimum(a, b)[keep].astype(np.int32), np.maximum(a, b)[keep].astype(np.int32)


@pytest.mark.parametrize("fluid", [di.DI_FLUID_F64, di.DI_FLUID_F32])
def test_dag_is_solved_by_the_prepass(fluid):
    lib()
    n = 20000
    src, dst = _dag(n, 6 * n, seed=4100)
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    assert g.stats["E"] == n
    B = workloads.uniform(4101, 1, n) * (1 - D) / n
    ref, _, oinfo, ok = oracle.di_e(og, B, D, 1e-300)
    assert ok and oinfo["cycles"] == 0
    tol = 1e-12 * B.sum()
    X, info = di.di_solve_ex(g, B, D, tol, schedule=di.DI_SOP, fluid=fluid, e_prediffuse=1)
    assert info["e_visits"] == n
    if fluid == di.DI_FLUID_F64:
        assert info["sweeps"] == 0            # nothing is left for the sweeps
        assert info["residual_l1"] == 0.0
        assert rel_l1(X, ref) <= 1e-12
    else:
        assert info["residual_l1"] <= tol
        assert rel_l1(X, ref) <= 1e-6


@pytest.mark.parametrize("schedule", [di.DI_CYC, di.DI_SOP])
@pytest.mark.parametrize("fluid", [di.DI_FLUID_F64, di.DI_FLUID_F32])
@pytest.mark.parametrize("seed", [0, 1])
def test_prediffused_solve_matches_oracle(schedule, fluid, seed):
    lib()
    spec = workloads.GraphSpec(n=60000, p_dangling=0.2, cap=500, mean_out=8.0, p_local=0.7, chain_frac=0.4,
                               seed=4200 + seed)
    n, src, dst = workloads.generate(spec)
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    e_mask = oracle.zero_in(og)[0].astype(bool)
    assert g.stats["E"] == int(e_mask.sum()) > 0
    B = workloads.uniform(4300 + seed, 1, n) * (1 - D) / n
    ref, _, _, ok = oracle.di_e(og, B, D, 1e-15 * B.sum(), oracle.SOP)
    assert ok
    plain_ref, _, _, ok = oracle.di(og, B, D, 1e-15 * B.sum(), oracle.SOP)
    assert ok and rel_l1(plain_ref, ref) <= 1e-12
    tol = (1e-13 if fluid == di.DI_FLUID_F64 else 1e-10) * B.sum()
    X, info = di.di_solve_ex(g, B, D, tol, schedule=schedule, fluid=fluid, e_prediffuse=1)
    assert info["e_visits"] == g.stats["E"]
    bar = 1e-10 if fluid == di.DI_FLUID_F64 else 1e-6
    assert rel_l1(X, ref) <= bar
    assert rel_l1(X[e_mask], ref[e_mask]) <= bar
    # the same solve without the pre-pass reaches the same fixed point
    X0, info0 = di.di_solve_ex(g, B, D, tol, schedule=schedule, fluid=fluid)
    assert info0["e_visits"] == 0 and rel_l1(X0, X) <= 2 * bar


def test_prediffusion_host_loop_and_profile_modes():
    lib()
    spec = workloads.GraphSpec(n=30000, p_dangling=0.2, cap=300, mean_out=6.0, p_local=0.7, chain_frac=0.3,
                               seed=4400)
    n, src, dst = workloads.generate(spec)
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    B = workloads.uniform(4401, 1, n) * (1 - D) / n
    ref, _, _, ok = oracle.di_e(og, B, D, 1e-15 * B.sum(), oracle.SOP)
    assert ok
    for kw in (dict(host_loop=1), dict(profile=1)):
        X, info = di.di_solve_ex(g, B, D, 1e-10 * B.sum(), schedule=di.DI_SOP, e_prediffuse=1, **kw)
        assert rel_l1(X, ref) <= 1e-6
        assert info["e_visits"] == g.stats["E"]
    # in profile mode the pre-pass launches (one per level of E) are counted
    assert info["refine_launches"] >= g.stats["e_levels"] + 1


def test_prediffusion_on_the_1m_node_workload():
    lib()
    cfg = workloads.WORKLOADS["web_n1m"]
    n, src, dst = workloads.generate(cfg["spec"])
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    B = np.full(n, (1 - cfg["d"]) / n)
    ref, _, _, ok = oracle.di(og, B, cfg["d"], 1e-13, oracle.SOP)
    assert ok
    X, info = di.di_solve_ex(g, B, cfg["d"], cfg["tol"], schedule=di.DI_SOP, e_prediffuse=1)
    assert info["residual_l1"] <= cfg["tol"] and info["e_visits"] == g.stats["E"]
    assert rel_l1(X, ref) <= 1e-6


def test_prediffusion_on_a_graph_where_E_dominates():
    # the web_n10m_e shape at 200k nodes: 87 % of the nodes in E, 22 levels
    lib()
    base = workloads.WORKLOADS["web_n10m_e"]["spec"]
    spec = workloads.GraphSpec(**dict(base.as_dict(), n=200_000, seed=base.seed + 100))
    n, src, dst = workloads.generate(spec)
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    st = g.stats
    assert st["E"] > 0.8 * n and st["e_levels"] >= 20
    B = oracle.uniform_B(n, D)
    ref, _, _, ok = oracle.di(og, B, D, 1e-13, oracle.SOP)
    assert ok
    X0, i0 = di.di_solve_ex(g, B, D, 1e-8, schedule=di.DI_SOP)
    X1, i1 = di.di_solve_ex(g, B, D, 1e-8, schedule=di.DI_SOP, e_prediffuse=1)
    assert rel_l1(X0, ref) <= 1e-6 and rel_l1(X1, ref) <= 1e-6
    assert i1["e_visits"] == st["E"]
    # the chains no longer feed the core one level per sweep
    assert i1["sweeps"] < i0["sweeps"]


@pytest.mark.parametrize("fluid", [di.DI_FLUID_F64, di.DI_FLUID_F32])
def test_large_levels_take_the_windowed_push(fluid):
    # links only from [0, h) to [h, n): level 0 holds h = 30000 nodes, above the size from which
    # a level is selected by id chunks and pushed through the sweep's windowed push (FP32 fluid)
    lib()
    n, h = 60000, 30000
    u = workloads.u64(4300, 1, 2 * 8 * h)
    src = (u[:8 * h] % np.uint64(h)).astype(np.int32)
    dst = (h + (u[8 * h:] % np.uint64(n - h))).astype(np.int32)
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    assert g.stats["E"] == n and g.stats["e_levels"] == 2
    B = workloads.uniform(4301, 1, n) * (1 - D) / n
    ref, _, oinfo, ok = oracle.di_e(og, B, D, 1e-300)
    assert ok and oinfo["cycles"] == 0
    X, info = di.di_solve_ex(g, B, D, 1e-12 * B.sum(), schedule=di.DI_SOP, fluid=fluid, e_prediffuse=1)
    assert info["e_visits"] == n
    assert rel_l1(X, ref) <= (1e-12 if fluid == di.DI_FLUID_F64 else 1e-6)


def test_prediffusion_on_the_e_dominated_shape_at_1m_nodes():
    # levels of about 40k nodes each: the chunked select and windowed push carry them
    lib()
    base = workloads.WORKLOADS["web_n10m_e"]["spec"]
    spec = workloads.GraphSpec(**dict(base.as_dict(), n=1_000_000, seed=base.seed + 200))
    n, src, dst = workloads.generate(spec)
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    B = oracle.uniform_B(n, D)
    ref, _, _, ok = oracle.di(og, B, D, 1e-12, oracle.SOP)
    assert ok
    for sched in (di.DI_SOP, di.DI_CYC):
        X, info = di.di_solve_ex(g, B, D, 1e-9, schedule=sched, e_prediffuse=1)
        assert rel_l1(X, ref) <= 1e-6 and info["e_visits"] == g.stats["E"]


@pytest.mark.parametrize("fluid", [di.DI_FLUID_F64, di.DI_FLUID_F32])
def test_long_rows_of_a_level_are_pushed_by_the_block(fluid):
    """Nodes of E with far more out-links than a warp takes alone (the block pushes rows above
    256 links after its warps): a layered DAG whose layers hold a few sources of 300 to 6000
    links each beside many short rows. The pre-pass alone must give the oracle's values."""
    lib()
    rng = workloads.u64(4300, 1, 1 << 20)
    pos = [0]

    def draw(k):
        v = rng[pos[0]:pos[0] + k]
        pos[0] += k
        return v

    layers, width = 4, 4000
    n = layers * width
    src, dst = [], []
    for layer in range(layers - 1):
        base, nxt = layer * width, (layer + 1) * width
        for i in range(width):
            deg = (300, 1200, 6000)[i % 3] if i < 9 else 1 + int(draw(1)[0] % np.uint64(12))
            deg = min(deg, width)
            t = nxt + (draw(deg) % np.uint64(width)).astype(np.int64)
            src.append(np.full(deg, base + i, dtype=np.int32))
            dst.append(t.astype(np.int32))
    src, dst = np.concatenate(src), np.concatenate(dst)
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    assert g.stats["E"] == n and g.stats["max_out"] > 256
    B = workloads.uniform(4301, 1, n) * (1 - D) / n
    ref, _, oinfo, ok = oracle.di_e(og, B, D, 1e-300)
    assert ok and oinfo["cycles"] == 0
    tol = 1e-12 * B.sum()
    X, info = di.di_solve_ex(g, B, D, tol, schedule=di.DI_SOP, fluid=fluid, e_prediffuse=1)
    assert info["e_visits"] == n
    assert rel_l1(X, ref) <= (1e-12 if fluid == di.DI_FLUID_F64 else 1e-6)
