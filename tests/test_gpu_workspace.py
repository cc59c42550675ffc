"""Caller-owned scratch at the C boundary: after di_graph_set_workspace every solve of that kind
lays its scratch out in the caller's buffer (a torch allocation here) and calls no allocator,
and its results are those of the same solves with library-allocated scratch."""
import numpy as np
import pytest

import oracle
import paper_1204_6255_gb300 as di
import workloads
from gpu_util import lib, rel_l1

pytestmark = pytest.mark.gpu
D = 0.85


def _graph(seed=4040, n=50_000):
    spec = workloads.GraphSpec(n=n, p_dangling=0.2, cap=2000, mean_out=10.0, p_local=0.7, chain_frac=0.1,
                               seed=workloads.BASE_SEED + seed)
    n, src, dst = workloads.generate(spec)
    return n, src, dst


def test_solves_in_a_torch_workspace_allocate_nothing():
    import torch
    lib()
    n, src, dst = _graph()
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    B = oracle.uniform_B(n, D)
    ref, _, _, ok = oracle.di(og, B, D, 1e-14, oracle.SOP)
    assert ok
    sizes = {(di.DI_WS_SOLVE, di.DI_FLUID_F32): di.di_workspace_size(g, di.DI_WS_SOLVE, di.DI_FLUID_F32),
             (di.DI_WS_SOLVE, di.DI_FLUID_F64): di.di_workspace_size(g, di.DI_WS_SOLVE, di.DI_FLUID_F64),
             (di.DI_WS_BATCH, 8): di.di_workspace_size(g, di.DI_WS_BATCH, 8),
             (di.DI_WS_BATCH, 32): di.di_workspace_size(g, di.DI_WS_BATCH, 32)}
    assert sizes[(di.DI_WS_SOLVE, di.DI_FLUID_F64)] > sizes[(di.DI_WS_SOLVE, di.DI_FLUID_F32)] > 40 * n
    assert sizes[(di.DI_WS_BATCH, 32)] > sizes[(di.DI_WS_BATCH, 8)] > 8 * 40 * n
    ws_solve = torch.empty(sizes[(di.DI_WS_SOLVE, di.DI_FLUID_F64)], dtype=torch.uint8, device="cuda")
    ws_batch = torch.empty(sizes[(di.DI_WS_BATCH, 8)], dtype=torch.uint8, device="cuda")
    di.di_graph_set_workspace(g, di.DI_WS_SOLVE, ws_solve)
    di.di_graph_set_workspace(g, di.DI_WS_BATCH, ws_batch)
    held = di.di_device_bytes_held()
    Bt = torch.from_numpy(B).cuda()
    # every solve kind, FP32 and FP64 fluid, power iteration both ways, a resumed solve
    for sched in (di.DI_SOP, di.DI_CYC):
        X, info = di.di_solve(g, Bt, D, 1e-9, sched)
        assert rel_l1(X.cpu().numpy(), ref) <= 1e-6
    X, _ = di.di_solve_ex(g, Bt, D, 1e-11, schedule=di.DI_SOP, fluid=di.DI_FLUID_F64)
    assert rel_l1(X.cpu().numpy(), ref) <= 1e-9
    X, _ = di.di_power_iter(g, Bt, D, 1e-9)
    assert rel_l1(X.cpu().numpy(), ref) <= 1e-6
    X, _ = di.di_power_iter_push(g, Bt, D, 1e-9)
    assert rel_l1(X.cpu().numpy(), ref) <= 1e-6
    H0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    X, _ = di.di_solve_resume(g, Bt, H0, D, 1e-9)
    assert rel_l1(X.cpu().numpy(), ref) <= 1e-6
    # batched: the autotuner only tries widths the 8-column workspace holds
    k = 11
    off, seeds = workloads.seed_sets(n, k, 200, seed=77)
    Xb, res, binfo = di.di_ppr_batch(g, off, seeds, D, 1e-7)
    assert binfo["rhs_tile"] <= 8 and np.all(res <= 1e-7)
    Bs = np.zeros((3, n))
    for r in range(3):
        Bs[r, np.arange(r, n, 7)] = 1.0 / len(range(r, n, 7)) * (1 - D)
    Xd, res, _ = di.di_solve_batch(g, Bs, D, 1e-8, rhs_tile=4)
    torch.cuda.synchronize()
    assert di.di_device_bytes_held() == held, "a solve with an attached workspace allocated device memory"
    for r in range(k):
        Br = oracle.ppr_B(n, seeds[off[r]:off[r + 1]], D)
        xr, _, _, ok = oracle.di(og, Br, D, 1e-14, oracle.SOP)
        assert rel_l1(Xb[r], xr) <= 1e-6
    xr, _, _, _ = oracle.di(og, Bs[2], D, 1e-14, oracle.SOP)
    assert rel_l1(Xd[2], xr) <= 1e-6
    # wider tiles than the workspace holds: an error, no allocation
    with pytest.raises(di.DiError) as e:
        di.di_ppr_batch(g, off, seeds, D, 1e-7, rhs_tile=32)
    assert e.value.status == 1 and "workspace" in e.value.message
    assert di.di_device_bytes_held() == held
    # detached: the library allocates its own scratch again
    di.di_graph_set_workspace(g, di.DI_WS_SOLVE, None)
    X, _ = di.di_solve(g, Bt, D, 1e-9, di.DI_SOP)
    assert rel_l1(X.cpu().numpy(), ref) <= 1e-6
    assert di.di_device_bytes_held() > held


def test_workspace_checks():
    import torch
    lib()
    n, src, dst = _graph(seed=4041, n=5_000)
    g = di.di_graph_create(n, src, dst)
    need = di.di_workspace_size(g, di.DI_WS_SOLVE, di.DI_FLUID_F32)
    small = torch.empty(need // 2, dtype=torch.uint8, device="cuda")
    di.di_graph_set_workspace(g, di.DI_WS_SOLVE, small)
    held = di.di_device_bytes_held()
    B = torch.full((n,), (1 - D) / n, dtype=torch.float64, device="cuda")
    with pytest.raises(di.DiError) as e:
        di.di_solve(g, B, D, 1e-9, di.DI_SOP)
    assert e.value.status == 1 and "workspace" in e.value.message
    assert di.di_device_bytes_held() == held
    # unaligned, host memory, unknown kind
    big = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    assert di.load().di_graph_set_workspace(g.handle, di.DI_WS_SOLVE, big.data_ptr() + 8, need) == 1
    host = np.zeros(need, dtype=np.uint8)
    assert di.load().di_graph_set_workspace(g.handle, di.DI_WS_SOLVE, host.ctypes.data, need) == 1
    assert di.load().di_graph_set_workspace(g.handle, 7, big.data_ptr(), need) == 1
    # the right size works
    di.di_graph_set_workspace(g, di.DI_WS_SOLVE, big)
    X, info = di.di_solve(g, B, D, 1e-9, di.DI_SOP)
    assert info["residual_l1"] <= 1e-9
