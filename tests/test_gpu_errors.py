"""Measured error of every result against the oracle's fixed point, and its certified bound.

For each method on the two oracle-sized workloads (pa_n10k: N=10k, FP64 workload, tol 1e-10;
web_n1m: N=1M web-like, tol 1e-8), the GPU result X is compared with the oracle's DI-SOP solved
to 1e-14. The contraction of P (Section 2: ||P||_1 <= 1, so ||(I - dP)^-1||_1 <= 1/(1 - d))
gives ||X - X*||_1 <= residual/(1 - d) for the exact residual the solver reports; each measured
error must sit under that bound (plus the oracle's own 1e-14/(1 - d) and the rounding of the
reported residual). Run with `-s` to print the table: one line per method with the relative L1
error, the reported residual and the bound.
"""
import numpy as np
import pytest

import oracle
import paper_1204_6255_gb300 as di
import workloads
from gpu_util import lib, rel_l1

pytestmark = pytest.mark.gpu

ORACLE_TOL = 1e-14
# the exact residual is itself summed in double-float (about 44 bits) over terms of size ||H||_1 = O(1)
RESID_ABS = 1e-12


def _methods(g, B, d, tol):
    F32, F64 = di.DI_FLUID_F32, di.DI_FLUID_F64
    return [
        ("di_sop_f32", lambda: di.di_solve_ex(g, B, d, tol, schedule=di.DI_SOP, fluid=F32)),
        ("di_cyc_f32", lambda: di.di_solve_ex(g, B, d, tol, schedule=di.DI_CYC, fluid=F32)),
        ("di_sop_f64", lambda: di.di_solve_ex(g, B, d, tol, schedule=di.DI_SOP, fluid=F64)),
        ("di_cyc_f64", lambda: di.di_solve_ex(g, B, d, tol, schedule=di.DI_CYC, fluid=F64)),
        ("di_sop_e_prediffused", lambda: di.di_solve_ex(g, B, d, tol, schedule=di.DI_SOP, e_prediffuse=1)),
        ("di_sop_r_refresh2", lambda: di.di_solve_ex(g, B, d, tol, schedule=di.DI_SOP, r_refresh=2)),
        ("di_sop_exact_r", lambda: di.di_solve_ex(g, B, d, tol, schedule=di.DI_SOP, exact_r=1)),
        ("pi_f32_increments", lambda: di.di_power_iter_ex(g, B, d, tol, fluid=F32)),
        ("pi_f64", lambda: di.di_power_iter_ex(g, B, d, tol, fluid=F64)),
        ("pi_push_f32", lambda: di.di_power_iter_push(g, B, d, tol, fluid=F32)),
        ("pi_push_f64", lambda: di.di_power_iter_push(g, B, d, tol, fluid=F64)),
    ]


def _line(name, label, err, residual, bound):
    res = "-" if residual is None else f"{residual:.3e}"
    print(f"\n{name:8s} {label:22s} rel_l1 {err:.3e}  residual {res:>9s}  bound_rel {bound:.3e}", end="")


@pytest.mark.parametrize("name", ["pa_n10k", "web_n1m"])
def test_errors_against_the_oracle(name):
    cfg = workloads.WORKLOADS[name]
    n, src, dst = workloads.generate(cfg["spec"])
    lib()
    g = di.di_graph_create(n, src, dst)
    og = oracle.build(n, src, dst)
    d, tol = cfg["d"], cfg["tol"]
    slack = (ORACLE_TOL + RESID_ABS) / (1 - d)

    B = oracle.uniform_B(n, d)
    ref, _, _, ok = oracle.di(og, B, d, ORACLE_TOL, oracle.SOP)
    assert ok
    norm = np.abs(ref).sum()
    for label, fn in _methods(g, B, d, tol):
        X, info = fn()
        assert info["residual_l1"] <= tol, label
        err = rel_l1(X, ref)
        bound = (info["residual_l1"] / (1 - d) + slack) / norm
        _line(name, label, err, info["residual_l1"], bound)
        assert err <= bound * (1 + 1e-9), label

    # personalised vectors: batched and served, each against its own oracle fixed point
    off, seeds = workloads.seed_sets(n, 8, 500, seed=99)
    refs = []
    for r in range(8):
        xr, _, _, ok = oracle.di(og, oracle.ppr_B(n, seeds[off[r]:off[r + 1]], d), d, ORACLE_TOL, oracle.SOP)
        assert ok
        refs.append(xr)
    Xb, res_b, _ = di.di_ppr_batch(g, off, seeds, d, tol)
    worst = max(range(8), key=lambda r: rel_l1(Xb[r], refs[r]))
    for r in range(8):
        assert res_b[r] <= tol
        bound = (res_b[r] / (1 - d) + slack) / np.abs(refs[r]).sum()
        assert rel_l1(Xb[r], refs[r]) <= bound * (1 + 1e-9), r
    _line(name, "ppr_batch (worst of 8)", rel_l1(Xb[worst], refs[worst]), float(res_b[worst]),
          (res_b[worst] / (1 - d) + slack) / np.abs(refs[worst]).sum())

    srv = di.di_server_create([g], d=d, slots=8)
    try:
        errs = []
        for r in range(4):
            rid = di.di_server_submit(srv, 0, seeds[off[r]:off[r + 1]], tol)
            X = np.empty(n)
            _, info = di.di_server_wait(srv, rid, X_out=X, timeout_ms=60000)
            assert info["status"] == 0 and info["residual_l1"] <= tol
            bound = (info["residual_l1"] / (1 - d) + slack) / np.abs(refs[r]).sum()
            errs.append((rel_l1(X, refs[r]), info["residual_l1"], bound))
            assert errs[-1][0] <= bound * (1 + 1e-9), r
    finally:
        srv.close()
    err, residual, bound = max(errs)
    _line(name, "served (worst of 4)", err, residual, bound)
