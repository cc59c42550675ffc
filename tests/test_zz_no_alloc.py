"""The zero-allocation residual entry point (di_residual_noalloc) agrees with the existing solve.

Callers that cannot allocate (hosts whose own pool owns all device memory, code that must not
add the device-wide synchronisation cudaMalloc may cause) use di_residual_noalloc, which keeps
its scratch in a static device array. di_solve with refinement reports the exact residual ||B + P.H - H||_1 of the
history it returns; the zero-allocation call on the same H must report the same norm, on two
calls in a row (the shared scratch must be left ready by the first call). This file is collected
last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest

import oracle
import paper_1204_6255_gb300 as di
import workloads
from gpu_util import lib

pytestmark = pytest.mark.gpu
TOL_REL = 1e-6
# F* = B + P.H - H is a difference of terms of size ||B||_1 + ||H||_1 that cancel to ~tol; its link
# sums are taken in double-float (unit roundoff 2^-44), so the computed F* carries an absolute
# error of about 2^-44 times the terms it cancels, however small F* itself is
DF_EPS = 2.0 ** -44


def _slack(B, X):
    return DF_EPS * (np.abs(B).sum() + 2.0 * np.abs(X).sum())


def _setup():
    import torch
    lib()
    spec = workloads.GraphSpec(n=60_000, p_dangling=0.2, cap=2000, mean_out=12.0, p_local=0.7, chain_frac=0.1,
                               seed=workloads.BASE_SEED + 777)
    n, src, dst = workloads.generate(spec)
    g = di.di_graph_create(n, src, dst)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    csr = (dev(di.di_graph_export(g, "rowptr_in")), dev(di.di_graph_export(g, "col_in")),
           dev(di.di_graph_export(g, "out_deg")))
    return torch, n, src, dst, g, csr


def test_noalloc_residual_matches_solve_twice():
    torch, n, src, dst, g, (rp_in, col_in, out_deg) = _setup()
    d = 0.85
    og = oracle.build(n, src, dst)
    cases = [(oracle.uniform_B(n, d), di.DI_SOP, 1e-9), (oracle.ppr_B(n, np.arange(0, n, 97), d), di.DI_CYC, 1e-7)]
    for B, sched, tol in cases:          # two calls in a row on the shared scratch
        Bt = torch.from_numpy(B).cuda()
        X, info = di.di_solve_ex(g, Bt, d, tol, schedule=sched)
        norm = torch.zeros(1, dtype=torch.float64, device="cuda")
        Fs = torch.empty(n, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        held, torch_held = di.di_device_bytes_held(), torch.cuda.memory_allocated()
        di.di_residual_noalloc(n, rp_in, col_in, out_deg, Bt, d, X, norm, Fstar_out=Fs)
        torch.cuda.synchronize()
        # neither the library nor torch's allocator gained device memory during the call
        assert di.di_device_bytes_held() == held and torch.cuda.memory_allocated() == torch_held
        got = float(norm.item())
        Xh = X.cpu().numpy()
        slack = _slack(B, Xh)
        assert abs(got - info["residual_l1"]) <= max(TOL_REL * info["residual_l1"], slack), (got, info["residual_l1"])
        ref, ref_norm = oracle.residual(og, B, d, Xh)
        assert abs(got - ref_norm) <= max(TOL_REL * ref_norm, slack)
        assert np.abs(Fs.cpu().numpy() - ref).sum() <= max(TOL_REL * ref_norm, slack)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    torch, n, src, dst, g, (rp_in, col_in, out_deg) = _setup()
    B = torch.zeros(n, dtype=torch.float64, device="cuda")
    norm = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(di.DiError) as e:
        di.di_residual_noalloc((1 << 20) + 1, rp_in, col_in, out_deg, B, 0.85, B, norm)
    assert e.value.status == 1 and "scratch" in e.value.message
    with pytest.raises(di.DiError) as e:
        di.di_residual_noalloc(n, rp_in, col_in, out_deg, B.cpu(), 0.85, B, norm)
    assert e.value.status == 1


def test_noalloc_rejects_short_or_misplaced_arrays():
    """The C call trusts n, so the binding checks every length against it before the call: a
    history, right-hand side or output shorter than n, or row pointers of the wrong length,
    raise DiError instead of reading or writing past the arrays."""
    torch, n, src, dst, g, (rp_in, col_in, out_deg) = _setup()
    B = torch.zeros(n, dtype=torch.float64, device="cuda")
    H = torch.zeros(n, dtype=torch.float64, device="cuda")
    norm = torch.zeros(1, dtype=torch.float64, device="cuda")
    bad = [dict(H=H[: n - 1]), dict(B=B[: n // 2]), dict(rp_in=rp_in[:n]), dict(out_deg=out_deg[:10]),
           dict(norm_out=norm[:0]), dict(Fstar_out=torch.empty(n - 3, dtype=torch.float64, device="cuda"))]
    for kw in bad:
        args = dict(rp_in=rp_in, col_in=col_in, out_deg=out_deg, B=B, H=H, norm_out=norm)
        args.update(kw)
        with pytest.raises(di.DiError) as e:
            di.di_residual_noalloc(n, args["rp_in"], args["col_in"], args["out_deg"], args["B"], 0.85, args["H"],
                                   args["norm_out"], Fstar_out=args.get("Fstar_out"))
        assert e.value.status == 1, kw
    # the checked call still works afterwards on the shared scratch
    di.di_residual_noalloc(n, rp_in, col_in, out_deg, B, 0.85, H, norm)
    torch.cuda.synchronize()
    assert float(norm.item()) == 0.0
