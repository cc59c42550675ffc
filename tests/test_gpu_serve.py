"""Serving (continuously batched personalised PageRank over resident graphs) through the C ABI.

Requests arrive while others are on the GPU; each one is admitted into a free slot of its
graph's tile (or, while few wait on an idle graph, solved alone on the single right-hand-side
path), retires at its own tolerance and is copied out. Every result must equal the same
request solved alone (and the oracle's solution) within its tolerance's error bound
||X - H||_1 <= tol / (1 - d), whatever was in the mix.
"""
import threading
import time

import numpy as np
import pytest

import oracle
import paper_1204_6255_gb300 as di
import workloads
from gpu_util import lib, rel_l1

pytestmark = pytest.mark.gpu
D = 0.85


def _graphs(sizes, seed):
    lib()
    out = []
    for k, n in enumerate(sizes):
        spec = workloads.GraphSpec(n=n, p_dangling=0.2, cap=1000, mean_out=10.0, p_local=0.7, chain_frac=0.1,
                                   seed=seed + 1000 * k)
        n, src, dst = workloads.generate(spec)
        out.append((di.di_graph_create(n, src, dst), oracle.build(n, src, dst)))
    return out


@pytest.mark.parametrize("tile_min_queue", [1, 4, 0, 1000], ids=["tile", "mixed", "default", "single"])
def test_served_results_match_solo_and_oracle(tile_min_queue):
    # tile_min_queue 1: every request shares the tile; 4: requests run one by one on the single
    # right-hand-side path until 4 wait on an idle graph; 0 (default 16): the same with 16 (the 40
    # requests submitted at once start on the tile); 1000: nearly always single
    graphs = _graphs((3000, 20000), seed=5151)
    srv = di.di_server_create([g for g, _ in graphs], d=D, slots=8, sweeps_per_step=3,
                              tile_min_queue=tile_min_queue)
    rng = workloads.u64(99, 1, 400)
    reqs = []
    tols = (1e-4, 1e-6, 1e-8)
    for i in range(40):
        gi = int(rng[i] % 2)
        n = graphs[gi][0].n
        off, seeds = workloads.seed_sets(n, 1, 200, seed=1000 + i)
        tol = tols[i % 3]
        rid = di.di_server_submit(srv, gi, seeds, tol)
        reqs.append((rid, gi, seeds, tol))
        if i % 7 == 0:
            time.sleep(0.002)           # staggered arrivals
    queue_ms = []
    for rid, gi, seeds, tol in reqs:
        g, og = graphs[gi]
        X = np.empty(g.n)
        _, info = di.di_server_wait(srv, rid, X_out=X, timeout_ms=60000)
        assert info["status"] == 0 and info["residual_l1"] <= tol
        queue_ms.append(info["queue_ms"])
        B = oracle.ppr_B(g.n, seeds, D)
        H, _, _, ok = oracle.di(og, B, D, 1e-13, oracle.SOP)
        assert ok
        bound = tol / (1 - D) * (1 + 1e-6) + 1e-12
        assert np.abs(H - X).sum() <= bound                  # against the oracle's fixed point
        solo, sinfo = di.di_solve(g, B, D, tol)
        assert np.abs(solo - X).sum() <= 2 * bound           # against the same request alone
    srv.close()
    # 40 requests over 2 workers: some of them waited while others were running
    assert max(queue_ms) > 0.0


def test_continuous_admission_under_a_request_stream():
    graphs = _graphs((20000,), seed=6161)
    g, og = graphs[0]
    srv = di.di_server_create([g], d=D, slots=4, sweeps_per_step=2, tile_min_queue=1)
    done = []
    lock = threading.Lock()

    def client(k):
        off, seeds = workloads.seed_sets(g.n, 1, 50, seed=2000 + k)
        rid = di.di_server_submit(srv, 0, seeds, 1e-7)
        X = np.empty(g.n)
        _, info = di.di_server_wait(srv, rid, X_out=X, timeout_ms=60000)
        with lock:
            done.append((seeds, X, info))

    threads = []
    for k in range(12):                  # 12 clients over 4 slots, arriving over time
        t = threading.Thread(target=client, args=(k,))
        t.start()
        threads.append(t)
        time.sleep(0.003)
    for t in threads:
        t.join(timeout=120)
    srv.close()
    assert len(done) == 12
    for seeds, X, info in done:
        assert info["status"] == 0
        ref, _, _, ok = oracle.di(og, oracle.ppr_B(g.n, seeds, D), D, 1e-13, oracle.SOP)
        assert np.abs(ref - X).sum() <= 1e-7 / (1 - D) * (1 + 1e-6) + 1e-12
    # later arrivals were admitted while earlier ones were still on the GPU: some request spent
    # time queued, and slots were reused (more requests than slots all completed)
    assert max(i["queue_ms"] for _, _, i in done) > 0.0


def test_server_errors():
    graphs = _graphs((2000,), seed=7171)
    g, og = graphs[0]
    srv = di.di_server_create([g], d=D, slots=4)
    with pytest.raises(di.DiError) as e:
        di.di_server_submit(srv, 1, np.array([0], np.int32), 1e-6)
    assert e.value.status == 1
    with pytest.raises(di.DiError) as e:
        di.di_server_submit(srv, 0, np.array([g.n], np.int32), 1e-6)
    assert e.value.status == 2
    with pytest.raises(di.DiError) as e:
        di.di_server_submit(srv, 0, np.array([1], np.int32), 0.0)
    assert e.value.status == 1
    with pytest.raises(di.DiError) as e:
        di.di_server_wait(srv, 123456, timeout_ms=10)
    assert e.value.status == 1
    # a request capped at one sweep with a tight tolerance ends NOT_CONVERGED, and the server
    # keeps working afterwards
    srv.close()
    srv = di.di_server_create([g], d=D, slots=4, max_request_sweeps=1)
    rid = di.di_server_submit(srv, 0, np.arange(0, 2000, 3, dtype=np.int32), 1e-12)
    with pytest.raises(di.DiError) as e:
        di.di_server_wait(srv, rid, timeout_ms=60000)
    assert e.value.status == 5
    srv.close()
    with pytest.raises(di.DiError) as e:
        di.di_server_create([g], d=D, slots=4, mem_budget=1000)
    assert e.value.status == 3


def test_destroy_with_requests_in_flight():
    # results being copied out and requests still queued when the server goes away: the
    # destructor drains the in-flight copies and fails the rest, and the graphs stay usable
    graphs = _graphs((50000, 8000), seed=8181)
    srv = di.di_server_create([g for g, _ in graphs], d=D, slots=4, sweeps_per_step=2)
    for i in range(24):
        gi = i % 2
        off, seeds = workloads.seed_sets(graphs[gi][0].n, 1, 100, seed=3000 + i)
        di.di_server_submit(srv, gi, seeds, 1e-8)
    time.sleep(0.05)
    t = time.perf_counter()
    srv.close()
    assert time.perf_counter() - t < 30.0
    g, og = graphs[1]
    srv = di.di_server_create([g], d=D, slots=4)
    seeds = np.array([1, 2, 3], np.int32)
    X = np.empty(g.n)
    rid = di.di_server_submit(srv, 0, seeds, 1e-8)
    _, info = di.di_server_wait(srv, rid, X_out=X, timeout_ms=60000)
    ref, _, _, ok = oracle.di(og, oracle.ppr_B(g.n, seeds, D), D, 1e-13, oracle.SOP)
    assert ok and np.abs(ref - X).sum() <= 1e-8 / (1 - D) * (1 + 1e-6) + 1e-12
    srv.close()


def test_result_into_device_memory():
    import torch
    graphs = _graphs((6000,), seed=9191)
    g, og = graphs[0]
    srv = di.di_server_create([g], d=D, slots=4)
    seeds = np.array([7, 70, 700], np.int32)
    Xd = torch.full((g.n,), -1.0, dtype=torch.float64, device="cuda")
    Xh = np.empty(g.n)
    a = di.di_server_submit(srv, 0, seeds, 1e-9)
    b = di.di_server_submit(srv, 0, seeds, 1e-9)
    di.di_server_wait(srv, a, X_out=Xd, timeout_ms=60000)
    di.di_server_wait(srv, b, X_out=Xh, timeout_ms=60000)
    srv.close()
    ref, _, _, ok = oracle.di(og, oracle.ppr_B(g.n, seeds, D), D, 1e-14, oracle.SOP)
    bound = 1e-9 / (1 - D) * (1 + 1e-6) + 1e-12
    assert ok and np.abs(Xd.cpu().numpy() - ref).sum() <= bound and np.abs(Xh - ref).sum() <= bound
