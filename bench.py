#!/usr/bin/env python
"""Benchmark of the GB300 D-iteration.

One step = one DI-SOP solve (Section 2.3) of X = P.X + B to ||F||_1 <= 1e-8 on the resident
10M-node / ~150M-link synthetic web graph (FP32 fluid, FP64 history and residual, exact FP64
refinement), B = (1-d)/N, d = 0.85. The metric is GTEPS = pushed links / solve time (the graph
build is timed apart, like the paper's "Init"). Inputs (CSR ~1.8 GB) are larger than L2 and L2 is
flushed between steps anyway.

Extra legs in the same JSON line: time-to-residual of DI-SOP, DI-CYC and power iteration at
d = 0.85 and DI-SOP at d = 0.95; graph build time; the roofline of the push kernel; the oracle
timed on the host cores (`cpu_baseline`).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Multi-GPU: the solve does not shard here, so N ranks run N independent replicas ("weak"
scaling); value = pushed links of all ranks / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "web_n10m"
D = 0.85
TOL = 1e-8
L2_FLUSH_BYTES = 512 << 20
MAX_SWEEPS = 20000


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    p.add_argument("--no-legs", action="store_true", help="skip the extra legs (DI-CYC, PI, d=0.95)")
    p.add_argument("--legs", default="all",
                   help="comma list of extra legs to run: solvers, small_graphs, transposed, e_dominated, "
                        "ppr_batch, serving")
    p.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    p.add_argument("--push-split", default="",
                   help="row,heavy_cut,heavy_chunk: use this push split instead of tuning it (profiling runs)")
    p.add_argument("--one-solve", action="store_true",
                   help="build the graph, run one DI-SOP solve and exit (the command the ncu captures profile)")
    p.add_argument("--one-pi", action="store_true",
                   help="build the graph, run one power iteration solve and exit (profiles the pull)")
    p.add_argument("--sweeps", default="",
                   help="with --one-solve: A,B runs the same solve capped at A and then at B sweeps and prints "
                        "the links and frontier entries that sweeps A+1..B push (scales a capture of those "
                        "push launches to algorithmic bytes)")
    return p.parse_args()


def world():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


def aggregate(dist, total_ms: float, pushed: float, launches: int, device=None):
    """Whole-job numbers over the ranks of a replica run: the slowest rank's time and the summed
    pushed links and kernel launches (each rank solves its own replica). Without a process
    group the rank's own numbers are returned."""
    if dist is None:
        return total_ms, pushed, launches
    import torch
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([float(pushed), float(launches)], dtype=torch.float64, device=device)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p[0].item()), int(p[1].item())


# ------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        # the timed region starts once the sampler has written its first line (nvidia-smi takes
        # a moment to start), so every timed step is covered
        t0 = time.time()
        while time.time() - t0 < 5.0 and os.path.getsize(self.path) == 0:
            time.sleep(0.02)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


PUSH_SRC = os.path.join(ROOT, "paper_1204_6255_gb300", "csrc", "di_solve.cu")
PUSH_PROFILE = os.path.join(ROOT, "profiles", "k_push_win_web_n10m.md")


def push_source_sha():
    """sha256 of the push kernel's source: the text from the comment that opens k_push_win's
    section of di_solve.cu to the kernel's closing brace (its constants included)."""
    import hashlib
    text = open(PUSH_SRC).read()
    start = text.index("// Push with a shared-memory window (FP32 fluid).")
    body = text.index("k_push_win(", start)
    end = text.index("\n}\n", body) + 3
    return hashlib.sha256(text[start:end].encode()).hexdigest()


def push_traffic():
    """DRAM bytes per push launch from the committed ncu summary, or None when the push kernel's
    source changed since that capture (the summary records its sha256)."""
    if not os.path.exists(PUSH_PROFILE):
        return None, None
    sha = push_source_sha()
    fields = {}
    for line in open(PUSH_PROFILE):
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            fields[k.strip()] = v.strip().strip("`")
    if fields.get("source_sha256") != sha:
        return None, "stale: kernel source changed since the capture"
    try:
        return float(fields["dram_bytes_per_launch"]), os.path.relpath(PUSH_PROFILE, ROOT)
    except (KeyError, ValueError):
        return None, None


def host_cpu(cpuinfo="/proc/cpuinfo"):
    """The host the oracle ran on: architecture, logical cores, and the CPU model when the
    kernel reports one."""
    import platform
    model, arm = None, {}
    try:
        for line in open(cpuinfo):
            key, _, val = line.partition(":")
            key = key.strip().lower()
            if key in ("model name", "cpu model") and model is None:
                model = val.strip()
            elif key in ("cpu implementer", "cpu part") and key not in arm:
                arm[key] = val.strip()   # Arm cores report these instead of a model name
    except OSError:
        pass
    if model is None and arm:
        model = "implementer {} part {}".format(arm.get("cpu implementer", "?"), arm.get("cpu part", "?"))
    return {"machine": platform.machine(), "nproc": os.cpu_count(), "model": model}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------------------------------
# CPU oracle legs (the only place bench.py runs oracle/)
# ------------------------------------------------------------------------------------------
def oracle_sample(n, src, dst, d, max_cycles):
    """The oracle's sequential DI-SOP on the same graph, bounded to `max_cycles` cycles from
    F = B. Returns (pushed links, seconds, cycles)."""
    import oracle
    og = oracle.build(n, src, dst)
    B = oracle.uniform_B(n, d)
    t = time.perf_counter()
    _, _, info, _ = oracle.di(og, B, d, TOL, oracle.SOP, max_cycles=max_cycles)
    sec = time.perf_counter() - t
    return info["pushed_edges"], sec, info["cycles"], og


def run_reference(args):
    rank, local_rank, ws = world()
    if ws > 1 and rank != 0:
        return
    import workloads
    cfg = workloads.WORKLOADS[WORKLOAD]
    n, src, dst = workloads.generate(cfg["spec"])
    import oracle
    og = oracle.build(n, src, dst)
    B = oracle.uniform_B(n, D)
    # each step: one DI-SOP cycle of the oracle from F = B (a bounded sample of the solve)
    times, pushed = [], []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        _, _, info, _ = oracle.di(og, B, D, TOL, oracle.SOP, max_cycles=1)
        dt = time.perf_counter() - t
        if i >= args.warmup:
            times.append(dt)
            pushed.append(info["pushed_edges"])
    total = sum(times)
    value = sum(pushed) / total / 1e9
    line = {
        "impl": "reference", "metric": "GTEPS (DI-SOP, N=10M, tol 1e-8)", "value": value, "unit": "GTEPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: N={n}, L={og.L}, d={D}, tol={TOL}, B=(1-d)/N",
                   "step": "one oracle DI-SOP cycle from F=B (bounded sample of the solve)", "fluid": "f64",
                   "history": "f64"},
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                         "sample": "one sequential DI-SOP cycle per step on the full 10M-node graph",
                         "host": host_cpu()},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------------------------------------
# PPR legs: batched solves and served requests, each against per-request plain solves
# ------------------------------------------------------------------------------------------
def pct(values, q):
    import numpy as np
    return float(np.percentile(np.asarray(values, dtype=float), q)) if values else None


def ppr_batch_leg(di, workloads, torch):
    """256 personalised PageRank requests on the 2M-node graph (seed sets of 1..1000 nodes,
    tol 1e-6): one batched call against the same requests solved one by one (a sample)."""
    import numpy as np
    cfg = workloads.WORKLOADS["ppr_n2m_k256"]
    n, src, dst = workloads.generate(cfg["spec"])
    g = di.di_graph_create(n, src, dst)
    k, d, tol = cfg["k"], cfg["d"], cfg["tol"]
    off, seeds = workloads.seed_sets(n, k, cfg["max_seeds"], seed=cfg["spec"].seed)
    off_d, seeds_d = torch.from_numpy(off).cuda(), torch.from_numpy(seeds).cuda()
    X = torch.empty((k, n), dtype=torch.float64, device="cuda")
    di.di_ppr_batch(g, off_d[:9], seeds_d, d, tol, X_out=X[:8])        # autotune + warm-up
    torch.cuda.synchronize()
    t = time.perf_counter()
    _, res, info = di.di_ppr_batch(g, off_d, seeds_d, d, tol, X_out=X)
    torch.cuda.synchronize()
    batch_s = time.perf_counter() - t
    # per-request plain solves (single right-hand side, FP32 fluid + refinement) of the same
    # 256 requests
    sample = k
    B = torch.zeros(n, dtype=torch.float64, device="cuda")
    Xs = torch.empty(n, dtype=torch.float64, device="cuda")
    for r in range(2):                                   # warm-up of the same path
        B.zero_()
        sr = seeds_d[off[r]:off[r + 1]].long()
        B.index_add_(0, sr, torch.full((sr.numel(),), (1 - d) / sr.numel(), dtype=torch.float64, device="cuda"))
        di.di_solve(g, B, d, tol, di.DI_SOP, MAX_SWEEPS, X_out=Xs)
    torch.cuda.synchronize()
    lat = []
    t0 = time.perf_counter()
    for r in range(sample):
        B.zero_()
        sr = seeds_d[off[r]:off[r + 1]].long()
        B.index_add_(0, sr, torch.full((sr.numel(),), (1 - d) / sr.numel(), dtype=torch.float64, device="cuda"))
        t = time.perf_counter()
        di.di_solve(g, B, d, tol, di.DI_SOP, MAX_SWEEPS, X_out=Xs)
        lat.append(1e3 * (time.perf_counter() - t))
    solo_s = time.perf_counter() - t0
    # the batched push's roofline, from one more batched call with each kernel timed alone:
    # per launch 4 B link index per link of a frontier node, 8 B read-modify-write of F per
    # link and column with a non-zero share, and per frontier entry 4 B id + 8 B row bounds +
    # 4 B share per column of the tile
    _, _, pinfo = di.di_ppr_batch(g, off_d, seeds_d, d, tol, X_out=X, profile=1)
    T = pinfo["rhs_tile"]
    launches = max(pinfo["push_launches"], 1)
    push_bytes = (4.0 * pinfo["pushed_edges"] + 8.0 * pinfo["column_links"]
                  + (12.0 + 4.0 * T) * pinfo["frontier_entries"]) / launches
    push_ms = pinfo["push_ms"] / launches
    peak, peak_kind = peaks()
    roof = {"kernel": f"kb_push<{T}>", "bound": "hbm", "bytes_per_launch": push_bytes, "ms_per_launch": push_ms,
            "achieved": push_bytes / (push_ms * 1e-3) / 1e9, "peak": peak, "unit": "GB/s", "peak_kind": peak_kind,
            "frac": push_bytes / (push_ms * 1e-3) / 1e9 / peak, "launches": pinfo["push_launches"],
            "column_links": pinfo["column_links"], "select_ms_per_launch": pinfo["select_ms"] / max(pinfo["select_launches"], 1)}
    return {"requests": k, "graph": f"N={n}, L={g.stats['L']}", "tol": tol, "rhs_tile": info["rhs_tile"],
            "push_split": di.di_autotune(g, d, what=0), "roofline": roof,
            "batched_qps": k / batch_s, "batched_ms": 1e3 * batch_s,
            "per_request_qps": sample / solo_s, "per_request_p50_ms": pct(lat, 50), "per_request_p99_ms": pct(lat, 99),
            "speedup": (k / batch_s) / (sample / solo_s), "max_residual": float(np.max(res))}


def small_graph_leg(di, workloads, torch, name, reps=7):
    """The paper's four solvers on a smaller workload, median of `reps` solves after warm-ups,
    inputs resident: pa_n10k (10k nodes, everything in FP64, tol 1e-10) and web_n1m (1M nodes,
    FP32 fluid with the exact FP64 refinement, tol 1e-8)."""
    import statistics
    cfg = workloads.WORKLOADS[name]
    n, src, dst = workloads.generate(cfg["spec"])
    g = di.di_graph_create(n, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda())
    d, tol = cfg["d"], cfg["tol"]
    fp64 = cfg["fluid"] == "f64"
    fluid = di.DI_FLUID_F64 if fp64 else di.DI_FLUID_F32
    B = torch.full((n,), (1.0 - d) / n, dtype=torch.float64, device="cuda")
    X = torch.empty(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    runs = {
        "di_sop": lambda: di.di_solve_ex(g, B, d, tol, schedule=di.DI_SOP, fluid=fluid, max_sweeps=MAX_SWEEPS, X_out=X)[1],
        "di_cyc": lambda: di.di_solve_ex(g, B, d, tol, schedule=di.DI_CYC, fluid=fluid, max_sweeps=MAX_SWEEPS, X_out=X)[1],
        "pi": lambda: di.di_power_iter_ex(g, B, d, tol, fluid=fluid, max_iters=MAX_SWEEPS, X_out=X)[1],
        "pi_push": lambda: di.di_power_iter_push(g, B, d, tol, max_iters=MAX_SWEEPS, fluid=fluid, X_out=X)[1],
    }
    out = {"graph": {k: g.stats[k] for k in ("n_nodes", "L", "D", "E", "O", "max_in", "max_out")}, "d": d, "tol": tol,
           "fluid": cfg["fluid"], "median_of": reps}
    for label, fn in runs.items():
        fn()
        fn()
        ms, inf = [], None
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            inf = fn()
            b.record(stream)
            b.synchronize()
            ms.append(a.elapsed_time(b))
        out[label] = {"ms_to_residual": statistics.median(ms), "iterations_or_sweeps": inf["sweeps"],
                      "pushed_per_L": inf["pushed_edges"] / g.stats["L"], "residual_l1": inf["residual_l1"]}
    return out


def transposed_leg(di, workloads, torch, flush, name="web_n10m_t"):
    """Another 10M-node graph: by default the benchmark graph with every link reversed (P
    transposed, the paper's Dataset 1bis pattern); `web_n10m_e` is the graph where E dominates
    (E/N about 0.87, like the paper's Dataset 2). DI-SOP with and without the E pre-diffusion,
    and PI, from resident inputs."""
    cfg = workloads.WORKLOADS[name]
    n, src, dst = workloads.generate(cfg["spec"])
    g = di.di_graph_create(n, torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda())
    del src, dst
    d, tol = cfg["d"], cfg["tol"]
    B = torch.full((n,), (1.0 - d) / n, dtype=torch.float64, device="cuda")
    X = torch.empty(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()                                                   # warm-up of the same call
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        inf = fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b), inf

    out = {"graph": {k: g.stats[k] for k in ("n_nodes", "L", "D", "E", "e_levels", "max_in", "max_out")}}
    for name, e in (("di_sop", 0), ("di_sop_e_prediffused", 1)):
        ms, inf = timed(lambda: di.di_solve_ex(g, B, d, tol, schedule=di.DI_SOP, max_sweeps=MAX_SWEEPS,
                                                e_prediffuse=e, X_out=X)[1])
        out[name] = {"ms_to_residual": ms, "GTEPS": inf["pushed_edges"] / (ms * 1e-3) / 1e9, "sweeps": inf["sweeps"],
                     "pushed_per_L": inf["pushed_edges"] / g.stats["L"], "residual_l1": inf["residual_l1"]}
    ms, inf = timed(lambda: di.di_power_iter(g, B, d, tol, max_iters=MAX_SWEEPS, X_out=X)[1])
    out["pi"] = {"ms_to_residual": ms, "iterations": inf["sweeps"], "residual_l1": inf["residual_l1"]}
    ms, inf = timed(lambda: di.di_power_iter_push(g, B, d, tol, max_iters=MAX_SWEEPS, X_out=X)[1])
    out["pi_push"] = {"ms_to_residual": ms, "iterations": inf["sweeps"], "residual_l1": inf["residual_l1"]}
    return out


def serving_leg(di, workloads, torch, n_req=1000, fracs=(0.25, 0.5, 0.75, 1.0, 1.25), slots=16,
                sweeps_per_step=8, tile_min_queue=0):
    """Poisson streams of personalised PageRank requests over four resident graphs (N = 100k,
    500k, 2M, 5M), tolerances 1e-4/1e-6/1e-8, seed sets of 1..1000 nodes, at arrival rates of
    25% to 125% of the plain path's capacity: the continuously batched server against
    per-request plain solves in arrival order (one at a time on the same GPU). Latency runs from
    arrival to the history in host memory on both sides.

    The plain path is a single FIFO server whose service times do not depend on the arrivals, so
    each request's plain service time (seed upload, solve, copy-out) is measured once, and its
    latency at every rate follows from the FIFO recursion finish = max(arrival, previous finish)
    + service. The served side runs in real time at each rate."""
    import numpy as np
    cfg = workloads.WORKLOADS["serve_4g"]
    d = cfg["d"]
    graphs = []
    for spec in cfg["specs"]:
        n, src, dst = workloads.generate(spec)
        graphs.append(di.di_graph_create(n, src, dst))
    u = workloads.uniform(4242, 1, 3 * n_req)
    gsel = (u[n_req:2 * n_req] * len(graphs)).astype(int)
    tsel = (u[2 * n_req:] * 3).astype(int)
    reqs = []
    for i in range(n_req):
        g = graphs[gsel[i]]
        off, seeds = workloads.seed_sets(g.n, 1, cfg["max_seeds"], seed=7000 + i)
        reqs.append((gsel[i], seeds, cfg["tols"][tsel[i]]))

    # plain service times, one request at a time (done when its history is in pinned host memory)
    Bs = [torch.zeros(g.n, dtype=torch.float64, device="cuda") for g in graphs]
    Xs = [torch.empty(g.n, dtype=torch.float64, device="cuda") for g in graphs]
    Xh = [torch.empty(g.n, dtype=torch.float64).pin_memory() for g in graphs]

    def plain(gi, seeds, tol):
        B = Bs[gi]
        B.zero_()
        sd = torch.from_numpy(seeds.astype(np.int64)).cuda()
        B.index_add_(0, sd, torch.full((sd.numel(),), (1 - d) / sd.numel(), dtype=torch.float64, device="cuda"))
        di.di_solve(graphs[gi], B, d, tol, di.DI_SOP, MAX_SWEEPS, X_out=Xs[gi])
        Xh[gi].copy_(Xs[gi], non_blocking=True)
        torch.cuda.current_stream().synchronize()

    for gi, g in enumerate(graphs):                                 # warm-up of the same path
        plain(gi, np.arange(8, dtype=np.int32), 1e-4)
    service = np.empty(n_req)
    for i, (gi, seeds, tol) in enumerate(reqs):
        t = time.perf_counter()
        plain(gi, seeds, tol)
        service[i] = time.perf_counter() - t
    capacity = n_req / service.sum()

    srv = di.di_server_create(graphs, d=d, slots=slots, sweeps_per_step=sweeps_per_step,
                              tile_min_queue=tile_min_queue)
    for gi in range(len(graphs)):                                   # warm every worker
        di.di_server_wait(srv, di.di_server_submit(srv, gi, np.array([0], np.int32), 1e-4), timeout_ms=60000)
    points = []
    for k, frac in enumerate(fracs):
        rate = frac * capacity
        gaps = -np.log(1.0 - workloads.uniform(4300 + k, 1, n_req)) / rate      # Poisson arrivals
        arrive = np.cumsum(gaps)
        # plain: FIFO recursion over the measured service times
        finish, lat_p = 0.0, np.empty(n_req)
        for i in range(n_req):
            finish = max(arrive[i], finish) + service[i]
            lat_p[i] = 1e3 * (finish - arrive[i])
        plain_qps = n_req / finish
        # served, in real time; a client thread collects results while requests arrive, so the
        # server's pinned result buffers are recycled as a serving front end would
        ids = [None] * n_req
        infos = [None] * n_req
        submitted = threading.Semaphore(0)

        def collect():
            for i in range(n_req):
                submitted.acquire()
                infos[i] = di.di_server_wait(srv, ids[i], timeout_ms=600000)[1]

        waiter = threading.Thread(target=collect)
        waiter.start()
        t0 = time.perf_counter()
        for i, (gi, seeds, tol) in enumerate(reqs):
            delay = arrive[i] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ids[i] = di.di_server_submit(srv, int(gi), seeds, tol)
            submitted.release()
        waiter.join()
        lat, worst, lone, by_graph = [], 0.0, 0, {}
        for i in range(n_req):
            info = infos[i]
            assert info is not None, f"request {i} was not collected"
            lat.append(info["total_ms"])
            lone += info["slot"] < 0
            by_graph.setdefault(int(reqs[i][0]), []).append(info["total_ms"])
            worst = max(worst, info["residual_l1"] / reqs[i][2])
        served_s = time.perf_counter() - t0
        plain_by_graph = {}
        for i in range(n_req):
            plain_by_graph.setdefault(int(reqs[i][0]), []).append(lat_p[i])
        points.append({"load": frac, "arrival_qps": rate, "served_qps": n_req / served_s,
                       "served_p50_ms": pct(lat, 50), "served_p99_ms": pct(lat, 99), "plain_qps": plain_qps,
                       "plain_p50_ms": pct(list(lat_p), 50), "plain_p99_ms": pct(list(lat_p), 99),
                       "served_single_path": lone / n_req,
                       "served_p99_ms_by_graph": [pct(by_graph.get(k, []), 99) for k in range(len(graphs))],
                       "plain_p99_ms_by_graph": [pct(plain_by_graph.get(k, []), 99) for k in range(len(graphs))],
                       "worst_residual_over_tol": worst})
    srv.close()
    return {"requests_per_point": n_req, "graphs": [g.n for g in graphs], "slots": slots,
            "sweeps_per_step": sweeps_per_step, "tile_min_queue": tile_min_queue or 16, "plain_capacity_qps": capacity,
            "plain_service_ms_mean": 1e3 * float(service.mean()), "points": points}


# ------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch

    import paper_1204_6255_gb300 as di
    import workloads

    rank, local_rank, ws = world()
    torch.cuda.set_device(local_rank)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    di.build()
    di.load()
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream(dev)

    cfg = workloads.WORKLOADS[WORKLOAD]
    n, src, dst = workloads.generate(cfg["spec"])

    # graph build from a device edge list (the paper's "Init", timed apart)
    src_d = torch.from_numpy(src).to(dev)
    dst_d = torch.from_numpy(dst).to(dev)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g = di.di_graph_create(n, src_d, dst_d)
    e1.record(stream)
    torch.cuda.synchronize()
    build_ms = e0.elapsed_time(e1)
    del src_d, dst_d
    st = g.stats

    B = torch.full((n,), (1.0 - D) / n, dtype=torch.float64, device=dev)
    X = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # the push split (row cut-off, heavy cut-off, chunk length) tuned once for this graph, like
    # the build: outside the timed region
    t_tune = time.perf_counter()
    if args.push_split:
        tuning = di.di_autotune(g, D, what=0, set_split=[int(x) for x in args.push_split.split(",")])
    else:
        tuning = di.di_autotune(g, D, what=1)
    tune_s = time.perf_counter() - t_tune

    def step(Bx=B, Xx=X, d=D, schedule=di.DI_SOP, **kw):
        return di.di_solve_ex(g, Bx, d, TOL, schedule=schedule, fluid=di.DI_FLUID_F32, max_sweeps=MAX_SWEEPS,
                              X_out=Xx, **kw)[1]

    if args.one_pi:
        info = di.di_power_iter_ex(g, B, D, TOL, max_iters=MAX_SWEEPS, profile=1, X_out=X)[1]
        torch.cuda.synchronize()
        print(json.dumps({"one_pi": {k: info[k] for k in ("sweeps", "refine_rounds", "kernel_launches", "ms")}}))
        return
    if args.one_solve and args.sweeps:
        a, b = (int(x) for x in args.sweeps.split(","))
        counts = []
        for cap in (a, b):
            try:
                info = di.di_solve_ex(g, B, D, TOL, schedule=di.DI_SOP, fluid=di.DI_FLUID_F32, max_sweeps=cap,
                                      X_out=X, profile=1)[1]
            except di.DiError as e:           # capped before the tolerance: the counts still come back
                info = e.info
            counts.append(info)
        print(json.dumps({"sweeps": [a + 1, b], "push_launches": counts[1]["push_launches"] - counts[0]["push_launches"],
                          "pushed_edges": counts[1]["pushed_edges"] - counts[0]["pushed_edges"],
                          "frontier_entries": counts[1]["frontier_entries"] - counts[0]["frontier_entries"]}))
        return
    if args.one_solve:
        info = step(profile=1)        # kernels launched one by one, so a profiler sees each
        torch.cuda.synchronize()
        print(json.dumps({"one_solve": {k: info[k] for k in ("sweeps", "pushed_edges", "frontier_entries",
                                                             "kernel_launches", "ms")}}))
        return

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    sampler = ClockSampler(vis.split(",")[local_rank] if vis else local_rank)
    sampler.start()
    step_ms, infos = [], []
    for _ in range(args.steps):
        flush.fill_(1)                      # evict the previous step's lines from L2
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        info = step()
        b.record(stream)
        b.synchronize()
        step_ms.append(a.elapsed_time(b))
        infos.append(info)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    if dist:
        dist.barrier()

    total_ms = sum(step_ms)
    pushed = sum(i["pushed_edges"] for i in infos)
    launches = sum(i["kernel_launches"] for i in infos)
    total_ms, pushed, launches = aggregate(dist, total_ms, pushed, launches, device=dev)
    value = pushed / (total_ms * 1e-3) / 1e9

    # end to end through the public API with host buffers: B from pinned host memory, X back
    Bh = torch.full((n,), (1.0 - D) / n, dtype=torch.float64).pin_memory()
    Xh = torch.empty(n, dtype=torch.float64).pin_memory()
    e2e_ms, e2e_pushed = [], 0
    for _ in range(max(1, min(args.steps, 20))):
        flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        info = di.di_solve_ex(g, Bh, D, TOL, schedule=di.DI_SOP, fluid=di.DI_FLUID_F32, max_sweeps=MAX_SWEEPS,
                              X_out=Xh)[1]
        b.record(stream)
        b.synchronize()
        e2e_ms.append(a.elapsed_time(b))
        e2e_pushed += info["pushed_edges"]
    e2e_value = e2e_pushed / (sum(e2e_ms) * 1e-3) / 1e9 * ws

    # per-kernel timing: one solve with CUDA events around every kernel launch
    prof = step(profile=1)
    push_ms = prof["push_ms"] / max(prof["push_launches"], 1)
    # algorithmic bytes of the push: 4 B link index + 8 B read-modify-write of F_j per pushed
    # link; per frontier entry 4 B id + 4 B share + 8 B row start (the row end is the next node's
    # row start, counted with that node)
    push_bytes = (12.0 * prof["pushed_edges"] + 16.0 * prof["frontier_entries"]) / max(prof["push_launches"], 1)
    peak, peak_kind = peaks()
    achieved = push_bytes / (push_ms * 1e-3) / 1e9
    kernel_total = prof["select_ms"] + prof["push_ms"] + prof["reduce_ms"] + prof["refine_ms"]
    traffic, traffic_src = push_traffic()
    # the whole solve's algorithmic bytes, the same solve: per sweep the select reads every
    # node's F and degree word (8 B); per visit it zeroes F_i (4 B), adds to H_i (16 B) and writes
    # a frontier entry (8 B); the push as above; each exact residual pass reads a link index and
    # gathers H_j (12 B per link) and per row its row start, B_i, H_i and writes F_i (28 B, 32 B
    # with d/out); setup and output: B read, F and H initialised, X written (28 B per node)
    solve_bytes = (8.0 * n * prof["sweeps"] + 28.0 * prof["visited_nodes"]
                   + 12.0 * prof["pushed_edges"] + 16.0 * prof["frontier_entries"]
                   + prof["refine_rounds"] * (12.0 * st["L"] + 32.0 * n) + 28.0 * n)

    legs = {}
    want = set(["solvers", "small_graphs", "transposed", "e_dominated", "ppr_batch", "serving"] if args.legs == "all"
               else args.legs.split(","))
    if args.no_legs:
        want = set()
    def median_of(fn, reps=5):
        """Median device time of `reps` runs of fn (after one warm-up), L2 flushed before each."""
        fn()
        times, inf = [], None
        for _ in range(reps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            inf = fn()
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        return statistics.median(times), inf

    if "solvers" in want:
        B95 = torch.full((n,), (1.0 - 0.95) / n, dtype=torch.float64, device=dev)
        for name, kw in (("di_cyc", dict(schedule=di.DI_CYC)), ("di_sop_d095", dict(d=0.95, Bx=B95)),
                         ("di_sop_e_prediffused", dict(e_prediffuse=1))):
            ms, inf = median_of(lambda: step(**kw))
            legs[name] = {"ms_to_residual": ms, "GTEPS": inf["pushed_edges"] / (ms * 1e-3) / 1e9,
                          "sweeps": inf["sweeps"], "pushed_per_L": inf["pushed_edges"] / st["L"],
                          "residual_l1": inf["residual_l1"], "median_of": 5}
        ms, pinf = median_of(lambda: di.di_power_iter(g, B, D, TOL, max_iters=MAX_SWEEPS, X_out=X)[1])
        legs["pi"] = {"ms_to_residual": ms, "GTEPS": pinf["pushed_edges"] / (ms * 1e-3) / 1e9,
                      "iterations": pinf["sweeps"], "refine_rounds": pinf["refine_rounds"],
                      "residual_l1": pinf["residual_l1"], "median_of": 5,
                      "form": "FP32 increments, FP64 X, exact FP64-certified residual"}
        ms, qinf = median_of(lambda: di.di_power_iter_push(g, B, D, TOL, max_iters=MAX_SWEEPS, X_out=X)[1])
        legs["pi_push"] = {"ms_to_residual": ms, "GTEPS": qinf["pushed_edges"] / (ms * 1e-3) / 1e9,
                           "iterations": qinf["sweeps"], "residual_l1": qinf["residual_l1"], "median_of": 5}
        # the pull's roofline: per pass 4 B index + 4 B FP32 increment gathered per link; per row
        # 8 B row start, 8 B FP64 X read and 8 B written, 4 B increment written, 4 B d/out
        pprof = di.di_power_iter_ex(g, B, D, TOL, max_iters=MAX_SWEEPS, profile=1, X_out=X)[1]
        if pprof["push_launches"]:
            pull_ms = pprof["push_ms"] / pprof["push_launches"]
            pull_bytes = 8.0 * st["L"] + 32.0 * n
            peak, peak_kind = peaks()
            legs["pi"]["roofline"] = {"kernel": "k_pull<PULL_INC>", "bound": "hbm", "bytes_per_launch": pull_bytes,
                                      "ms_per_launch": pull_ms, "achieved": pull_bytes / (pull_ms * 1e-3) / 1e9,
                                      "peak": peak, "unit": "GB/s",
                                      "frac": pull_bytes / (pull_ms * 1e-3) / 1e9 / peak, "peak_kind": peak_kind}
    if "small_graphs" in want:
        legs["pa_n10k"] = small_graph_leg(di, workloads, torch, "pa_n10k")
        legs["web_n1m"] = small_graph_leg(di, workloads, torch, "web_n1m")
    if "transposed" in want:
        legs["transposed"] = transposed_leg(di, workloads, torch, flush)
    if "e_dominated" in want:
        legs["e_dominated"] = transposed_leg(di, workloads, torch, flush, name="web_n10m_e")
    if "ppr_batch" in want:
        legs["ppr_batch"] = ppr_batch_leg(di, workloads, torch)
    if "serving" in want:
        legs["serving"] = serving_leg(di, workloads, torch)
    legs["di_sop"] = {"ms_to_residual": statistics.median(step_ms), "sweeps": infos[-1]["sweeps"],
                      "pushed_per_L": infos[-1]["pushed_edges"] / st["L"], "refine_rounds": infos[-1]["refine_rounds"],
                      "residual_l1": infos[-1]["residual_l1"]}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cyc = 6
        cp, csec, ccyc, _ = oracle_sample(n, src, dst, D, cyc)
        cpu = {"value": cp / csec / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
               "sample": f"first {ccyc} sequential DI-SOP cycles of the oracle on the same 10M-node graph "
                         f"({cp} pushed links in {csec:.1f} s; oracle build excluded)",
               "host": host_cpu()}

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    line = {
        "metric": "GTEPS (DI-SOP, N=10M, tol 1e-8)",
        "value": value,
        "unit": "GTEPS",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: N={n}, L={st['L']}, d={D}, tol={TOL}, B=(1-d)/N",
                   "fluid": "f32", "history": "f64", "residual": "f64 exact (refined)",
                   "parallelism": f"replicas x{ws}", "l2": "flushed between steps (512 MB write)",
                   "graph_build_ms": build_ms,
                   "push_tune": {"row": tuning["push_row"], "heavy_cut": tuning["heavy_cut"],
                                 "heavy_chunk": tuning["heavy_chunk"], "tuning_s": tune_s}},
        "e2e": {"value": e2e_value, "unit": "GTEPS", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
                "ms_per_step": statistics.mean(e2e_ms)},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": traffic, "traffic_source": traffic_src, "kernel": "k_push_win", "peak_kind": peak_kind,
                     "bytes_per_launch": push_bytes, "ms_per_launch": push_ms,
                     "kernel_share": prof["push_ms"] / kernel_total if kernel_total else None,
                     "profiled_solve_kernel_ms": {k: prof[k + "_ms"] for k in ("select", "push", "reduce", "refine")}},
        "roofline_solve": {"bound": "hbm", "bytes_per_solve": solve_bytes,
                           "ms_per_solve": statistics.median(step_ms),
                           "achieved": solve_bytes / (statistics.median(step_ms) * 1e-3) / 1e9, "peak": peak,
                           "unit": "GB/s",
                           "frac": solve_bytes / (statistics.median(step_ms) * 1e-3) / 1e9 / peak,
                           "peak_kind": peak_kind, "sweeps": prof["sweeps"],
                           "refine_rounds": prof["refine_rounds"]},
        "cpu_baseline": cpu,
        "clocks": clocks,
        "legs": legs,
        "graph": {k: st[k] for k in ("n_nodes", "L", "D", "E", "O", "max_in", "max_out", "e_levels")},
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
