// Batched D-iteration: k independent right-hand sides on one graph, solved T at a time in the
// tiles of di_tile.cuh. With FP32 fluid, retirement is followed by the exact FP64 residual of
// every column; a column whose exact residual is above its tolerance re-enters the sweep loop
// from F*_c, aiming at half its tolerance.
//
// The tile width T is a template parameter (4, 8, 16, 32). The autotuner times a short probe of
// each width on the graph itself and keeps the fastest (cached per graph).
#include <algorithm>
#include <cmath>
#include <cstring>

#include "di_tile.cuh"

namespace di {

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
BatchWorkspace::~BatchWorkspace() {
    for (auto &e : exec)
        if (e) cudaGraphExecDestroy(e);
    if (capture_stream) cudaStreamDestroy(capture_stream);
    if (ctl_host) cudaFreeHost(ctl_host);
}

void destroy_batch_workspace(BatchWorkspace *w) { delete w; }

// Solves one tile of up to T columns [c0, c0 + ncols): right-hand sides already in w.Bn.
// Accumulates the report into `acc`; writes per-column residuals into res_host[c0 + c].
template <int T>
static void solve_tile(di_graph *g, int c0, int ncols, double d, const double *tol_host, int schedule, int max_sweeps,
                       bool refine, double *X_out, bool X_dev, double *res_host, di_solve_info *acc, cudaStream_t s) {
    BatchWorkspace &w = *g->bws;
    const BLaunch l = blaunch<T>(g);
    BatchCtl *ctl = w.ctl.as<BatchCtl>();
    BatchCtl &hc = *(BatchCtl *)w.ctl_host;
    memset(&hc, 0, sizeof(BatchCtl));
    hc.d = d;
    hc.L = (double)g->L;
    hc.ncols = ncols;
    hc.schedule = schedule;
    hc.max_sweeps = max_sweeps;
    hc.last_selected = -1;
    hc.split_mask = refine ? (ncols == 32 ? 0xffffffffu : ((1u << ncols) - 1u)) : 0u;
    for (int c = 0; c < ncols; c++) {
        hc.tol[c] = tol_host[c0 + c];
        hc.active[c] = 1;
        hc.retire_sweep[c] = -1;
    }
    DI_CHECK_CUDA(cudaMemcpyAsync(ctl, &hc, sizeof(BatchCtl), cudaMemcpyHostToDevice, s));
    kb_init<T><<<l.ew, 256, 0, s>>>(w.Bn.as<double>(), g->n, w.F.as<float>(), w.H.as<double>(), ctl);
    int64_t launches = 1;
    cudaGraphExec_t ex = batch_graph<T>(g, w, l);
    int rounds = 0;
    for (;;) {
        kb_reduce<T><<<l.red, 256, 0, s>>>(w.F.as<float>(), g->n, w.partials.as<double>(), ctl,
                                           cudaGraphConditionalHandle(0), 0);
        DI_CHECK_CUDA(cudaGetLastError());
        if (w.host_loop) {
            // host-driven sweeps (one sync per sweep), for profiling the kernels one by one
            for (;;) {
                read_bctl(w, s);
                if (hc.done) break;
                batch_body<T>(g, w, l, s, cudaGraphConditionalHandle(0), 0, w.clock);
                launches += 3;
            }
        } else {
            DI_CHECK_CUDA(cudaGraphLaunch(ex, s));
        }
        launches += 1;
        if (!refine) {
            read_bctl(w, s);
            break;
        }
        batch_resid<T>(g, w, l, d, s);
        launches += g->n_heavy_in_chunks > 0 ? 2 : 1;
        read_bctl(w, s);
        rounds++;
        // reactivate the columns whose exact residual is above their tolerance
        bool again = false;
        for (int c = 0; c < ncols; c++) {
            const bool a = hc.r[c] > tol_host[c0 + c];
            hc.active[c] = a ? 1 : 0;
            again = again || a;
        }
        if (!again || hc.status || hc.sweeps >= max_sweeps || rounds >= 4) break;
        // continuation sweeps aim just under the tolerance after a column's halfway refinement
        // (its fluid's rounding since then is far below tol), else at half of it
        for (int c = 0; c < ncols; c++) {
            const bool after_split = rounds == 1 && hc.tol[c] > tol_host[c0 + c];
            hc.tol[c] = (after_split ? kAimAfterSplit : 0.5) * tol_host[c0 + c];
        }
        DI_CHECK_CUDA(cudaMemcpyAsync(ctl->tol, hc.tol, sizeof(hc.tol), cudaMemcpyHostToDevice, s));
        DI_CHECK_CUDA(cudaMemcpyAsync(ctl->active, hc.active, sizeof(hc.active), cudaMemcpyHostToDevice, s));
        int zero = 0;
        DI_CHECK_CUDA(cudaMemcpyAsync(&ctl->done, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
    }
    // X columns out
    if (X_dev) {
        kb_extract<T><<<l.ew, 256, 0, s>>>(w.H.as<double>(), g->n, ncols, X_out + (int64_t)c0 * g->n);
    } else {
        kb_extract<T><<<l.ew, 256, 0, s>>>(w.H.as<double>(), g->n, ncols, w.stage.as<double>());
        from_device(X_out + (int64_t)c0 * g->n, w.stage.p, sizeof(double) * (size_t)g->n * ncols, s);
    }
    launches += 1;
    DI_CHECK_CUDA(cudaGetLastError());
    DI_CHECK_CUDA(cudaStreamSynchronize(s));
    DI_REQUIRE(hc.status != 1, DI_ERR_INVALID_ARG, "B has a negative or non-finite entry");
    for (int c = 0; c < ncols; c++) res_host[c0 + c] = hc.r[c];
    acc->sweeps += hc.sweeps;
    acc->refine_rounds += rounds;
    acc->pushed_edges += (int64_t)hc.pushed;
    acc->visited_nodes += (int64_t)hc.visited;
    acc->frontier_entries += (int64_t)hc.front_total;
    acc->column_links += (int64_t)hc.col_pushed;
    acc->kernel_launches += launches + 3 * (int64_t)hc.body_runs;
    for (int c = 0; c < ncols; c++) acc->dangling_mass_e += hc.e[c];
}

// ------------------------------------------------------------------------------------------
// autotuner: time a short probe of every tile width on this graph and keep the fastest
// ------------------------------------------------------------------------------------------
template <int T>
static double probe(di_graph *g, double d, cudaStream_t s, int sweeps = 6) {
    BatchWorkspace &w = *g->bws;
    const BLaunch l = blaunch<T>(g);
    // probe right-hand sides: uniform (1-d)/N in every column, a few sweeps
    std::vector<double> tol(T, 1e-300);
    kb_fill<T><<<l.ew, 256, 0, s>>>(w.Bn.as<double>(), (int64_t)g->n * T, (1.0 - d) / g->n);
    cudaEvent_t a, b;
    DI_CHECK_CUDA(cudaEventCreate(&a));
    DI_CHECK_CUDA(cudaEventCreate(&b));
    di_solve_info acc;
    memset(&acc, 0, sizeof(acc));
    std::vector<double> res(T);
    DI_CHECK_CUDA(cudaEventRecord(a, s));
    solve_tile<T>(g, 0, T, d, tol.data(), DI_SOP, sweeps, false, w.stage.as<double>(), true, res.data(), &acc, s);
    DI_CHECK_CUDA(cudaEventRecord(b, s));
    DI_CHECK_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    // column-link updates per second
    return (double)acc.pushed_edges * T / (ms * 1e-3);
}

// The batched push split (PushTune heavy cut-off and chunk length, i.e. how many warps share a
// high-degree row) for tiles of T columns: coordinate descent over 24-sweep probes, long enough
// for the sweeps to select high-degree nodes (the first sweeps from a uniform B select only nodes
// with fewer than L / N links).
static void tune_batch_split(di_graph *g, double d, cudaStream_t s, int T) {
    auto rate = [&](const PushTune &t) {
        g->tune_batch = t;
        double best = 0.0;
        for (int rep = 0; rep < 2; rep++) {
            const double v = T == 4 ? probe<4>(g, d, s, 24) : T == 8 ? probe<8>(g, d, s, 24)
                           : T == 16 ? probe<16>(g, d, s, 24) : probe<32>(g, d, s, 24);
            best = v > best ? v : best;
        }
        return best;
    };
    PushTune best = g->tune_batch;
    double brate = rate(best);
    for (int heavy : {1024, 2048, 4096, 8192}) {
        PushTune t = best;
        t.heavy = heavy;
        if (t == best || t.chunk > t.heavy) continue;
        const double v = rate(t);
        if (v > brate) { brate = v; best = t; }
    }
    for (int chunk : {256, 512, 1024, 2048}) {
        PushTune t = best;
        t.chunk = chunk;
        if (t == best || t.chunk > t.heavy) continue;
        const double v = rate(t);
        if (v > brate) { brate = v; best = t; }
    }
    g->tune_batch = best;
    g->bws->split_rate = brate;
}

static int autotune(di_graph *g, double d, cudaStream_t s) {
    if (g->bws && g->bws->tuned_T) return g->bws->tuned_T;
    if (!g->bws) g->bws = new BatchWorkspace();
    // the widest tile the workspace holds (an attached one may hold fewer than 32 columns)
    int widest = 32;
    if (g->bws->ext)
        while (widest > 4 && batch_bytes(g, widest) > g->bws->ext_bytes) widest /= 2;
    ensure_batch(g, *g->bws, widest);
    double best = -1.0;
    int bestT = 4;
    const int cands[4] = {4, 8, 16, 32};
    for (int T : cands) {
        if (T > widest) break;
        double v = T == 4 ? probe<4>(g, d, s) : T == 8 ? probe<8>(g, d, s) : T == 16 ? probe<16>(g, d, s) : probe<32>(g, d, s);
        g->bws->probe_rate[tile_index(T)] = v;
        if (v > best) {
            best = v;
            bestT = T;
        }
    }
    g->bws->tuned_T = bestT;
    tune_batch_split(g, d, s, bestT);
    return bestT;
}

// The k right-hand sides run through one tile of T column slots. Each step admits the next
// requests into the free slots (in cohorts of at least half the tile), runs at most kBatchStepSweeps sweeps from the CUDA graph (the
// WHILE loop also ends once every occupied slot has retired), then retires the columns that
// reached their tolerance: with refinement, after an exact FP64 residual of just those columns
// (a column still above its tolerance keeps sweeping from that residual, first from its
// halfway point, then aiming under its tolerance). A retired column's history goes out and the
// column is zeroed for the next request, so requests of uneven difficulty share sweeps instead
// of one slow column holding a whole tile.
constexpr int kBatchStepSweeps = 8;

template <int T>
static void batch_refill(di_graph *g, int k, const double *B, bool B_dev, const int64_t *off_h, const int32_t *seeds,
                         bool seeds_dev, double d, const double *tol_host, int schedule, int max_sweeps, bool refine,
                         double *X_out, bool X_dev, double *res_host, di_solve_info *acc, cudaStream_t s) {
    if (!g->bws) g->bws = new BatchWorkspace();
    ensure_batch(g, *g->bws, T);
    BatchWorkspace &w = *g->bws;
    const BLaunch l = blaunch<T>(g);
    const int32_t n = g->n;
    BatchCtl *ctl = w.ctl.as<BatchCtl>();
    BatchCtl &hc = *(BatchCtl *)w.ctl_host;
    memset(&hc, 0, sizeof(BatchCtl));
    hc.d = d;
    hc.L = (double)g->L;
    hc.ncols = T;
    hc.schedule = schedule;
    hc.last_selected = -1;
    for (int c = 0; c < T; c++) hc.retire_sweep[c] = -1;
    // a clean control block on the device too (an earlier call may have left a status there)
    DI_CHECK_CUDA(cudaMemcpyAsync(ctl, &hc, sizeof(BatchCtl), cudaMemcpyHostToDevice, s));
    DI_CHECK_CUDA(cudaMemsetAsync(w.F.p, 0, sizeof(float) * (size_t)n * T, s));
    DI_CHECK_CUDA(cudaMemsetAsync(w.H.p, 0, sizeof(double) * (size_t)n * T, s));
    DI_CHECK_CUDA(cudaMemsetAsync(w.Bn.p, 0, sizeof(double) * (size_t)n * T, s));
    cudaGraphExec_t ex = batch_graph<T>(g, w, l);
    struct Slot {
        int req = -1;        // request in the slot, -1 when free
        int admit = 0;       // tile sweep count at admission
        int rounds = 0;      // exact residuals taken
        bool halfway = false;
    };
    std::vector<Slot> slot(T);
    int next = 0, finished = 0;
    int64_t launches = 0, rounds_total = 0;
    double *stage = w.stage.as<double>();
    while (finished < k) {
        // 1. admission into the free slots (their columns are zero), in cohorts: only once half
        //    the slots are free (or nothing runs), so the tile mixes at most two stages of
        //    columns; columns far apart in their solves widen every sweep's set of visited nodes
        int free_slots = 0;
        for (int c = 0; c < T; c++) free_slots += slot[c].req < 0 ? 1 : 0;
        const bool admit_now = free_slots == T || 2 * free_slots >= T;
        bool admitted = false;
        for (int c = 0; c < T && next < k && admit_now; c++) {
            if (slot[c].req >= 0) continue;
            const int r = next++;
            if (off_h) {
                const int64_t e0 = off_h[r], e1 = off_h[r + 1];
                const double share = (1.0 - d) / (double)(e1 - e0);
                const int64_t piece = seeds_dev ? e1 - e0 : (int64_t)(w.stage.bytes / sizeof(int32_t)) / T;
                for (int64_t e = e0; e < e1; e += piece) {
                    const int64_t cnt = std::min(piece, e1 - e);
                    const int32_t *src = seeds + e;
                    if (!seeds_dev) {   // staged in column c's share of the staging buffer
                        int32_t *st = reinterpret_cast<int32_t *>(stage + (size_t)c * n);
                        to_device(st, seeds + e, sizeof(int32_t) * (size_t)cnt, s);
                        src = st;
                    }
                    kb_seed_col<T><<<(int)std::min<int64_t>((cnt + 255) / 256, (int64_t)g->dev.sms * 4), 256, 0, s>>>(
                        src, cnt, c, share, n, w.F.as<float>(), w.Bn.as<double>(), ctl);
                    launches++;
                }
            } else {
                const double *col = B + (int64_t)r * n;
                if (!B_dev) {
                    to_device(stage + (size_t)c * n, col, sizeof(double) * (size_t)n, s);
                    col = stage + (size_t)c * n;
                }
                kb_load_col<T><<<l.ew, 256, 0, s>>>(col, n, c, w.F.as<float>(), w.Bn.as<double>(), ctl);
                launches++;
            }
            slot[c].req = r;
            slot[c].admit = hc.sweeps;
            slot[c].rounds = 0;
            slot[c].halfway = refine;
            hc.active[c] = 1;
            hc.tol[c] = tol_host[r];
            hc.r[c] = 0.0;
            hc.e[c] = 0.0;
            if (refine) hc.split_mask |= 1u << c;   // its first stop is halfway to its tolerance
            admitted = true;
        }
        if (admitted) {
            // status of the admission kernels (a bad right-hand side or seed)
            int st = 0;
            DI_CHECK_CUDA(cudaMemcpyAsync(&st, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost, s));
            DI_CHECK_CUDA(cudaStreamSynchronize(s));
            DI_REQUIRE(st != 1, DI_ERR_INVALID_ARG, "B has a negative or non-finite entry");
            DI_REQUIRE(st != 2, DI_ERR_OUT_OF_RANGE_ID, "a seed is outside [0, %d)", n);
        }
        // 2. a bounded number of sweeps
        hc.max_sweeps = hc.sweeps + kBatchStepSweeps;
        hc.done = 0;
        hc.ticket = 0;
        hc.status = 0;
        DI_CHECK_CUDA(cudaMemcpyAsync(ctl, &hc, sizeof(BatchCtl), cudaMemcpyHostToDevice, s));
        kb_reduce<T><<<l.red, 256, 0, s>>>(w.F.as<float>(), n, w.partials.as<double>(), ctl,
                                           cudaGraphConditionalHandle(0), 0);
        launches++;
        if (w.host_loop) {
            for (;;) {   // host-driven sweeps (one sync per sweep), for profiling kernels one by one
                read_bctl(w, s);
                if (hc.done) break;
                batch_body<T>(g, w, l, s, cudaGraphConditionalHandle(0), 0, w.clock);
                launches += 3;
            }
        } else {
            DI_CHECK_CUDA(cudaGraphLaunch(ex, s));
            launches++;
            read_bctl(w, s);
        }
        // 3. retirement: columns whose stop test fired, or whose sweep budget is spent
        uint32_t cand = 0;
        for (int c = 0; c < T; c++) {
            if (slot[c].req < 0) continue;
            const bool capped = hc.sweeps - slot[c].admit >= max_sweeps;
            if (!hc.active[c] || capped) cand |= 1u << c;
        }
        if (!cand) continue;
        if (refine) {
            batch_resid<T>(g, w, l, d, s, cand);
            launches += g->n_heavy_in_chunks > 0 ? 3 : 2;
            read_bctl(w, s);
        }
        for (int c = 0; c < T; c++) {
            if (!(cand >> c & 1u)) continue;
            Slot &sl = slot[c];
            const int r = sl.req;
            const bool capped = hc.sweeps - sl.admit >= max_sweeps;
            if (refine) {
                sl.rounds++;
                rounds_total++;
                if (hc.r[c] > tol_host[r] && !capped && sl.rounds < 4) {
                    // keeps sweeping from the exact residual: after the halfway point just under
                    // its tolerance (the fluid's rounding since then is far below it), else at half
                    hc.active[c] = 1;
                    hc.tol[c] = (sl.halfway ? kAimAfterSplit : 0.5) * tol_host[r];
                    sl.halfway = false;
                    continue;
                }
            }
            // 4. the column's history goes out and the column is zeroed for the next request
            double *out = X_dev ? X_out + (int64_t)r * n : stage + (size_t)c * n;
            kb_col_retire<T><<<l.ew, 256, 0, s>>>(w.F.as<float>(), w.H.as<double>(), w.Bn.as<double>(), n, c, out);
            launches++;
            if (!X_dev) from_device(X_out + (int64_t)r * n, out, sizeof(double) * (size_t)n, s);
            res_host[r] = hc.r[c];
            acc->dangling_mass_e += hc.e[c];
            hc.active[c] = 0;
            sl.req = -1;
            finished++;
        }
        DI_CHECK_CUDA(cudaGetLastError());
    }
    DI_CHECK_CUDA(cudaStreamSynchronize(s));
    acc->sweeps += hc.sweeps;
    acc->refine_rounds += (int32_t)rounds_total;
    acc->pushed_edges += (int64_t)hc.pushed;
    acc->visited_nodes += (int64_t)hc.visited;
    acc->frontier_entries += (int64_t)hc.front_total;
    acc->column_links += (int64_t)hc.col_pushed;
    acc->kernel_launches += launches + 3 * (int64_t)hc.body_runs;
}

static di_status batch_entry(di_graph *g, int32_t k, const double *B, const int64_t *seed_off, const int32_t *seeds,
                             double d, const double *tol, const di_solve_opts *opts, double *X_out, double *res_out,
                             di_solve_info *info, cudaStream_t s) {
    return guarded([&] {
        DI_REQUIRE(g != nullptr, DI_ERR_INVALID_ARG, "graph is NULL");
        DI_REQUIRE(k >= 1, DI_ERR_INVALID_ARG, "k must be >= 1 (got %d)", k);
        DI_REQUIRE(tol && X_out && (B || (seed_off && seeds)), DI_ERR_INVALID_ARG, "NULL argument");
        DI_REQUIRE(d >= 0.0 && d < 1.0, DI_ERR_INVALID_ARG, "d must be in [0, 1) (got %g)", d);
        di_solve_opts o;
        memset(&o, 0, sizeof(o));
        if (opts) o = *opts;
        DI_REQUIRE(o.schedule == DI_CYC || o.schedule == DI_SOP, DI_ERR_INVALID_ARG, "unknown schedule %d", o.schedule);
        DI_REQUIRE(o.fluid == DI_FLUID_F32, DI_ERR_INVALID_ARG, "batched solves keep the fluid in FP32");
        DI_REQUIRE(o.rhs_tile == 0 || o.rhs_tile == 4 || o.rhs_tile == 8 || o.rhs_tile == 16 || o.rhs_tile == 32,
                   DI_ERR_INVALID_ARG, "rhs_tile must be 0 (autotune), 4, 8, 16 or 32 (got %d)", o.rhs_tile);
        const int max_sweeps = o.max_sweeps <= 0 ? 100000 : (o.max_sweeps > 1000000 ? 1000000 : o.max_sweeps);
        const bool refine = o.refine >= 0;   // FP32 fluid: on unless switched off
        std::unique_lock<std::mutex> lk(g->mu, std::try_to_lock);
        DI_REQUIRE(lk.owns_lock(), DI_ERR_BUSY, "graph workspace is in use by another call");
        DeviceGuard dg(g->dev.device);
        // tolerances and seed offsets on the host
        std::vector<double> tol_h((size_t)k);
        from_device(tol_h.data(), tol, sizeof(double) * (size_t)k, s);
        std::vector<int64_t> off_h;
        if (!B) {
            off_h.resize((size_t)k + 1);
            from_device(off_h.data(), seed_off, sizeof(int64_t) * ((size_t)k + 1), s);
            DI_CHECK_CUDA(cudaStreamSynchronize(s));
            DI_REQUIRE(off_h[0] == 0, DI_ERR_INVALID_ARG, "seed_offsets[0] must be 0");
            for (int c = 0; c < k; c++)
                DI_REQUIRE(off_h[c + 1] > off_h[c], DI_ERR_INVALID_ARG, "seed set %d is empty or offsets decrease", c);
        }
        DI_CHECK_CUDA(cudaStreamSynchronize(s));
        for (int c = 0; c < k; c++)
            DI_REQUIRE(tol_h[c] > 0.0 && std::isfinite(tol_h[c]), DI_ERR_INVALID_ARG, "tol[%d] must be positive", c);
        const bool B_dev = B && is_device_ptr(B);
        const bool X_dev = is_device_ptr(X_out);
        const bool seeds_dev = seeds && is_device_ptr(seeds);
        int T = o.rhs_tile ? o.rhs_tile : autotune(g, d, s);
        if (!g->bws) g->bws = new BatchWorkspace();
        g->bws->host_loop = o.host_loop != 0 || o.profile != 0;
        // profile: host-driven sweeps with each select, push and reduce timed alone
        KernelClock kc(o.profile != 0, s);
        g->bws->clock = o.profile ? &kc : nullptr;
        struct ClockReset {
            BatchWorkspace *w;
            ~ClockReset() { w->clock = nullptr; }
        } clock_reset{g->bws};
        std::vector<double> res((size_t)k, 0.0);
        di_solve_info acc;
        memset(&acc, 0, sizeof(acc));
        cudaEvent_t e0, e1;
        DI_CHECK_CUDA(cudaEventCreate(&e0));
        DI_CHECK_CUDA(cudaEventCreate(&e1));
        DI_CHECK_CUDA(cudaEventRecord(e0, s));
        try {
            switch (T) {
                case 4: batch_refill<4>(g, k, B, B_dev, B ? nullptr : off_h.data(), seeds, seeds_dev, d, tol_h.data(), o.schedule, max_sweeps, refine, X_out, X_dev, res.data(), &acc, s); break;
                case 8: batch_refill<8>(g, k, B, B_dev, B ? nullptr : off_h.data(), seeds, seeds_dev, d, tol_h.data(), o.schedule, max_sweeps, refine, X_out, X_dev, res.data(), &acc, s); break;
                case 16: batch_refill<16>(g, k, B, B_dev, B ? nullptr : off_h.data(), seeds, seeds_dev, d, tol_h.data(), o.schedule, max_sweeps, refine, X_out, X_dev, res.data(), &acc, s); break;
                default: batch_refill<32>(g, k, B, B_dev, B ? nullptr : off_h.data(), seeds, seeds_dev, d, tol_h.data(), o.schedule, max_sweeps, refine, X_out, X_dev, res.data(), &acc, s); break;
            }
        } catch (...) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            throw;
        }
        DI_CHECK_CUDA(cudaEventRecord(e1, s));
        DI_CHECK_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (res_out) from_device(res_out, res.data(), sizeof(double) * (size_t)k, s);
        DI_CHECK_CUDA(cudaStreamSynchronize(s));
        double worst = 0.0;
        int bad = -1;
        for (int c = 0; c < k; c++)
            if (res[c] > tol_h[c] && (bad < 0 || res[c] / tol_h[c] > worst)) {
                worst = res[c] / tol_h[c];
                bad = c;
            }
        acc.ms = ms;
        acc.residual_l1 = 0.0;
        for (int c = 0; c < k; c++) acc.residual_l1 = res[c] > acc.residual_l1 ? res[c] : acc.residual_l1;
        acc.paper_error = acc.residual_l1 / (1.0 - d);
        acc.rhs_tile = T;
        if (o.profile) {
            acc.select_ms = kc.ms[KC_SELECT];
            acc.push_ms = kc.ms[KC_PUSH];
            acc.reduce_ms = kc.ms[KC_REDUCE];
            acc.select_launches = kc.count[KC_SELECT];
            acc.push_launches = kc.count[KC_PUSH];
            acc.reduce_launches = kc.count[KC_REDUCE];
        }
        if (info) *info = acc;
        DI_REQUIRE(bad < 0, DI_ERR_NOT_CONVERGED, "column %d not converged: ||F||_1 = %g > tol = %g", bad, res[bad],
                   tol_h[bad]);
    });
}

}  // namespace di

extern "C" {

di_status di_workspace_size(const di_graph *g, int32_t kind, int32_t param, int64_t *bytes) {
    using namespace di;
    return guarded([&] {
        DI_REQUIRE(g && bytes, DI_ERR_INVALID_ARG, "graph or bytes is NULL");
        di_graph *gm = const_cast<di_graph *>(g);   // sizing reads the graph only
        if (kind == DI_WS_SOLVE) {
            DI_REQUIRE(param == DI_FLUID_F32 || param == DI_FLUID_F64, DI_ERR_INVALID_ARG, "unknown fluid %d", param);
            *bytes = (int64_t)solve_workspace_bytes(gm, param);
        } else if (kind == DI_WS_BATCH) {
            const int T = param == 0 ? 32 : param;
            DI_REQUIRE(T == 4 || T == 8 || T == 16 || T == 32, DI_ERR_INVALID_ARG,
                       "tile width must be 0 (32), 4, 8, 16 or 32 (got %d)", param);
            *bytes = (int64_t)batch_bytes(gm, T);
        } else {
            DI_REQUIRE(false, DI_ERR_INVALID_ARG, "unknown workspace kind %d", kind);
        }
    });
}

di_status di_graph_set_workspace(di_graph *g, int32_t kind, void *workspace, int64_t bytes) {
    using namespace di;
    return guarded([&] {
        DI_REQUIRE(g != nullptr, DI_ERR_INVALID_ARG, "graph is NULL");
        DI_REQUIRE(kind == DI_WS_SOLVE || kind == DI_WS_BATCH, DI_ERR_INVALID_ARG, "unknown workspace kind %d", kind);
        std::unique_lock<std::mutex> lk(g->mu, std::try_to_lock);
        DI_REQUIRE(lk.owns_lock(), DI_ERR_BUSY, "graph workspace is in use by another call");
        DeviceGuard dg(g->dev.device);
        if (workspace) {
            DI_REQUIRE(bytes > 0, DI_ERR_INVALID_ARG, "workspace bytes must be positive (got %lld)", (long long)bytes);
            DI_REQUIRE(((uintptr_t)workspace & 255u) == 0, DI_ERR_INVALID_ARG, "the workspace must be 256-byte aligned");
            cudaPointerAttributes a;
            const bool ok = cudaPointerGetAttributes(&a, workspace) == cudaSuccess &&
                            ((a.type == cudaMemoryTypeDevice && a.device == g->dev.device) ||
                             a.type == cudaMemoryTypeManaged);
            cudaGetLastError();
            DI_REQUIRE(ok, DI_ERR_INVALID_ARG, "the workspace must be device memory of the graph's GPU (%d)",
                       g->dev.device);
        }
        DI_CHECK_CUDA(cudaDeviceSynchronize());   // no earlier call's work still uses the old buffers
        if (kind == DI_WS_SOLVE) {
            solve_workspace_attach(g, workspace, workspace ? (size_t)bytes : 0);
        } else {
            if (!g->bws) g->bws = new BatchWorkspace();
            BatchWorkspace &w = *g->bws;
            for (auto &e : w.exec)
                if (e) cudaGraphExecDestroy(e);
            for (auto &e : w.exec) e = nullptr;
            batch_layout(g, w, 32, [&](DevBuf &b, size_t) { b.release(); });
            w.ext = workspace;
            w.ext_bytes = workspace ? (size_t)bytes : 0;
            w.T_alloc = 0;
            w.tuned_T = 0;   // the widest tile may differ now
            if (!w.ctl_host) DI_CHECK_CUDA(cudaMallocHost(&w.ctl_host, sizeof(BatchCtl)));
        }
    });
}

int64_t di_device_bytes_held(void) { return (int64_t)di::g_device_bytes.load(); }

di_status di_autotune(di_graph *g, double d, int32_t what, di_tuning *out, void *stream) {
    using namespace di;
    return guarded([&] {
        DI_REQUIRE(g != nullptr, DI_ERR_INVALID_ARG, "graph is NULL");
        DI_REQUIRE(d >= 0.0 && d < 1.0, DI_ERR_INVALID_ARG, "d must be in [0, 1) (got %g)", d);
        DI_REQUIRE(what >= 0 && what <= 7, DI_ERR_INVALID_ARG, "what must be 0..7 (got %d)", what);
        if (what & 4) {
            DI_REQUIRE(out != nullptr, DI_ERR_INVALID_ARG, "setting a split needs the values in out");
            const bool row_ok = out->push_row >= 1 && out->push_row <= 1 << 20;
            const bool heavy_ok = out->heavy_cut >= kPushHeavyMin && out->heavy_cut <= 1 << 30;
            const bool chunk_ok = out->heavy_chunk >= kHeavyChunkMin && out->heavy_chunk <= out->heavy_cut;
            DI_REQUIRE(row_ok && heavy_ok && chunk_ok, DI_ERR_INVALID_ARG,
                       "push split out of range (row %d, heavy cut %d >= %d, chunk %d in [%d, heavy cut])",
                       out->push_row, out->heavy_cut, kPushHeavyMin, out->heavy_chunk, kHeavyChunkMin);
        }
        std::unique_lock<std::mutex> lk(g->mu, std::try_to_lock);
        DI_REQUIRE(lk.owns_lock(), DI_ERR_BUSY, "graph workspace is in use by another call");
        DeviceGuard dg(g->dev.device);
        cudaStream_t s = (cudaStream_t)stream;
        double single_ms = 0.0;
        if (what & 4) {
            g->tune_single.row = out->push_row;
            g->tune_single.heavy = out->heavy_cut;
            g->tune_single.chunk = out->heavy_chunk;
        }
        if (what & 1) autotune_single(g, d, s, &single_ms);
        if (what & 2) {
            if (g->bws) g->bws->tuned_T = 0;   // tune again
            autotune(g, d, s);
        }
        DI_CHECK_CUDA(cudaStreamSynchronize(s));
        if (out) {
            memset(out, 0, sizeof(*out));
            out->push_row = g->tune_single.row;
            out->heavy_cut = g->tune_single.heavy;
            out->heavy_chunk = g->tune_single.chunk;
            out->rhs_tile = g->bws ? g->bws->tuned_T : 0;
            out->batch_heavy_cut = g->tune_batch.heavy;
            out->batch_heavy_chunk = g->tune_batch.chunk;
            out->single_probe_ms = single_ms;
            out->batch_rate = g->bws ? g->bws->split_rate : 0.0;
        }
    });
}

di_status di_solve_batch(di_graph *g, int32_t k, const double *B, double d, const double *tol,
                         const di_solve_opts *opts, double *X_out, double *res_out, di_solve_info *info, void *stream) {
    return di::batch_entry(g, k, B, nullptr, nullptr, d, tol, opts, X_out, res_out, info, (cudaStream_t)stream);
}

di_status di_ppr_batch(di_graph *g, int32_t k, const int64_t *seed_offsets, const int32_t *seeds, double d,
                       const double *tol, const di_solve_opts *opts, double *X_out, double *res_out,
                       di_solve_info *info, void *stream) {
    return di::batch_entry(g, k, nullptr, seed_offsets, seeds, d, tol, opts, X_out, res_out, info, (cudaStream_t)stream);
}

}  // extern "C"
