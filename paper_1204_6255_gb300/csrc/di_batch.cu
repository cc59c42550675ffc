// Batched D-iteration: k independent right-hand sides on one graph, solved T at a time in the
// tiles of di_tile.cuh. With FP32 fluid, retirement is followed by the exact FP64 residual of
// every column; a column whose exact residual is above its tolerance re-enters the sweep loop
// from F*_c, aiming at half its tolerance.
//
// The tile width T is a template parameter (4, 8, 16, 32). The autotuner times a short probe of
// each width on the graph itself and keeps the fastest (cached per graph).
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
    hc.split = refine ? 1 : 0;
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
                batch_body<T>(g, w, l, s, cudaGraphConditionalHandle(0), 0);
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
    acc->kernel_launches += launches + 3 * (int64_t)hc.body_runs;
    for (int c = 0; c < ncols; c++) acc->dangling_mass_e += hc.e[c];
}

// ------------------------------------------------------------------------------------------
// autotuner: time a short probe of every tile width on this graph and keep the fastest
// ------------------------------------------------------------------------------------------
template <int T>
static double probe(di_graph *g, double d, cudaStream_t s) {
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
    solve_tile<T>(g, 0, T, d, tol.data(), DI_SOP, 6, false, w.stage.as<double>(), true, res.data(), &acc, s);
    DI_CHECK_CUDA(cudaEventRecord(b, s));
    DI_CHECK_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    // column-link updates per second
    return (double)acc.pushed_edges * T / (ms * 1e-3);
}

static int autotune(di_graph *g, double d, cudaStream_t s) {
    if (g->bws && g->bws->tuned_T) return g->bws->tuned_T;
    if (!g->bws) g->bws = new BatchWorkspace();
    ensure_batch(g, *g->bws, 32);
    double best = -1.0;
    int bestT = 8;
    const int cands[4] = {4, 8, 16, 32};
    for (int T : cands) {
        double v = T == 4 ? probe<4>(g, d, s) : T == 8 ? probe<8>(g, d, s) : T == 16 ? probe<16>(g, d, s) : probe<32>(g, d, s);
        g->bws->probe_rate[tile_index(T)] = v;
        if (v > best) {
            best = v;
            bestT = T;
        }
    }
    g->bws->tuned_T = bestT;
    return bestT;
}

template <int T>
static void batch_all(di_graph *g, int k, const double *B, bool B_dev, const int64_t *off_dev, const int32_t *seeds_dev,
                      double d, const double *tol_host, int schedule, int max_sweeps, bool refine, double *X_out,
                      bool X_dev, double *res_host, di_solve_info *acc, cudaStream_t s) {
    if (!g->bws) g->bws = new BatchWorkspace();
    ensure_batch(g, *g->bws, T);
    BatchWorkspace &w = *g->bws;
    const BLaunch l = blaunch<T>(g);
    BatchCtl *ctl = w.ctl.as<BatchCtl>();
    for (int c0 = 0; c0 < k; c0 += T) {
        const int ncols = k - c0 < T ? k - c0 : T;
        if (off_dev) {
            DI_CHECK_CUDA(cudaMemsetAsync(w.Bn.p, 0, sizeof(double) * (size_t)g->n * T, s));
            int zero = 0;
            DI_CHECK_CUDA(cudaMemcpyAsync(&ctl->status, &zero, sizeof(int), cudaMemcpyHostToDevice, s));
            kb_seed_B<T><<<g->dev.sms * 4, 256, 0, s>>>(off_dev, seeds_dev, g->n, c0, ncols, d, w.Bn.as<double>(), ctl);
            int st = 0;
            DI_CHECK_CUDA(cudaMemcpyAsync(&st, &ctl->status, sizeof(int), cudaMemcpyDeviceToHost, s));
            DI_CHECK_CUDA(cudaStreamSynchronize(s));
            DI_REQUIRE(st == 0, DI_ERR_OUT_OF_RANGE_ID, "a seed of columns %d..%d is outside [0, %d)", c0, c0 + ncols - 1,
                       g->n);
            acc->kernel_launches += 1;
        } else {
            const double *src = B;
            if (!B_dev) {
                to_device(w.stage.p, B + (int64_t)c0 * g->n, sizeof(double) * (size_t)g->n * ncols, s);
                src = w.stage.as<double>() - (int64_t)c0 * g->n;   // kb_load_B indexes by c0 + c
            }
            kb_load_B<T><<<l.ew, 256, 0, s>>>(src, g->n, c0, ncols, w.Bn.as<double>());
            acc->kernel_launches += 1;
        }
        solve_tile<T>(g, c0, ncols, d, tol_host, schedule, max_sweeps, refine, X_out, X_dev, res_host, acc, s);
    }
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
        DevBuf off_d, seeds_d;
        const int64_t *off_dev = nullptr;
        const int32_t *seeds_dev = nullptr;
        if (!B) {
            std::vector<int64_t> off_h((size_t)k + 1);
            from_device(off_h.data(), seed_off, sizeof(int64_t) * ((size_t)k + 1), s);
            DI_CHECK_CUDA(cudaStreamSynchronize(s));
            DI_REQUIRE(off_h[0] == 0, DI_ERR_INVALID_ARG, "seed_offsets[0] must be 0");
            for (int c = 0; c < k; c++)
                DI_REQUIRE(off_h[c + 1] > off_h[c], DI_ERR_INVALID_ARG, "seed set %d is empty or offsets decrease", c);
            off_d.ensure(sizeof(int64_t) * ((size_t)k + 1));
            to_device(off_d.p, off_h.data(), sizeof(int64_t) * ((size_t)k + 1), s);
            const int64_t ns = off_h[k];
            if (is_device_ptr(seeds)) {
                seeds_dev = seeds;
            } else {
                seeds_d.ensure(sizeof(int32_t) * (size_t)ns);
                to_device(seeds_d.p, seeds, sizeof(int32_t) * (size_t)ns, s);
                seeds_dev = seeds_d.as<int32_t>();
            }
            off_dev = off_d.as<int64_t>();
        }
        DI_CHECK_CUDA(cudaStreamSynchronize(s));
        for (int c = 0; c < k; c++)
            DI_REQUIRE(tol_h[c] > 0.0 && std::isfinite(tol_h[c]), DI_ERR_INVALID_ARG, "tol[%d] must be positive", c);
        const bool B_dev = B && is_device_ptr(B);
        const bool X_dev = is_device_ptr(X_out);
        int T = o.rhs_tile ? o.rhs_tile : autotune(g, d, s);
        if (!g->bws) g->bws = new BatchWorkspace();
        g->bws->host_loop = o.host_loop != 0;
        std::vector<double> res((size_t)k, 0.0);
        di_solve_info acc;
        memset(&acc, 0, sizeof(acc));
        cudaEvent_t e0, e1;
        DI_CHECK_CUDA(cudaEventCreate(&e0));
        DI_CHECK_CUDA(cudaEventCreate(&e1));
        DI_CHECK_CUDA(cudaEventRecord(e0, s));
        try {
            switch (T) {
                case 4: batch_all<4>(g, k, B, B_dev, off_dev, seeds_dev, d, tol_h.data(), o.schedule, max_sweeps, refine, X_out, X_dev, res.data(), &acc, s); break;
                case 8: batch_all<8>(g, k, B, B_dev, off_dev, seeds_dev, d, tol_h.data(), o.schedule, max_sweeps, refine, X_out, X_dev, res.data(), &acc, s); break;
                case 16: batch_all<16>(g, k, B, B_dev, off_dev, seeds_dev, d, tol_h.data(), o.schedule, max_sweeps, refine, X_out, X_dev, res.data(), &acc, s); break;
                default: batch_all<32>(g, k, B, B_dev, off_dev, seeds_dev, d, tol_h.data(), o.schedule, max_sweeps, refine, X_out, X_dev, res.data(), &acc, s); break;
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
        if (info) *info = acc;
        DI_REQUIRE(bad < 0, DI_ERR_NOT_CONVERGED, "column %d not converged: ||F||_1 = %g > tol = %g", bad, res[bad],
                   tol_h[bad]);
    });
}

}  // namespace di

extern "C" {

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
