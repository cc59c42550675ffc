// Serving personalised-PageRank requests over resident graphs with continuous batching.
//
// Every graph has a worker thread with its own CUDA stream and one tile of T request slots
// (di_tile.cuh: node-major FP32 fluid, FP64 history, per-column DI-SOP selection and
// retirement). The worker repeats one step:
//   1. admit queued requests into free slots (reset the slot's columns, scatter the seeds'
//      mass (1 - d) / |S| into B and F);
//   2. run at most `sweeps_per_step` sweeps of the tile from one CUDA-graph launch (the WHILE
//      loop also ends as soon as every occupied slot has retired);
//   3. retire: a slot whose ||F_c||_1 fell to its tolerance is finished; for tolerances below
//      1e-6 the exact FP64 residual of the tile (B + P.H - H) is recomputed first and a slot
//      whose exact residual is still above its tolerance keeps sweeping from it (such a
//      request first stops halfway, on a log scale, between ||B||_1 and its tolerance, so that
//      one exact residual clears the FP32 rounding early);
//   4. copy each finished column's history out and zero the column, so the slot is clean for the
//      next request; the copy to pinned host memory is followed on the stream by a host function
//      that marks the request done, so the worker never waits for the copy.
// Requests that arrive while others are on the GPU are admitted at the next step as slots
// free up, so requests of different arrival times share sweeps, and the workers of different
// graphs run concurrently on the device. Each column is an independent problem; batch-mates
// only change which nodes a sweep visits, not the fixed point.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <memory>
#include <thread>
#include <unordered_map>

#include "di_tile.cuh"

namespace di {

namespace {

double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}


__global__ void ks_seed_dense(const int32_t *seeds, int cnt, double share, double *B) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += gridDim.x * blockDim.x)
        atomicAdd(&B[seeds[e]], share);
}

// Requests with a tolerance below this get an exact FP64 residual before they retire.
constexpr double kServeExactTol = 1e-6;

constexpr int kPoolStart = 4;   // pinned result buffers per worker made at server creation

struct Request {
    int64_t id = 0;
    int graph = 0;
    std::vector<int32_t> seeds;
    double tol = 0.0;
    double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
    int slot = -1;
    int admit_sweep = 0;
    bool halfway = false;           // sweeping towards the halfway refinement point
    double *X = nullptr;            // pinned host copy of the history (from the worker's pool)
    di_status status = DI_OK;
    int sweeps = 0;
    double residual = 0.0;
    bool done = false;
};

}  // namespace

struct Worker;

}  // namespace di

struct di_server {
    double d = 0.85;
    int sweeps_per_step = 8;
    int max_request_sweeps = 100000;
    int tile_min_queue = 16;             // requests waiting on an idle graph before the tile runs
    std::vector<std::unique_ptr<di::Worker>> workers;
    std::mutex mu;                       // requests map, completion signalling
    std::condition_variable done_cv;
    std::unordered_map<int64_t, std::shared_ptr<di::Request>> requests;
    int64_t next_id = 1;
    std::atomic<bool> stop{false};
    std::mutex copy_mu;                  // results copied to device memory by di_server_wait
    cudaStream_t copy_stream = nullptr;  // non-blocking: such a copy waits on no other work
    ~di_server();
};

namespace di {

struct Worker {
    di_server *srv = nullptr;
    di_graph *g = nullptr;
    int index = 0;
    int T = 32;
    BatchWorkspace w;
    cudaStream_t s = nullptr;
    DevBuf seeds_dev, col_out, lone_B;
    Workspace lone_ws;                   // single-solve workspace of the worker's lone requests
    std::mutex pool_mu;
    std::vector<double *> pool;          // free pinned host buffers of n doubles
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> queue;
    std::vector<std::shared_ptr<Request>> slot;
    std::thread th;
    std::atomic<bool> failed{false};

    ~Worker() {
        if (s) {
            cudaStreamSynchronize(s);   // pending copies and their host functions
            cudaStreamDestroy(s);
        }
        for (double *p : pool) cudaFreeHost(p);
    }

    double *take_buffer() {
        {
            std::lock_guard<std::mutex> lk(pool_mu);
            if (!pool.empty()) {
                double *p = pool.back();
                pool.pop_back();
                return p;
            }
        }
        double *p = nullptr;
        DI_CHECK_CUDA(cudaMallocHost(&p, sizeof(double) * (size_t)g->n));
        return p;
    }
    void give_buffer(double *p) {
        std::lock_guard<std::mutex> lk(pool_mu);
        pool.push_back(p);
    }

    template <int TT>
    void step_loop();
    void run();
    bool solve_lone(const std::shared_ptr<Request> &r);

    // runs on the CUDA runtime's thread once a result's copy to host memory has completed; it
    // only takes the server's lock (no CUDA call)
    struct Copied {
        di_server *srv;
        std::shared_ptr<Request> r;
    };
    static void CUDART_CB copied(void *p) {
        std::unique_ptr<Copied> c(static_cast<Copied *>(p));
        {
            std::lock_guard<std::mutex> lk(c->srv->mu);
            c->r->t_done = now_ms();
            c->r->done = true;
        }
        c->srv->done_cv.notify_all();
    }
};

template <int TT>
void Worker::step_loop() {
    const int32_t n = g->n;
    const BLaunch l = blaunch<TT>(g);
    BatchCtl *ctl = w.ctl.as<BatchCtl>();
    BatchCtl &hc = *(BatchCtl *)w.ctl_host;
    memset(&hc, 0, sizeof(BatchCtl));
    hc.d = srv->d;
    hc.L = (double)g->L;
    hc.ncols = TT;
    hc.schedule = DI_SOP;
    hc.last_selected = -1;
    for (int c = 0; c < TT; c++) hc.retire_sweep[c] = -1;
    DI_CHECK_CUDA(cudaMemsetAsync(w.F.p, 0, sizeof(float) * (size_t)n * TT, s));
    DI_CHECK_CUDA(cudaMemsetAsync(w.H.p, 0, sizeof(double) * (size_t)n * TT, s));
    DI_CHECK_CUDA(cudaMemsetAsync(w.Bn.p, 0, sizeof(double) * (size_t)n * TT, s));
    cudaGraphExec_t ex = batch_graph<TT>(g, w, l);
    slot.assign(TT, nullptr);
    while (!srv->stop.load()) {
        // 1. admission
        std::vector<std::shared_ptr<Request>> admitted;
        std::shared_ptr<Request> lone;
        {
            std::unique_lock<std::mutex> lk(mu);
            bool any_busy = false;
            for (auto &r : slot) any_busy = any_busy || (r != nullptr);
            if (!any_busy && queue.empty()) {
                cv.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
            // while few requests wait on an idle tile, they run one by one on the single
            // right-hand-side path: a tile sweep moves all TT columns' state, a single solve only
            // its own, so the tile pays only once enough requests share its sweeps
            if (!any_busy && (int)queue.size() < srv->tile_min_queue) {
                lone = queue.front();
                queue.pop_front();
                lone->t_admit = now_ms();
            }
            // (a pass that takes a lone request admits nothing into the tile)
            for (int c = 0; c < TT && !queue.empty() && !lone; c++) {
                if (slot[c]) continue;
                auto r = queue.front();
                queue.pop_front();
                r->slot = c;
                r->t_admit = now_ms();
                slot[c] = r;
                admitted.push_back(r);
            }
        }
        if (lone) {
            solve_lone(lone);
            continue;
        }
        if (!admitted.empty()) {
            // free slots are clean (a retiring column is zeroed), so admission only scatters the
            // seeds; all admitted seed lists go up in one copy
            std::vector<int32_t> all_seeds;
            for (auto &r : admitted) all_seeds.insert(all_seeds.end(), r->seeds.begin(), r->seeds.end());
            seeds_dev.ensure(sizeof(int32_t) * all_seeds.size());
            DI_CHECK_CUDA(cudaMemcpyAsync(seeds_dev.p, all_seeds.data(), sizeof(int32_t) * all_seeds.size(),
                                          cudaMemcpyHostToDevice, s));
            DI_CHECK_CUDA(cudaStreamSynchronize(s));   // all_seeds is a local buffer
            size_t at = 0;
            for (auto &r : admitted) {
                const int cnt = (int)r->seeds.size();
                kb_seed_col<TT><<<(cnt + 255) / 256, 256, 0, s>>>(seeds_dev.as<int32_t>() + at, cnt, r->slot,
                                                                   (1.0 - srv->d) / cnt, n, w.F.as<float>(),
                                                                   w.Bn.as<double>(), ctl);
                at += (size_t)cnt;
                const int c = r->slot;
                hc.active[c] = 1;
                hc.tol[c] = r->tol;
                // a tight request (refined at retirement) first stops halfway, on a log scale,
                // between ||B||_1 = 1 - d and its tol, where an exact residual replaces its
                // fluid before the FP32 rounding grows comparable to tol
                const double mid = sqrt(r->tol * (1.0 - srv->d));
                r->halfway = r->tol < kSplitBelow * (1.0 - srv->d);
                if (r->halfway) hc.tol[c] = mid;
                hc.r[c] = 0.0;
                hc.e[c] = 0.0;
                hc.retire_sweep[c] = -1;
                r->admit_sweep = hc.sweeps;
            }
            DI_CHECK_CUDA(cudaGetLastError());
        }
        // 2. a bounded number of sweeps
        hc.max_sweeps = hc.sweeps + srv->sweeps_per_step;
        hc.done = 0;
        hc.ticket = 0;
        DI_CHECK_CUDA(cudaMemcpyAsync(ctl, &hc, sizeof(BatchCtl), cudaMemcpyHostToDevice, s));
        kb_reduce<TT><<<l.red, 256, 0, s>>>(w.F.as<float>(), n, w.partials.as<double>(), ctl,
                                            cudaGraphConditionalHandle(0), 0);
        DI_CHECK_CUDA(cudaGraphLaunch(ex, s));
        DI_CHECK_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
        DI_CHECK_CUDA(cudaStreamSynchronize(s));
        // 3. retirement
        std::vector<int> retired;
        uint32_t exact_mask = 0;
        for (int c = 0; c < TT; c++) {
            if (!slot[c]) continue;
            const bool capped = hc.sweeps - slot[c]->admit_sweep >= srv->max_request_sweeps;
            if (!hc.active[c] || capped) {
                retired.push_back(c);
                if (slot[c]->tol < kServeExactTol) exact_mask |= 1u << c;
            }
        }
        if (retired.empty()) continue;
        if (exact_mask) {
            // exact residual of just the retiring tight-tolerance columns
            batch_resid<TT>(g, w, l, srv->d, s, exact_mask);
            DI_CHECK_CUDA(cudaMemcpyAsync(&hc, ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
            DI_CHECK_CUDA(cudaStreamSynchronize(s));
        }
        for (int c : retired) {
            auto r = slot[c];
            const bool capped = hc.sweeps - r->admit_sweep >= srv->max_request_sweeps;
            if (hc.r[c] > r->tol && !capped) {
                hc.active[c] = 1;            // keeps sweeping from the exact residual
                hc.tol[c] = (r->halfway ? kAimAfterSplit : 0.5) * r->tol;
                r->halfway = false;
                continue;
            }
            // 4. the column's history goes to a pinned buffer of the request, the column is zeroed
            // for its next request, and a host function marks the request done after the copy
            r->X = take_buffer();
            kb_col_retire<TT><<<l.ew, 256, 0, s>>>(w.F.as<float>(), w.H.as<double>(), w.Bn.as<double>(), n, c,
                                                   col_out.as<double>());
            DI_CHECK_CUDA(cudaMemcpyAsync(r->X, col_out.p, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, s));
            r->sweeps = hc.sweeps - r->admit_sweep;
            r->residual = hc.r[c];
            r->status = hc.r[c] <= r->tol ? DI_OK : DI_ERR_NOT_CONVERGED;
            hc.active[c] = 0;
            DI_CHECK_CUDA(cudaLaunchHostFunc(s, &Worker::copied, new Copied{srv, r}));
            {
                std::lock_guard<std::mutex> lk(mu);
                slot[c] = nullptr;
            }
        }
    }
}

// One request alone: B = (1 - d) / |S| on its seeds, a single right-hand-side DI-SOP solve into
// a pinned buffer, in the worker's own workspace.
bool Worker::solve_lone(const std::shared_ptr<Request> &r) {
    const int32_t n = g->n;
    const int cnt = (int)r->seeds.size();
    lone_B.ensure(sizeof(double) * (size_t)n);
    seeds_dev.ensure(sizeof(int32_t) * (size_t)cnt);
    DI_CHECK_CUDA(cudaMemsetAsync(lone_B.p, 0, sizeof(double) * (size_t)n, s));
    DI_CHECK_CUDA(cudaMemcpyAsync(seeds_dev.p, r->seeds.data(), sizeof(int32_t) * (size_t)cnt, cudaMemcpyHostToDevice, s));
    ks_seed_dense<<<(cnt + 255) / 256, 256, 0, s>>>(seeds_dev.as<int32_t>(), cnt, (1.0 - srv->d) / cnt,
                                                    lone_B.as<double>());
    DI_CHECK_CUDA(cudaGetLastError());
    double *X = take_buffer();
    di_solve_opts o;
    memset(&o, 0, sizeof(o));
    o.schedule = DI_SOP;
    o.max_sweeps = srv->max_request_sweeps;
    di_solve_info info;
    double res = 0.0;
    // the worker's own single-solve workspace, so callers' solves on the same graph never wait
    const di_status st = solve_single_in(g, lone_ws, lone_B.as<double>(), srv->d, r->tol, &o, X, &res, &info, s);
    DI_REQUIRE(st == DI_OK || st == DI_ERR_NOT_CONVERGED, st, "single solve of request %lld failed", (long long)r->id);
    r->X = X;
    r->sweeps = info.sweeps;
    r->residual = res;
    r->status = st;
    r->slot = -1;
    {
        std::lock_guard<std::mutex> lk(srv->mu);   // the history is in host memory already
        r->t_done = now_ms();
        r->done = true;
    }
    srv->done_cv.notify_all();
    return true;
}

void Worker::run() {
    try {
        DI_CHECK_CUDA(cudaSetDevice(g->dev.device));
        switch (T) {
            case 4: step_loop<4>(); break;
            case 8: step_loop<8>(); break;
            case 16: step_loop<16>(); break;
            default: step_loop<32>(); break;
        }
    } catch (const Fail &) {
        failed.store(true);
    }
    // fail whatever is left
    std::vector<std::shared_ptr<Request>> left;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (auto &r : slot)
            if (r) left.push_back(r);
        for (auto &r : queue) left.push_back(r);
        queue.clear();
    }
    {
        std::lock_guard<std::mutex> lk(srv->mu);
        for (auto &r : left)
            if (!r->done) {
                r->status = srv->stop.load() ? DI_ERR_BUSY : DI_ERR_CUDA;
                r->done = true;
                r->t_done = now_ms();
            }
    }
    srv->done_cv.notify_all();
}

}  // namespace di

di_server::~di_server() {
    stop.store(true);
    for (auto &w : workers) {
        w->cv.notify_all();
        if (w->th.joinable()) w->th.join();
    }
    // copies still in flight and their host functions use this server's lock: finish them
    // while the lock exists, then hand back the buffers of results nobody collected
    for (auto &w : workers)
        if (w->s) cudaStreamSynchronize(w->s);
    for (auto &kv : requests)
        if (kv.second->X) {
            workers[kv.second->graph]->give_buffer(kv.second->X);
            kv.second->X = nullptr;
        }
    workers.clear();
    if (copy_stream) cudaStreamDestroy(copy_stream);
}

using namespace di;

extern "C" {

di_status di_server_create(di_graph *const *graphs, int32_t n_graphs, const di_server_opts *opts, di_server **out) {
    return guarded([&] {
        DI_REQUIRE(out != nullptr, DI_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        DI_REQUIRE(graphs != nullptr && n_graphs >= 1, DI_ERR_INVALID_ARG, "need at least one graph");
        di_server_opts o;
        memset(&o, 0, sizeof(o));
        if (opts) o = *opts;
        const double d = o.d == 0.0 ? 0.85 : o.d;
        DI_REQUIRE(d > 0.0 && d < 1.0, DI_ERR_INVALID_ARG, "d must be in (0, 1) (got %g)", d);
        int T = o.slots == 0 ? 32 : o.slots;
        DI_REQUIRE(T == 4 || T == 8 || T == 16 || T == 32, DI_ERR_INVALID_ARG, "slots must be 4, 8, 16 or 32");
        // request state per slot and node: F (4) + H (8) + B (8) + frontier share (4) bytes
        auto state_bytes = [&](int t) {
            int64_t b = 0;
            for (int i = 0; i < n_graphs; i++) b += (int64_t)graphs[i]->n * t * 24;
            return b;
        };
        if (o.mem_budget > 0) {
            while (T > 4 && state_bytes(T) > o.mem_budget) T /= 2;
            DI_REQUIRE(state_bytes(T) <= o.mem_budget, DI_ERR_OOM,
                       "request state needs %lld bytes for 4 slots per graph; budget is %lld",
                       (long long)state_bytes(T), (long long)o.mem_budget);
        }
        std::unique_ptr<di_server> srv(new di_server());
        srv->d = d;
        srv->sweeps_per_step = o.sweeps_per_step > 0 ? o.sweeps_per_step : 8;
        srv->max_request_sweeps = o.max_request_sweeps > 0 ? o.max_request_sweeps : 100000;
        srv->tile_min_queue = o.tile_min_queue > 0 ? o.tile_min_queue : 16;
        for (int i = 0; i < n_graphs; i++) {
            DI_REQUIRE(graphs[i] != nullptr, DI_ERR_INVALID_ARG, "graph %d is NULL", i);
            std::unique_ptr<Worker> w(new Worker());
            w->srv = srv.get();
            w->g = graphs[i];
            w->index = i;
            w->T = T;
            DeviceGuard dg(graphs[i]->dev.device);
            ensure_batch(graphs[i], w->w, T);
            w->col_out.ensure(sizeof(double) * (size_t)graphs[i]->n);
            // pinned result buffers made up front: pinning host memory takes milliseconds for a
            // large graph, which a request finishing on an empty pool would otherwise wait for
            for (int b = 0; b < kPoolStart; b++) {
                double *p = nullptr;
                DI_CHECK_CUDA(cudaMallocHost(&p, sizeof(double) * (size_t)graphs[i]->n));
                w->give_buffer(p);
            }
            // stream priority by graph size: the largest graph's kernels are scheduled first when
            // workers overlap on the device, since its requests are the longest and make the
            // latency tail; the others are short whatever their priority
            int lo = 0, hi = 0;   // least and greatest priority (greatest is the smaller number)
            DI_CHECK_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
            int rank = 0;         // graphs larger than this one
            for (int j = 0; j < n_graphs; j++) rank += graphs[j]->n > graphs[i]->n ? 1 : 0;
            const int prio = std::max(hi, std::min(lo, hi + rank));
            DI_CHECK_CUDA(cudaStreamCreateWithPriority(&w->s, cudaStreamNonBlocking, prio));
            srv->workers.push_back(std::move(w));
        }
        for (auto &w : srv->workers) {
            Worker *wp = w.get();
            w->th = std::thread([wp] { wp->run(); });
        }
        *out = srv.release();
    });
}

di_status di_server_submit(di_server *srv, int32_t graph, const int32_t *seeds, int32_t n_seeds, double tol,
                           int64_t *request_id) {
    return guarded([&] {
        DI_REQUIRE(srv && request_id, DI_ERR_INVALID_ARG, "server or request_id is NULL");
        DI_REQUIRE(graph >= 0 && graph < (int32_t)srv->workers.size(), DI_ERR_INVALID_ARG, "graph %d out of range",
                   graph);
        DI_REQUIRE(seeds && n_seeds >= 1, DI_ERR_INVALID_ARG, "a request needs at least one seed");
        DI_REQUIRE(tol > 0.0 && std::isfinite(tol), DI_ERR_INVALID_ARG, "tol must be positive (got %g)", tol);
        Worker &w = *srv->workers[graph];
        DI_REQUIRE(!w.failed.load(), DI_ERR_CUDA, "the worker of graph %d stopped on a CUDA error", graph);
        auto r = std::make_shared<Request>();
        r->graph = graph;
        r->seeds.assign(seeds, seeds + n_seeds);
        for (int32_t v : r->seeds)
            DI_REQUIRE(v >= 0 && v < w.g->n, DI_ERR_OUT_OF_RANGE_ID, "seed %d outside [0, %d)", v, w.g->n);
        r->tol = tol;
        r->t_submit = now_ms();
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            r->id = srv->next_id++;
            srv->requests[r->id] = r;
        }
        {
            std::lock_guard<std::mutex> lk(w.mu);
            w.queue.push_back(r);
        }
        w.cv.notify_one();
        *request_id = r->id;
    });
}

di_status di_server_wait(di_server *srv, int64_t request_id, double *X_out, di_request_info *info,
                         int32_t timeout_ms) {
    return guarded([&] {
        DI_REQUIRE(srv != nullptr, DI_ERR_INVALID_ARG, "server is NULL");
        std::shared_ptr<Request> r;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            auto it = srv->requests.find(request_id);
            DI_REQUIRE(it != srv->requests.end(), DI_ERR_INVALID_ARG, "unknown request %lld", (long long)request_id);
            r = it->second;
            const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
            while (!r->done) {
                if (srv->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && !r->done) {
                    set_error("request %lld not finished after %d ms", (long long)request_id, timeout_ms);
                    throw Fail{DI_ERR_TIMEOUT};
                }
            }
            srv->requests.erase(it);
        }
        if (info) {
            memset(info, 0, sizeof(*info));
            info->status = r->status;
            info->sweeps = r->sweeps;
            info->graph = r->graph;
            info->slot = r->slot;
            info->residual_l1 = r->residual;
            info->queue_ms = r->t_admit > 0 ? r->t_admit - r->t_submit : 0.0;
            info->service_ms = r->t_admit > 0 ? r->t_done - r->t_admit : 0.0;
            info->total_ms = r->t_done - r->t_submit;
        }
        if (r->X) {
            Worker &w = *srv->workers[r->graph];
            double *buf = r->X;
            r->X = nullptr;
            const size_t bytes = sizeof(double) * (size_t)w.g->n;
            cudaError_t e = cudaSuccess;
            if (X_out) {
                cudaPointerAttributes a;
                const bool device = cudaPointerGetAttributes(&a, X_out) == cudaSuccess &&
                                    (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
                cudaGetLastError();
                if (!device) {
                    std::memcpy(X_out, buf, bytes);   // pinned host buffer to host memory
                } else {
                    std::lock_guard<std::mutex> lk(srv->copy_mu);
                    DeviceGuard dg(w.g->dev.device);
                    if (!srv->copy_stream) e = cudaStreamCreateWithFlags(&srv->copy_stream, cudaStreamNonBlocking);
                    if (e == cudaSuccess) e = cudaMemcpyAsync(X_out, buf, bytes, cudaMemcpyHostToDevice, srv->copy_stream);
                    if (e == cudaSuccess) e = cudaStreamSynchronize(srv->copy_stream);
                }
            }
            w.give_buffer(buf);
            DI_CHECK_CUDA(e);
        }
        DI_REQUIRE(r->status == DI_OK, r->status, "request %lld ended with status %d", (long long)request_id,
                   (int)r->status);
    });
}

void di_server_destroy(di_server *srv) { delete srv; }

}  // extern "C"
