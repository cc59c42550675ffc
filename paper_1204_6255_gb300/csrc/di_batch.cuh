// Batched (multi-RHS) workspace of a graph (di_batch.cu).
#pragma once

#include "di_internal.cuh"

namespace di {

struct BatchWorkspace {
    int T_alloc = 0;                 // widest tile the buffers hold
    void *ext = nullptr;             // caller's workspace (di_graph_set_workspace), or NULL
    size_t ext_bytes = 0;
    int tuned_T = 0;                 // autotuned tile width (0 = not tuned yet)
    double probe_rate[4] = {0, 0, 0, 0};   // column-link updates per second of each width
    double split_rate = 0.0;         // the same for the tuned push split at the tuned width
    DevBuf F, H, Bn, front_id, front_s, heavy_partial, partials, ctl, stage, y;
    DevBuf heavy_cstart, heavy_chunk;   // entry -> first chunk; chunk -> entry (heavy nodes)
    cudaGraphExec_t exec[4] = {nullptr, nullptr, nullptr, nullptr};   // per tile width
    PushTune exec_tune[4];           // push split each graph was captured with
    cudaStream_t capture_stream = nullptr;
    void *ctl_host = nullptr;
    bool host_loop = false;          // drive the sweeps from the host instead of the graph
    KernelClock *clock = nullptr;    // a profiled call's kernel timer (host-driven sweeps)
    ~BatchWorkspace();
};

}  // namespace di
