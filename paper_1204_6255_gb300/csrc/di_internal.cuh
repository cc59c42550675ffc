// Internal declarations of the GB300 D-iteration library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "di.h"

namespace di {

// ------------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------------
void set_error(const char *fmt, ...);
void clear_error();

struct Fail {
    di_status status;
};

#define DI_CHECK_CUDA(expr)                                                                     \
    do {                                                                                        \
        cudaError_t _e = (expr);                                                                \
        if (_e != cudaSuccess) {                                                                \
            ::di::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__,   \
                            __LINE__);                                                          \
            throw ::di::Fail{_e == cudaErrorMemoryAllocation ? DI_ERR_OOM : DI_ERR_CUDA};       \
        }                                                                                       \
    } while (0)

#define DI_REQUIRE(cond, status, ...)                                                           \
    do {                                                                                        \
        if (!(cond)) {                                                                          \
            ::di::set_error(__VA_ARGS__);                                                       \
            throw ::di::Fail{status};                                                           \
        }                                                                                       \
    } while (0)

// Runs `body` and converts a thrown Fail into its status; also catches allocation failures.
template <class F>
di_status guarded(F &&body) {
    clear_error();
    try {
        body();
        return DI_OK;
    } catch (const Fail &f) {
        return f.status;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return DI_ERR_OOM;
    }
}

// ------------------------------------------------------------------------------------------
// device memory: owned by the library (cudaMalloc) or borrowed from a caller's workspace
// ------------------------------------------------------------------------------------------
// Bytes of device memory the library currently holds from cudaMalloc, over every graph (the
// graphs' CSR arrays included; a caller's workspace is not counted).
extern std::atomic<long long> g_device_bytes;

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    bool borrowed = false;         // p points into a caller's workspace: never freed here
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p && !borrowed) {
            cudaFree(p);
            g_device_bytes -= (long long)bytes;
        }
        p = nullptr;
        bytes = 0;
        borrowed = false;
    }
    // (Re)allocates to at least `n` bytes; contents are not preserved.
    void ensure(size_t n) {
        if (n <= bytes && p && !borrowed) return;
        release();
        size_t b = n ? n : 16;
        DI_CHECK_CUDA(cudaMalloc(&p, b));
        g_device_bytes += (long long)b;
        bytes = b;
    }
    // Points at `n` bytes of a caller's workspace (whatever it held is released first).
    void bind(void *q, size_t n) {
        release();
        p = q;
        bytes = n;
        borrowed = true;
    }
    template <class T>
    T *as() const { return static_cast<T *>(p); }
};

// Hands out consecutive 256-byte-aligned pieces of a caller's workspace (or, with base NULL,
// only adds up the bytes the pieces need).
struct Carve {
    char *base = nullptr;
    size_t cap = 0, used = 0;
    static size_t round(size_t n) { return (n + 255) & ~(size_t)255; }
    void take(DevBuf &b, size_t n) {
        const size_t a = round(n ? n : 16);
        if (base) {
            DI_REQUIRE(used + a <= cap, DI_ERR_INVALID_ARG,
                       "the attached workspace holds %zu bytes; this call needs more (see di_workspace_size)", cap);
            b.bind(base + used, a);
        }
        used += a;
    }
};

// True when `ptr` is device (or managed) memory.
bool is_device_ptr(const void *ptr);

// Copies `bytes` from src (host or device) into device buffer dst on `s`.
void to_device(void *dst, const void *src, size_t bytes, cudaStream_t s);
// Copies device src into dst (host or device) on `s`.
void from_device(void *dst, const void *src, size_t bytes, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// launch geometry
// ------------------------------------------------------------------------------------------
struct DeviceInfo {
    int device = 0;
    int sms = 0;
    int max_threads_per_sm = 0;
    size_t l2_bytes = 0;
};
DeviceInfo query_device();

// ------------------------------------------------------------------------------------------
// solve control block (device resident; one per workspace)
// ------------------------------------------------------------------------------------------
struct SolveCtl {
    // parameters written by the host before a launch
    double d;
    double tol;
    double L;                 // links (DI-SOP threshold is (r / L) * out_i)
    int32_t schedule;
    int32_t max_sweeps;
    // state
    double r;                 // ||F||_1 after the latest reduction
    double e;                 // dangling mass sum_{out=0} H
    unsigned long long pushed;
    unsigned long long visited;
    int32_t sweeps;
    int32_t force_cyc;        // next selection ignores the DI-SOP threshold
    int32_t last_selected;    // nodes selected by the latest sweep, -1 before the first
    // light frontier entries (low 40 bits) and frontier segments (high 24 bits) written by the
    // latest selection: one atomic reserves both for a select chunk
    unsigned long long front_chunks;
    int32_t heavy_count;      // heavy frontier entries written by the latest selection
    int32_t heavy_chunks;     // PushTune::chunk-link chunks of those entries
    int32_t done;             // 1 when the stop test has fired
    int32_t status;           // 0 ok; 1 bad right-hand side
    uint32_t ticket;          // last-block-done counter of the reductions
    int32_t body_runs;        // executions of the WHILE body (kernel-launch accounting)
    int32_t chunk_next;       // dynamic work counter over the segments
    double absorbed;          // fluid the visits of the current sweep removed from sum F (FP64)
    int32_t track;            // 1: F >= 0 throughout, so sum F after a sweep = before - absorbed
    int32_t reduce_est;       // 1: this sweep's reduction may take r from the tracked sum
    int32_t plain_loops;      // 1: a self-link is a plain link (power iteration per column), no
                              //    closed form for loop nodes
    unsigned long long front_total;  // frontier entries over all sweeps
    int32_t split;            // 1: the first reduction raises tol to sqrt(tol * r), the point of
                              //    the first refinement of a refined FP32 solve
    int32_t big_segs;         // frontier segments of at least kBigSegment entries (latest selection)
    int32_t small_segs;       // the other segments
    int32_t subs;             // selections so far (a sweep is r_refresh selections, one per
                              //    part of the node range)
    int32_t sweep_selected;   // nodes the parts of the current sweep selected so far
    int32_t halfway;          // 1: these sweeps end in that halfway refinement, whose exact
                              //    residual replaces the fluid, so the stop test may use the
                              //    tracked sum all the way down
};

// Fixed tuning of the single-RHS kernels.
constexpr int kFrontBits = 40;
__host__ __device__ inline int32_t front_entries(unsigned long long fc) {
    return (int32_t)(fc & ((1ull << kFrontBits) - 1));
}
__host__ __device__ inline int32_t front_segments(unsigned long long fc) { return (int32_t)(fc >> kFrontBits); }

// Push work split, picked per graph by the autotuner (di_autotune), defaults below: rows of at
// least `row` links are pushed one at a time by a whole warp; nodes with more than `heavy` links
// are pushed in `chunk`-link pieces spread over all warps (so out / chunk warps share such a row).
struct PushTune {
    int32_t row = 64;
    int32_t heavy = 4096;
    int32_t chunk = 1024;
    bool operator==(const PushTune &o) const { return row == o.row && heavy == o.heavy && chunk == o.chunk; }
};
constexpr int kPushHeavyMin = 1024;   // smallest `heavy` the tuner tries (buffers are sized for it)
constexpr int kHeavyChunkMin = 256;   // smallest `chunk` the tuner tries
// A refined FP32 solve refines first where ||F||_1 reaches sqrt(tol * ||F_0||_1) (halfway on a log
// scale); its continuation sweeps then aim at kAimAfterSplit * tol.
constexpr double kAimAfterSplit = 0.9;
// ... and only when tol is below kSplitBelow * ||F_0||_1: the FP32 rounding of a whole solve was
// measured near 7e-8 of ||F_0||_1, so above that bound it stays a few percent of tol and the
// halfway refinement would only cost an extra exact residual.
constexpr double kSplitBelow = 1e-6;
constexpr int kPullHeavy = 8192;    // in-degree above which a row's edges are split over warps
constexpr int kPullChunk = 4096;    // edges per heavy-row chunk of the pull
constexpr int kPullSamples = 4096;  // samples of the pull's link prefix (di_graph::pull_sample)
constexpr int kColInPad = 8;        // int32 slots allocated past col_in's L links (pull vector reads)
constexpr int kReduceBlocks = 1024; // partial sums of the last-block-done reductions
constexpr int kHubSlots = 2048;     // shared-memory hub cache of the push kernels
constexpr int kWinReach = 4096;     // push window: every source-target pair it takes is closer

// Per-graph state for single-RHS solves and power iteration.
struct Workspace {
    int fluid = -1;                 // di_fluid the buffers were sized for
    void *ext = nullptr;            // caller's workspace (di_graph_set_workspace), or NULL
    size_t ext_bytes = 0;
    DevBuf F, H, B, front_id, front_s, heavy_id, heavy_s, partials, ctl, y0, y1, chunks;
    DevBuf heavy_cstart, heavy_chunk;   // heavy entry -> first chunk; chunk -> heavy entry
    DevBuf Bdf, cdf, Xdf;           // power iteration: d/out (FP32 or FP64) in Bdf, X in Xdf;
                                    // cdf: d/out as double-float for the exact residual
    double cdf_d = -1.0;            // damping factor cdf currently holds (-1: none)
    cudaGraphExec_t sweep_exec = nullptr;   // reduce -> WHILE{(select, push, reduce) x sweep_parts}
    int sweep_parts = 1;
    PushTune sweep_tune;                    // push split the sweep graph was captured with
    cudaGraphExec_t pi_exec = nullptr;      // WHILE{[heavy chunk sums,] pull}
    int pi_fp64 = 0;                        // mode pi_exec was built for
    cudaStream_t capture_stream = nullptr;
    cudaStream_t out_stream = nullptr;      // copies X out beside the last refinement
    cudaEvent_t out_ready = nullptr, out_done = nullptr;
    SolveCtl *ctl_host = nullptr;           // pinned mirror for readback
    void reset_graphs();
    ~Workspace();
};

// Makes the graph's device current for the lifetime of the guard.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            DI_CHECK_CUDA(cudaSetDevice(dev));
        } else {
            prev = -1;
        }
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// Counts the kernels a call launches from the host and, in profile mode, brackets each launch
// with CUDA events on the launching stream (synchronising after it) to time it alone.
enum { KC_SELECT = 0, KC_PUSH = 1, KC_REDUCE = 2, KC_REFINE = 3 };
struct KernelClock {
    bool on = false;
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    double ms[4] = {0, 0, 0, 0};
    int count[4] = {0, 0, 0, 0};
    int64_t host_launches = 0;
    KernelClock(bool profile, cudaStream_t st) : on(profile), s(st) {
        if (on) {
            DI_CHECK_CUDA(cudaEventCreate(&a));
            DI_CHECK_CUDA(cudaEventCreate(&b));
        }
    }
    ~KernelClock() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
    template <class F>
    void run(int slot, int launches, F &&launch) {
        host_launches += launches;
        if (!on) {
            launch();
            return;
        }
        DI_CHECK_CUDA(cudaEventRecord(a, s));
        launch();
        DI_CHECK_CUDA(cudaEventRecord(b, s));
        DI_CHECK_CUDA(cudaEventSynchronize(b));
        float t = 0.f;
        DI_CHECK_CUDA(cudaEventElapsedTime(&t, a, b));
        ms[slot] += t;
        count[slot] += 1;
    }
};

struct BatchWorkspace;
void destroy_batch_workspace(BatchWorkspace *);

}  // namespace di

struct di_graph {
    int32_t n = 0;
    int64_t L = 0;
    int bits = 1;                  // bits per node id in packed keys
    di::DeviceInfo dev;
    di_graph_stats stats{};
    di::DevBuf rp_out, col_out, rp_in, col_in;   // int64 / int32
    di::DevBuf out_info;           // int32: out-degree | loop << 31
    di::DevBuf out_deg, in_deg;    // int32
    di::DevBuf loop;               // uint8
    di::DevBuf e_mask;             // uint8
    di::DevBuf e_level;            // int32
    di::DevBuf e_order;            // int32[N]: its first |E| entries list E grouped by level
    std::vector<int64_t> e_level_off;  // host: level l of E is e_order[off[l], off[l + 1])
    std::vector<int64_t> e_level_span; // host: ids spanned by level l (last - first + 1)
    // heavy rows of the in-CSR (in-degree > kPullHeavy), for the pull kernels
    int32_t n_heavy_in = 0;
    int32_t n_heavy_in_chunks = 0;
    std::vector<int64_t> pull_sample;  // host: light in-links of the rows below k * n / kPullSamples
    di::DevBuf heavy_in_rows;      // int32[n_heavy_in], ascending
    di::DevBuf heavy_in_chunk_off; // int32[n_heavy_in + 1]
    di::DevBuf heavy_in_chunk_row; // int32[n_heavy_in_chunks]: heavy index of each chunk
    di::DevBuf heavy_in_partial;   // float2[n_heavy_in_chunks] (double-float partial sums)
    int64_t n_heavy_out = 0;       // nodes with out-degree > kPushHeavyMin
    di::PushTune tune_single;      // single right-hand-side push split (autotuned or default)
    di::PushTune tune_batch;       // batched push split
    di::DevBuf hub_ids;            // int32[kHubSlots]: hub node per hash slot, -1 when empty
    int32_t win_reach_max = 0;     // most in-links of a non-hub node from sources < kWinReach ids away
    int32_t win_qbits = 20;        // push window: |fixed-point share| < 2^win_qbits (no int32 overflow)
    di::DevBuf col_push;           // int32[L]: col_out with bit 31 set on links into a hub
    di::DevBuf rp_push;            // int32[n+1]: rp_out narrowed (L < 2^31), the push's row bounds;
                                   //   bit 31 of entry u + 1: node u has a self-link (last in its row)
    std::mutex mu;                 // serialises use of the workspaces
    di::Workspace ws;
    di::BatchWorkspace *bws = nullptr;   // batched solves (created on first use)
    ~di_graph() { if (bws) di::destroy_batch_workspace(bws); }
};

namespace di {
// Solve entry used by the C ABI functions (di_solve.cu).
di_status solve_single(di_graph *g, const double *B, double d, double tol, const di_solve_opts *opts,
                       double *X_out, double *residual_out, di_solve_info *info, cudaStream_t s);
di_status power_iter(di_graph *g, const double *B, double d, double tol, int32_t max_iters,
                     double *X_out, double *residual_out, di_solve_info *info, cudaStream_t s);
// A single solve in a workspace the caller owns (not the graph's): no graph lock is taken, so
// the caller keeps that workspace to itself (the server's workers do).
di_status solve_single_in(di_graph *g, Workspace &ws, const double *B, double d, double tol,
                          const di_solve_opts *opts, double *X_out, double *residual_out, di_solve_info *info,
                          cudaStream_t s);
// Autotuning of the single right-hand-side push split (di_solve.cu); the caller holds g->mu.
PushTune autotune_single(di_graph *g, double d, cudaStream_t s, double *best_ms);
// Caller-provided solve workspace (di_solve.cu): bytes a fluid needs, and attaching one.
size_t solve_workspace_bytes(di_graph *g, int fluid);
void solve_workspace_attach(di_graph *g, void *ext, size_t bytes);
}  // namespace di

// ------------------------------------------------------------------------------------------
// small device helpers
// ------------------------------------------------------------------------------------------
#ifdef __CUDACC__
namespace di {
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Inclusive prefix sum across the warp.
template <class T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
    const unsigned lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(kFull, v, o);
        if (lane >= (unsigned)o) v += u;
    }
    return v;
}

// Block-wide sum; every thread receives the total. `scratch` holds one T per warp.
template <class T>
__device__ __forceinline__ T block_sum(T v, T *scratch) {
    const int warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane_id() == 0) scratch[warp] = v;
    __syncthreads();
    T t = 0;
    for (int w = 0; w < nw; w++) t += scratch[w];
    return t;
}

// Hash slot of a node in the hub table.
__device__ __forceinline__ int hub_slot(int32_t v) { return (int)(((uint32_t)v * 0x9E3779B1u) >> 21); }

// Largest lane k with off_k <= q, for lane offsets that are non-decreasing across the warp.
// Every lane of the warp must call it.
__device__ __forceinline__ int warp_owner(int off, int q) {
    int pos = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        int o = __shfl_sync(kFull, off, pos + s);
        if (o <= q) pos += s;
    }
    return pos;
}

// Exact FP32 -> FP64 widening on the integer units (IEEE 754 binary32 to binary64: the exponent
// is rebiased from 127 to 1023 and the fraction extended with zeros; a subnormal is normalised
// first; infinities and NaN keep the all-ones exponent).
__device__ __forceinline__ double widen(float x) {
    const uint32_t b = __float_as_uint(x);
    uint32_t e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
    if (e == 0xffu) {
        e = 0x7ffu - 896u;
    } else if (e == 0u) {
        if (m == 0u) {
            e = 0u - 896u;   // signed zero
        } else {
            const int s = __clz(m) - 8;   // moves the leading one to bit 23
            m = (m << s) & 0x7fffffu;
            e = 1u - (uint32_t)s;
        }
    }
    const uint32_t hi = (b & 0x80000000u) | ((e + 896u) << 20) | (m >> 3);
    return __hiloint2double((int)hi, (int)(m << 29));
}
__device__ __forceinline__ void red_add(float *p, float v) { atomicAdd(p, v); }
__device__ __forceinline__ void red_add(double *p, double v) { atomicAdd(p, v); }
}  // namespace di
#endif
