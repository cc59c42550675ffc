// Single right-hand-side D-iteration and power iteration on the GPU.
//
// A sweep (Section 2.3 DI-CYC / DI-SOP, Section 2.5) is three kernels:
//   k_select    reads F and out[], picks the nodes of the sweep (DI-CYC: F_i != 0; DI-SOP:
//               |F_i| > (r / L) * out_i with r = ||F||_1 taken at the sweep start), and performs
//               the node part of every visit: F_i -> 0, transit (F_i * out_i / (out_i - d) for a
//               loop node), H_i += transit, dangling mass e. Each warp packs the selected nodes
//               of its 256-node range first, so the visits run on full warps; with FP32 fluid
//               the next range's F and degrees arrive by cp.async meanwhile. Visited nodes with
//               out-links become frontier entries (node id, per-link share d * transit / out_i),
//               id-sorted within segments of kSelChunk nodes; nodes with more links than the
//               graph's heavy cut-off go to a separate heavy list.
//   k_push_win  (FP32 fluid) scatters the shares onto the out-neighbours j != i (the l_out loop
//               of Section 2.5): a block takes a segment, adds the links that land near it into
//               a shared-memory window and the links into hubs into a shared-memory hub cache,
//               and sends the rest to F with L2 reductions. Long rows go warp-wide; heavy
//               nodes are spread over every warp of the grid in chunks (PushTune: the lengths
//               are autotuned per graph). k_push does the same for FP64 fluid without the caches.
//   k_reduce    r = sum |F_i| in FP64 (FP32 runs, warp shuffle, block, then the last block to
//               finish sums the block partials in a fixed order), and the stop test r <= tol.
//               It writes the WHILE-node condition, so the whole sweep loop runs from one CUDA
//               graph launch.
// All selected nodes diffuse concurrently; the result is a valid D-iteration in another
// diffusion order, which reaches the same fixed point. Around the sweeps: k_e_visit (the E-level
// pre-diffusion, one launch per level of E), the exact FP64 residual refinement (an FP32 solve
// refines halfway, on a log scale, between ||B||_1 and tol, and at the end), and resumed solves
// from a given (H, F).
//
// Power iteration (Section 2.5 "PI", Jacobi on X = P.X + B) and the exact FP64 residual
// F* = B + P.H - H both use k_pull: a warp takes 32 consecutive rows of the in-CSR; each lane
// walks a run of kPullVT contiguous in-links, and a segmented scan joins the rows that span
// lanes. Rows with more than kPullHeavy in-links are summed chunk-wise by k_pull_heavy first.
// Power iteration per column (PI') runs the sweep kernels above with self-links as plain links.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include "di_internal.cuh"

namespace di {

// ------------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------------
template <class T>
__global__ void k_init(const double *B, int32_t n, T *F, double *H, SolveCtl *ctl) {
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double b = B[i];
        if (!(b >= 0.0) || isinf(b)) bad = true;
        F[i] = (T)b;
        H[i] = 0.0;
    }
    if (bad) ctl->status = 1;
}

// Resumed solve: B is checked like k_init does, H already holds the given history, and F takes
// the given fluid (staged as FP64) unless F0 is NULL (the caller then forms the exact residual).
template <class T>
__global__ void k_resume_init(const double *B, const double *F0, int32_t n, T *F, const double *H, SolveCtl *ctl) {
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double b = B[i];
        if (!(b >= 0.0) || isinf(b) || !isfinite(H[i])) bad = true;
        if (F0) {
            const double f = F0[i];
            if (!isfinite(f)) bad = true;
            F[i] = (T)f;
        }
    }
    if (bad) ctl->status = 1;
}

template <class T>
__global__ void k_fluid_to_double(const T *F, int32_t n, double *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)F[i];
}

// Last-block-done FP64 sum of the per-block partials; returns true in the finishing block,
// where `total` holds the grand total (thread 0 only needs it).
__device__ __forceinline__ bool finish_sum(double s, double *partials, SolveCtl *ctl, double *scratch, double &total) {
    __shared__ bool is_last;
    s = block_sum(s, scratch);
    if (threadIdx.x == 0) {
        partials[blockIdx.x] = s;
        __threadfence();
        unsigned t = atomicAdd(&ctl->ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return false;
    __threadfence();
    double acc = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) acc += __ldcg(&partials[b]);
    total = block_sum(acc, scratch);
    return true;
}

// This thread's share of sum |F_i| (grid-stride). FP32 fluid is summed in FP32 runs of 16
// entries that are then added in FP64 (FP64 throughput on this part is a small fraction of FP32).
__device__ __forceinline__ double abs_sum(const float *F, int32_t n) {
    // four float4 loads in flight per thread and step; the 16-entry FP32 run is then widened
    const int64_t n4 = n >> 2;
    const float4 *F4 = reinterpret_cast<const float4 *>(F);
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double s = 0.0;
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (; q + 3 * stride < n4; q += 4 * stride) {
        float4 a = __ldcg(F4 + q), b = __ldcg(F4 + q + stride), c = __ldcg(F4 + q + 2 * stride),
               d = __ldcg(F4 + q + 3 * stride);
        const float run = ((fabsf(a.x) + fabsf(a.y)) + (fabsf(a.z) + fabsf(a.w))) +
                          ((fabsf(b.x) + fabsf(b.y)) + (fabsf(b.z) + fabsf(b.w))) +
                          ((fabsf(c.x) + fabsf(c.y)) + (fabsf(c.z) + fabsf(c.w))) +
                          ((fabsf(d.x) + fabsf(d.y)) + (fabsf(d.z) + fabsf(d.w)));
        s += (double)run;
    }
    for (; q < n4; q += stride) {
        const float4 a = __ldcg(F4 + q);
        s += (double)((fabsf(a.x) + fabsf(a.y)) + (fabsf(a.z) + fabsf(a.w)));
    }
    // tail entries n4*4 .. n-1
    const int64_t t = (n4 << 2) + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) s += (double)fabsf(__ldcg(F + t));
    return s;
}
__device__ __forceinline__ double abs_sum(const double *F, int32_t n) {
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s += fabs(__ldcg(F + i));
    return s;
}

// r = ||F||_1, stop test, and bookkeeping for the next selection.
template <class T>
__global__ void k_reduce(const T *F, int32_t n, double *partials, SolveCtl *ctl, cudaGraphConditionalHandle h,
                         int set_cond, int sweep_end) {
    __shared__ double scratch[32];
    double tot;
    if (ctl->done) {
        // an earlier part of this sweep already stopped the loop: keep the WHILE condition at 0
        if (set_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(h, 0u);
        return;
    }
    if (ctl->reduce_est) {
        // with nonnegative fluid, sum |F| after the sweep is the sum before it less what the
        // visits absorbed (the select decided this per sweep; see there for when)
        if (blockIdx.x != 0 || threadIdx.x != 0) return;
        tot = ctl->r - ctl->absorbed;
        if (tot < 0.0) tot = 0.0;
    } else {
        const double s = abs_sum(F, n);
        if (!finish_sum(s, partials, ctl, scratch, tot)) return;
    }
    if (threadIdx.x == 0) {
        ctl->ticket = 0;
        ctl->r = tot;
        ctl->absorbed = 0.0;
        ctl->reduce_est = 0;
        // a DI-SOP sweep whose parts together found no node is followed by a DI-CYC sweep
        if (sweep_end) {
            const int sel = ctl->last_selected < 0 ? -1 : ctl->sweep_selected + ctl->last_selected;
            ctl->force_cyc = (sel == 0 && tot > 0.0) ? 1 : 0;
            ctl->sweep_selected = 0;
        } else {
            ctl->sweep_selected += ctl->last_selected > 0 ? ctl->last_selected : 0;
        }
        ctl->last_selected = 0;
        ctl->front_total += (unsigned long long)(front_entries(ctl->front_chunks) + ctl->heavy_count);
        ctl->front_chunks = 0;
        ctl->big_segs = 0;
        ctl->small_segs = 0;
        ctl->heavy_count = 0;
        ctl->heavy_chunks = 0;
        ctl->chunk_next = 0;
        if (set_cond) ctl->body_runs++;
        if (ctl->split) {
            // first reduction of a refined FP32 solve: its sweeps stop halfway (geometrically)
            // between ||B||_1 and tol, where an exact residual replaces the fluid
            ctl->split = 0;
            const double mid = sqrt(ctl->tol * tot);
            if (ctl->tol < kSplitBelow * tot) {
                ctl->tol = mid;
                ctl->halfway = 1;
            }
        }
        bool cont = ctl->status == 0 && tot > ctl->tol && ctl->sweeps < ctl->max_sweeps;
        ctl->done = cont ? 0 : 1;
        if (set_cond) cudaGraphSetConditional(h, cont ? 1u : 0u);
    }
}

// ------------------------------------------------------------------------------------------
// cache-policy helpers: F (the scatter target) should stay in L2 while everything else streams
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
// link indices: each lane reads a run of consecutive links, so the line is kept in L1 for the
// lane's next reads, and marked for early eviction in L2
__device__ __forceinline__ int32_t ld_stream(const int32_t *p, uint64_t pol) {
    int32_t v;
    asm volatile("ld.global.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}
// four consecutive link indices from a 16-byte aligned address, same cache policy
__device__ __forceinline__ int4 ld_stream4(const int32_t *p, uint64_t pol) {
    int4 v;
    asm volatile("ld.global.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void red_keep_v4(float *p, float4 v, uint64_t pol) {
    asm volatile("red.global.add.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w), "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void red_keep(float *p, float v, uint64_t pol) {
    asm volatile("red.global.add.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void red_keep(double *p, double v, uint64_t pol) {
    asm volatile("red.global.add.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ float ld_keep(const float *p, uint64_t pol) {
    float v;
    asm volatile("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double ld_keep(const double *p, uint64_t pol) {
    double v;
    asm volatile("ld.global.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_keep(float *p, float v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(p), "f"(v), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_keep(double *p, double v, uint64_t pol) {
    asm volatile("st.global.L2::cache_hint.f64 [%0], %1, %2;" ::"l"(p), "d"(v), "l"(pol) : "memory");
}

__device__ __forceinline__ double widen(double x) { return x; }

// Node part of a visit: transit (loop closed form) and the per-link share d * transit / out.
// FP32 fluid: the arithmetic stays in FP32 (this part's FP64 rate is a small fraction of its
// FP32 rate); the transit is widened to FP64 only to be added to H. One quotient serves both:
// q = f / (out - d) for a loop node (transit q * out, share q * d), q = f / out otherwise
// (transit f, share q * d); the fast FP32 division is within 2 ulp.
__device__ __forceinline__ void visit_math(float f, int32_t o, bool lp, double, float d_f, float &t, float &share) {
    const float of = (float)o;
    const float q = o ? __fdividef(f, lp ? of - d_f : of) : 0.f;
    share = q * d_f;
    t = lp ? q * of : f;
}
__device__ __forceinline__ void visit_math(double f, int32_t o, bool lp, double d, float, double &t, double &share) {
    t = lp ? f * (double)o / ((double)o - d) : f;
    share = o ? t * d / (double)o : 0.0;
}
// DI-SOP's test |F_i| > (r / L) * out_i, decided as in FP64 (r / L is an FP64 value). The FP32
// product thr_f * out differs from the FP64 one by less than 2^-22 of it, so FP32 decides every
// node whose fluid is more than 2^-20 (relative) away from its threshold, and FP64 the near ties
// (and every node when r / L is too small for FP32's normal range).
constexpr float kThrBand = 1.0f / (1 << 20);
__device__ __forceinline__ bool sop_selects(float a, int32_t o, double thr, float thr_f) {
    const float p = thr_f * (float)o;
    if (thr_f >= 1e-30f) {
        if (a > p * (1.f + kThrBand)) return true;
        if (a < p * (1.f - kThrBand)) return false;
    }
    return (double)a > thr * (double)o;
}
__device__ __forceinline__ bool selects(float f, int32_t o, bool cyc, double thr, float thr_f) {
    return cyc ? (f != 0.f) : sop_selects(fabsf(f), o, thr, thr_f);
}
__device__ __forceinline__ bool selects(double f, int32_t o, bool cyc, double thr, float) {
    return cyc ? (f != 0.0) : (fabs(f) > thr * (double)o);
}

// cp.async (16-byte pieces into shared memory, zero-filled past src_bytes) and its groups
__device__ __forceinline__ void cp_async16(void *dst, const void *src, unsigned src_bytes, uint64_t pol) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2, %3;" ::"r"(d), "l"(src), "r"(src_bytes),
                 "l"(pol)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all_but_newest() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Copies F and the degree words of the nodes [wb, wb + 256) (those below n) into a warp's
// shared-memory slots: 64 16-byte pieces per array, two per lane. wb is a multiple of 256, so
// every piece is 16-byte aligned.
__device__ __forceinline__ void sel_prefetch(float *dst_f, int32_t *dst_i, const float *F, const int32_t *info,
                                             uint32_t wb, int32_t n, unsigned lane, uint64_t keep, uint64_t stream) {
#pragma unroll
    for (int q = 0; q < 2; q++) {
        const uint32_t piece = lane + 32 * q, first = wb + 4 * piece;
        if (first < (uint32_t)n) {
            const unsigned bytes = 4u * min(4u, (uint32_t)n - first);
            cp_async16(dst_f + 4 * piece, F + first, bytes, keep);
            cp_async16(dst_i + 4 * piece, info + first, bytes, stream);
        }
    }
}
__device__ __forceinline__ void sel_prefetch(double *, int32_t *, const double *, const int32_t *, uint32_t, int32_t,
                                             unsigned, uint64_t, uint64_t) {}

// Fixed-point scale of a segment's shared-memory push window (k_push_win). FP32 atomics on
// shared memory are compare-and-swap loops on this part, integer ones are native, so the window
// adds integers: q = round(share * 2^k) for each frontier entry. A window slot sums at most
// win_reach_max shares per segment (at most one link per source, and only from sources within
// kWinReach ids: a bound the graph build measures), so shares with |q| < 2^win_qbits cannot
// overflow its int32. k puts the segment's mean |share| just below 2^(win_qbits - kWinHeadBits):
// shares up to 2^kWinHeadBits times the mean stay in the window, larger ones skip it, and a unit
// is 2^-(win_qbits - kWinHeadBits) of the mean share.
constexpr int kWinHeadBits = 4;
__device__ __forceinline__ int window_exponent(float mean_abs, int mean_bits) {
    if (!(mean_abs > 0.f) || isinf(mean_abs)) return 0;
    int e;
    frexpf(mean_abs, &e);   // mean_abs < 2^e
    const int k = mean_bits - e;
    return k < -126 ? -126 : (k > 126 ? 126 : k);
}
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }   // -126 <= k <= 127

// Frontier segment records: the push takes segments in record order, so segments of at least
// kBigSegment entries are written from the front of the record array and the others from its
// back (index seg_cap - 1 downward); the push reads the front ones first, so the long segments
// start early and the short ones fill the end of the kernel.
constexpr int kBigSegment = 512;
__device__ __forceinline__ int segment_slot(SolveCtl *ctl, int entries, int seg_cap) {
    return entries >= kBigSegment ? atomicAdd(&ctl->big_segs, 1) : seg_cap - 1 - atomicAdd(&ctl->small_segs, 1);
}
__device__ __forceinline__ int segment_at(const SolveCtl *ctl, int ci, int seg_cap) {
    const int big = ctl->big_segs;
    return ci < big ? ci : seg_cap - 1 - (ci - big);
}

// Nodes are visited in chunks of kSelChunk consecutive ids per block iteration; warp w of the
// block owns the kSelWarpNodes consecutive ids from base + w * kSelWarpNodes. The frontier
// entries of a chunk are compacted with one atomic per chunk, so the frontier is id-sorted
// within each chunk (the push then walks neighbouring rows together). An entry is the node id
// and its share (8 bytes); the push reads the row bounds itself, from neighbouring row pointers
// (whose bit 31 marks a loop node, see k_push_win).
constexpr int kSelItems = 8;
constexpr int kTrackResync = 8;      // an exact reduction at least every kTrackResync sweeps
constexpr double kTrackBand = 16.0;  // ... and at every sweep once r <= kTrackBand * tol
constexpr int kSelWarpNodes = 32 * kSelItems;
constexpr int kSelChunk = 8 * kSelWarpNodes;   // 256 threads
constexpr int kSelMinBlocks = 4;
template <class T>
constexpr int kSelBatch = sizeof(T) == 4 ? 4 : 2;   // packed rounds of 32 visits whose history loads fly together

template <class T>
__global__ void __launch_bounds__(256, kSelMinBlocks) k_select(T *F, double *H, const int32_t *out_info,
                                                            int32_t n, SolveCtl *ctl, int32_t *front_id, T *front_s,
                                                            int32_t *heavy_id, T *heavy_s, int32_t *heavy_cstart,
                                                            int32_t *heavy_chunk, int4 *chunks, int win_mean_bits,
                                                            int32_t node_lo, int32_t node_hi, int sweep_end,
                                                            int heavy_cut, int heavy_len, int seg_cap) {
    __shared__ double scratch[32];
    __shared__ unsigned long long scratch_u[32];
    // Per warp, the selected nodes of its range packed in id order: fluid, degree word and
    // offset within the range. After their visits the same slots hold the warp's frontier
    // entries (share, offset), again in id order.
    // With FP32 fluid the slots are double-buffered: the next chunk's F and degree words are
    // copied in (cp.async) while the current chunk is visited.
    constexpr bool kPre = sizeof(T) == 4;
    __shared__ __align__(16) T s_f[kPre ? 2 : 1][8][kSelWarpNodes];
    __shared__ __align__(16) int32_t s_info[kPre ? 2 : 1][8][kSelWarpNodes];
    __shared__ uint8_t s_off[8][kSelWarpNodes];
    __shared__ int s_wcount[8], s_wbase[8];
    __shared__ float s_wabs[8];
    __shared__ int s_chunk_base;
    __shared__ double s_thr;
    if (ctl->done) return;
    if (threadIdx.x == 0) s_thr = ctl->L > 0.0 ? ctl->r / ctl->L : 0.0;
    __syncthreads();
    const double r = ctl->r, d = ctl->d, thr = s_thr;
    const bool cyc = ctl->schedule == DI_CYC || ctl->force_cyc;
    const bool plain_loops = ctl->plain_loops != 0;
    const float thr_f = (float)thr, d_f = (float)d;
    const uint64_t keep = policy_evict_last(), stream = policy_evict_first();
    const unsigned lane = lane_id(), lt = lanemask_lt();
    const int warp = threadIdx.x >> 5;
    uint8_t *woff = s_off[warp];
    int cur = 0;
    // this launch selects among the nodes [node_lo, node_hi) (node_lo a multiple of kSelChunk):
    // the whole range, or one part of it when r is refreshed within a sweep
    n = node_hi;
    if (kPre) {
        if (node_lo + blockIdx.x * kSelChunk < (uint32_t)n)
            sel_prefetch(s_f[0][warp], s_info[0][warp], F, out_info,
                         node_lo + blockIdx.x * kSelChunk + warp * kSelWarpNodes, n, lane, keep, stream);
        cp_async_commit();
    }
    T e_run = (T)0;      // dangling mass of this thread
    float ab_run = 0.f;  // fluid absorbed by this thread's visits (FP32: FP64 is slow here)
    unsigned long long pushed = 0;
    unsigned visited = 0;
    // 32-bit node arithmetic: ids stay below 2^31 and a stride below 2^31, so nothing wraps
    for (uint32_t base = node_lo + blockIdx.x * kSelChunk; base < (uint32_t)n; base += gridDim.x * kSelChunk) {
        const uint32_t wb = base + warp * kSelWarpNodes;
        T *wf = s_f[cur][warp];
        int32_t *winfo = s_info[cur][warp];
        // F and the degree word of the warp's nodes: every load is issued before any is used
        T f[kSelItems];
        int32_t info[kSelItems];
        if (kPre) {
            const uint32_t nb = base + gridDim.x * kSelChunk;
            if (nb < (uint32_t)n)
                sel_prefetch(s_f[cur ^ 1][warp], s_info[cur ^ 1][warp], F, out_info, nb + warp * kSelWarpNodes, n,
                             lane, keep, stream);
            cp_async_commit();
            cp_async_wait_all_but_newest();   // this chunk's copies are in
            __syncwarp();
        }
#pragma unroll
        for (int j = 0; j < kSelItems; j++) {
            const uint32_t i = wb + j * 32 + lane;
            f[j] = (T)0;
            info[j] = 0;
            if (i < (uint32_t)n) {
                if (kPre) {
                    f[j] = wf[j * 32 + lane];
                    info[j] = winfo[j * 32 + lane];
                } else {
                    f[j] = ld_keep(F + i, keep);
                    info[j] = __ldcs(out_info + i);
                }
            }
        }
        if (kPre) __syncwarp();   // all read before the packing below overwrites the slots
        // pack the selected nodes, so the visits below run on full warps
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < kSelItems; j++) {
            const bool s = wb + j * 32 + lane < (uint32_t)n && selects(f[j], info[j] & 0x7fffffff, cyc, thr, thr_f);
            const unsigned b = __ballot_sync(kFull, s);
            if (s) {
                const int p = cnt + __popc(b & lt);
                wf[p] = f[j];
                winfo[p] = info[j];
                woff[p] = (uint8_t)(j * 32 + lane);
            }
            cnt += __popc(b);
        }
        __syncwarp();
        int nlight = 0;
        float sh_abs = 0.f;   // sum of |share| over this lane's light entries of the chunk
        for (int r0 = 0; r0 < cnt; r0 += 32 * kSelBatch<T>) {
            T pf[kSelBatch<T>];
            int32_t pinfo[kSelBatch<T>];
            int poff[kSelBatch<T>];
            double ph[kSelBatch<T>];
#pragma unroll
            for (int v = 0; v < kSelBatch<T>; v++) {
                const int k = r0 + v * 32 + lane;
                pf[v] = (T)0;
                pinfo[v] = 0;
                poff[v] = 0;
                ph[v] = 0.0;
                if (k < cnt) {
                    pf[v] = wf[k];
                    pinfo[v] = winfo[k];
                    poff[v] = woff[k];
                    ph[v] = __ldcs(H + wb + poff[v]);
                }
            }
            // every slot of these rounds is in registers before entries overwrite slots below
            __syncwarp();
#pragma unroll
            for (int v = 0; v < kSelBatch<T>; v++) {
                const int k = r0 + v * 32 + lane;
                const uint32_t i = wb + poff[v];
                bool light = false, heavy = false;
                T share = (T)0;
                const int32_t o = pinfo[v] & 0x7fffffff;
                if (k < cnt) {
                    const bool lp = !plain_loops && pinfo[v] < 0;
                    st_keep(F + i, (T)0, keep);
                    T t;
                    visit_math(pf[v], o, lp, d, d_f, t, share);
                    __stcs(H + i, ph[v] + widen(t));
                    visited++;
                    pushed += (unsigned long long)o;
                    // F loses f and regains the share on each link pushed (all but a closed-form loop)
                    ab_run += (float)pf[v] - (float)share * (float)(o - (lp ? 1 : 0));
                    if (o == 0) {
                        e_run += t;
                    } else if (o > heavy_cut) {
                        heavy = true;
                    } else if (o - (lp ? 1 : 0) > 0) {
                        light = true;
                    }
                }
                const unsigned bl = __ballot_sync(kFull, light);
                if (light) {
                    const int p = nlight + __popc(bl & lt);
                    wf[p] = share;
                    woff[p] = (uint8_t)poff[v];
                    sh_abs += fabsf((float)share);
                }
                nlight += __popc(bl);
                // heavy nodes are rare: one atomic per warp that has any
                const unsigned bh = __ballot_sync(kFull, heavy);
                if (bh) {
                    const int leader = __ffs(bh) - 1;
                    int p0 = 0;
                    if ((int)lane == leader) p0 = atomicAdd(&ctl->heavy_count, __popc(bh));
                    p0 = __shfl_sync(kFull, p0, leader);
                    if (heavy) {
                        // the node's links are pushed in heavy_len-link chunks over all warps;
                        // the chunk list maps each chunk back to its entry
                        const int p = p0 + __popc(bh & lt);
                        heavy_id[p] = (int32_t)i;
                        heavy_s[p] = share;
                        const int nch = (o + heavy_len - 1) / heavy_len;
                        const int cs = atomicAdd(&ctl->heavy_chunks, nch);
                        heavy_cstart[p] = cs;
                        for (int c = 0; c < nch; c++) heavy_chunk[cs + c] = p;
                    }
                }
            }
        }
        // one atomic reserves the chunk's frontier entries and its segment slot
        const float wabs = kPre ? warp_sum(sh_abs) : 0.f;
        if (lane == 0) {
            s_wcount[warp] = nlight;
            s_wabs[warp] = wabs;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = 0;
#pragma unroll
            for (int w = 0; w < 8; w++) {
                s_wbase[w] = run;
                run += s_wcount[w];
            }
            s_chunk_base = 0;
            if (run) {
                float abs_tot = 0.f;
#pragma unroll
                for (int w = 0; w < 8; w++) abs_tot += s_wabs[w];
                const unsigned long long fc = atomicAdd(&ctl->front_chunks, (1ull << kFrontBits) | (unsigned)run);
                s_chunk_base = front_entries(fc);
                chunks[segment_slot(ctl, run, seg_cap)] =
                    make_int4((int)base, s_chunk_base, run, window_exponent(abs_tot / (float)run, win_mean_bits));
            }
        }
        __syncthreads();
        const int cb = s_chunk_base + s_wbase[warp];
        for (int k = lane; k < nlight; k += 32) {
            __stcs(front_id + cb + k, (int32_t)(wb + woff[k]));
            __stcs(front_s + cb + k, wf[k]);
        }
        __syncwarp();   // the slots are reused: by the next chunk's copies or packing
        if (kPre) cur ^= 1;
    }
    // warp sums in the fluid's type, block sums in FP64 by one thread
    const T e_w = warp_sum(e_run);
    const float ab_w = warp_sum(ab_run);
    if (lane == 0) {
        scratch[warp] = (double)e_w;
        scratch[8 + warp] = (double)ab_w;
    }
    pushed = block_sum(pushed, scratch_u);
    const unsigned long long nvis = block_sum((unsigned long long)visited, scratch_u);
    double e_loc = 0.0, absorbed = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < 8; w++) {
            e_loc += scratch[w];
            absorbed += scratch[8 + w];
        }
    if (threadIdx.x == 0) {
        if (e_loc != 0.0) atomicAdd(&ctl->e, e_loc);
        if (absorbed != 0.0) atomicAdd(&ctl->absorbed, absorbed);
        if (pushed) atomicAdd(&ctl->pushed, pushed);
        if (nvis) {
            atomicAdd(&ctl->visited, nvis);
            atomicAdd(&ctl->last_selected, (int)nvis);
        }
        if (blockIdx.x == 0) {
            const int sw = atomicAdd(&ctl->subs, 1) + 1;
            if (sweep_end) atomicAdd(&ctl->sweeps, 1);
            // this sweep's reduction takes r from the tracked sum while r is well above tol,
            // except every kTrackResync-th sweep (the FP32 atomics' rounding is not tracked);
            // near the tolerance every reduction sums F, so the stop test is on the exact sum.
            // Sweeps that end in the halfway refinement stop on the tracked sum all the way
            // down: that refinement's exact residual replaces the fluid in any case.
            ctl->reduce_est =
                (ctl->track && (ctl->halfway || r > kTrackBand * ctl->tol) && sw % kTrackResync != 0) ? 1 : 0;
        }
    }
}

// E-level pre-diffusion (Section 2.4: E, the recursively zero-in-degree set, converges in
// finitely many steps). One launch per level of E: every in-neighbour of a node of the level is
// in E at a lower level and was visited by an earlier launch, so the node's fluid is final, and
// no two nodes of a level are linked. One lane per node visits it (E holds no loop node) and
// pushes its share over at most kEWarpLinks out-links itself; the warp pushes the links of
// nodes with up to kEBlockLinks, one node at a time; the whole block pushes the links of larger
// nodes after its warps are done, so no single warp carries a long row at the kernel's tail.
// All keep kEUnroll index loads in flight before their additions. As in the push, links into
// hubs (bit 31 of col_push) collect in a per-block shared-memory cache, flushed once per block,
// and the L2 keeps F (the additions' target) while the links and the history stream through it.
constexpr int kEWarpLinks = 32;
constexpr int kEBlockLinks = 256;
constexpr int kEBlockRows = 256;   // large rows a block collects (more: the warp pushes them)
constexpr int kEUnroll = 8;   // index loads in flight before their additions

template <class T>
__global__ void __launch_bounds__(256) k_e_visit(const int32_t *nodes, int32_t count, const int32_t *out_info,
                                                 const int64_t *rp_out, const int32_t *col_push,
                                                 const int32_t *hub_ids, T *F, double *H, SolveCtl *ctl) {
    __shared__ double scratch[32];
    __shared__ unsigned long long scratch_u[32];
    __shared__ T s_hacc[kHubSlots];
    __shared__ int64_t s_rb[kEBlockRows];   // the block's large rows: first link, links, share
    __shared__ int32_t s_rd[kEBlockRows];
    __shared__ T s_rs[kEBlockRows];
    __shared__ int s_nrows;
    for (int q = threadIdx.x; q < kHubSlots; q += blockDim.x) s_hacc[q] = (T)0;
    if (threadIdx.x == 0) s_nrows = 0;
    __syncthreads();
    const uint64_t keep = policy_evict_last(), stream = policy_evict_first();
    auto add = [&](int32_t jr, T v) {
        if (jr < 0) atomicAdd(&s_hacc[hub_slot(jr & 0x7fffffff)], v);
        else red_keep(&F[jr], v, keep);
    };
    const double d = ctl->d;
    const float d_f = (float)d;
    const int lane = (int)lane_id();
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double e_loc = 0.0;
    unsigned long long pushed = 0, visited = 0;
    for (int64_t w0 = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * 32; w0 < count; w0 += nwarps * 32) {
        const int64_t idx = w0 + lane;
        int32_t u = 0, o = 0;
        int64_t b = 0;
        T share = (T)0;
        if (idx < count) {
            u = nodes[idx];
            const T f = ld_keep(F + u, keep);
            o = __ldcs(out_info + u) & 0x7fffffff;
            b = __ldcs(rp_out + u);
            T t;
            visit_math(f, o, false, d, d_f, t, share);
            st_keep(F + u, (T)0, keep);
            __stcs(H + u, __ldcs(H + u) + widen(t));
            if (o == 0) e_loc += widen(t);
            visited++;
            pushed += (unsigned long long)o;
            if (o <= kEWarpLinks)
                for (int64_t k0 = b; k0 < b + o; k0 += kEUnroll) {
                    int32_t jr[kEUnroll];
#pragma unroll
                    for (int v = 0; v < kEUnroll; v++) jr[v] = k0 + v < b + o ? ld_stream(col_push + k0 + v, stream) : 0;
#pragma unroll
                    for (int v = 0; v < kEUnroll; v++)
                        if (k0 + v < b + o) add(jr[v], share);
                }
        }
        // rows above kEBlockLinks go to the block's list (while it has room)
        bool later = false;
        if (idx < count && o > kEBlockLinks) {
            const int slot = atomicAdd(&s_nrows, 1);
            if (slot < kEBlockRows) {
                s_rb[slot] = b;
                s_rd[slot] = o;
                s_rs[slot] = share;
                later = true;
            }
        }
        unsigned big = __ballot_sync(kFull, idx < count && o > kEWarpLinks && !later);
        while (big) {
            const int src = __ffs(big) - 1;
            big &= big - 1;
            const int64_t bb = __shfl_sync(kFull, b, src);
            const int32_t oo = __shfl_sync(kFull, o, src);
            const T ss = __shfl_sync(kFull, share, src);
            for (int64_t k0 = bb + lane; k0 < bb + oo; k0 += 32 * kEUnroll) {
                int32_t jr[kEUnroll];
#pragma unroll
                for (int v = 0; v < kEUnroll; v++) jr[v] = k0 + 32 * v < bb + oo ? ld_stream(col_push + k0 + 32 * v, stream) : 0;
#pragma unroll
                for (int v = 0; v < kEUnroll; v++)
                    if (k0 + 32 * v < bb + oo) add(jr[v], ss);
            }
        }
    }
    __syncthreads();
    // the block's large rows, each over all of its threads
    const int nrows = min(s_nrows, kEBlockRows);
    for (int r = 0; r < nrows; r++) {
        const int64_t bb = s_rb[r];
        const int32_t oo = s_rd[r];
        const T ss = s_rs[r];
        for (int64_t k0 = bb + threadIdx.x; k0 < bb + oo; k0 += (int64_t)blockDim.x * kEUnroll) {
            int32_t jr[kEUnroll];
#pragma unroll
            for (int v = 0; v < kEUnroll; v++)
                jr[v] = k0 + (int64_t)blockDim.x * v < bb + oo ? ld_stream(col_push + k0 + blockDim.x * v, stream) : 0;
#pragma unroll
            for (int v = 0; v < kEUnroll; v++)
                if (k0 + (int64_t)blockDim.x * v < bb + oo) add(jr[v], ss);
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kHubSlots; q += blockDim.x)
        if (s_hacc[q] != (T)0) red_keep(&F[__ldg(hub_ids + q)], s_hacc[q], keep);
    e_loc = block_sum(e_loc, scratch);
    pushed = block_sum(pushed, scratch_u);
    visited = block_sum(visited, scratch_u);
    if (threadIdx.x == 0) {
        if (e_loc != 0.0) atomicAdd(&ctl->e, e_loc);
        if (pushed) atomicAdd(&ctl->pushed, pushed);
        if (visited) atomicAdd(&ctl->visited, visited);
    }
}

// E-level pre-diffusion of a large level through the windowed push: the level's nodes are
// id-sorted (the graph build sorts E by level, then id), so a block takes kSelChunk-id chunks,
// finds the level's nodes in each by binary search, visits them (no node of E has a self-loop:
// transit = F_i, share d F_i / out_i) and writes their frontier entries as one id-sorted segment
// per chunk, with the same records the sweep's selection writes; k_push_win then pushes them.
// Nodes above the heavy cut-off go to the heavy list as in the selection.
__global__ void __launch_bounds__(256) k_e_select(const int32_t *nodes, int32_t count, float *F, double *H,
                                                  const int32_t *out_info, int32_t n, SolveCtl *ctl,
                                                  int32_t *front_id, float *front_s, int32_t *heavy_id,
                                                  float *heavy_s, int32_t *heavy_cstart, int32_t *heavy_chunk,
                                                  int4 *chunks, int win_mean_bits, int heavy_cut, int heavy_len,
                                                  int seg_cap) {
    constexpr int kPerWarp = kSelChunk / 8;   // a chunk holds at most kSelChunk nodes of a level
    __shared__ int32_t s_id[8][kPerWarp];
    __shared__ float s_sh[8][kPerWarp];
    __shared__ int s_range[2];
    __shared__ int s_wcount[8], s_wbase[8];
    __shared__ float s_wabs[8];
    __shared__ int s_base;
    __shared__ double scratch[32];
    __shared__ unsigned long long scratch_u[32];
    const float d_f = (float)ctl->d;
    const unsigned lane = lane_id(), lt = lanemask_lt();
    const int warp = threadIdx.x >> 5;
    float e_run = 0.f;
    unsigned long long pushed = 0, visited = 0;
    const int nchunk = (n + kSelChunk - 1) / kSelChunk;
    for (int c = blockIdx.x; c < nchunk; c += gridDim.x) {
        if (threadIdx.x < 2) {
            // first list entry with id >= (c + threadIdx.x) * kSelChunk
            const int64_t key = (int64_t)(c + (int)threadIdx.x) * kSelChunk;
            int lo = 0, hi = count;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (nodes[mid] < key) lo = mid + 1; else hi = mid;
            }
            s_range[threadIdx.x] = lo;
        }
        __syncthreads();
        const int e0 = s_range[0], e1 = s_range[1];
        if (e1 <= e0) {
            __syncthreads();   // s_range is rewritten for the next chunk
            continue;
        }
        // warp w visits the contiguous run [w0, w1) of the chunk's entries, in order
        const int per = (e1 - e0 + 7) / 8;
        const int w0 = min(e1, e0 + warp * per), w1 = min(e1, w0 + per);
        int nl = 0;
        float wabs = 0.f;
        for (int k0 = w0; k0 < w1; k0 += 32) {
            const int k = k0 + (int)lane;
            bool light = false;
            int32_t u = 0;
            float share = 0.f;
            if (k < w1) {
                u = nodes[k];
                const float f = F[u];
                const int32_t o = out_info[u] & 0x7fffffff;
                F[u] = 0.f;
                H[u] += widen(f);
                visited++;
                pushed += (unsigned long long)o;
                share = o ? __fdividef(f, (float)o) * d_f : 0.f;
                if (o == 0) {
                    e_run += f;
                } else if (o > heavy_cut) {
                    const int p = atomicAdd(&ctl->heavy_count, 1);
                    heavy_id[p] = u;
                    heavy_s[p] = share;
                    const int nch = (o + heavy_len - 1) / heavy_len;
                    const int cs = atomicAdd(&ctl->heavy_chunks, nch);
                    heavy_cstart[p] = cs;
                    for (int q = 0; q < nch; q++) heavy_chunk[cs + q] = p;
                } else {
                    light = true;
                }
            }
            const unsigned bl = __ballot_sync(kFull, light);
            if (light) {
                const int p = nl + __popc(bl & lt);
                s_id[warp][p] = u;
                s_sh[warp][p] = share;
                wabs += fabsf(share);
            }
            nl += __popc(bl);
        }
        wabs = warp_sum(wabs);
        if (lane == 0) {
            s_wcount[warp] = nl;
            s_wabs[warp] = wabs;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int run = 0;
            float abs_tot = 0.f;
            for (int w = 0; w < 8; w++) {
                s_wbase[w] = run;
                run += s_wcount[w];
                abs_tot += s_wabs[w];
            }
            s_base = 0;
            if (run) {
                // one atomic reserves the chunk's frontier entries and its segment slot
                const unsigned long long fc = atomicAdd(&ctl->front_chunks, (1ull << kFrontBits) | (unsigned)run);
                s_base = front_entries(fc);
                chunks[segment_slot(ctl, run, seg_cap)] = make_int4(c * kSelChunk, s_base, run,
                                                       window_exponent(abs_tot / (float)run, win_mean_bits));
            }
        }
        __syncthreads();
        const int cb = s_base + s_wbase[warp];
        for (int k = (int)lane; k < nl; k += 32) {
            front_id[cb + k] = s_id[warp][k];
            front_s[cb + k] = s_sh[warp][k];
        }
        __syncthreads();   // staging and s_range are reused by the next chunk
    }
    const double e_loc = block_sum((double)e_run, scratch);
    pushed = block_sum(pushed, scratch_u);
    visited = block_sum(visited, scratch_u);
    if (threadIdx.x == 0) {
        if (e_loc != 0.0) atomicAdd(&ctl->e, e_loc);
        if (pushed) atomicAdd(&ctl->pushed, pushed);
        if (visited) atomicAdd(&ctl->visited, visited);
    }
}

constexpr int64_t kELevelSelectMin = 16384;   // levels of E at least this large ...
constexpr int64_t kELevelDensity = 512;        // ... and this dense (nodes per kSelChunk ids) take k_e_select

// Clears the frontier counters after a pre-diffusion level's push (the sweeps' reduction does
// this after every sweep).
__global__ void k_front_reset(SolveCtl *ctl) {
    ctl->front_total += (unsigned long long)(front_entries(ctl->front_chunks) + ctl->heavy_count);
    ctl->front_chunks = 0;
    ctl->big_segs = 0;
    ctl->small_segs = 0;
    ctl->heavy_count = 0;
    ctl->heavy_chunks = 0;
    ctl->chunk_next = 0;
}

// Push, one warp per batch of 32 frontier entries (no block barriers). Rows of PushTune::row links or
// more go one at a time over the whole warp, 32 consecutive links per load. For the others the
// warp scans their degrees, then each lane takes kPushVT contiguous links of their concatenated
// links per round, finds their owner once (binary search over the warp's 33 offsets in shared
// memory) and keeps kPushVT independent index loads in flight before its atomic adds.
constexpr int kPushVT = 4;   // measured on GB300: 4 beats 2, 8 and 16 (fewer registers, more blocks)
constexpr int kHeavyPushUnroll = 4;   // index loads in flight per lane in a heavy node's chunk

template <class T>
__global__ void __launch_bounds__(256) k_push(const int32_t *__restrict__ front_id, const T *__restrict__ front_s,
                                              const int32_t *__restrict__ heavy_id, const T *__restrict__ heavy_s,
                                              const int32_t *__restrict__ heavy_cstart,
                                              const int32_t *__restrict__ heavy_chunk,
                                              const int64_t *__restrict__ rp_out, const int32_t *__restrict__ col_out,
                                              T *F, SolveCtl *ctl, int heavy_len) {
    __shared__ int s_off[8][33];
    __shared__ int64_t s_beg[8][32];
    __shared__ int32_t s_u[8][32];
    __shared__ T s_s[8][32];
    if (ctl->done) return;
    const bool loops = ctl->plain_loops != 0;   // self-links pushed as plain links
    const uint64_t pol = policy_evict_last();
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + tid) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;

    // nodes with more than the heavy cut-off of links: their chunks over all warps
    const int hch = ctl->heavy_chunks;
    for (int64_t c = gwarp; c < hch; c += nwarps) {
        const int p = heavy_chunk[c];
        const int32_t u = heavy_id[p];
        const T sh = heavy_s[p];
        const int64_t cb = rp_out[u] + (int64_t)(c - heavy_cstart[p]) * heavy_len;
        const int64_t ce = min(cb + (int64_t)heavy_len, rp_out[u + 1]);
        for (int64_t k0 = cb + lane; k0 < ce; k0 += 32 * kHeavyPushUnroll) {
            int32_t j[kHeavyPushUnroll];
#pragma unroll
            for (int v = 0; v < kHeavyPushUnroll; v++) j[v] = k0 + 32 * v < ce ? __ldcs(col_out + k0 + 32 * v) : -1;
#pragma unroll
            for (int v = 0; v < kHeavyPushUnroll; v++)
                if (j[v] >= 0 && (j[v] != u || loops)) red_keep(&F[j[v]], sh, pol);
        }
    }

    const int count = front_entries(ctl->front_chunks);
    for (int64_t b0 = gwarp * 32; b0 < count; b0 += nwarps * 32) {
        const int64_t idx = b0 + lane;
        int deg = 0;
        if (idx < count) {
            const int32_t u = __ldcs(front_id + idx);
            const int64_t rb = __ldg(rp_out + u);
            deg = (int)(__ldg(rp_out + u + 1) - rb);
            s_u[w][lane] = u;
            s_s[w][lane] = __ldcs(front_s + idx);
            s_beg[w][lane] = rb;
        }
        const int inc = warp_inclusive_scan(deg);
        const int total = __shfl_sync(kFull, inc, 31);
        s_off[w][lane] = inc - deg;
        if (lane == 31) s_off[w][32] = total;
        __syncwarp();
        for (int e0 = lane * kPushVT; e0 < total; e0 += 32 * kPushVT) {
            int lo = 0, hi = 31;   // last entry k with s_off[k] <= e0
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_off[w][mid] <= e0) lo = mid; else hi = mid - 1;
            }
            int k = lo;
            int next = s_off[w][k + 1];
            int32_t j[kPushVT];
            int own[kPushVT];
#pragma unroll
            for (int v = 0; v < kPushVT; v++) {
                const int e = e0 + v;
                own[v] = -1;
                if (e < total) {
                    while (next <= e) next = s_off[w][++k + 1];
                    own[v] = k;
                    j[v] = __ldcs(col_out + s_beg[w][k] + (e - s_off[w][k]));
                }
            }
#pragma unroll
            for (int v = 0; v < kPushVT; v++)
                if (own[v] >= 0 && (j[v] != s_u[w][own[v]] || loops)) red_keep(&F[j[v]], s_s[w][own[v]], pol);
        }
        __syncwarp();
    }
}

// Push with a shared-memory window (FP32 fluid). The select emits the frontier as id-sorted
// segments of kSelChunk consecutive source nodes; a block takes one segment at a time and adds
// every link whose target lies within kHalo ids of the segment (host locality: most web links
// stay near their source) into a window of kWin slots in shared memory, sending only the other
// links straight to F. The window holds integers: each entry's share in the segment's fixed
// point (window_exponent), added with native 32-bit shared atomics; FP32 shared atomics would be
// compare-and-swap loops. The window then goes to F, converted back to FP32, with one four-float
// atomic per non-zero group, so a dense segment issues a fraction of the global atomics of a
// link-by-link push. Shares too large for the segment's fixed point take the direct path, and
// links into hubs always go to the hub cache (the window's overflow bound leaves hubs out).
constexpr int kHubCopies = 1;   // copies of the push's shared-memory hub cache
constexpr int kHalo = 768;
constexpr int kWin = kSelChunk + 2 * kHalo;     // 3584 int32 slots, 14 KB
constexpr int kWinMinEntries = 24;              // sparser segments push link by link
// Resident blocks per SM the registers are capped for: the kernel waits on memory and gains from
// more warps in flight. Measured on GB300: 7 blocks (32 registers) beat 6 and 5, and 8 blocks,
// which the 14 KB window of a 768-id halo fits in shared memory, beat 7 with the 16 KB window of
// a 1024-id halo (149.0 against 153.1 us per launch; the narrower halo misses few local links).
constexpr int kPushWinBlocks = 8;

__global__ void __launch_bounds__(256, kPushWinBlocks) k_push_win(const int32_t *__restrict__ front_id, const float *__restrict__ front_s,
                                                  const int32_t *__restrict__ heavy_id, const float *__restrict__ heavy_s,
                                                  const int32_t *__restrict__ heavy_cstart,
                                                  const int32_t *__restrict__ heavy_chunk,
                                                  const int32_t *__restrict__ rp_push,
                                                  const int32_t *__restrict__ col_push, const int4 *__restrict__ chunks,
                                                  const int32_t *__restrict__ hub_ids, float *F, SolveCtl *ctl,
                                                  int win_qmax, int push_row, int heavy_len, int seg_cap) {
    __shared__ __align__(16) int s_win[kWin];
    // this block's pending additions to the hubs, kHubCopies copies for alternating warps (the
    // hubs are the hottest addresses, and FP32 shared atomics retry when another lane wrote first)
    __shared__ float s_hacc[kHubCopies][kHubSlots];
    __shared__ int s_off[8][33];
    // per entry of a warp's batch: {row start - link offset, share, fixed-point share, unused}
    __shared__ int4 s_rec[8][32];
    __shared__ int s_chunk, s_batch;
    if (ctl->done) return;
    const bool loops = ctl->plain_loops != 0;   // self-links pushed as plain links
    const uint64_t keep = policy_evict_last(), stream = policy_evict_first();
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + tid) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int q = tid; q < kHubCopies * kHubSlots; q += 256) (&s_hacc[0][0])[q] = 0.f;
    __syncthreads();
    float *my_hacc = s_hacc[w % kHubCopies];
    // a link to a far target (jr: target id with bit 31 set when the target is a hub): hubs
    // (high in-degree nodes) collect in shared memory, the rest goes to F directly
    auto far_add = [&](int32_t jr, float v) {
        if (jr < 0) atomicAdd(&my_hacc[hub_slot(jr & 0x7fffffff)], v);
        else red_keep(&F[jr], v, keep);
    };
    // The hub cache stays FP32 (compare-and-swap atomics): integer hub slots, folded into FP32
    // at every segment's end so that a per-segment bound keeps them from overflowing, were
    // measured slower (the fold of every slot per segment costs more than the loops it saves).

    // nodes with more than the heavy cut-off of links: their chunks over all warps
    const int hch = ctl->heavy_chunks;
    for (int64_t c = gwarp; c < hch; c += nwarps) {
        const int p = heavy_chunk[c];
        const int32_t u = heavy_id[p];
        const float sh = heavy_s[p];
        const int64_t cb = (__ldg(rp_push + u) & 0x7fffffff) + (int64_t)(c - heavy_cstart[p]) * heavy_len;
        const int64_t ce = min(cb + (int64_t)heavy_len, (int64_t)(__ldg(rp_push + u + 1) & 0x7fffffff));
        for (int64_t k0 = cb + lane; k0 < ce; k0 += 32 * kHeavyPushUnroll) {
            int32_t jr[kHeavyPushUnroll];
#pragma unroll
            for (int v = 0; v < kHeavyPushUnroll; v++) jr[v] = k0 + 32 * v < ce ? ld_stream(col_push + k0 + 32 * v, stream) : 0;
#pragma unroll
            for (int v = 0; v < kHeavyPushUnroll; v++)
                if (k0 + 32 * v < ce && ((jr[v] & 0x7fffffff) != u || loops)) far_add(jr[v], sh);
        }
    }

    const int nchunks = front_segments(ctl->front_chunks);
    for (;;) {
        if (tid == 0) {
            s_chunk = atomicAdd(&ctl->chunk_next, 1);
            s_batch = 0;
        }
        __syncthreads();
        const int ci = s_chunk;
        if (ci >= nchunks) break;
        const int4 ch = chunks[segment_at(ctl, ci, seg_cap)];
        const int cstart = ch.y, clen = ch.z;
        const bool use_win = clen >= kWinMinEntries;
        const float win_scale = pow2f(ch.w), win_unit = pow2f(-ch.w);   // fixed point <-> FP32
        const int lo = max(0, ch.x - kHalo) & ~3;
        if (use_win) {
            for (int q = tid; q < kWin / 4; q += 256) reinterpret_cast<int4 *>(s_win)[q] = make_int4(0, 0, 0, 0);
            __syncthreads();
        }
        for (;;) {
            // warps claim 32-entry batches of the segment
            int b0 = 0;
            if (lane == 0) b0 = atomicAdd(&s_batch, 32);
            b0 = __shfl_sync(kFull, b0, 0);
            if (b0 >= clen) break;
            const int idx = cstart + b0 + lane;
            int deg = 0;
            int32_t eu = 0;
            float es = 0.f;
            int ebeg = 0;   // links stay below 2^31
            if (b0 + lane < clen) {
                eu = __ldcs(front_id + idx);
                es = __ldcs(front_s + idx);
                // bit 31 of the row end: a loop node, whose row ends with its self-link; diffused
                // in closed form (the self-link is not a plain link), the row stops one link short
                ebeg = __ldg(rp_push + eu) & 0x7fffffff;
                const int32_t end = __ldg(rp_push + eu + 1);
                deg = (end & 0x7fffffff) - ebeg - (loops ? 0 : (int)((uint32_t)end >> 31));
            }
            // the share in the segment's fixed point; 0 (never added to the window) when it
            // does not fit, so its local links go to F directly
            int eq = __float2int_rn(es * win_scale);
            const bool ewin = use_win && eq > -win_qmax && eq < win_qmax;
            if (!ewin) eq = 0;
            // rows of push_row links or more: one row at a time over the whole warp, 32
            // consecutive links per load, no owner lookup
            const bool row = deg >= push_row;
            for (unsigned rows = __ballot_sync(kFull, row); rows; rows &= rows - 1) {
                const int src = __ffs(rows) - 1;
                const int rb = __shfl_sync(kFull, ebeg, src);
                const int rd = __shfl_sync(kFull, deg, src);
                const float rs = __shfl_sync(kFull, es, src);
                const int rq = __shfl_sync(kFull, eq, src);
                for (int k0 = lane; k0 < rd; k0 += 32 * kPushVT) {
                    int32_t jr[kPushVT];
#pragma unroll
                    for (int v = 0; v < kPushVT; v++) jr[v] = k0 + 32 * v < rd ? ld_stream(col_push + rb + k0 + 32 * v, stream) : 0;
#pragma unroll
                    for (int v = 0; v < kPushVT; v++) {
                        if (k0 + 32 * v >= rd) continue;
                        const unsigned off = (unsigned)((jr[v] & 0x7fffffff) - lo);
                        if (rq != 0 && jr[v] >= 0 && off < (unsigned)kWin) atomicAdd(&s_win[off], rq);
                        else far_add(jr[v], rs);
                    }
                }
            }
            // the other entries, compacted (each has at least one link): kPushVT contiguous links
            // per lane over their concatenated rows
            const int dsm = row ? 0 : deg;
            const unsigned small = __ballot_sync(kFull, dsm > 0);
            if (!small) continue;
            const int inc = warp_inclusive_scan(dsm);
            const int total = __shfl_sync(kFull, inc, 31);
            const int rbase = (int)ebeg - (inc - dsm);   // link e of the batch sits at col_push[rbase + e]
            s_off[w][lane + 1] = INT_MAX;
            __syncwarp();
            if (dsm > 0) {
                const int pos = __popc(small & lanemask_lt());
                s_off[w][pos] = inc - dsm;
                s_rec[w][pos] = make_int4(rbase, __float_as_int(es), eq, 0);
            }
            if (lane == 0) s_off[w][__popc(small)] = total;
            __syncwarp();
            for (int e0 = lane * kPushVT; e0 < total; e0 += 32 * kPushVT) {
                int k = 0;   // last entry with s_off[k] <= e0
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                    if (s_off[w][k + step] <= e0) k += step;
                // the owner's record in registers; every entry has at least one link, so moving
                // to the next link crosses at most one entry boundary
                int next = s_off[w][k + 1];
                int4 rec = s_rec[w][k];
                int32_t jr[kPushVT], qq[kPushVT];
                float ss[kPushVT];
#pragma unroll
                for (int v = 0; v < kPushVT; v++) {
                    const int e = e0 + v;
                    jr[v] = 0;
                    ss[v] = 0.f;
                    qq[v] = 0;
                    if (e < total) {
                        if (e >= next) {
                            ++k;
                            next = s_off[w][k + 1];
                            rec = s_rec[w][k];
                        }
                        jr[v] = ld_stream(col_push + rec.x + e, stream);
                        ss[v] = __int_as_float(rec.y);
                        qq[v] = rec.z;
                    }
                }
#pragma unroll
                for (int v = 0; v < kPushVT; v++) {
                    if (e0 + v >= total) continue;
                    const unsigned off = (unsigned)((jr[v] & 0x7fffffff) - lo);
                    if (qq[v] != 0 && jr[v] >= 0 && off < (unsigned)kWin) atomicAdd(&s_win[off], qq[v]);
                    else far_add(jr[v], ss[v]);
                }
            }
            __syncwarp();
        }
        __syncthreads();
        if (use_win) {
            for (int q = tid; q < kWin / 4; q += 256) {
                const int4 v = reinterpret_cast<const int4 *>(s_win)[q];
                if (v.x != 0 || v.y != 0 || v.z != 0 || v.w != 0)
                    red_keep_v4(F + lo + 4 * q, make_float4((float)v.x * win_unit, (float)v.y * win_unit,
                                                            (float)v.z * win_unit, (float)v.w * win_unit), keep);
            }
            __syncthreads();
        }
    }
    // one atomic per hub that received something from this block
    for (int q = tid; q < kHubSlots; q += 256) {
        float v = 0.f;
#pragma unroll
        for (int c = 0; c < kHubCopies; c++) v += s_hacc[c][q];
        if (v != 0.f) red_keep(&F[__ldg(hub_ids + q)], v, keep);
    }
}

// ------------------------------------------------------------------------------------------
// double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32 numbers (about 44
// significant bits). Sums use Knuth's error-free two-sum, products an FMA-based exact product
// (Dekker's double-length arithmetic); both renormalise with a fast two-sum. The pull kernels
// accumulate this way instead of in FP64, whose throughput on this part is a small fraction of
// the FP32 rate.
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float bb = s - a.x;
    float e = (a.x - (s - bb)) + (b.x - bb);
    e += a.y + b.y;
    const float hi = s + e;
    return make_float2(hi, e - (hi - s));
}
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float hi = p + e;
    return make_float2(hi, e - (hi - p));
}
__device__ __forceinline__ float2 df_from(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}
__device__ __forceinline__ double df_to(float2 a) { return (double)a.x + (double)a.y; }

// c[j] = d / out_j as double-float (0 for a dangling node)
__global__ void k_link_weight(const int32_t *out_info, int32_t n, double d, float2 *c) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = out_info[i] & 0x7fffffff;
        c[i] = df_from(o ? d / (double)o : 0.0);
    }
}

// y[j] = v[j] * c[j] in double-float (refinement: v = H, c = d / out)
__global__ void k_scale(const double *v, const float2 *c, int32_t n, float2 *y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = df_mul(df_from(v[i]), c[i]);
}

__global__ void k_df_to_double(const float2 *X, int32_t n, double *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = df_to(X[i]);
}

// Accumulation types of the pull kernels: the gathered value y and the row sums are FP32
// (power iteration's increments), double-float (the exact residual) or FP64 (power iteration in
// FP64). Heavy-row chunk sums are always formed in the Wide type (double-float for the FP32 and
// double-float values, FP64 for FP64) and narrowed when the row is finished.
struct AccDF {
    using V = float2;
    using Wide = AccDF;
    __device__ static V zero() { return make_float2(0.f, 0.f); }
    __device__ static V add(V a, V b) { return df_add(a, b); }
    __device__ static V shfl_up(V v, int off) {
        return make_float2(__shfl_up_sync(kFull, v.x, off), __shfl_up_sync(kFull, v.y, off));
    }
    __device__ static V shfl(V v, int src) { return make_float2(__shfl_sync(kFull, v.x, src), __shfl_sync(kFull, v.y, src)); }
    __device__ static V shfl_xor(V v, int o) {
        return make_float2(__shfl_xor_sync(kFull, v.x, o), __shfl_xor_sync(kFull, v.y, o));
    }
    __device__ static float2 widen(V v) { return v; }
    __device__ static V narrow(float2 w) { return w; }
};
struct AccF32 {
    using V = float;
    using Wide = AccDF;
    __device__ static V zero() { return 0.f; }
    __device__ static V add(V a, V b) { return a + b; }
    __device__ static V shfl_up(V v, int off) { return __shfl_up_sync(kFull, v, off); }
    __device__ static V shfl(V v, int src) { return __shfl_sync(kFull, v, src); }
    __device__ static V shfl_xor(V v, int o) { return __shfl_xor_sync(kFull, v, o); }
    __device__ static float2 widen(V v) { return make_float2(v, 0.f); }
    __device__ static V narrow(float2 w) { return w.x + w.y; }
};
struct AccF64 {
    using V = double;
    using Wide = AccF64;
    __device__ static V zero() { return 0.0; }
    __device__ static V add(V a, V b) { return a + b; }
    __device__ static V shfl_up(V v, int off) { return __shfl_up_sync(kFull, v, off); }
    __device__ static V shfl(V v, int src) { return __shfl_sync(kFull, v, src); }
    __device__ static V shfl_xor(V v, int o) { return __shfl_xor_sync(kFull, v, o); }
    __device__ static double widen(V v) { return v; }
    __device__ static V narrow(double w) { return w; }
};

// partial[c] = sum of y over the in-links of heavy-row chunk c, in Acc's wide type
constexpr int kHeavyPullUnroll = 8;

template <class Acc>
__global__ void k_pull_heavy(const int64_t *rp_in, const int32_t *col_in, const int32_t *heavy_rows,
                             const int32_t *chunk_off, const int32_t *chunk_row, int32_t n_chunks,
                             const typename Acc::V *y0, const typename Acc::V *y1, const SolveCtl *ctl, int alternate,
                             typename Acc::Wide::V *partial) {
    using V = typename Acc::V;
    using W = typename Acc::Wide;
    const V *y = (alternate && (ctl->sweeps & 1)) ? y1 : y0;
    const int lane = (int)lane_id();
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < n_chunks; c += nwarps) {
        const int32_t h = chunk_row[c];
        const int32_t row = heavy_rows[h];
        const int64_t b = rp_in[row] + (int64_t)(c - chunk_off[h]) * kPullChunk;
        const int64_t e = min(b + (int64_t)kPullChunk, rp_in[row + 1]);
        typename W::V s = W::zero();
        // kHeavyPullUnroll index loads, then as many gathers, in flight before the additions
        for (int64_t k0 = b + lane; k0 < e; k0 += 32 * kHeavyPullUnroll) {
            int32_t j[kHeavyPullUnroll];
#pragma unroll
            for (int v = 0; v < kHeavyPullUnroll; v++) j[v] = k0 + 32 * v < e ? __ldcs(col_in + k0 + 32 * v) : -1;
            V val[kHeavyPullUnroll];
#pragma unroll
            for (int v = 0; v < kHeavyPullUnroll; v++) val[v] = j[v] >= 0 ? y[j[v]] : Acc::zero();
#pragma unroll
            for (int v = 0; v < kHeavyPullUnroll; v++) s = W::add(s, Acc::widen(val[v]));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = W::add(s, W::shfl_xor(s, o));
        if (lane == 0) partial[c] = s;
    }
}

enum { PULL_RESID = 1, PULL_INC = 2, PULL_PI64 = 3 };

// Row sums acc_i = sum_{j in in(i)} y_j for 32 consecutive rows per warp (Acc's arithmetic), then:
//   PULL_RESID (double-float): F*_i = B_i + acc_i - H_i (FP64) -> F_i (as T); sum |F*| -> ctl->r.
//   PULL_INC   (FP32): power iteration in increment form, X_(k+1) - X_k = P (X_k - X_(k-1)):
//               y_j = d (X_k - X_(k-1))_j / out_j, so acc_i is the next increment; X_i (FP64)
//               += acc_i, y'_i = acc_i * c_i (c_i = d / out_i in FP32); sum |acc| ->
//               ctl->r (PI's ||X_(k+1) - X_k||_1), iteration count and the WHILE condition.
//   PULL_PI64  (FP64): X'_i = B_i + acc_i, delta_i = |X'_i - X_i|, X_i = X'_i, y'_i = X'_i * c_i
//               (c_i = d / out_i in FP64); sum delta -> ctl->r, iteration count, WHILE condition.
// Segmented sum over the links of 32 consecutive rows per warp. The rows' links are contiguous
// in col_in (unless the group holds a heavy row, below), so a round gives each lane VT
// contiguous links, read as 16-byte vectors, with their VT gathers in flight together:
//   1. the rows that start in the round mark their first link in a per-lane bit mask;
//   2. each lane forms the prefix sums of its links, restarting at every marked link;
//   3. one segmented scan across the lanes gives each lane the sum of the row that runs into
//      it from the left (and the round's carry into the next round);
//   4. the lane that holds a row's last link publishes that link's prefix (with the incoming sum
//      added when the row started before the lane) in shared memory, where the row's owner lane
//      reads it.
// A group holding a heavy row (summed apart in chunks) sums its other rows one at a time over
// the whole warp.
// Links per lane per round (a multiple of 4, at most 32), per accumulator.
constexpr int kPullVT = 8;
constexpr int kPullVTF32 = 8;
template <class Acc>
struct PullVT {
    static constexpr int value = sizeof(typename Acc::V) == 4 ? kPullVTF32 : kPullVT;
};
// Resident blocks per SM the registers are capped for (0: the compiler's own count). Measured on
// GB300: double-float 5 (a small spill) beats 4 by 1.4 %; FP32 at the compiler's own 64 registers
// (4 blocks) beats caps for 5 (3.5 %) and 6.
template <class Acc>
struct PullCfg {
    static constexpr int min_blocks = 5;
};
template <>
struct PullCfg<AccF32> {
    static constexpr int min_blocks = 0;
};
template <>
struct PullCfg<AccF64> {
    static constexpr int min_blocks = 3;
};

template <int MODE, class Acc, class T>
__global__ void __launch_bounds__(256, PullCfg<Acc>::min_blocks) k_pull(const int64_t *__restrict__ rp_in, const int32_t *__restrict__ col_in,
                                              const typename Acc::V *y0, typename Acc::V *y1, int32_t n,
                                              const int32_t *heavy_rows, const int32_t *heavy_chunk_off,
                                              const typename Acc::Wide::V *heavy_partial, int32_t n_heavy,
                                              const double *__restrict__ B, const void *__restrict__ cvec, void *Xvec,
                                              const double *H, T *F, double *partials, SolveCtl *ctl,
                                              cudaGraphConditionalHandle hcond, int set_cond, int stripes) {
    using V = typename Acc::V;
    using W = typename Acc::Wide;
    constexpr int VT = PullVT<Acc>::value;     // links per lane per round
    constexpr int RL = 32 * VT;                // links per warp per round
    static_assert(VT % 4 == 0 && VT <= 32, "a lane's links are 16-byte vectors of indices, its starts one word");
    __shared__ __align__(16) V s_pre[8][RL];   // at a row's last link: the row's sum
    __shared__ unsigned s_bits[8][32];                 // per lane: bit v set when its link v starts a row
    __shared__ double scratch[32];
    const int lane = (int)lane_id(), warp = threadIdx.x >> 5;
    const bool odd = (MODE != PULL_RESID) && (ctl->sweeps & 1);
    const V *y_in = odd ? y1 : y0;
    V *y_out = odd ? const_cast<V *>(y0) : y1;
    const uint64_t stream = policy_evict_first();
    double sum = 0.0;
    float run = 0.f;
    int runs = 0;
    // stripes = 1: each block walks its own contiguous stripe of row groups, its warps side by
    // side, so the gathers of nearby rows (most links stay near their source) find y in the SM's
    // L1; the host picks this when the stripes carry even numbers of links. stripes = 0: the
    // row groups are interleaved over the grid, which balances graphs whose links crowd into a
    // few id ranges. Every warp runs the same number of row groups, so the block stays converged.
    const int64_t groups = ((int64_t)n + 31) >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * 8;
    const int64_t per_block = (groups + gridDim.x - 1) / gridDim.x;
    const int64_t g_lo = stripes ? blockIdx.x * per_block : 0;
    const int64_t g_hi = stripes ? min(groups, g_lo + per_block) : groups;
    const int64_t rounds = stripes ? (per_block + 7) / 8 : (groups + nwarps - 1) / nwarps;
    for (int64_t rd = 0; rd < rounds; rd++) {
        const int64_t grp = stripes ? g_lo + rd * 8 + warp : rd * nwarps + blockIdx.x * 8 + warp;
        const int64_t row = grp * 32 + lane;
        const bool valid = grp < g_hi && row < n;
        int64_t beg = 0;
        int deg = 0;
        bool heavy = false;
        if (valid) {
            beg = rp_in[row];
            const int64_t dd = rp_in[row + 1] - beg;
            heavy = dd > kPullHeavy;
            deg = heavy ? 0 : (int)dd;
        }
        V a = Acc::zero();
        if (!__any_sync(kFull, heavy)) {
            const int inc = warp_inclusive_scan(deg);
            const int total = __shfl_sync(kFull, inc, 31);
            const int start = inc - deg, last = inc - 1;   // the row's first and last link in the group
            // link e of the group sits at col_in[gbase + e]; rounds start pre links early so that
            // every lane's run is 16-byte aligned (col_in is padded past L; links before 0 or
            // from total on are read but not used)
            const int64_t gbase = __shfl_sync(kFull, beg, 0);
            const int pre = total > 0 ? (int)(gbase & 3) : 0;
            V carry = Acc::zero();
            for (int e0 = -pre; e0 < total; e0 += RL) {
                const int first = e0 + lane * VT;
                s_bits[warp][lane] = 0u;
                __syncwarp();
                if (deg > 0 && start >= e0 && start < e0 + RL)
                    atomicOr(&s_bits[warp][(start - e0) / VT], 1u << ((start - e0) % VT));
                int32_t j[VT];
                if (first < total) {
#pragma unroll
                    for (int q = 0; q < VT / 4; q++) {
                        const int4 jq = ld_stream4(col_in + gbase + first + 4 * q, stream);
                        j[4 * q] = jq.x;
                        j[4 * q + 1] = jq.y;
                        j[4 * q + 2] = jq.z;
                        j[4 * q + 3] = jq.w;
                    }
                }
                V val[VT];
#pragma unroll
                for (int v = 0; v < VT; v++)
                    val[v] = (first + v >= 0 && first + v < total) ? y_in[j[v]] : Acc::zero();
                __syncwarp();
                const unsigned m = s_bits[warp][lane];
                // prefix sums of the lane's links, restarting where a row starts
#pragma unroll
                for (int v = 1; v < VT; v++)
                    if (!(m >> v & 1u)) val[v] = Acc::add(val[v - 1], val[v]);
                // segmented inclusive scan of the lanes' last prefixes: S = the open row's sum at
                // the lane's end; f = some row starts in this lane or one to its left
                V S = val[VT - 1];
                bool f = m != 0u;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const V o = Acc::shfl_up(S, off);
                    const bool fo = __shfl_up_sync(kFull, f, off);
                    if (lane >= off) {
                        if (!f) S = Acc::add(o, S);
                        f = f || fo;
                    }
                }
                if (!f) S = Acc::add(carry, S);   // still the row carried in from the last round
                V cin = Acc::shfl_up(S, 1);
                if (lane == 0) cin = carry;
                carry = Acc::shfl(S, 31);
                // a row ends before every start, at the group's last link, and possibly at the
                // lane's last link: those positions publish the row's sum
                unsigned ends = (m >> 1) | (1u << (VT - 1));
                if (total - 1 >= first && total - 1 < first + VT) ends |= 1u << (total - 1 - first);
                const int fs = m ? __ffs(m) - 1 : VT;   // links before it continue the row from the left
#pragma unroll
                for (int v = 0; v < VT; v++)
                    if (ends >> v & 1u) s_pre[warp][lane * VT + v] = v < fs ? Acc::add(cin, val[v]) : val[v];
                __syncwarp();
                // the row whose last link is in this round takes its sum there
                if (deg > 0 && last >= e0 && last < e0 + RL) a = s_pre[warp][last - e0];
                __syncwarp();
            }
        } else {
            // a heavy row's links are not in the run: the other rows one at a time over the warp
            for (unsigned rows = __ballot_sync(kFull, deg > 0); rows; rows &= rows - 1) {
                const int k = __ffs(rows) - 1;
                const int64_t b = __shfl_sync(kFull, beg, k);
                const int dk = __shfl_sync(kFull, deg, k);
                V s = Acc::zero();
                for (int t = lane; t < dk; t += 32) s = Acc::add(s, y_in[ld_stream(col_in + b + t, stream)]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) s = Acc::add(s, Acc::shfl_xor(s, o));
                if (lane == k) a = s;
            }
        }
        if (heavy) {
            int lo = 0, hi = n_heavy - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (heavy_rows[mid] < row) lo = mid + 1; else hi = mid;
            }
            typename W::V wa = W::zero();
            for (int c = heavy_chunk_off[lo]; c < heavy_chunk_off[lo + 1]; c++) wa = W::add(wa, heavy_partial[c]);
            a = Acc::narrow(wa);
        }
        if (valid) {
            if constexpr (MODE == PULL_RESID) {
                const double fs = B[row] + df_to(AccDF::widen(a)) - H[row];
                F[row] = (T)fs;
                sum += fabs(fs);
            } else if constexpr (MODE == PULL_INC) {
                double *X = static_cast<double *>(Xvec);
                X[row] += (double)a;
                run += fabsf(a);
                y_out[row] = a * static_cast<const float *>(cvec)[row];
            } else {
                double *X = static_cast<double *>(Xvec);
                const double xn = B[row] + a;
                sum += fabs(xn - X[row]);
                X[row] = xn;
                y_out[row] = xn * static_cast<const double *>(cvec)[row];
            }
            if (++runs == 16) {
                sum += (double)run;
                run = 0.f;
                runs = 0;
            }
        }
    }
    sum += (double)run;
    double tot;
    if (!finish_sum(sum, partials, ctl, scratch, tot)) return;
    if (threadIdx.x == 0) {
        ctl->ticket = 0;
        ctl->r = tot;
        if (MODE != PULL_RESID) {
            const int it = ctl->sweeps + 1;
            ctl->sweeps = it;
            if (set_cond) ctl->body_runs++;
            const bool cont = tot > ctl->tol && it < ctl->max_sweeps;
            ctl->done = cont ? 0 : 1;
            if (set_cond) cudaGraphSetConditional(hcond, cont ? 1u : 0u);
        }
    }
}

// Power iteration in increment form, set-up: c_i = d / out_i (FP32, 0 for a dangling node),
// X_1 = B (the first iteration from X_0 = 0, FP64), y = c * B (the first increment
// X_1 - X_0 = B, scaled for the next pull); r = ||B||_1, one iteration done, and the halfway
// point of a refined solve (as the D-iteration's: sqrt(tol * r) when tol is well below r).
__global__ void k_pi_inc_init(const double *B, const int32_t *out_info, int32_t n, double d, float *c, double *X,
                              float *y, double *partials, SolveCtl *ctl) {
    __shared__ double scratch[32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = out_info[i] & 0x7fffffff;
        const float ci = o ? (float)(d / (double)o) : 0.f;
        const double b = B[i];
        c[i] = ci;
        X[i] = b;
        y[i] = (float)b * ci;
        s += fabs(b);
    }
    double tot;
    if (!finish_sum(s, partials, ctl, scratch, tot)) return;
    if (threadIdx.x == 0) {
        ctl->ticket = 0;
        ctl->r = tot;
        ctl->sweeps = 1;
        if (ctl->split && ctl->tol < kSplitBelow * tot) {
            ctl->tol = sqrt(ctl->tol * tot);
            ctl->halfway = 1;
        }
        ctl->split = 0;
        ctl->done = (tot > ctl->tol && 1 < ctl->max_sweeps) ? 0 : 1;
    }
}

// Continuation of the increment form from an exact residual F* = B + P.X - X (the next
// increment, computed exactly): X += F*, y = c * F*, one more iteration; y goes to the buffer
// the next pull reads (it alternates on the iteration count).
__global__ void k_pi_inc_resume(const float *Fs, int32_t n, const float *c, double *X, float *y0, float *y1,
                                SolveCtl *ctl) {
    const int it = ctl->sweeps + 1;
    float *y = (it & 1) ? y1 : y0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float f = Fs[i];
        X[i] += (double)f;
        y[i] = f * c[i];
    }
}

// FP64 power iteration set-up: c_i = d / out_i (FP64), X_0 = 0, y_0 = 0.
__global__ void k_pi64_init(const int32_t *out_info, int32_t n, double d, double *c, double *X, double *y0) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = out_info[i] & 0x7fffffff;
        c[i] = o ? d / (double)o : 0.0;
        X[i] = 0.0;
        y0[i] = 0.0;
    }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
Workspace::~Workspace() {
    reset_graphs();
    if (capture_stream) cudaStreamDestroy(capture_stream);
    if (out_stream) cudaStreamDestroy(out_stream);
    if (out_ready) cudaEventDestroy(out_ready);
    if (out_done) cudaEventDestroy(out_done);
    if (ctl_host) cudaFreeHost(ctl_host);
}

void Workspace::reset_graphs() {
    if (sweep_exec) cudaGraphExecDestroy(sweep_exec);
    if (pi_exec) cudaGraphExecDestroy(pi_exec);
    sweep_exec = nullptr;
    pi_exec = nullptr;
}

struct Launch {
    int sel_blocks, red_blocks, push_blocks, win_blocks, pull_blocks, pi_blocks, pi64_blocks, ew_blocks;
};

template <class T>
static Launch launch_shape(const di_graph *g) {
    Launch l;
    const int sms = g->dev.sms;
    int occ = 0;
    DI_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_push<T>, 256, 0));
    l.push_blocks = sms * (occ > 0 ? occ : 1);
    DI_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_push_win, 256, 0));
    l.win_blocks = sms * (occ > 0 ? occ : 1);
    DI_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pull<PULL_RESID, AccDF, T>, 256, 0));
    l.pull_blocks = sms * (occ > 0 ? occ : 1);
    DI_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pull<PULL_INC, AccF32, float>, 256, 0));
    l.pi_blocks = sms * (occ > 0 ? occ : 1);
    DI_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pull<PULL_PI64, AccF64, double>, 256, 0));
    l.pi64_blocks = sms * (occ > 0 ? occ : 1);
    const int64_t n = g->n;
    auto cap = [&](int64_t want, int64_t lim) { return (int)(want < 1 ? 1 : (want < lim ? want : lim)); };
    DI_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_select<T>, 256, 0));
    l.sel_blocks = cap((n + kSelChunk - 1) / kSelChunk, (int64_t)sms * (occ > 0 ? occ : 1));
    // two blocks per SM: most sweeps' reductions take r from the tracked sum, and a smaller grid
    // costs less to launch (measured: 2 per SM beat 4 and 1)
    l.red_blocks = cap((n + 255) / 256, (int64_t)(kReduceBlocks < sms * 2 ? kReduceBlocks : sms * 2));
    l.ew_blocks = cap((n + 255) / 256, (int64_t)sms * 8);
    // a pull block never needs more row groups than exist
    for (int *b : {&l.pull_blocks, &l.pi_blocks, &l.pi64_blocks}) {
        *b = cap(((n + 31) / 32 + 7) / 8, *b);
        if (*b > kReduceBlocks) *b = kReduceBlocks;
    }
    return l;
}

// 1 when `blocks` contiguous stripes of row groups carry even numbers of light in-links (the
// busiest stripe within kPullStripeSlack of the mean, from the build's samples of the link
// prefix), so each pull block may walk its own stripe; 0 keeps the groups interleaved.
constexpr double kPullStripeSlack = 1.5;
static int pull_stripes(const di_graph *g, int blocks) {
    const int64_t n = g->n, groups = (n + 31) / 32;
    const size_t S = g->pull_sample.size();
    if (blocks < 2 || groups < 8 * (int64_t)blocks || S < 2) return 0;
    const int64_t per = (groups + blocks - 1) / blocks;
    auto links_below = [&](int64_t row) {   // nearest sample at or below the row
        size_t k = (size_t)((double)row * (double)(S - 1) / (double)n);
        return g->pull_sample[k < S - 1 ? k : S - 1];
    };
    const double total = (double)(g->pull_sample[S - 1] - g->pull_sample[0]);
    if (total <= 0.0) return 0;
    double busiest = 0.0;
    for (int b = 0; b < blocks; b++) {
        const int64_t r0 = std::min(n, (int64_t)b * per * 32), r1 = std::min(n, ((int64_t)b + 1) * per * 32);
        busiest = std::max(busiest, (double)(links_below(r1) - links_below(r0)));
    }
    return busiest <= kPullStripeSlack * total / blocks ? 1 : 0;
}

// Records of frontier segments a selection can write (one per kSelChunk nodes, and one more).
static int seg_capacity(const di_graph *g) { return (int)(g->n / kSelChunk + 2); }

// The solve workspace's buffers in a fixed order, each with its size for a fluid of
// `fb` bytes per value (4: FP32, 8: FP64); `take(buffer, bytes)` allocates, binds or counts it.
template <class Take>
static void solve_layout(di_graph *g, Workspace &ws, size_t fb, Take &&take) {
    const size_t n = (size_t)g->n, nh = (size_t)g->n_heavy_out + 1;
    take(ws.F, fb * (n + 8));   // padded: window flushes write four floats at a time
    take(ws.chunks, sizeof(int4) * (size_t)seg_capacity(g));
    take(ws.H, sizeof(double) * n);
    take(ws.B, sizeof(double) * n);
    take(ws.front_id, sizeof(int32_t) * n);
    take(ws.front_s, fb * n);
    take(ws.heavy_id, sizeof(int32_t) * nh);
    take(ws.heavy_s, fb * nh);
    take(ws.heavy_cstart, sizeof(int32_t) * nh);
    // a heavy node has at most out / chunk + 1 chunks, chunk >= kHeavyChunkMin
    take(ws.heavy_chunk, sizeof(int32_t) * ((size_t)g->L / kHeavyChunkMin + nh));
    take(ws.partials, sizeof(double) * kReduceBlocks);
    take(ws.ctl, sizeof(SolveCtl));
    take(ws.y0, sizeof(float2) * n);   // also stages an FP64 vector (resume, final fluid)
    take(ws.y1, sizeof(float2) * n);
    take(ws.Bdf, sizeof(float2) * n);
    take(ws.cdf, sizeof(float2) * n);
    take(ws.Xdf, sizeof(float2) * n);
}

size_t solve_workspace_bytes(di_graph *g, int fluid) {
    Carve c;
    solve_layout(g, g->ws, fluid == DI_FLUID_F64 ? 8 : 4, [&](DevBuf &b, size_t n) { c.take(b, n); });
    return c.used;
}

// Attaches a caller's workspace (NULL: back to library allocations). The library's own solve
// buffers are freed at once, and the next solve lays its buffers out in the new memory.
void solve_workspace_attach(di_graph *g, void *ext, size_t bytes) {
    Workspace &ws = g->ws;
    ws.reset_graphs();   // the captured sweep graphs hold the old addresses
    solve_layout(g, ws, 8, [&](DevBuf &b, size_t) { b.release(); });
    ws.ext = ext;
    ws.ext_bytes = ext ? bytes : 0;
    ws.fluid = -1;
    ws.cdf_d = -1.0;
}

template <class T>
static void ensure_workspace(di_graph *g, Workspace &ws) {
    const int fl = sizeof(T) == 4 ? DI_FLUID_F32 : DI_FLUID_F64;
    if (ws.fluid == fl) return;
    ws.reset_graphs();
    if (ws.ext) {
        const size_t need = solve_workspace_bytes(g, fl);
        DI_REQUIRE(ws.ext_bytes >= need, DI_ERR_INVALID_ARG,
                   "the attached solve workspace holds %zu bytes; %s fluid needs %zu (di_workspace_size)",
                   ws.ext_bytes, fl == DI_FLUID_F64 ? "FP64" : "FP32", need);
        Carve c{static_cast<char *>(ws.ext), ws.ext_bytes};
        solve_layout(g, ws, sizeof(T), [&](DevBuf &b, size_t n) { c.take(b, n); });
    } else {
        solve_layout(g, ws, sizeof(T), [&](DevBuf &b, size_t n) { b.ensure(n); });
    }
    ws.cdf_d = -1.0;
    if (!ws.capture_stream) DI_CHECK_CUDA(cudaStreamCreateWithFlags(&ws.capture_stream, cudaStreamNonBlocking));
    if (!ws.out_stream) {
        DI_CHECK_CUDA(cudaStreamCreateWithFlags(&ws.out_stream, cudaStreamNonBlocking));
        DI_CHECK_CUDA(cudaEventCreateWithFlags(&ws.out_ready, cudaEventDisableTiming));
        DI_CHECK_CUDA(cudaEventCreateWithFlags(&ws.out_done, cudaEventDisableTiming));
    }
    if (!ws.ctl_host) DI_CHECK_CUDA(cudaMallocHost(&ws.ctl_host, sizeof(SolveCtl)));
    ws.fluid = fl;
}

template <class T>
static void launch_sweep_body(di_graph *g, Workspace &ws, const Launch &l, cudaStream_t s, cudaGraphConditionalHandle h, int set_cond,
                              KernelClock *kc, int parts) {
    SolveCtl *ctl = ws.ctl.as<SolveCtl>();
    KernelClock none(false, s);
    KernelClock &c = kc ? *kc : none;
    // a sweep is `parts` selections, each over a kSelChunk-aligned part of the node range with r
    // taken again before it (one part: r once per sweep, the paper's rule)
    const int64_t n = g->n;
    const int64_t chunks = (n + kSelChunk - 1) / kSelChunk;
    const int64_t per = (chunks + parts - 1) / parts;
    const PushTune tune = g->tune_single;
    for (int p = 0; p < parts; p++) {
        const int64_t lo = std::min(n, p * per * kSelChunk), hi = std::min(n, (p + 1) * per * kSelChunk);
        const bool last = p == parts - 1;
        const int64_t want = (hi - lo + kSelChunk - 1) / kSelChunk;
        const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>(want, l.sel_blocks));
        c.run(KC_SELECT, 1, [&] {
            k_select<T><<<blocks, 256, 0, s>>>(ws.F.as<T>(), ws.H.as<double>(), g->out_info.as<int32_t>(), g->n, ctl,
                                               ws.front_id.as<int32_t>(), ws.front_s.as<T>(), ws.heavy_id.as<int32_t>(),
                                               ws.heavy_s.as<T>(), ws.heavy_cstart.as<int32_t>(),
                                               ws.heavy_chunk.as<int32_t>(), ws.chunks.as<int4>(),
                                               g->win_qbits - kWinHeadBits, (int32_t)lo, (int32_t)hi, last ? 1 : 0,
                                               tune.heavy, tune.chunk, seg_capacity(g));
        });
        c.run(KC_PUSH, 1, [&] {
            if (sizeof(T) == 4) {
                k_push_win<<<l.win_blocks, 256, 0, s>>>(
                    ws.front_id.as<int32_t>(), ws.front_s.as<float>(), ws.heavy_id.as<int32_t>(), ws.heavy_s.as<float>(),
                    ws.heavy_cstart.as<int32_t>(), ws.heavy_chunk.as<int32_t>(), g->rp_push.as<int32_t>(),
                    g->col_push.as<int32_t>(), ws.chunks.as<int4>(), g->hub_ids.as<int32_t>(), ws.F.as<float>(), ctl,
                    1 << g->win_qbits, tune.row, tune.chunk, seg_capacity(g));
            } else {
                k_push<T><<<l.push_blocks, 256, 0, s>>>(ws.front_id.as<int32_t>(), ws.front_s.as<T>(),
                                                        ws.heavy_id.as<int32_t>(), ws.heavy_s.as<T>(),
                                                        ws.heavy_cstart.as<int32_t>(), ws.heavy_chunk.as<int32_t>(),
                                                        g->rp_out.as<int64_t>(), g->col_out.as<int32_t>(), ws.F.as<T>(),
                                                        ctl, tune.chunk);
            }
        });
        c.run(KC_REDUCE, 1, [&] {
            k_reduce<T><<<l.red_blocks, 256, 0, s>>>(ws.F.as<T>(), g->n, ws.partials.as<double>(), ctl, h, set_cond,
                                                     last ? 1 : 0);
        });
    }
}

// Graph: WHILE(cond, default 1 at every launch) { select; push; reduce -> cond }.
template <class T>
static void build_sweep_graph(di_graph *g, Workspace &ws, const Launch &l, int parts) {
    cudaGraph_t graph;
    DI_CHECK_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h;
    DI_CHECK_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    DI_CHECK_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    DI_CHECK_CUDA(cudaStreamBeginCaptureToGraph(ws.capture_stream, body, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal));
    launch_sweep_body<T>(g, ws, l, ws.capture_stream, h, 1, nullptr, parts);
    cudaGraph_t captured;
    DI_CHECK_CUDA(cudaStreamEndCapture(ws.capture_stream, &captured));
    DI_CHECK_CUDA(cudaGraphInstantiate(&ws.sweep_exec, graph, 0));
    DI_CHECK_CUDA(cudaGraphDestroy(graph));
    ws.sweep_parts = parts;
    ws.sweep_tune = g->tune_single;
}

// One power iteration: the heavy rows' chunk sums, then the pull. fp64: X_(k+1) = B + P X_k in
// FP64; otherwise the FP32 increment form.
static void launch_pi_body(di_graph *g, Workspace &ws, const Launch &l, cudaStream_t s, cudaGraphConditionalHandle h, int set_cond,
                           bool fp64, KernelClock *kc) {
    SolveCtl *ctl = ws.ctl.as<SolveCtl>();
    KernelClock none(false, s);
    KernelClock &c = kc ? *kc : none;
    if (g->n_heavy_in_chunks > 0) {
        int blocks = (int)((g->n_heavy_in_chunks + 7) / 8);
        if (blocks > g->dev.sms * 8) blocks = g->dev.sms * 8;
        c.run(KC_SELECT, 1, [&] {
            if (fp64)
                k_pull_heavy<AccF64><<<blocks, 256, 0, s>>>(
                    g->rp_in.as<int64_t>(), g->col_in.as<int32_t>(), g->heavy_in_rows.as<int32_t>(),
                    g->heavy_in_chunk_off.as<int32_t>(), g->heavy_in_chunk_row.as<int32_t>(), g->n_heavy_in_chunks,
                    ws.y0.as<double>(), ws.y1.as<double>(), ctl, 1, g->heavy_in_partial.as<double>());
            else
                k_pull_heavy<AccF32><<<blocks, 256, 0, s>>>(
                    g->rp_in.as<int64_t>(), g->col_in.as<int32_t>(), g->heavy_in_rows.as<int32_t>(),
                    g->heavy_in_chunk_off.as<int32_t>(), g->heavy_in_chunk_row.as<int32_t>(), g->n_heavy_in_chunks,
                    ws.y0.as<float>(), ws.y1.as<float>(), ctl, 1, g->heavy_in_partial.as<float2>());
        });
    }
    c.run(KC_PUSH, 1, [&] {
        if (fp64)
            k_pull<PULL_PI64, AccF64, double><<<l.pi64_blocks, 256, 0, s>>>(
                g->rp_in.as<int64_t>(), g->col_in.as<int32_t>(), ws.y0.as<double>(), ws.y1.as<double>(), g->n,
                g->heavy_in_rows.as<int32_t>(), g->heavy_in_chunk_off.as<int32_t>(), g->heavy_in_partial.as<double>(),
                g->n_heavy_in, ws.B.as<double>(), ws.Bdf.p, ws.Xdf.p, nullptr, (double *)nullptr,
                ws.partials.as<double>(), ctl, h, set_cond, pull_stripes(g, l.pi64_blocks));
        else
            k_pull<PULL_INC, AccF32, float><<<l.pi_blocks, 256, 0, s>>>(
                g->rp_in.as<int64_t>(), g->col_in.as<int32_t>(), ws.y0.as<float>(), ws.y1.as<float>(), g->n,
                g->heavy_in_rows.as<int32_t>(), g->heavy_in_chunk_off.as<int32_t>(), g->heavy_in_partial.as<float2>(),
                g->n_heavy_in, ws.B.as<double>(), ws.Bdf.p, ws.H.p, nullptr, (float *)nullptr,
                ws.partials.as<double>(), ctl, h, set_cond, pull_stripes(g, l.pi_blocks));
    });
}

// Graph: WHILE(cond) { [heavy chunk sums;] pull -> cond }, one per mode.
static void build_pi_graph(di_graph *g, Workspace &ws, const Launch &l, bool fp64) {
    cudaGraph_t graph;
    DI_CHECK_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h;
    DI_CHECK_CUDA(cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    DI_CHECK_CUDA(cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    DI_CHECK_CUDA(cudaStreamBeginCaptureToGraph(ws.capture_stream, body, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal));
    launch_pi_body(g, ws, l, ws.capture_stream, h, 1, fp64, nullptr);
    cudaGraph_t captured;
    DI_CHECK_CUDA(cudaStreamEndCapture(ws.capture_stream, &captured));
    DI_CHECK_CUDA(cudaGraphInstantiate(&ws.pi_exec, graph, 0));
    DI_CHECK_CUDA(cudaGraphDestroy(graph));
    ws.pi_fp64 = fp64 ? 1 : 0;
}

// F <- B + P.H - H (as T), ctl->r <- ||F*||_1 (exact residual of the history H: FP64 H and
// B, double-float link sums). Launches 2 or 3 kernels.
template <class T>
static void launch_refine(di_graph *g, Workspace &ws, const Launch &l, double d, cudaStream_t s) {
    SolveCtl *ctl = ws.ctl.as<SolveCtl>();
    if (ws.cdf_d != d) {   // d / out is formed once per damping factor
        k_link_weight<<<l.ew_blocks, 256, 0, s>>>(g->out_info.as<int32_t>(), g->n, d, ws.cdf.as<float2>());
        ws.cdf_d = d;
    }
    k_scale<<<l.ew_blocks, 256, 0, s>>>(ws.H.as<double>(), ws.cdf.as<float2>(), g->n, ws.y0.as<float2>());
    if (g->n_heavy_in_chunks > 0) {
        int blocks = (int)((g->n_heavy_in_chunks + 7) / 8);
        if (blocks > g->dev.sms * 8) blocks = g->dev.sms * 8;
        k_pull_heavy<AccDF><<<blocks, 256, 0, s>>>(g->rp_in.as<int64_t>(), g->col_in.as<int32_t>(),
                                                   g->heavy_in_rows.as<int32_t>(), g->heavy_in_chunk_off.as<int32_t>(),
                                                   g->heavy_in_chunk_row.as<int32_t>(), g->n_heavy_in_chunks,
                                                   ws.y0.as<float2>(), ws.y1.as<float2>(), ctl, 0,
                                                   g->heavy_in_partial.as<float2>());
    }
    k_pull<PULL_RESID, AccDF, T><<<l.pull_blocks, 256, 0, s>>>(
        g->rp_in.as<int64_t>(), g->col_in.as<int32_t>(), ws.y0.as<float2>(), ws.y1.as<float2>(), g->n,
        g->heavy_in_rows.as<int32_t>(), g->heavy_in_chunk_off.as<int32_t>(), g->heavy_in_partial.as<float2>(),
        g->n_heavy_in, ws.B.as<double>(), nullptr, nullptr, ws.H.as<double>(), ws.F.as<T>(), ws.partials.as<double>(),
        ctl, cudaGraphConditionalHandle(0), 0, pull_stripes(g, l.pull_blocks));
    DI_CHECK_CUDA(cudaGetLastError());
}

static void write_ctl(di_graph *g, Workspace &ws, double d, double tol, int schedule, int max_sweeps, int plain_loops,
                      cudaStream_t s, int track = 0, int split = 0) {
    SolveCtl &c = *ws.ctl_host;
    memset(&c, 0, sizeof(c));
    c.plain_loops = plain_loops;
    c.track = track;
    c.split = split;
    c.d = d;
    c.tol = tol;
    c.L = (double)g->L;
    c.schedule = schedule;
    c.max_sweeps = max_sweeps;
    c.last_selected = -1;
    DI_CHECK_CUDA(cudaMemcpyAsync(ws.ctl.p, &c, sizeof(SolveCtl), cudaMemcpyHostToDevice, s));
}

static void read_ctl(di_graph *g, Workspace &ws, cudaStream_t s) {
    DI_CHECK_CUDA(cudaMemcpyAsync(ws.ctl_host, ws.ctl.p, sizeof(SolveCtl), cudaMemcpyDeviceToHost, s));
    DI_CHECK_CUDA(cudaStreamSynchronize(s));
}

static void check_common(di_graph *g, const double *B, double d, double tol, const double *X_out) {
    DI_REQUIRE(g != nullptr, DI_ERR_INVALID_ARG, "graph is NULL");
    DI_REQUIRE(B != nullptr && X_out != nullptr, DI_ERR_INVALID_ARG, "B or X_out is NULL");
    DI_REQUIRE(d >= 0.0 && d < 1.0, DI_ERR_INVALID_ARG, "d must be in [0, 1) (got %g)", d);
    DI_REQUIRE(tol > 0.0 && std::isfinite(tol), DI_ERR_INVALID_ARG, "tol must be positive and finite (got %g)", tol);
}

// X may be copied on a second stream when it is device memory or pinned host memory (a copy to
// pageable memory would block the host thread before the refinement is launched).
static bool async_copy_target(const void *p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeManaged;
}

// A refined FP32 solve is split (write_ctl), so its first refinement is the halfway one.
static bool ctl_split_expected(bool fp32, int refine) { return fp32 && refine; }

template <class T>
static void solve_impl(di_graph *g, Workspace &ws, const double *B, double d, double tol, int schedule, int max_sweeps, int refine,
                       int host_loop, int profile, int e_prediffuse, int plain_loops, double *X_out,
                       double *residual_out, di_solve_info *info, cudaStream_t s, const double *H0 = nullptr,
                       const double *F0 = nullptr, double *F_out = nullptr, int parts = 1, int exact_r = 0) {
    ensure_workspace<T>(g, ws);
    const Launch l = launch_shape<T>(g);
    SolveCtl *ctl = ws.ctl.as<SolveCtl>();
    to_device(ws.B.p, B, sizeof(double) * (size_t)g->n, s);
    // r may be tracked between exact reductions while the fluid is nonnegative or nearly so:
    // FP32 sweeps from (0, B), up to and after their halfway refinement (see k_reduce: that
    // refinement comes before the fluid's rounding has grown comparable to tol). A refined
    // solve's final residual is exact in any case.
    write_ctl(g, ws, d, tol, schedule, max_sweeps, plain_loops, s, (sizeof(T) == 4 && refine && !H0 && !exact_r) ? 1 : 0,
              (sizeof(T) == 4 && refine) ? 1 : 0);
    if (profile) host_loop = 1;
    KernelClock kc(profile != 0, s);
    cudaEvent_t e0, e1;
    DI_CHECK_CUDA(cudaEventCreate(&e0));
    DI_CHECK_CUDA(cudaEventCreate(&e1));
    int rounds = 0;
    try {
        DI_CHECK_CUDA(cudaEventRecord(e0, s));
        if (!H0) {
            kc.run(KC_REFINE, 1, [&] {
                k_init<T><<<l.ew_blocks, 256, 0, s>>>(ws.B.as<double>(), g->n, ws.F.as<T>(), ws.H.as<double>(), ctl);
            });
        } else {
            // resumed state: H from the caller; F from the caller (staged as FP64 in y0) or, when
            // F0 is NULL, the exact residual B + P.H - H of the given history
            to_device(ws.H.p, H0, sizeof(double) * (size_t)g->n, s);
            double *stage = nullptr;
            if (F0) {
                stage = reinterpret_cast<double *>(ws.y0.p);
                to_device(stage, F0, sizeof(double) * (size_t)g->n, s);
            }
            kc.run(KC_REFINE, 1, [&] {
                k_resume_init<T><<<l.ew_blocks, 256, 0, s>>>(ws.B.as<double>(), stage, g->n, ws.F.as<T>(),
                                                             ws.H.as<double>(), ctl);
            });
            if (!F0) kc.run(KC_REFINE, g->n_heavy_in_chunks > 0 ? 3 : 2, [&] { launch_refine<T>(g, ws, l, d, s); });
        }
        if (e_prediffuse) {
            const PushTune tune = g->tune_single;
            for (size_t lv = 0; lv + 1 < g->e_level_off.size(); lv++) {
                const int64_t at = g->e_level_off[lv], cnt = g->e_level_off[lv + 1] - at;
                // (a level's ids span g->e_level_span[lv]: dense levels only, else the chunks
                // would hold a few nodes each and the push's segments would be tiny)
                if (sizeof(T) == 4 && cnt >= kELevelSelectMin &&
                    cnt * kSelChunk >= kELevelDensity * g->e_level_span[lv]) {
                    // a large level: select by id chunks, then the sweep's windowed push
                    const int64_t nchunk = (g->n + kSelChunk - 1) / kSelChunk;
                    const int blocks = (int)std::min<int64_t>(nchunk, (int64_t)g->dev.sms * 4);
                    kc.run(KC_SELECT, 1, [&] {
                        k_e_select<<<blocks, 256, 0, s>>>(
                            g->e_order.as<int32_t>() + at, (int32_t)cnt, ws.F.as<float>(), ws.H.as<double>(),
                            g->out_info.as<int32_t>(), g->n, ctl, ws.front_id.as<int32_t>(), ws.front_s.as<float>(),
                            ws.heavy_id.as<int32_t>(), ws.heavy_s.as<float>(), ws.heavy_cstart.as<int32_t>(),
                            ws.heavy_chunk.as<int32_t>(), ws.chunks.as<int4>(), g->win_qbits - kWinHeadBits,
                            tune.heavy, tune.chunk, seg_capacity(g));
                    });
                    kc.run(KC_PUSH, 1, [&] {
                        k_push_win<<<l.win_blocks, 256, 0, s>>>(
                            ws.front_id.as<int32_t>(), ws.front_s.as<float>(), ws.heavy_id.as<int32_t>(),
                            ws.heavy_s.as<float>(), ws.heavy_cstart.as<int32_t>(), ws.heavy_chunk.as<int32_t>(),
                            g->rp_push.as<int32_t>(), g->col_push.as<int32_t>(), ws.chunks.as<int4>(),
                            g->hub_ids.as<int32_t>(), ws.F.as<float>(), ctl, 1 << g->win_qbits, tune.row, tune.chunk, seg_capacity(g));
                    });
                    kc.run(KC_REFINE, 1, [&] { k_front_reset<<<1, 1, 0, s>>>(ctl); });
                } else {
                    const int64_t want = (cnt + 255) / 256, lim = (int64_t)g->dev.sms * 8;
                    const int blocks = (int)(want < lim ? want : lim);
                    kc.run(KC_REFINE, 1, [&] {
                        k_e_visit<T><<<blocks, 256, 0, s>>>(g->e_order.as<int32_t>() + at, (int32_t)cnt,
                                                            g->out_info.as<int32_t>(), g->rp_out.as<int64_t>(),
                                                            g->col_push.as<int32_t>(), g->hub_ids.as<int32_t>(),
                                                            ws.F.as<T>(), ws.H.as<double>(), ctl);
                    });
                }
            }
            DI_CHECK_CUDA(cudaGetLastError());
        }
        auto run_sweeps = [&]() {
            // a new phase of sweeps: the reduction below decides again whether to stop
            static const int32_t not_done = 0;
            DI_CHECK_CUDA(cudaMemcpyAsync(&ctl->done, &not_done, sizeof(int32_t), cudaMemcpyHostToDevice, s));
            kc.run(KC_REDUCE, 1, [&] {
                k_reduce<T><<<l.red_blocks, 256, 0, s>>>(ws.F.as<T>(), g->n, ws.partials.as<double>(), ctl,
                                                         cudaGraphConditionalHandle(0), 0, 1);
            });
            DI_CHECK_CUDA(cudaGetLastError());
            if (host_loop) {
                for (;;) {
                    read_ctl(g, ws, s);
                    if (ws.ctl_host->done) break;
                    launch_sweep_body<T>(g, ws, l, s, cudaGraphConditionalHandle(0), 0, &kc, parts);
                    DI_CHECK_CUDA(cudaGetLastError());
                }
            } else {
                if (ws.sweep_exec && (ws.sweep_parts != parts || !(ws.sweep_tune == g->tune_single))) ws.reset_graphs();
                if (!ws.sweep_exec) build_sweep_graph<T>(g, ws, l, parts);
                DI_CHECK_CUDA(cudaGraphLaunch(ws.sweep_exec, s));
            }
        };
        run_sweeps();
        // every refinement round ends on an exact residual, so the reported one is exact
        const size_t x_bytes = sizeof(double) * (size_t)g->n;
        const bool x_async = async_copy_target(X_out);
        bool x_copied = false;
        while (refine) {
            // A refinement leaves H as it is. When this round is likely the last (not the halfway
            // one of a split solve), X goes out on a second stream while the refinement runs; if
            // more sweeps follow after all, they wait for that copy and X is copied again.
            x_copied = x_async && (rounds > 0 || !ctl_split_expected(sizeof(T) == 4, refine));
            if (x_copied) {
                DI_CHECK_CUDA(cudaEventRecord(ws.out_ready, s));
                DI_CHECK_CUDA(cudaStreamWaitEvent(ws.out_stream, ws.out_ready, 0));
                from_device(X_out, ws.H.p, x_bytes, ws.out_stream);
                DI_CHECK_CUDA(cudaEventRecord(ws.out_done, ws.out_stream));
            }
            kc.run(KC_REFINE, g->n_heavy_in_chunks > 0 ? 3 : 2, [&] { launch_refine<T>(g, ws, l, d, s); });
            read_ctl(g, ws, s);
            rounds++;
            if (ws.ctl_host->status || ws.ctl_host->r <= tol || ws.ctl_host->sweeps >= max_sweeps || rounds >= 4) break;
            if (x_copied) {
                DI_CHECK_CUDA(cudaStreamWaitEvent(s, ws.out_done, 0));
                x_copied = false;
            }
            // Continuation sweeps start from the exact residual. After the halfway refinement of
            // a split solve the fluid's rounding since then is far below tol, so they aim just
            // under it; otherwise at half the tolerance, so the next exact residual lands below.
            const bool after_split = rounds == 1 && ws.ctl_host->tol > tol;
            const double aim = (after_split ? kAimAfterSplit : 0.5) * tol;
            DI_CHECK_CUDA(cudaMemcpyAsync(&ctl->tol, &aim, sizeof(double), cudaMemcpyHostToDevice, s));
            static const int32_t final_phase = 0;   // the next refinement may be the last
            DI_CHECK_CUDA(cudaMemcpyAsync(&ctl->halfway, &final_phase, sizeof(int32_t), cudaMemcpyHostToDevice, s));
            // An exact residual may have negative entries. After the halfway refinement they are
            // of the size of the rounding it replaced, a fraction of a percent of sum |F|, so the
            // tracked total (which follows sum F) stays on between exact reductions; otherwise
            // every reduction sums |F|.
            if (!after_split) {
                static const int32_t no_track = 0;
                DI_CHECK_CUDA(cudaMemcpyAsync(&ctl->track, &no_track, sizeof(int32_t), cudaMemcpyHostToDevice, s));
            }
            run_sweeps();
        }
        DI_CHECK_CUDA(cudaEventRecord(e1, s));
        if (x_copied)
            DI_CHECK_CUDA(cudaStreamWaitEvent(s, ws.out_done, 0));
        else
            from_device(X_out, ws.H.p, x_bytes, s);
        if (F_out) {
            // the final fluid (after refinement: the exact residual, rounded to the fluid's type)
            double *stage = reinterpret_cast<double *>(ws.y0.p);
            k_fluid_to_double<T><<<l.ew_blocks, 256, 0, s>>>(ws.F.as<T>(), g->n, stage);
            DI_CHECK_CUDA(cudaGetLastError());
            from_device(F_out, stage, sizeof(double) * (size_t)g->n, s);
        }
        read_ctl(g, ws, s);
    } catch (...) {
        if (ws.out_stream) cudaStreamSynchronize(ws.out_stream);   // no copy outlives the call
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const SolveCtl &c = *ws.ctl_host;
    if (info) {
        memset(info, 0, sizeof(*info));
        info->sweeps = c.sweeps;
        info->refine_rounds = rounds;
        info->pushed_edges = (int64_t)c.pushed;
        info->visited_nodes = (int64_t)c.visited;
        info->residual_l1 = c.r;
        info->dangling_mass_e = c.e;
        info->paper_error = c.r / (1.0 - d - d * c.e);
        info->ms = ms;
        info->kernel_launches = kc.host_launches + 3 * (int64_t)parts * (int64_t)c.body_runs;
        info->frontier_entries = (int64_t)c.front_total;
        info->select_ms = kc.ms[KC_SELECT];
        info->push_ms = kc.ms[KC_PUSH];
        info->reduce_ms = kc.ms[KC_REDUCE];
        info->refine_ms = kc.ms[KC_REFINE];
        info->select_launches = kc.count[KC_SELECT];
        info->push_launches = kc.count[KC_PUSH];
        info->reduce_launches = kc.count[KC_REDUCE];
        info->refine_launches = kc.count[KC_REFINE];
        info->e_visits = e_prediffuse ? (int32_t)g->stats.E : 0;
    }
    if (residual_out) *residual_out = c.r;
    DI_REQUIRE(c.status == 0, DI_ERR_INVALID_ARG, "B has a negative or non-finite entry");
    DI_REQUIRE(c.r <= tol, DI_ERR_NOT_CONVERGED, "not converged after %d sweeps: ||F||_1 = %g > tol = %g", c.sweeps,
               c.r, tol);
}

// ------------------------------------------------------------------------------------------
// autotuning of the single right-hand-side push split (PushTune)
// ------------------------------------------------------------------------------------------
__global__ void k_fill(double *v, int32_t n, double x) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) v[i] = x;
}

// Device time of a probe solve with split t: DI-SOP from B = (1 - d) / N, FP32 fluid without
// refinement, to ||F||_1 <= 1e-3 (1 - d) (about 40% of a full solve's sweeps), median of 3 after
// a warm-up. The caller holds the graph's lock.
static double probe_single_ms(di_graph *g, Workspace &ws, double d, const PushTune &t, cudaStream_t s) {
    ensure_workspace<float>(g, ws);
    g->tune_single = t;
    const Launch l = launch_shape<float>(g);
    double *Bp = ws.Xdf.as<double>();       // neither buffer is used by a D-iteration solve
    double *Xp = ws.Bdf.as<double>();
    k_fill<<<l.ew_blocks, 256, 0, s>>>(Bp, g->n, (1.0 - d) / g->n);
    DI_CHECK_CUDA(cudaGetLastError());
    std::vector<double> ms;
    for (int rep = 0; rep < 4; rep++) {
        di_solve_info info;
        solve_impl<float>(g, ws, Bp, d, 1e-3 * (1.0 - d), DI_SOP, 100000, 0, 0, 0, 0, 0, Xp, nullptr, &info, s);
        if (rep) ms.push_back(info.ms);
    }
    std::sort(ms.begin(), ms.end());
    return ms[ms.size() / 2];
}

// Coordinate descent over the row cut-off, then the heavy cut-off, then the chunk length.
PushTune autotune_single(di_graph *g, double d, cudaStream_t s, double *best_ms) {
    Workspace &ws = g->ws;
    PushTune best = g->tune_single;
    double bms = probe_single_ms(g, ws, d, best, s);
    auto try_one = [&](PushTune t) {
        if (t.chunk > t.heavy) return;
        const double ms = probe_single_ms(g, ws, d, t, s);
        if (ms < bms) {
            bms = ms;
            best = t;
        }
    };
    for (int row : {32, 64, 128, 256}) {
        PushTune t = best;
        t.row = row;
        if (!(t == best)) try_one(t);
    }
    for (int heavy : {1024, 2048, 4096, 8192}) {
        PushTune t = best;
        t.heavy = heavy;
        if (!(t == best)) try_one(t);
    }
    for (int chunk : {256, 512, 1024, 2048}) {
        PushTune t = best;
        t.chunk = chunk;
        if (!(t == best)) try_one(t);
    }
    g->tune_single = best;
    if (best_ms) *best_ms = bms;
    return best;
}

// Parts of a DI-SOP sweep, each selecting with r taken again (opts.r_refresh; 1 = the paper's
// r once per sweep). DI-CYC does not use r, so it always sweeps in one part.
constexpr int kMaxSweepParts = 16;
static int sweep_parts(const di_solve_opts &o) {
    return (o.schedule == DI_SOP && o.r_refresh > 1) ? o.r_refresh : 1;
}

// Checks and dispatch shared by solve_single and solve_single_in; the caller owns ws.
static void solve_single_body(di_graph *g, Workspace &ws, const double *B, double d, double tol,
                              const di_solve_opts *opts, double *X_out, double *residual_out, di_solve_info *info,
                              cudaStream_t s, bool lock) {
    check_common(g, B, d, tol, X_out);
    di_solve_opts o;
    memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    DI_REQUIRE(o.schedule == DI_CYC || o.schedule == DI_SOP, DI_ERR_INVALID_ARG, "unknown schedule %d", o.schedule);
    DI_REQUIRE(o.fluid == DI_FLUID_F32 || o.fluid == DI_FLUID_F64, DI_ERR_INVALID_ARG, "unknown fluid %d", o.fluid);
    DI_REQUIRE(o.r_refresh >= 0 && o.r_refresh <= kMaxSweepParts, DI_ERR_INVALID_ARG,
               "r_refresh must be in [0, %d] (got %d)", kMaxSweepParts, o.r_refresh);
    int max_sweeps = o.max_sweeps <= 0 ? 100000 : (o.max_sweeps > 1000000 ? 1000000 : o.max_sweeps);
    int refine = o.refine == 0 ? (o.fluid == DI_FLUID_F32) : (o.refine > 0);
    std::unique_lock<std::mutex> lk(g->mu, std::defer_lock);
    if (lock) {
        DI_REQUIRE(lk.try_lock(), DI_ERR_BUSY, "graph workspace is in use by another call");
    }
    DeviceGuard dg(g->dev.device);
    if (o.fluid == DI_FLUID_F32)
        solve_impl<float>(g, ws, B, d, tol, o.schedule, max_sweeps, refine, o.host_loop, o.profile,
                          o.e_prediffuse != 0, 0, X_out, residual_out, info, s, nullptr, nullptr, nullptr,
                          sweep_parts(o), o.exact_r != 0);
    else
        solve_impl<double>(g, ws, B, d, tol, o.schedule, max_sweeps, refine, o.host_loop, o.profile,
                           o.e_prediffuse != 0, 0, X_out, residual_out, info, s, nullptr, nullptr, nullptr,
                           sweep_parts(o), o.exact_r != 0);
}

di_status solve_single(di_graph *g, const double *B, double d, double tol, const di_solve_opts *opts, double *X_out,
                       double *residual_out, di_solve_info *info, cudaStream_t s) {
    return guarded([&] {
        DI_REQUIRE(g != nullptr, DI_ERR_INVALID_ARG, "graph is NULL");
        solve_single_body(g, g->ws, B, d, tol, opts, X_out, residual_out, info, s, true);
    });
}

di_status solve_single_in(di_graph *g, Workspace &ws, const double *B, double d, double tol, const di_solve_opts *opts,
                          double *X_out, double *residual_out, di_solve_info *info, cudaStream_t s) {
    return guarded([&] {
        DI_REQUIRE(g != nullptr, DI_ERR_INVALID_ARG, "graph is NULL");
        solve_single_body(g, ws, B, d, tol, opts, X_out, residual_out, info, s, false);
    });
}

// Power iteration per column (PI', Section 2.5): in increment form the Jacobi iterate obeys
// X_(k+1) - X_k = P (X_k - X_(k-1)), so a DI-CYC sweep that pushes every node's increment over
// its out-links, the self-link as a plain link (no loop closed form), is PI' iteration k: H holds
// X_k and ||F||_1 is PI's ||X_(k+1) - X_k||_1. FP64 increments give PI's iterates and counts;
// FP32 increments are followed by the exact FP64 residual B + P.H - H (that same difference
// computed exactly) and continuation sweeps from it.
di_status solve_resume(di_graph *g, const double *B, const double *H0, const double *F0, double d, double tol,
                       const di_solve_opts *opts, double *X_out, double *F_out, double *residual_out,
                       di_solve_info *info, cudaStream_t s) {
    return guarded([&] {
        check_common(g, B, d, tol, X_out);
        DI_REQUIRE(H0 != nullptr, DI_ERR_INVALID_ARG, "H0 is NULL");
        di_solve_opts o;
        memset(&o, 0, sizeof(o));
        if (opts) o = *opts;
        DI_REQUIRE(o.schedule == DI_CYC || o.schedule == DI_SOP, DI_ERR_INVALID_ARG, "unknown schedule %d", o.schedule);
        DI_REQUIRE(o.fluid == DI_FLUID_F32 || o.fluid == DI_FLUID_F64, DI_ERR_INVALID_ARG, "unknown fluid %d", o.fluid);
        DI_REQUIRE(o.r_refresh >= 0 && o.r_refresh <= kMaxSweepParts, DI_ERR_INVALID_ARG,
                   "r_refresh must be in [0, %d] (got %d)", kMaxSweepParts, o.r_refresh);
        int max_sweeps = o.max_sweeps <= 0 ? 100000 : (o.max_sweeps > 1000000 ? 1000000 : o.max_sweeps);
        int refine = o.refine == 0 ? (o.fluid == DI_FLUID_F32) : (o.refine > 0);
        std::unique_lock<std::mutex> lk(g->mu, std::try_to_lock);
        DI_REQUIRE(lk.owns_lock(), DI_ERR_BUSY, "graph workspace is in use by another call");
        DeviceGuard dg(g->dev.device);
        Workspace &ws = g->ws;
        if (o.fluid == DI_FLUID_F32)
            solve_impl<float>(g, ws, B, d, tol, o.schedule, max_sweeps, refine, o.host_loop, o.profile,
                              o.e_prediffuse != 0, 0, X_out, residual_out, info, s, H0, F0, F_out, sweep_parts(o),
                              o.exact_r != 0);
        else
            solve_impl<double>(g, ws, B, d, tol, o.schedule, max_sweeps, refine, o.host_loop, o.profile,
                               o.e_prediffuse != 0, 0, X_out, residual_out, info, s, H0, F0, F_out, sweep_parts(o),
                               o.exact_r != 0);
    });
}

di_status power_iter_push(di_graph *g, const double *B, double d, double tol, int32_t max_iters, int32_t fluid,
                          double *X_out, double *residual_out, di_solve_info *info, cudaStream_t s) {
    return guarded([&] {
        check_common(g, B, d, tol, X_out);
        DI_REQUIRE(fluid == DI_FLUID_F32 || fluid == DI_FLUID_F64, DI_ERR_INVALID_ARG, "unknown fluid %d", fluid);
        int mi = max_iters <= 0 ? 100000 : (max_iters > 1000000 ? 1000000 : max_iters);
        std::unique_lock<std::mutex> lk(g->mu, std::try_to_lock);
        DI_REQUIRE(lk.owns_lock(), DI_ERR_BUSY, "graph workspace is in use by another call");
        DeviceGuard dg(g->dev.device);
        Workspace &ws = g->ws;
        if (fluid == DI_FLUID_F32)
            solve_impl<float>(g, ws, B, d, tol, DI_CYC, mi, 1, 0, 0, 0, 1, X_out, residual_out, info, s);
        else
            solve_impl<double>(g, ws, B, d, tol, DI_CYC, mi, 0, 0, 0, 0, 1, X_out, residual_out, info, s);
    });
}

// Power iteration (Jacobi on X = P.X + B, Section 2.5 "PI"), from X_0 = 0 until
// ||X_(k+1) - X_k||_1 <= tol. fp64: FP64 throughout. Otherwise in increment form with FP32
// increments: X_(k+1) - X_k = P (X_k - X_(k-1)), pulled over the in-links, X accumulated in
// FP64 (in the history buffer, which the exact residual reads). The increments' FP32 rounding is relative to the increments, which shrink
// geometrically; with refinement the iteration stops halfway (on a log scale) and at the end
// to take the exact next increment B + P.X - X (double-float link sums, FP64 B and X), which
// certifies the reported residual and, when above tol, restarts the increments from it.
static void power_iter_impl(di_graph *g, Workspace &ws, const double *B, double d, double tol, int max_iters, bool fp64, bool refine,
                            int profile, double *X_out, double *residual_out, di_solve_info *info, cudaStream_t s) {
    using T = float;   // the single-solve workspace in its FP32 layout
    ensure_workspace<T>(g, ws);
    const Launch l = launch_shape<T>(g);
    SolveCtl *ctl = ws.ctl.as<SolveCtl>();
    to_device(ws.B.p, B, sizeof(double) * (size_t)g->n, s);
    write_ctl(g, ws, d, tol, DI_CYC, max_iters, 0, s, 0, (!fp64 && refine) ? 1 : 0);
    KernelClock kc(profile != 0, s);
    cudaEvent_t e0, e1;
    DI_CHECK_CUDA(cudaEventCreate(&e0));
    DI_CHECK_CUDA(cudaEventCreate(&e1));
    int rounds = 0;
    try {
        DI_CHECK_CUDA(cudaEventRecord(e0, s));
        if (fp64) {
            kc.run(KC_REFINE, 1, [&] {
                k_pi64_init<<<l.ew_blocks, 256, 0, s>>>(g->out_info.as<int32_t>(), g->n, d, ws.Bdf.as<double>(),
                                                        ws.Xdf.as<double>(), ws.y0.as<double>());
            });
        } else {
            kc.run(KC_REFINE, 1, [&] {
                // one iteration is done after the set-up, so the next pull reads y1 (see k_pull)
                k_pi_inc_init<<<l.red_blocks, 256, 0, s>>>(ws.B.as<double>(), g->out_info.as<int32_t>(), g->n, d,
                                                           ws.Bdf.as<float>(), ws.H.as<double>(), ws.y1.as<float>(),
                                                           ws.partials.as<double>(), ctl);
            });
        }
        DI_CHECK_CUDA(cudaGetLastError());
        auto run_iters = [&]() {
            if (profile) {
                for (;;) {
                    read_ctl(g, ws, s);
                    if (ws.ctl_host->done) break;
                    launch_pi_body(g, ws, l, s, cudaGraphConditionalHandle(0), 0, fp64, &kc);
                    DI_CHECK_CUDA(cudaGetLastError());
                }
            } else {
                if (ws.pi_exec && ws.pi_fp64 != (fp64 ? 1 : 0)) ws.reset_graphs();
                if (!ws.pi_exec) build_pi_graph(g, ws, l, fp64);
                DI_CHECK_CUDA(cudaGraphLaunch(ws.pi_exec, s));
            }
        };
        // the set-up counts as the first iteration (X_1 = B), so the loop may already be done
        read_ctl(g, ws, s);
        if (!ws.ctl_host->done) run_iters();
        if (fp64) {
            kc.run(KC_REFINE, 1, [&] {
                k_fluid_to_double<double><<<l.ew_blocks, 256, 0, s>>>(ws.Xdf.as<double>(), g->n, ws.H.as<double>());
            });
        }
        while (!fp64 && refine) {
            // the exact next increment of X (in ws.F as FP32, its norm in ctl->r)
            kc.run(KC_REFINE, g->n_heavy_in_chunks > 0 ? 3 : 2, [&] { launch_refine<T>(g, ws, l, d, s); });
            read_ctl(g, ws, s);
            rounds++;
            if (ws.ctl_host->r <= tol || ws.ctl_host->sweeps >= max_iters || rounds >= 4) break;
            // continue the increments from it: after the halfway stop at tol itself (the exact
            // check follows, and the fluid's rounding since that stop is far below tol), else at
            // half of it
            const bool after_split = ws.ctl_host->halfway != 0;
            SolveCtl &c = *ws.ctl_host;
            c.tol = (after_split ? 1.0 : 0.5) * tol;
            c.halfway = 0;
            c.done = 0;
            DI_CHECK_CUDA(cudaMemcpyAsync(&ctl->tol, &c.tol, sizeof(double), cudaMemcpyHostToDevice, s));
            DI_CHECK_CUDA(cudaMemcpyAsync(&ctl->halfway, &c.halfway, sizeof(int32_t), cudaMemcpyHostToDevice, s));
            DI_CHECK_CUDA(cudaMemcpyAsync(&ctl->done, &c.done, sizeof(int32_t), cudaMemcpyHostToDevice, s));
            kc.run(KC_REFINE, 1, [&] {
                k_pi_inc_resume<<<l.ew_blocks, 256, 0, s>>>(ws.F.as<float>(), g->n, ws.Bdf.as<float>(),
                                                            ws.H.as<double>(), ws.y0.as<float>(), ws.y1.as<float>(),
                                                            ctl);
            });
            // applying the exact increment is one more iteration
            c.sweeps += 1;
            DI_CHECK_CUDA(cudaMemcpyAsync(&ctl->sweeps, &c.sweeps, sizeof(int32_t), cudaMemcpyHostToDevice, s));
            if (c.sweeps < max_iters) run_iters();
        }
        DI_CHECK_CUDA(cudaGetLastError());
        DI_CHECK_CUDA(cudaEventRecord(e1, s));
        from_device(X_out, ws.H.p, sizeof(double) * (size_t)g->n, s);
        read_ctl(g, ws, s);
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        throw;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const SolveCtl &c = *ws.ctl_host;
    if (info) {
        memset(info, 0, sizeof(*info));
        info->sweeps = c.sweeps;
        info->refine_rounds = rounds;
        info->pushed_edges = (int64_t)c.sweeps * g->L;
        info->visited_nodes = (int64_t)c.sweeps * g->n;
        info->residual_l1 = c.r;
        info->ms = ms;
        const int per = g->n_heavy_in_chunks > 0 ? 2 : 1;
        info->kernel_launches = kc.host_launches + (int64_t)c.body_runs * per;
        info->select_ms = kc.ms[KC_SELECT];
        info->push_ms = kc.ms[KC_PUSH];
        info->refine_ms = kc.ms[KC_REFINE];
        info->select_launches = kc.count[KC_SELECT];
        info->push_launches = kc.count[KC_PUSH];
        info->refine_launches = kc.count[KC_REFINE];
    }
    if (residual_out) *residual_out = c.r;
    DI_REQUIRE(c.r <= tol, DI_ERR_NOT_CONVERGED, "PI not converged after %d iterations: %g > %g", c.sweeps, c.r, tol);
}

di_status power_iter_ex(di_graph *g, const double *B, double d, double tol, const di_solve_opts *opts, double *X_out,
                        double *residual_out, di_solve_info *info, cudaStream_t s) {
    return guarded([&] {
        check_common(g, B, d, tol, X_out);
        di_solve_opts o;
        memset(&o, 0, sizeof(o));
        if (opts) o = *opts;
        DI_REQUIRE(o.fluid == DI_FLUID_F32 || o.fluid == DI_FLUID_F64, DI_ERR_INVALID_ARG, "unknown fluid %d", o.fluid);
        const int mi = o.max_sweeps <= 0 ? 100000 : (o.max_sweeps > 1000000 ? 1000000 : o.max_sweeps);
        const bool fp64 = o.fluid == DI_FLUID_F64;
        const bool refine = o.refine >= 0;
        std::unique_lock<std::mutex> lk(g->mu, std::try_to_lock);
        DI_REQUIRE(lk.owns_lock(), DI_ERR_BUSY, "graph workspace is in use by another call");
        DeviceGuard dg(g->dev.device);
        power_iter_impl(g, g->ws, B, d, tol, mi, fp64, refine, o.profile, X_out, residual_out, info, s);
    });
}

di_status power_iter(di_graph *g, const double *B, double d, double tol, int32_t max_iters, double *X_out,
                     double *residual_out, di_solve_info *info, cudaStream_t s) {
    di_solve_opts o;
    memset(&o, 0, sizeof(o));
    o.max_sweeps = max_iters;
    return power_iter_ex(g, B, d, tol, &o, X_out, residual_out, info, s);
}

}  // namespace di

extern "C" {

di_status di_solve(di_graph *g, const double *B, double d, double tol, int32_t schedule, int32_t max_sweeps,
                   double *X_out, double *residual_out, di_solve_info *info, void *stream) {
    di_solve_opts o;
    memset(&o, 0, sizeof(o));
    o.schedule = schedule;
    o.max_sweeps = max_sweeps;
    return di::solve_single(g, B, d, tol, &o, X_out, residual_out, info, (cudaStream_t)stream);
}

di_status di_solve_ex(di_graph *g, const double *B, double d, double tol, const di_solve_opts *opts, double *X_out,
                      double *residual_out, di_solve_info *info, void *stream) {
    return di::solve_single(g, B, d, tol, opts, X_out, residual_out, info, (cudaStream_t)stream);
}

di_status di_solve_resume(di_graph *g, const double *B, const double *H0, const double *F0, double d, double tol,
                          const di_solve_opts *opts, double *X_out, double *F_out, double *residual_out,
                          di_solve_info *info, void *stream) {
    return di::solve_resume(g, B, H0, F0, d, tol, opts, X_out, F_out, residual_out, info, (cudaStream_t)stream);
}

di_status di_power_iter_push(di_graph *g, const double *B, double d, double tol, int32_t max_iters,
                             int32_t fluid, double *X_out, double *residual_out, di_solve_info *info,
                             void *stream) {
    return di::power_iter_push(g, B, d, tol, max_iters, fluid, X_out, residual_out, info, (cudaStream_t)stream);
}

di_status di_power_iter(di_graph *g, const double *B, double d, double tol, int32_t max_iters, double *X_out,
                        double *residual_out, di_solve_info *info, void *stream) {
    return di::power_iter(g, B, d, tol, max_iters, X_out, residual_out, info, (cudaStream_t)stream);
}

di_status di_power_iter_ex(di_graph *g, const double *B, double d, double tol, const di_solve_opts *opts,
                           double *X_out, double *residual_out, di_solve_info *info, void *stream) {
    return di::power_iter_ex(g, B, d, tol, opts, X_out, residual_out, info, (cudaStream_t)stream);
}

}  // extern "C"
