// Multi-RHS tile machinery shared by the batched solver (di_batch.cu) and the server
// (di_server.cu): a tile holds T right-hand sides ("columns") of one graph with the fluid
// node-major, F[i*T + c] (FP32), so one pass over the out-links of a visited node serves all T
// fluids: the push loads each link index once and adds four columns per vector atomic
// (red.global.add.v4.f32). H[i*T + c] is FP64. Every column keeps its own DI-SOP rule
// (Section 2.3): column c of node i is diffused when |F_ic| > (r_c / L) * out_i with
// r_c = ||F_c||_1 at the sweep start, and a node is pushed when any of its columns was diffused
// (columns that were not send 0, and skip their atomics). A column retires when r_c <= tol_c.
// The exact FP64 residual of every column (F*_c = B_c + P.H_c - H_c) replaces F when asked for.
#pragma once

#include <cmath>
#include <cstring>

#include "di_batch.cuh"

namespace di {

constexpr int kMaxT = 32;

struct BatchCtl {
    double d;
    double L;
    double tol[kMaxT];
    double r[kMaxT];
    double e[kMaxT];
    int32_t active[kMaxT];
    int32_t retire_sweep[kMaxT];
    unsigned long long pushed;       // sum of out_i over node visits (a node counted once per sweep)
    unsigned long long visited;      // node visits
    unsigned long long col_visits;   // (node, column) diffusions
    unsigned long long col_pushed;   // links pushed per (node, column) diffusion with a share,
                                     //    summed: the push's link-column updates
    unsigned long long front_total;
    int32_t ncols;
    int32_t schedule;
    int32_t max_sweeps;
    int32_t sweeps;
    int32_t done;
    int32_t status;                  // 0 ok, 1 bad right-hand side, 2 seed out of range
    int32_t force_cyc;
    int32_t last_selected;
    int32_t front_count;
    int32_t heavy_chunks;            // chunks of the entries with more than PushTune::heavy links
    int32_t batch_next;
    int32_t body_runs;
    uint32_t ticket;
    uint32_t split_mask;             // columns whose next stop test raises their tol to
                                     //    sqrt(tol * r), their first refinement point
    int64_t seed_off[kMaxT + 1];     // seed sets of the tile's columns: column c holds the seeds
                                     //    at positions [seed_off[c], seed_off[c+1]) of the list
};

// ------------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------------

// Bn[i*T + c] = B[(c0 + c) * n + i] for c < ncols (0 for padding columns)
template <int T>
__global__ void kb_load_B(const double *B, int32_t n, int c0, int ncols, double *Bn) {
    const int64_t total = (int64_t)n * T;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / T;
        const int c = (int)(idx % T);
        Bn[idx] = c < ncols ? B[(int64_t)(c0 + c) * n + i] : 0.0;
    }
}

// Bn[s*T + c] += (1 - d) / |S_c| for every seed s of column c: seeds[e - e0] is the seed at list
// position e, for e in [e0, e1), and ctl->seed_off holds the tile's column ranges
template <int T>
__global__ void kb_seed_B(const int32_t *seeds, int64_t e0, int64_t e1, int32_t n, int ncols, double d, double *Bn,
                          BatchCtl *ctl) {
    const int64_t *off = ctl->seed_off;
    for (int64_t e = e0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < e1; e += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = ncols - 1;          // column whose range holds e
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (off[mid] <= e) lo = mid; else hi = mid - 1;
        }
        const int32_t s = seeds[e - e0];
        if (s < 0 || s >= n) {
            ctl->status = 2;
            continue;
        }
        const double cnt = (double)(off[lo + 1] - off[lo]);
        atomicAdd(&Bn[(int64_t)s * T + lo], (1.0 - d) / cnt);
    }
}

template <int T>
__global__ void kb_init(const double *Bn, int32_t n, float *F, double *H, BatchCtl *ctl) {
    bool bad = false;
    const int64_t total = (int64_t)n * T;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const double b = Bn[idx];
        if (!(b >= 0.0) || isinf(b)) bad = true;
        F[idx] = (float)b;
        H[idx] = 0.0;
    }
    if (bad) ctl->status = 1;
}

// Per-column sums of |v| over a node-major [n][T] array into `out[c]` (FP64, fixed order);
// the finishing block then runs `tail(total)` on thread 0 after writing the sums.
template <int T, class V, class Tail>
__device__ __forceinline__ void column_l1(const V *v, int32_t n, double *partials, BatchCtl *ctl, double *out,
                                          Tail &&tail) {
    __shared__ double ssum[8][T];
    __shared__ bool is_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double s = 0.0;
    const int64_t total = (int64_t)n * T;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // blockDim (256) and the grid stride are multiples of T, so a thread always sees column
    // tid % T; four independent loads per step, summed in FP32 and widened to FP64 (this
    // part's FP64 rate is low)
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + tid;
    for (; idx + 3 * stride < total; idx += 4 * stride) {
        const float a = fabsf((float)__ldcg(v + idx)), b = fabsf((float)__ldcg(v + idx + stride));
        const float c2 = fabsf((float)__ldcg(v + idx + 2 * stride)), e2 = fabsf((float)__ldcg(v + idx + 3 * stride));
        s += (double)((a + b) + (c2 + e2));
    }
    for (; idx < total; idx += stride) s += (double)fabsf((float)__ldcg(v + idx));
#pragma unroll
    for (int o = 16; o >= T; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if (lane < T) ssum[warp][lane] = s;
    __syncthreads();
    if (tid < T) {
        double b = 0.0;
        for (int w = 0; w < 8; w++) b += ssum[w][tid];
        partials[(int64_t)blockIdx.x * T + tid] = b;
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) is_last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (tid < T) {
        double tot = 0.0;
        for (int b = 0; b < (int)gridDim.x; b++) tot += __ldcg(&partials[(int64_t)b * T + tid]);
        out[tid] = tot;
    }
    __syncthreads();
    if (tid == 0) {
        ctl->ticket = 0;
        tail();
    }
}

// Column retirement and the stop test (thread 0 of the finishing block).
static __device__ __forceinline__ void batch_stop_test(BatchCtl *ctl, cudaGraphConditionalHandle h, int set_cond) {
    if (ctl->split_mask) {
        for (int c = 0; c < ctl->ncols; c++) {
            const double mid = sqrt(ctl->tol[c] * ctl->r[c]);
            if ((ctl->split_mask >> c & 1u) && ctl->active[c] && ctl->tol[c] < kSplitBelow * ctl->r[c])
                ctl->tol[c] = mid;
        }
        ctl->split_mask = 0;
    }
    bool any = false;
    double rsum = 0.0;
    for (int c = 0; c < ctl->ncols; c++) {
        if (ctl->active[c] && !(ctl->r[c] > ctl->tol[c])) {
            ctl->active[c] = 0;
            ctl->retire_sweep[c] = ctl->sweeps;
        }
        any = any || ctl->active[c];
        rsum += ctl->r[c];
    }
    const int sel = ctl->last_selected;
    ctl->force_cyc = (sel == 0 && rsum > 0.0) ? 1 : 0;
    ctl->last_selected = 0;
    ctl->front_total += (unsigned long long)ctl->front_count;
    ctl->front_count = 0;
    ctl->heavy_chunks = 0;
    ctl->batch_next = 0;
    if (set_cond) ctl->body_runs++;
    const bool cont = ctl->status == 0 && any && ctl->sweeps < ctl->max_sweeps;
    ctl->done = cont ? 0 : 1;
    if (set_cond) cudaGraphSetConditional(h, cont ? 1u : 0u);
}

template <int T>
__global__ void __launch_bounds__(256) kb_reduce(const float *F, int32_t n, double *partials, BatchCtl *ctl,
                                                 cudaGraphConditionalHandle h, int set_cond) {
    column_l1<T>(F, n, partials, ctl, ctl->r, [&] { batch_stop_test(ctl, h, set_cond); });
}

// A column's DI-SOP test |F_ic| > (r_c / L) * out_i, decided as in FP64: FP32 unless the fluid
// is within 2^-20 (relative) of the threshold, where the FP32 product's rounding (below 2^-22)
// could matter, or r_c / L is too small for FP32's normal range.
static __device__ __forceinline__ bool tile_sop_selects(float a, float o_f, double thr, float thr_f) {
    const float p = thr_f * o_f;
    if (thr_f >= 1e-30f) {
        if (a > p * (1.f + 1.0f / (1 << 20))) return true;
        if (a < p * (1.f - 1.0f / (1 << 20))) return false;
    }
    return (double)a > thr * (double)o_f;
}

// A block handles 256 consecutive nodes per iteration in T sub-steps of 256/T nodes (T lanes per
// node, one lane per column); the pushed nodes of the 256 are compacted with one atomic, so the
// frontier is id-sorted within each 256-node chunk.
template <int T>
__global__ void __launch_bounds__(256) kb_select(float *F, double *H, const int32_t *out_info, int32_t n,
                                                 BatchCtl *ctl, int32_t *front_id, float *front_s,
                                                 int32_t *heavy_cstart, int32_t *heavy_chunk, int heavy_cut,
                                                 int heavy_len) {
    constexpr int kNodesPerStep = 256 / T;
    __shared__ double s_thr[T];
    __shared__ int s_act[T];
    __shared__ double s_e[8][T];
    __shared__ unsigned long long s_cnt[4][8];
    __shared__ int wcount[T][8];
    __shared__ int chunk_base;
    __shared__ float s_share[T][256];       // per sub-step share of every lane
    __shared__ unsigned s_lbs[T][8];        // per sub-step leader ballot of every warp
    __shared__ int32_t s_hdeg[T][256 / T];  // per sub-step and node: out-degree if above heavy_cut, else 0
    if (ctl->done) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool cyc = ctl->schedule == DI_CYC || ctl->force_cyc;
    const double d = ctl->d;
    if (tid < T) {
        s_thr[tid] = ctl->L > 0.0 ? ctl->r[tid] / ctl->L : 0.0;
        s_act[tid] = tid < ctl->ncols ? ctl->active[tid] : 0;
    }
    __syncthreads();
    const int c = tid % T;
    const int gbase = lane & ~(T - 1);                         // first lane of this node's group
    const unsigned gmask = (T == 32) ? kFull : (((1u << T) - 1u) << gbase);
    const unsigned below = gbase ? ((1u << gbase) - 1u) : 0u;  // lanes before this group
    const bool leader = lane == gbase;
    const float thr_f = (float)s_thr[c];
    const float d_f = (float)d;
    const bool act = s_act[c] != 0;
    float e_run = 0.f;
    unsigned long long pushed = 0, visited = 0, colv = 0, colp = 0;
    for (int64_t base = (int64_t)blockIdx.x * 256; base < n; base += (int64_t)gridDim.x * 256) {
        // sub-steps in groups of kGroup: the F and degree loads of a group are issued before any
        // of its stores, then H of the selected entries, so the loads of a group overlap
        constexpr int kGroup = T < 8 ? T : 8;
        for (int j0 = 0; j0 < T; j0 += kGroup) {
            float f[kGroup];
            int32_t info[kGroup];
#pragma unroll
            for (int q = 0; q < kGroup; q++) {
                const int64_t i = base + (j0 + q) * kNodesPerStep + tid / T;
                f[q] = 0.f;
                info[q] = 0;
                if (i < n) {
                    f[q] = F[i * T + c];
                    info[q] = out_info[i];
                }
            }
            unsigned selm = 0;
#pragma unroll
            for (int q = 0; q < kGroup; q++) {
                const int64_t i = base + (j0 + q) * kNodesPerStep + tid / T;
                const float o_f = (float)(info[q] & 0x7fffffff);
                if (i < n && act && (cyc ? (f[q] != 0.f) : tile_sop_selects(fabsf(f[q]), o_f, s_thr[c], thr_f)))
                    selm |= 1u << q;
            }
            double h[kGroup];
#pragma unroll
            for (int q = 0; q < kGroup; q++) {
                const int64_t i = base + (j0 + q) * kNodesPerStep + tid / T;
                h[q] = (selm >> q & 1u) ? H[i * T + c] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < kGroup; q++) {
                const int j = j0 + q;
                const int64_t i = base + j * kNodesPerStep + tid / T;
                const bool sel = selm >> q & 1u;
                bool pushable = false;
                const int32_t o = info[q] & 0x7fffffff;
                float share = 0.f;
                if (sel) {
                    const int64_t idx = i * T + c;
                    const bool lp = info[q] < 0;
                    F[idx] = 0.f;
                    // FP32 transit and share; FP64 only for H += transit
                    const float of = (float)o;
                    const float tf = lp ? f[q] * of / (of - d_f) : f[q];
                    H[idx] = h[q] + widen(tf);   // exact, on the integer units
                    colv++;
                    if (o == 0) e_run += tf;
                    else {
                        share = tf * d_f / of;
                        pushable = (o - (lp ? 1 : 0)) > 0;
                        if (pushable && share != 0.f) colp += (unsigned long long)(o - (lp ? 1 : 0));
                    }
                }
                const unsigned bsel = __ballot_sync(kFull, sel) & gmask;
                const unsigned bpush = __ballot_sync(kFull, pushable) & gmask;
                if (leader && bsel) {
                    visited++;
                    pushed += (unsigned long long)o;
                }
                const unsigned lb = __ballot_sync(kFull, leader && bpush != 0);
                if (leader) s_hdeg[j][tid / T] = o > heavy_cut ? o : 0;
                s_share[j][tid] = share;
                if (lane == 0) {
                    s_lbs[j][warp] = lb;
                    wcount[j][warp] = __popc(lb);
                }
            }
        }
        __syncthreads();
        if (tid == 0) {
            int run = 0;
            for (int j = 0; j < T; j++)
                for (int w = 0; w < 8; w++) {
                    const int v = wcount[j][w];
                    wcount[j][w] = run;
                    run += v;
                }
            chunk_base = run ? atomicAdd(&ctl->front_count, run) : 0;
        }
        __syncthreads();
        const int cb = chunk_base;
#pragma unroll 4
        for (int j = 0; j < T; j++) {
            const unsigned lb = s_lbs[j][warp];
            if (lb & (1u << gbase)) {
                const int pos = cb + wcount[j][warp] + __popc(lb & below);
                front_s[(int64_t)pos * T + c] = s_share[j][tid];
                if (leader) {
                    const int32_t node = (int32_t)(base + j * kNodesPerStep + tid / T);
                    front_id[pos] = node;
                    // a node with many links is pushed in chunks over all warps (see kb_push)
                    const int32_t o = s_hdeg[j][tid / T];
                    if (o > 0) {
                        const int nch = (o + heavy_len - 1) / heavy_len;
                        const int cs = atomicAdd(&ctl->heavy_chunks, nch);
                        heavy_cstart[pos] = cs;
                        for (int q = 0; q < nch; q++) heavy_chunk[cs + q] = pos;
                    }
                }
            }
        }
        __syncthreads();
    }
    // per-column dangling mass
    double e_loc = (double)e_run;
#pragma unroll
    for (int o2 = 16; o2 >= T; o2 >>= 1) e_loc += __shfl_xor_sync(kFull, e_loc, o2);
    if (lane < T) s_e[warp][lane] = e_loc;
    pushed = warp_sum(pushed);
    visited = warp_sum(visited);
    colv = warp_sum(colv);
    colp = warp_sum(colp);
    if (lane == 0) { s_cnt[0][warp] = pushed; s_cnt[1][warp] = visited; s_cnt[2][warp] = colv; s_cnt[3][warp] = colp; }
    __syncthreads();
    if (tid < T) {
        double sum = 0.0;
        for (int w = 0; w < 8; w++) sum += s_e[w][tid];
        if (sum != 0.0) atomicAdd(&ctl->e[tid], sum);
    }
    if (tid == 0) {
        unsigned long long a = 0, b = 0, cc = 0, cp = 0;
        for (int w = 0; w < 8; w++) { a += s_cnt[0][w]; b += s_cnt[1][w]; cc += s_cnt[2][w]; cp += s_cnt[3][w]; }
        if (a) atomicAdd(&ctl->pushed, a);
        if (b) {
            atomicAdd(&ctl->visited, b);
            atomicAdd(&ctl->last_selected, (int)b);
        }
        if (cc) atomicAdd(&ctl->col_visits, cc);
        if (cp) atomicAdd(&ctl->col_pushed, cp);
        if (blockIdx.x == 0) atomicAdd(&ctl->sweeps, 1);
    }
}

// Slot kernels of a tile whose columns are refilled (the batched solver and the server):
// scattering a request's seeds into a free column, loading a dense right-hand side into one,
// and handing a finished column's history out while zeroing the column for its next request.
template <int T>
__global__ void kb_seed_col(const int32_t *seeds, int64_t cnt, int c, double share, int32_t n, float *F, double *Bn,
                            BatchCtl *ctl) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = seeds[e];
        if (s < 0 || s >= n) {
            ctl->status = 2;
            continue;
        }
        atomicAdd(&Bn[(int64_t)s * T + c], share);
        atomicAdd(&F[(int64_t)s * T + c], (float)share);
    }
}

template <int T>
__global__ void kb_load_col(const double *B, int32_t n, int c, float *F, double *Bn, BatchCtl *ctl) {
    bool bad = false;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double b = B[i];
        if (!(b >= 0.0) || isinf(b)) bad = true;
        Bn[i * T + c] = b;
        F[i * T + c] = (float)b;
    }
    if (bad) ctl->status = 1;
}

template <int T>
__global__ void kb_col_retire(float *F, double *H, double *Bn, int32_t n, int c, double *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t idx = i * T + c;
        out[i] = H[idx];
        H[idx] = 0.0;
        F[idx] = 0.f;
        Bn[idx] = 0.0;
    }
}

template <int T>
__global__ void kb_fill(double *Bn, int64_t count, double v) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        Bn[i] = v;
}

static __device__ __forceinline__ void red_add_v4(float *p, float4 v) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// One frontier node at a time per warp: T/4 lanes cover the T columns of one link, so a warp
// walks 128/T links per step, each link index loaded once for its T fluids.
template <int T>
__global__ void __launch_bounds__(256) kb_push(const int32_t *__restrict__ front_id, const float *__restrict__ front_s,
                                               const int32_t *__restrict__ heavy_cstart,
                                               const int32_t *__restrict__ heavy_chunk,
                                               const int64_t *__restrict__ rp_out, const int32_t *__restrict__ col_out,
                                               float *F, BatchCtl *ctl, int heavy_cut, int heavy_len) {
    if (ctl->done) return;
    constexpr int LPE = T / 4;          // lanes per link
    constexpr int EPI = 32 / LPE;       // links per warp step
    const int lane = (int)lane_id();
    const int q = lane % LPE, es = lane / LPE;
    const int count = ctl->front_count;
    constexpr int kGrab = 32;
    for (;;) {
        int c0 = 0;
        if (lane == 0) c0 = atomicAdd(&ctl->batch_next, kGrab);
        c0 = __shfl_sync(kFull, c0, 0);
        if (c0 >= count) break;
        const int cend = min(c0 + kGrab, count);
        for (int p = c0; p < cend; p++) {
            const int32_t u = front_id[p];
            const int64_t beg = rp_out[u];
            const int deg = (int)(rp_out[u + 1] - beg);
            if (deg > heavy_cut) continue;   // pushed below, in chunks over all warps
            const float4 s = reinterpret_cast<const float4 *>(front_s + (int64_t)p * T)[q];
            const bool any = (s.x != 0.f) || (s.y != 0.f) || (s.z != 0.f) || (s.w != 0.f);
            if (!any) continue;
            for (int e0 = es; e0 < deg; e0 += EPI * 4) {
                int32_t j[4];   // four index loads in flight before the reductions
#pragma unroll
                for (int v = 0; v < 4; v++) j[v] = e0 + EPI * v < deg ? col_out[beg + e0 + EPI * v] : u;
#pragma unroll
                for (int v = 0; v < 4; v++)
                    if (j[v] != u) red_add_v4(F + (int64_t)j[v] * T + 4 * q, s);
            }
        }
    }
    // nodes with more than heavy_cut links: heavy_len-link chunks over all warps
    const int hch = ctl->heavy_chunks;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < hch; c += nwarps) {
        const int p = heavy_chunk[c];
        const int32_t u = front_id[p];
        const float4 s = reinterpret_cast<const float4 *>(front_s + (int64_t)p * T)[q];
        const bool any = (s.x != 0.f) || (s.y != 0.f) || (s.z != 0.f) || (s.w != 0.f);
        const int64_t cb = rp_out[u] + (int64_t)(c - heavy_cstart[p]) * heavy_len;
        const int64_t ce = min(cb + (int64_t)heavy_len, rp_out[u + 1]);
        if (!any) continue;
        for (int64_t e0 = cb + es; e0 < ce; e0 += EPI * 4) {
            int32_t j[4];   // four index loads in flight before the reductions
#pragma unroll
            for (int v = 0; v < 4; v++) j[v] = e0 + EPI * v < ce ? col_out[e0 + EPI * v] : u;
#pragma unroll
            for (int v = 0; v < 4; v++)
                if (j[v] != u) red_add_v4(F + (int64_t)j[v] * T + 4 * q, s);
        }
    }
}

// Double-float helpers (an unevaluated sum hi + lo of two FP32 numbers; Knuth two-sum and an
// FMA-based exact product) so the link sums of the residual need no FP64 arithmetic.
static __device__ __forceinline__ float2 tdf_add(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float bb = s - a.x;
    float e = (a.x - (s - bb)) + (b.x - bb);
    e += a.y + b.y;
    const float hi = s + e;
    return make_float2(hi, e - (hi - s));
}
static __device__ __forceinline__ float2 tdf_mul(float2 a, float2 b) {
    const float p = a.x * b.x;
    float e = fmaf(a.x, b.x, -p);
    e = fmaf(a.x, b.y, e);
    e = fmaf(a.y, b.x, e);
    const float hi = p + e;
    return make_float2(hi, e - (hi - p));
}
static __device__ __forceinline__ float2 tdf_from(double v) {
    const float hi = (float)v;
    return make_float2(hi, (float)(v - (double)hi));
}

// y[i*T + c] = d * H_ic / out_i as double-float (0 for a dangling node); d / out_i is formed
// once per node and shared by the T columns.
template <int T>
__global__ void kb_resid_y(const double *H, const int32_t *out_info, int32_t n, double d, uint32_t mask, float2 *y) {
    const int64_t total = (int64_t)n * T;
    const int lane = threadIdx.x & 31, leader = lane & ~(T - 1);
    // whole warps iterate together (total is a multiple of T, blocks of 256 threads)
    for (int64_t base = (blockIdx.x * (int64_t)blockDim.x) & ~31ll; base < total;
         base += (int64_t)gridDim.x * blockDim.x) {
        const int64_t idx = base + (threadIdx.x & ~31) + lane;
        float2 c = make_float2(0.f, 0.f);
        if (lane == leader && idx < total) {
            const int32_t o = out_info[idx / T] & 0x7fffffff;
            if (o) c = tdf_from(d / (double)o);           // one division per node
        }
        c.x = __shfl_sync(kFull, c.x, leader);
        c.y = __shfl_sync(kFull, c.y, leader);
        if (idx < total && (mask >> (lane & (T - 1)) & 1u)) y[idx] = tdf_mul(tdf_from(H[idx]), c);
    }
}

// Exact residual of the history, per column: F*_ic = B_ic + sum_{j in in(i)} d H_jc / out_j - H_ic.
// (32/T) link slots x T columns per warp; rows with more than kPullHeavy links take their
// chunk partial sums from kb_resid_heavy.
template <int T>
__global__ void kb_resid_heavy(const int64_t *rp_in, const int32_t *col_in, const int32_t *heavy_rows,
                               const int32_t *chunk_off, const int32_t *chunk_row, int32_t n_chunks,
                               const float2 *y, uint32_t mask, float2 *partial) {
    constexpr int SL = 32 / T;
    constexpr int kUnroll = 8;
    const int lane = (int)lane_id(), c = lane % T, slot = lane / T;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t ch = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; ch < n_chunks; ch += nwarps) {
        const int32_t h = chunk_row[ch];
        const int32_t row = heavy_rows[h];
        const int64_t b = rp_in[row] + (int64_t)(ch - chunk_off[h]) * kPullChunk;
        const int64_t e = min(b + (int64_t)kPullChunk, rp_in[row + 1]);
        float2 acc = make_float2(0.f, 0.f);
        if (mask >> c & 1u)
            // kUnroll index loads, then as many gathers, in flight before the additions
            for (int64_t k0 = b + slot; k0 < e; k0 += SL * kUnroll) {
                int32_t j[kUnroll];
#pragma unroll
                for (int v = 0; v < kUnroll; v++) j[v] = k0 + SL * v < e ? __ldcs(col_in + k0 + SL * v) : -1;
                float2 val[kUnroll];
#pragma unroll
                for (int v = 0; v < kUnroll; v++) val[v] = j[v] >= 0 ? y[(int64_t)j[v] * T + c] : make_float2(0.f, 0.f);
#pragma unroll
                for (int v = 0; v < kUnroll; v++) acc = tdf_add(acc, val[v]);
            }
#pragma unroll
        for (int o = 16; o >= T; o >>= 1) {
            float2 t;
            t.x = __shfl_xor_sync(kFull, acc.x, o);
            t.y = __shfl_xor_sync(kFull, acc.y, o);
            acc = tdf_add(acc, t);
        }
        if (lane < T) partial[ch * T + c] = acc;
    }
}

template <int T>
__global__ void __launch_bounds__(256) kb_resid(const int64_t *rp_in, const int32_t *col_in, const float2 *y,
                                                const int32_t *heavy_rows, const int32_t *heavy_chunk_off,
                                                const float2 *heavy_partial, int32_t n_heavy, const double *Bn,
                                                const double *H, int32_t n, uint32_t mask, float *F,
                                                double *out_l1, double *partials, BatchCtl *ctl) {
    constexpr int SL = 32 / T;
    __shared__ double ssum[8][T];
    __shared__ bool is_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int c = lane % T, slot = lane / T;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double colsum = 0.0;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + tid) >> 5; i < n; i += nwarps) {
        const int64_t b = rp_in[i], e = rp_in[i + 1];
        float2 acc = make_float2(0.f, 0.f);
        const bool mine = (mask >> c & 1u) != 0;
        if (!mine) {
            // this column keeps its fluid
        } else if (e - b > kPullHeavy) {
            if (slot == 0) {
                int lo = 0, hi = n_heavy - 1;
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (heavy_rows[mid] < i) lo = mid + 1; else hi = mid;
                }
                for (int ch = heavy_chunk_off[lo]; ch < heavy_chunk_off[lo + 1]; ch++)
                    acc = tdf_add(acc, heavy_partial[(int64_t)ch * T + c]);
            }
        } else {
            for (int64_t k = b + slot; k < e; k += SL) acc = tdf_add(acc, y[(int64_t)__ldcs(col_in + k) * T + c]);
        }
#pragma unroll
        for (int o = 16; o >= T; o >>= 1) {
            float2 t;
            t.x = __shfl_xor_sync(kFull, acc.x, o);
            t.y = __shfl_xor_sync(kFull, acc.y, o);
            acc = tdf_add(acc, t);
        }
        if (lane < T && mine) {
            const int64_t idx = i * T + c;
            const double fs = Bn[idx] + ((double)acc.x + (double)acc.y) - H[idx];
            F[idx] = (float)fs;
            colsum += fabs(fs);
        }
    }
    if (lane < T) ssum[warp][lane] = colsum;
    __syncthreads();
    if (tid < T) {
        double s = 0.0;
        for (int w = 0; w < 8; w++) s += ssum[w][tid];
        partials[(int64_t)blockIdx.x * T + tid] = s;
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) is_last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    if (tid < T && (mask >> tid & 1u)) {
        double tot = 0.0;
        for (int bb = 0; bb < (int)gridDim.x; bb++) tot += __ldcg(&partials[(int64_t)bb * T + tid]);
        out_l1[tid] = tot;
    }
    __syncthreads();
    if (tid == 0) ctl->ticket = 0;
}

// X[(c0 + c) * n + i] = H[i*T + c] for c < ncols   (column-major output block)
template <int T>
__global__ void kb_extract(const double *H, int32_t n, int ncols, double *X) {
    const int64_t total = (int64_t)n * ncols;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = idx / n, i = idx % n;
        X[idx] = H[i * T + c];
    }
}

static int tile_index(int T) { return T == 4 ? 0 : T == 8 ? 1 : T == 16 ? 2 : 3; }

// The batched workspace's buffers for tiles of up to T columns, in a fixed order; `take(buffer,
// bytes)` allocates, binds or counts each.
template <class Take>
static void batch_layout(di_graph *g, BatchWorkspace &w, int T, Take &&take) {
    const size_t n = (size_t)g->n, t = (size_t)T;
    take(w.F, sizeof(float) * n * t);
    take(w.H, sizeof(double) * n * t);
    take(w.Bn, sizeof(double) * n * t);
    take(w.front_id, sizeof(int32_t) * n);
    take(w.heavy_cstart, sizeof(int32_t) * n);
    // a heavy node has at most out / chunk + 1 chunks (chunk >= kHeavyChunkMin), and each node is
    // one entry per sweep
    take(w.heavy_chunk, sizeof(int32_t) * (size_t)(g->L / kHeavyChunkMin + g->n_heavy_out + 1));
    take(w.front_s, sizeof(float) * n * t);
    take(w.heavy_partial, sizeof(float2) * (size_t)(g->n_heavy_in_chunks + 1) * t);
    take(w.y, sizeof(float2) * n * t);
    take(w.partials, sizeof(double) * kReduceBlocks * kMaxT);
    take(w.ctl, sizeof(BatchCtl));
    take(w.stage, sizeof(double) * n * t);   // host <-> device staging of B, X and seed lists
}

static size_t batch_bytes(di_graph *g, int T) {
    BatchWorkspace scratch;   // only counted, never allocated
    Carve c;
    batch_layout(g, scratch, T, [&](DevBuf &b, size_t n) { c.take(b, n); });
    return c.used;
}

static void ensure_batch(di_graph *g, BatchWorkspace &w, int T) {
    if (w.T_alloc < T) {
        for (auto &e : w.exec)
            if (e) cudaGraphExecDestroy(e);
        for (auto &e : w.exec) e = nullptr;
        if (w.ext) {
            const size_t need = batch_bytes(g, T);
            DI_REQUIRE(w.ext_bytes >= need, DI_ERR_INVALID_ARG,
                       "the attached batch workspace holds %zu bytes; tiles of %d columns need %zu (di_workspace_size)",
                       w.ext_bytes, T, need);
            Carve c{static_cast<char *>(w.ext), w.ext_bytes};
            batch_layout(g, w, T, [&](DevBuf &b, size_t n) { c.take(b, n); });
        } else {
            batch_layout(g, w, T, [&](DevBuf &b, size_t n) { b.ensure(n); });
        }
        w.T_alloc = T;
    }
    if (!w.capture_stream) DI_CHECK_CUDA(cudaStreamCreateWithFlags(&w.capture_stream, cudaStreamNonBlocking));
    if (!w.ctl_host) DI_CHECK_CUDA(cudaMallocHost(&w.ctl_host, sizeof(BatchCtl)));
}

struct BLaunch {
    int ew, sel, push, red, pull;
};

template <int T>
static BLaunch blaunch(const di_graph *g) {
    BLaunch l;
    const int sms = g->dev.sms;
    const int64_t n = g->n;
    auto cap = [&](int64_t want, int64_t lim) { return (int)(want < 1 ? 1 : (want < lim ? want : lim)); };
    l.ew = cap((n * T + 255) / 256, (int64_t)sms * 8);
    int occ = 0;
    DI_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_select<T>, 256, 0));
    l.sel = cap((n + 255) / 256, (int64_t)sms * (occ > 0 ? occ : 1));   // one wave of 256-node chunks
    DI_CHECK_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kb_push<T>, 256, 0));
    l.push = sms * (occ > 0 ? occ : 1);
    l.red = cap((n * T + 255) / 256, (int64_t)(sms * 4 < kReduceBlocks ? sms * 4 : kReduceBlocks));
    l.pull = cap((n + 7) / 8, (int64_t)(sms * 8 < kReduceBlocks ? sms * 8 : kReduceBlocks));
    return l;
}

// One sweep of a tile: select, push, reduce. `kc` (host-driven sweeps only) times each kernel.
template <int T>
static void batch_body(di_graph *g, BatchWorkspace &w, const BLaunch &l, cudaStream_t s, cudaGraphConditionalHandle h,
                       int set_cond, KernelClock *kc = nullptr) {
    BatchCtl *ctl = w.ctl.as<BatchCtl>();
    const PushTune tune = g->tune_batch;
    KernelClock none(false, s);
    KernelClock &c = kc ? *kc : none;
    c.run(KC_SELECT, 1, [&] {
        kb_select<T><<<l.sel, 256, 0, s>>>(w.F.as<float>(), w.H.as<double>(), g->out_info.as<int32_t>(), g->n, ctl,
                                           w.front_id.as<int32_t>(), w.front_s.as<float>(),
                                           w.heavy_cstart.as<int32_t>(), w.heavy_chunk.as<int32_t>(), tune.heavy,
                                           tune.chunk);
    });
    c.run(KC_PUSH, 1, [&] {
        kb_push<T><<<l.push, 256, 0, s>>>(w.front_id.as<int32_t>(), w.front_s.as<float>(), w.heavy_cstart.as<int32_t>(),
                                          w.heavy_chunk.as<int32_t>(), g->rp_out.as<int64_t>(),
                                          g->col_out.as<int32_t>(), w.F.as<float>(), ctl, tune.heavy, tune.chunk);
    });
    c.run(KC_REDUCE, 1, [&] {
        kb_reduce<T><<<l.red, 256, 0, s>>>(w.F.as<float>(), g->n, w.partials.as<double>(), ctl, h, set_cond);
    });
}

template <int T>
static cudaGraphExec_t batch_graph(di_graph *g, BatchWorkspace &w, const BLaunch &l) {
    cudaGraphExec_t &ex = w.exec[tile_index(T)];
    if (ex && !(w.exec_tune[tile_index(T)] == g->tune_batch)) {
        cudaGraphExecDestroy(ex);
        ex = nullptr;
    }
    if (ex) return ex;
    w.exec_tune[tile_index(T)] = g->tune_batch;
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
    DI_CHECK_CUDA(cudaStreamBeginCaptureToGraph(w.capture_stream, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                cudaStreamCaptureModeThreadLocal));
    batch_body<T>(g, w, l, w.capture_stream, h, 1);
    cudaGraph_t captured;
    DI_CHECK_CUDA(cudaStreamEndCapture(w.capture_stream, &captured));
    DI_CHECK_CUDA(cudaGraphInstantiate(&ex, graph, 0));
    DI_CHECK_CUDA(cudaGraphDestroy(graph));
    return ex;
}

// Exact residual of the columns in `mask`: F_c <- F*_c and ctl->r[c] <- ||F*_c||_1; other
// columns are untouched, and their lanes issue no loads.
template <int T>
static void batch_resid(di_graph *g, BatchWorkspace &w, const BLaunch &l, double d, cudaStream_t s,
                        uint32_t mask = 0xffffffffu) {
    BatchCtl *ctl = w.ctl.as<BatchCtl>();
    kb_resid_y<T><<<l.ew, 256, 0, s>>>(w.H.as<double>(), g->out_info.as<int32_t>(), g->n, d, mask, w.y.as<float2>());
    if (g->n_heavy_in_chunks > 0) {
        int blocks = (g->n_heavy_in_chunks + 7) / 8;
        if (blocks > g->dev.sms * 8) blocks = g->dev.sms * 8;
        kb_resid_heavy<T><<<blocks, 256, 0, s>>>(g->rp_in.as<int64_t>(), g->col_in.as<int32_t>(),
                                                 g->heavy_in_rows.as<int32_t>(), g->heavy_in_chunk_off.as<int32_t>(),
                                                 g->heavy_in_chunk_row.as<int32_t>(), g->n_heavy_in_chunks,
                                                 w.y.as<float2>(), mask, w.heavy_partial.as<float2>());
    }
    kb_resid<T><<<l.pull, 256, 0, s>>>(g->rp_in.as<int64_t>(), g->col_in.as<int32_t>(), w.y.as<float2>(),
                                       g->heavy_in_rows.as<int32_t>(), g->heavy_in_chunk_off.as<int32_t>(),
                                       w.heavy_partial.as<float2>(), g->n_heavy_in, w.Bn.as<double>(),
                                       w.H.as<double>(), g->n, mask, w.F.as<float>(), ctl->r, w.partials.as<double>(),
                                       ctl);
}

static void read_bctl(BatchWorkspace &w, cudaStream_t s) {
    DI_CHECK_CUDA(cudaMemcpyAsync(w.ctl_host, w.ctl.p, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
    DI_CHECK_CUDA(cudaStreamSynchronize(s));
}


}  // namespace di
