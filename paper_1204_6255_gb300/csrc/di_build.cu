// Graph build on the GPU: the paper's iterator "Init" (Section 2.1, Section 2.5 out[], in[],
// l_out, l_in) and the statistics of Section 2.4 (L, D, E, O, max_in, max_out).
//
// Pipeline (all integer work, bit-exact and deterministic):
//   validate ids and pack each link as key = src << bits | dst
//   -> stable LSD radix sort of the keys (8-bit digits, tile histograms + scan + ranked scatter)
//   -> drop repeated keys (flag scan + compaction)
//   -> out-CSR (rows by origin, destinations ascending) + loop flags
//   -> re-pack as dst << bits | src and stable-sort on the dst field only, which keeps origins
//      ascending inside each row -> in-CSR
//   -> degrees, statistics, and E by level-synchronous peeling (Section 2.4), recording E grouped
//      by level for the E pre-diffusion
//   -> for the push kernels: a hash table of the highest in-degree nodes (hubs) and a copy of
//      the out-links with bit 31 set on links into a hub; for the pull kernels: the rows with
//      more in-links than one warp should walk, split into chunks.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "di_internal.cuh"

namespace di {

// ------------------------------------------------------------------------------------------
// errors and small host utilities
// ------------------------------------------------------------------------------------------
static thread_local std::string g_last_error;
std::atomic<long long> g_device_bytes{0};

void set_error(const char *fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
}
void clear_error() { g_last_error.clear(); }
const char *last_error() { return g_last_error.c_str(); }

bool is_device_ptr(const void *ptr) {
    if (!ptr) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void to_device(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (!bytes) return;
    DI_CHECK_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
}
void from_device(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    if (!bytes) return;
    DI_CHECK_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, s));
}

DeviceInfo query_device() {
    DeviceInfo d;
    DI_CHECK_CUDA(cudaGetDevice(&d.device));
    DI_CHECK_CUDA(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, d.device));
    DI_CHECK_CUDA(cudaDeviceGetAttribute(&d.max_threads_per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, d.device));
    int l2 = 0;
    DI_CHECK_CUDA(cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, d.device));
    d.l2_bytes = (size_t)l2;
    return d;
}

static int grid_for(int64_t items, int threads, const DeviceInfo &dev, int per_sm = 8) {
    int64_t want = (items + threads - 1) / threads;
    int64_t cap = (int64_t)dev.sms * per_sm;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

// ------------------------------------------------------------------------------------------
// tile scans (warp-striped: warp w owns items [w*32*ITEMS, (w+1)*32*ITEMS) of the tile and
// visits them 32 consecutive items at a time, so loads are coalesced)
// ------------------------------------------------------------------------------------------
constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;   // 4096
constexpr int kWarps = kThreads / 32;

// Exclusive scan of v[] across the tile; returns the tile total to every thread.
__device__ __forceinline__ uint32_t tile_exclusive_scan(uint32_t (&v)[kItems], uint32_t *wsum) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t carry = 0;
#pragma unroll
    for (int j = 0; j < kItems; j++) {
        uint32_t x = v[j];
        uint32_t inc = warp_inclusive_scan(x);
        v[j] = carry + inc - x;
        carry += __shfl_sync(kFull, inc, 31);
    }
    __syncthreads();
    if (lane == 0) wsum[warp] = carry;
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < kWarps; w++) {
        if (w < warp) before += wsum[w];
        total += wsum[w];
    }
#pragma unroll
    for (int j = 0; j < kItems; j++) v[j] += before;
    return total;
}

__device__ __forceinline__ int64_t tile_index(int j) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    return (int64_t)blockIdx.x * kTile + warp * (32 * kItems) + j * 32 + lane;
}

// ---- generic exclusive scan of uint32 values (length n), writing n+1 outputs (last = total)
__global__ void k_scan_reduce(const uint32_t *in, int64_t n, uint32_t *tile_sums) {
    __shared__ uint32_t scratch[kWarps];
    uint32_t s = 0;
    for (int j = 0; j < kItems; j++) {
        int64_t i = tile_index(j);
        if (i < n) s += in[i];
    }
    s = block_sum(s, scratch);
    if (threadIdx.x == 0) tile_sums[blockIdx.x] = s;
}

// Single block: exclusive scan of tile sums in place; writes the grand total to *total.
__global__ void k_scan_tiles(uint32_t *tile_sums, int64_t ntiles, uint32_t *total) {
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry_s;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t base = 0; base < ntiles; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        uint32_t x = i < ntiles ? tile_sums[i] : 0;
        uint32_t inc = warp_inclusive_scan(x);
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        uint32_t before = 0, all = 0;
        for (int w = 0; w < nw; w++) {
            if (w < warp) before += wsum[w];
            all += wsum[w];
        }
        uint32_t c = carry_s;
        if (i < ntiles) tile_sums[i] = c + before + inc - x;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = c + all;
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry_s;
}

__global__ void k_scan_apply(const uint32_t *in, int64_t n, const uint32_t *tile_offs, uint32_t *out) {
    __shared__ uint32_t wsum[kWarps];
    uint32_t v[kItems];
#pragma unroll
    for (int j = 0; j < kItems; j++) {
        int64_t i = tile_index(j);
        v[j] = i < n ? in[i] : 0;
    }
    tile_exclusive_scan(v, wsum);
    const uint32_t base = tile_offs[blockIdx.x];
#pragma unroll
    for (int j = 0; j < kItems; j++) {
        int64_t i = tile_index(j);
        if (i < n) out[i] = base + v[j];
    }
}

// out[0..n] = exclusive scan of in[0..n), out[n] = total. tmp holds ceil(n/kTile)+1 values.
static void exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n, DevBuf &tmp, cudaStream_t s) {
    int64_t ntiles = (n + kTile - 1) / kTile;
    if (ntiles == 0) {
        DI_CHECK_CUDA(cudaMemsetAsync(out, 0, sizeof(uint32_t), s));
        return;
    }
    tmp.ensure(sizeof(uint32_t) * (size_t)(ntiles + 1));
    uint32_t *ts = tmp.as<uint32_t>();
    k_scan_reduce<<<(unsigned)ntiles, kThreads, 0, s>>>(in, n, ts);
    k_scan_tiles<<<1, 1024, 0, s>>>(ts, ntiles, out + n);
    k_scan_apply<<<(unsigned)ntiles, kThreads, 0, s>>>(in, n, ts, out);
    DI_CHECK_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------------------------------
// stable LSD radix sort of uint64 keys on bits [lo_bit, hi_bit)
// ------------------------------------------------------------------------------------------
constexpr int kBins = 256;

__global__ void k_rs_hist(const uint64_t *keys, int64_t m, int shift, uint32_t *hist, int64_t ntiles) {
    __shared__ uint32_t h[kWarps][kBins];
    for (int i = threadIdx.x; i < kWarps * kBins; i += blockDim.x) (&h[0][0])[i] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5;
#pragma unroll 4
    for (int j = 0; j < kItems; j++) {
        int64_t i = tile_index(j);
        if (i < m) atomicAdd(&h[warp][(unsigned)(keys[i] >> shift) & 0xffu], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) {
        uint32_t s = 0;
        for (int w = 0; w < kWarps; w++) s += h[w][b];
        hist[(int64_t)b * ntiles + blockIdx.x] = s;   // digit-major
    }
}

__global__ void k_rs_scatter(const uint64_t *in, uint64_t *out, int64_t m, int shift, const uint32_t *offs,
                             int64_t ntiles) {
    __shared__ uint32_t wcnt[kWarps][kBins];
    __shared__ uint32_t gbase[kBins];
    for (int i = threadIdx.x; i < kWarps * kBins; i += blockDim.x) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt = lanemask_lt();
    uint64_t key[kItems];
    uint32_t rank[kItems];
#pragma unroll
    for (int j = 0; j < kItems; j++) {
        int64_t i = tile_index(j);
        bool valid = i < m;
        uint64_t k = valid ? in[i] : 0;
        unsigned digit = valid ? ((unsigned)(k >> shift) & 0xffu) : 0x100u;
        unsigned peers = __match_any_sync(kFull, digit);
        uint32_t before = valid ? wcnt[warp][digit] : 0;
        __syncwarp();
        if (valid && lane == 31 - __clz(peers)) wcnt[warp][digit] = before + __popc(peers);
        __syncwarp();
        key[j] = k;
        rank[j] = before + __popc(peers & lt);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kBins; b += blockDim.x) {
        uint32_t run = 0;
        for (int w = 0; w < kWarps; w++) {
            uint32_t c = wcnt[w][b];
            wcnt[w][b] = run;
            run += c;
        }
        gbase[b] = offs[(int64_t)b * ntiles + blockIdx.x];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kItems; j++) {
        int64_t i = tile_index(j);
        if (i < m) {
            unsigned digit = (unsigned)(key[j] >> shift) & 0xffu;
            out[gbase[digit] + wcnt[warp][digit] + rank[j]] = key[j];
        }
    }
}

// Sorts keys (length m) on bits [lo_bit, hi_bit); the result is in *keys (buffers may swap).
static void radix_sort(DevBuf &keys, DevBuf &alt, int64_t m, int lo_bit, int hi_bit, DevBuf &hist,
                       DevBuf &scan_tmp, cudaStream_t s) {
    if (m <= 1 || hi_bit <= lo_bit) return;
    int64_t ntiles = (m + kTile - 1) / kTile;
    int64_t nh = ntiles * kBins;
    hist.ensure(sizeof(uint32_t) * (size_t)(2 * nh + 1));
    uint32_t *h = hist.as<uint32_t>();
    uint32_t *offs = h + nh;
    alt.ensure(sizeof(uint64_t) * (size_t)m);
    for (int shift = lo_bit; shift < hi_bit; shift += 8) {
        k_rs_hist<<<(unsigned)ntiles, kThreads, 0, s>>>(keys.as<uint64_t>(), m, shift, h, ntiles);
        exclusive_scan_u32(h, offs, nh, scan_tmp, s);
        k_rs_scatter<<<(unsigned)ntiles, kThreads, 0, s>>>(keys.as<uint64_t>(), alt.as<uint64_t>(), m, shift,
                                                           offs, ntiles);
        DI_CHECK_CUDA(cudaGetLastError());
        std::swap(keys.p, alt.p);
        std::swap(keys.bytes, alt.bytes);
    }
}

// ------------------------------------------------------------------------------------------
// link packing, dedupe, CSR
// ------------------------------------------------------------------------------------------
__global__ void k_pack(const int32_t *src, const int32_t *dst, int64_t m, int32_t n, int bits, uint64_t *keys,
                       unsigned long long *first_bad) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        int32_t a = src[e], b = dst[e];
        if (a < 0 || a >= n || b < 0 || b >= n) {
            atomicMin(first_bad, (unsigned long long)e);
            keys[e] = 0;
        } else {
            keys[e] = ((uint64_t)(uint32_t)a << bits) | (uint64_t)(uint32_t)b;
        }
    }
}

// flag[i] = 1 when key i starts a run of equal keys
__global__ void k_unique_flags(const uint64_t *keys, int64_t m, uint32_t *flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void k_compact(const uint64_t *keys, const uint32_t *flag, const uint32_t *pos, int64_t m, uint64_t *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        if (flag[i]) out[pos[i]] = keys[i];
}

// Sorted unique keys hi << bits | lo  ->  col[e] = lo, loop flags (optional).
__global__ void k_csr_cols(const uint64_t *keys, int64_t L, int bits, int32_t *col, uint8_t *loop) {
    const uint64_t mask = (1ull << bits) - 1;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L; e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[e];
        uint32_t hi = (uint32_t)(k >> bits), lo = (uint32_t)(k & mask);
        col[e] = (int32_t)lo;
        if (loop && hi == lo) loop[hi] = 1;
    }
}

// rp[v] = first e with (keys[e] >> bits) >= v, for v in [0, n]  (lower bound by binary search)
__global__ void k_csr_rowptr(const uint64_t *keys, int64_t L, int bits, int32_t n, int64_t *rp) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v <= n; v += (int64_t)gridDim.x * blockDim.x) {
        uint64_t target = (uint64_t)v << bits;
        int64_t lo = 0, hi = L;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (keys[mid] < target) lo = mid + 1; else hi = mid;
        }
        rp[v] = lo;
    }
}

__global__ void k_repack_in(const uint64_t *keys, int64_t L, int bits, uint64_t *out) {
    const uint64_t mask = (1ull << bits) - 1;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L; e += (int64_t)gridDim.x * blockDim.x) {
        uint64_t k = keys[e];
        out[e] = ((k & mask) << bits) | (k >> bits);
    }
}

struct BuildStats {
    unsigned long long D, O;
    int max_in, max_out;
};

__global__ void k_degrees(const int64_t *rp_out, const int64_t *rp_in, const uint8_t *loop, int32_t n,
                          int32_t *out_deg, int32_t *in_deg, int32_t *out_info, BuildStats *st) {
    __shared__ unsigned long long sD[32], sO[32];
    __shared__ int smi[32], smo[32];
    unsigned long long D = 0, O = 0;
    int mi = 0, mo = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t o = (int32_t)(rp_out[v + 1] - rp_out[v]);
        int32_t i = (int32_t)(rp_in[v + 1] - rp_in[v]);
        uint8_t lp = loop[v];
        out_deg[v] = o;
        in_deg[v] = i;
        out_info[v] = o | (lp ? (int32_t)0x80000000u : 0);
        D += (o == 0);
        O += (lp != 0);
        mi = max(mi, i);
        mo = max(mo, o);
    }
    D = warp_sum(D);
    O = warp_sum(O);
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        mi = max(mi, __shfl_xor_sync(kFull, mi, s));
        mo = max(mo, __shfl_xor_sync(kFull, mo, s));
    }
    const int warp = threadIdx.x >> 5;
    if (lane_id() == 0) { sD[warp] = D; sO[warp] = O; smi[warp] = mi; smo[warp] = mo; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
            sD[0] += sD[w]; sO[0] += sO[w];
            smi[0] = max(smi[0], smi[w]); smo[0] = max(smo[0], smo[w]);
        }
        atomicAdd(&st->D, sD[0]);
        atomicAdd(&st->O, sO[0]);
        atomicMax(&st->max_in, smi[0]);
        atomicMax(&st->max_out, smo[0]);
    }
}

// ------------------------------------------------------------------------------------------
// E: level-synchronous peeling (Section 2.4)
// ------------------------------------------------------------------------------------------
__global__ void k_e_init(const int32_t *in_deg, int32_t n, int32_t *left, uint8_t *e_mask, int32_t *e_level,
                         int32_t *frontier, int32_t *count) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t d = in_deg[v];
        left[v] = d;
        bool z = d == 0;
        e_mask[v] = z ? 1 : 0;
        e_level[v] = z ? 0 : -1;
        if (z) frontier[atomicAdd(count, 1)] = (int32_t)v;
    }
}

// One level: every member u of the frontier removes its out-links; a node whose remaining
// in-degree reaches zero joins E at level `level`. One warp per frontier node.
__global__ void k_e_peel(const int32_t *frontier, const int32_t *count, const int64_t *rp_out, const int32_t *col_out,
                         int32_t *left, uint8_t *e_mask, int32_t *e_level, int32_t level, int32_t *next,
                         int32_t *next_count) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t cnt = *count;
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < cnt; w += nwarps) {
        int32_t u = frontier[w];
        for (int64_t k = rp_out[u] + lane; k < rp_out[u + 1]; k += 32) {
            int32_t x = col_out[k];
            if (atomicSub(&left[x], 1) == 1) {
                e_mask[x] = 1;
                e_level[x] = level;
                next[atomicAdd(next_count, 1)] = x;
            }
        }
    }
}

// The pull's links per row (rows above kPullHeavy in-links count 0: they are summed apart), and
// samples of their prefix at rows k * n / samples, k = 0..samples.
__global__ void k_pull_links(const int32_t *in_deg, int32_t n, uint32_t *links) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = in_deg[v];
        links[v] = d > kPullHeavy ? 0u : (uint32_t)d;
    }
}
__global__ void k_sample_prefix(const uint32_t *prefix, int32_t n, int samples, int64_t *out) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k <= samples; k += gridDim.x * blockDim.x)
        out[k] = (int64_t)prefix[(int64_t)k * n / samples];
}

// Heavy rows of the in-CSR (in-degree > kPullHeavy) and their chunk lists.
__global__ void k_heavy_in_flags(const int32_t *in_deg, int32_t n, uint32_t *flag, uint32_t *nchunks) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t d = in_deg[v];
        bool h = d > kPullHeavy;
        flag[v] = h ? 1u : 0u;
        nchunks[v] = h ? (uint32_t)((d + kPullChunk - 1) / kPullChunk) : 0u;
    }
}

__global__ void k_heavy_in_lists(const uint32_t *flag, const uint32_t *flag_pos, const uint32_t *chunk_pos, int32_t n,
                                 int32_t *rows, int32_t *chunk_off, int32_t *chunk_row, const int32_t *in_deg) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        if (!flag[v]) continue;
        uint32_t h = flag_pos[v];
        rows[h] = (int32_t)v;
        uint32_t c0 = chunk_pos[v];
        chunk_off[h] = (int32_t)c0;
        int32_t nc = (in_deg[v] + kPullChunk - 1) / kPullChunk;
        for (int32_t c = 0; c < nc; c++) chunk_row[c0 + c] = (int32_t)h;
    }
}

__global__ void k_count_heavy_out(const int32_t *out_deg, int32_t n, unsigned long long *cnt) {
    unsigned long long c = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        c += out_deg[v] > kPushHeavyMin;
    c = warp_sum(c);
    if (lane_id() == 0 && c) atomicAdd(cnt, c);
}

// Hub table: the nodes of highest in-degree, by open hashing into kHubSlots slots; a slot keeps
// the candidate with the larger in-degree (packed in-degree << 32 | id, atomicMax).
__global__ void k_indeg_hist(const int32_t *in_deg, int32_t n, unsigned long long *hist) {
    __shared__ unsigned int h[32];
    if (threadIdx.x < 32) h[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = in_deg[v];
        if (d > 0) atomicAdd(&h[31 - __clz(d)], 1u);
    }
    __syncthreads();
    if (threadIdx.x < 32 && h[threadIdx.x]) atomicAdd(&hist[threadIdx.x], (unsigned long long)h[threadIdx.x]);
}

__global__ void k_hub_insert(const int32_t *in_deg, int32_t n, int32_t min_deg, unsigned long long *slots) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t d = in_deg[v];
        if (d >= min_deg) atomicMax(&slots[hub_slot((int32_t)v)], ((unsigned long long)(uint32_t)d << 32) | (uint32_t)v);
    }
}

__global__ void k_hub_finalize(const unsigned long long *slots, int32_t *ids) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kHubSlots) ids[i] = slots[i] ? (int32_t)(uint32_t)(slots[i] & 0xffffffffu) : -1;
}

// Largest number of in-links that a node which is not a hub receives from sources less than
// `reach` ids away (the rows of col_in are sorted, so two binary searches per node). The push
// window adds at most one link per source of a segment into a slot, and only from sources that
// near, so this bounds the adds into any window slot per segment.
__global__ void k_window_reach(const int64_t *rp_in, const int32_t *col_in, int32_t n, const int32_t *hub_ids,
                               int32_t reach, unsigned int *max_cnt) {
    unsigned int best = 0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        if (__ldg(hub_ids + hub_slot((int32_t)j)) == (int32_t)j) continue;
        const int64_t b = rp_in[j], e = rp_in[j + 1];
        const int64_t lo_id = j - reach + 1, hi_id = j + reach - 1;
        int64_t a = b, z = e;   // first link with id >= lo_id
        while (a < z) {
            const int64_t m = (a + z) >> 1;
            if (col_in[m] < lo_id) a = m + 1; else z = m;
        }
        int64_t c = a, y = e;   // first link with id > hi_id
        while (c < y) {
            const int64_t m = (c + y) >> 1;
            if (col_in[m] <= hi_id) c = m + 1; else y = m;
        }
        const unsigned int cnt = (unsigned int)(c - a);
        best = cnt > best ? cnt : best;
    }
    atomicMax(max_cnt, best);
}

// (level << bits | id) keys of the nodes of E, and back to ids after sorting
__global__ void k_e_keys(const int32_t *order, int64_t cnt, const int32_t *level, int bits, uint64_t *keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = order[i];
        keys[i] = ((uint64_t)(uint32_t)level[v] << bits) | (uint64_t)(uint32_t)v;
    }
}
__global__ void k_e_unkey(const uint64_t *keys, int64_t cnt, int bits, int32_t *order) {
    const uint64_t mask = (1ull << bits) - 1;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        order[i] = (int32_t)(keys[i] & mask);
}

// the push kernels' copy of the link targets: bit 31 marks a target that owns its hub slot
__global__ void k_mark_hub_links(const int32_t *col_out, int64_t L, const int32_t *hub_ids, int32_t *col_push) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < L; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = col_out[k];
        col_push[k] = __ldg(hub_ids + hub_slot(j)) == j ? (int32_t)((uint32_t)j | 0x80000000u) : j;
    }
}

// In the push kernels' copy, a loop node's self-link is swapped with the last link of its row, so
// a push that diffuses the loop in closed form simply stops one link short of the row's end
// instead of comparing every link with the source.
__global__ void k_loop_last(const int64_t *rp, const uint8_t *loop, int32_t n, int32_t *col_push) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        if (!loop[u]) continue;
        int64_t lo = rp[u], hi = rp[u + 1] - 1;   // rows are sorted, and the self-link is in the row
        const int64_t last = hi;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((col_push[mid] & 0x7fffffff) < (int32_t)u) lo = mid + 1; else hi = mid;
        }
        const int32_t self = col_push[lo];
        col_push[lo] = col_push[last];
        col_push[last] = self;
    }
}

// the push kernels' row bounds: rp_out narrowed to 32 bits (L < 2^31), so one 32-byte sector
// holds eight nodes' bounds instead of four. Bit 31 of a node's row end (the next node's entry)
// marks a loop node, whose self-link k_loop_last moved to the row's last link.
__global__ void k_narrow_rows(const int64_t *rp, const uint8_t *loop, int64_t count, int32_t *out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count; k += (int64_t)gridDim.x * blockDim.x)
        out[k] = (int32_t)((uint32_t)rp[k] | (k > 0 && loop[k - 1] ? 0x80000000u : 0u));
}

static int ceil_log2(int64_t x) {
    int b = 0;
    while ((int64_t(1) << b) < x) b++;
    return b < 1 ? 1 : b;
}

}  // namespace di

using namespace di;

static void build_graph(di_graph *g, const int32_t *src_in, const int32_t *dst_in, int64_t m, cudaStream_t s) {
    const int32_t n = g->n;
    g->dev = query_device();
    const DeviceInfo &dev = g->dev;
    g->bits = ceil_log2(n);
    const int bits = g->bits;

    // link arrays on the device
    DevBuf d_src, d_dst;
    const int32_t *src = src_in, *dst = dst_in;
    if (m > 0 && !is_device_ptr(src_in)) {
        d_src.ensure(sizeof(int32_t) * (size_t)m);
        to_device(d_src.p, src_in, sizeof(int32_t) * (size_t)m, s);
        src = d_src.as<int32_t>();
    }
    if (m > 0 && !is_device_ptr(dst_in)) {
        d_dst.ensure(sizeof(int32_t) * (size_t)m);
        to_device(d_dst.p, dst_in, sizeof(int32_t) * (size_t)m, s);
        dst = d_dst.as<int32_t>();
    }

    DevBuf keys, alt, hist, scan_tmp, misc;
    misc.ensure(256);
    unsigned long long *first_bad = misc.as<unsigned long long>();
    BuildStats *bst = reinterpret_cast<BuildStats *>(misc.as<char>() + 64);
    int32_t *counts = reinterpret_cast<int32_t *>(misc.as<char>() + 128);
    DI_CHECK_CUDA(cudaMemsetAsync(misc.p, 0, 256, s));
    DI_CHECK_CUDA(cudaMemsetAsync(first_bad, 0xff, sizeof(unsigned long long), s));

    int64_t L = 0;
    if (m > 0) {
        keys.ensure(sizeof(uint64_t) * (size_t)m);
        k_pack<<<grid_for(m, 256, dev), 256, 0, s>>>(src, dst, m, n, bits, keys.as<uint64_t>(), first_bad);
        DI_CHECK_CUDA(cudaGetLastError());
        unsigned long long bad = 0;
        DI_CHECK_CUDA(cudaMemcpyAsync(&bad, first_bad, sizeof(bad), cudaMemcpyDeviceToHost, s));
        DI_CHECK_CUDA(cudaStreamSynchronize(s));
        d_src.release();
        d_dst.release();
        if (bad != ~0ull) {
            int32_t a = 0, b = 0;
            // report the offending pair (read back from the caller's arrays)
            from_device(&a, src_in + bad, sizeof(int32_t), s);
            from_device(&b, dst_in + bad, sizeof(int32_t), s);
            cudaStreamSynchronize(s);
            set_error("edge %llu (%d -> %d) has an id outside [0, %d)", bad, a, b, n);
            throw Fail{DI_ERR_OUT_OF_RANGE_ID};
        }
        radix_sort(keys, alt, m, 0, 2 * bits, hist, scan_tmp, s);

        // drop repeated links
        DevBuf flag, pos;
        flag.ensure(sizeof(uint32_t) * (size_t)m);
        pos.ensure(sizeof(uint32_t) * (size_t)(m + 1));
        k_unique_flags<<<grid_for(m, 256, dev), 256, 0, s>>>(keys.as<uint64_t>(), m, flag.as<uint32_t>());
        exclusive_scan_u32(flag.as<uint32_t>(), pos.as<uint32_t>(), m, scan_tmp, s);
        uint32_t Lu = 0;
        DI_CHECK_CUDA(cudaMemcpyAsync(&Lu, pos.as<uint32_t>() + m, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        alt.ensure(sizeof(uint64_t) * (size_t)m);
        k_compact<<<grid_for(m, 256, dev), 256, 0, s>>>(keys.as<uint64_t>(), flag.as<uint32_t>(), pos.as<uint32_t>(), m,
                                                      alt.as<uint64_t>());
        DI_CHECK_CUDA(cudaGetLastError());
        DI_CHECK_CUDA(cudaStreamSynchronize(s));
        std::swap(keys.p, alt.p);
        std::swap(keys.bytes, alt.bytes);
        L = Lu;
    }
    g->L = L;

    // out-CSR
    g->rp_out.ensure(sizeof(int64_t) * ((size_t)n + 1));
    g->col_out.ensure(sizeof(int32_t) * (size_t)(L > 0 ? L : 1));
    g->loop.ensure((size_t)n);
    DI_CHECK_CUDA(cudaMemsetAsync(g->loop.p, 0, (size_t)n, s));
    if (L > 0) {
        k_csr_cols<<<grid_for(L, 256, dev), 256, 0, s>>>(keys.as<uint64_t>(), L, bits, g->col_out.as<int32_t>(),
                                                       g->loop.as<uint8_t>());
    }
    k_csr_rowptr<<<grid_for((int64_t)n + 1, 256, dev), 256, 0, s>>>(keys.as<uint64_t>(), L, bits, n,
                                                                   g->rp_out.as<int64_t>());
    DI_CHECK_CUDA(cudaGetLastError());

    // in-CSR: stable sort on the destination field keeps origins ascending within each row
    g->rp_in.ensure(sizeof(int64_t) * ((size_t)n + 1));
    // padded by kColInPad: the pull reads whole 16-byte vectors of links around a group's range
    g->col_in.ensure(sizeof(int32_t) * ((size_t)L + kColInPad));
    DI_CHECK_CUDA(cudaMemsetAsync(g->col_in.as<int32_t>() + L, 0, sizeof(int32_t) * kColInPad, s));
    if (L > 0) {
        alt.ensure(sizeof(uint64_t) * (size_t)L);
        k_repack_in<<<grid_for(L, 256, dev), 256, 0, s>>>(keys.as<uint64_t>(), L, bits, alt.as<uint64_t>());
        std::swap(keys.p, alt.p);
        std::swap(keys.bytes, alt.bytes);
        radix_sort(keys, alt, L, bits, 2 * bits, hist, scan_tmp, s);
        k_csr_cols<<<grid_for(L, 256, dev), 256, 0, s>>>(keys.as<uint64_t>(), L, bits, g->col_in.as<int32_t>(), nullptr);
    }
    k_csr_rowptr<<<grid_for((int64_t)n + 1, 256, dev), 256, 0, s>>>(keys.as<uint64_t>(), L, bits, n,
                                                                   g->rp_in.as<int64_t>());
    DI_CHECK_CUDA(cudaGetLastError());
    keys.release();
    alt.release();
    hist.release();

    // degrees, flags, statistics
    g->out_deg.ensure(sizeof(int32_t) * (size_t)n);
    g->in_deg.ensure(sizeof(int32_t) * (size_t)n);
    g->out_info.ensure(sizeof(int32_t) * (size_t)n);
    k_degrees<<<grid_for(n, 256, dev), 256, 0, s>>>(g->rp_out.as<int64_t>(), g->rp_in.as<int64_t>(),
                                                  g->loop.as<uint8_t>(), n, g->out_deg.as<int32_t>(),
                                                  g->in_deg.as<int32_t>(), g->out_info.as<int32_t>(), bst);
    unsigned long long *heavy_out_cnt = reinterpret_cast<unsigned long long *>(misc.as<char>() + 192);
    k_count_heavy_out<<<grid_for(n, 256, dev), 256, 0, s>>>(g->out_deg.as<int32_t>(), n, heavy_out_cnt);
    DI_CHECK_CUDA(cudaGetLastError());

    // hub table (highest in-degree nodes) for the push kernels' shared-memory hub cache
    {
        DevBuf hist, slots;
        hist.ensure(sizeof(unsigned long long) * 32);
        DI_CHECK_CUDA(cudaMemsetAsync(hist.p, 0, sizeof(unsigned long long) * 32, s));
        k_indeg_hist<<<grid_for(n, 256, dev), 256, 0, s>>>(g->in_deg.as<int32_t>(), n, hist.as<unsigned long long>());
        unsigned long long hh[32];
        DI_CHECK_CUDA(cudaMemcpyAsync(hh, hist.p, sizeof(hh), cudaMemcpyDeviceToHost, s));
        DI_CHECK_CUDA(cudaStreamSynchronize(s));
        // smallest power-of-two in-degree bound that leaves at most 2 * kHubSlots candidates
        int b = 31;
        unsigned long long above = 0;
        while (b > 6 && above + hh[b - 1] <= 2ull * kHubSlots) above += hh[--b];
        const int32_t min_deg = (int32_t)1 << b;
        slots.ensure(sizeof(unsigned long long) * kHubSlots);
        DI_CHECK_CUDA(cudaMemsetAsync(slots.p, 0, sizeof(unsigned long long) * kHubSlots, s));
        k_hub_insert<<<grid_for(n, 256, dev), 256, 0, s>>>(g->in_deg.as<int32_t>(), n, min_deg,
                                                         slots.as<unsigned long long>());
        g->hub_ids.ensure(sizeof(int32_t) * kHubSlots);
        k_hub_finalize<<<(kHubSlots + 255) / 256, 256, 0, s>>>(slots.as<unsigned long long>(), g->hub_ids.as<int32_t>());
        g->col_push.ensure(sizeof(int32_t) * (size_t)(L > 0 ? L : 1));
        if (L > 0)
            k_mark_hub_links<<<grid_for(L, 256, dev), 256, 0, s>>>(g->col_out.as<int32_t>(), L, g->hub_ids.as<int32_t>(),
                                                                 g->col_push.as<int32_t>());
        if (L > 0)
            k_loop_last<<<grid_for(n, 256, dev), 256, 0, s>>>(g->rp_out.as<int64_t>(), g->loop.as<uint8_t>(), n,
                                                            g->col_push.as<int32_t>());
        g->rp_push.ensure(sizeof(int32_t) * (size_t)(n + 1));
        k_narrow_rows<<<grid_for((int64_t)n + 1, 256, dev), 256, 0, s>>>(g->rp_out.as<int64_t>(), g->loop.as<uint8_t>(),
                                                                       (int64_t)n + 1, g->rp_push.as<int32_t>());
        // fixed-point width of the push window: a slot sums at most `reach_cnt` shares per
        // segment, each below 2^win_qbits in magnitude, and the sum must stay an int32
        unsigned int *reach_cnt = reinterpret_cast<unsigned int *>(slots.as<char>());
        DI_CHECK_CUDA(cudaMemsetAsync(reach_cnt, 0, sizeof(unsigned int), s));
        k_window_reach<<<grid_for(n, 256, dev), 256, 0, s>>>(g->rp_in.as<int64_t>(), g->col_in.as<int32_t>(), n,
                                                           g->hub_ids.as<int32_t>(), kWinReach, reach_cnt);
        unsigned int rc = 0;
        DI_CHECK_CUDA(cudaMemcpyAsync(&rc, reach_cnt, sizeof(rc), cudaMemcpyDeviceToHost, s));
        DI_CHECK_CUDA(cudaGetLastError());
        DI_CHECK_CUDA(cudaStreamSynchronize(s));
        g->win_reach_max = (int32_t)rc;
        int qb = 30;
        while (qb > 1 && (uint64_t)(rc ? rc : 1) * ((1ull << qb) - 1) > 0x7fffffffull) qb--;
        g->win_qbits = qb;

    }

    // E by peeling; each level's frontier is appended to e_order, so e_order lists E grouped by
    // level (level 0 first) for the pre-diffusion
    g->e_mask.ensure((size_t)n);
    g->e_level.ensure(sizeof(int32_t) * (size_t)n);
    g->e_order.ensure(sizeof(int32_t) * (size_t)n);
    g->e_level_off.assign(1, 0);
    DevBuf left;
    left.ensure(sizeof(int32_t) * (size_t)n);
    int32_t *cnt_a = counts, *cnt_b = counts + 1;
    int32_t *eo = g->e_order.as<int32_t>();
    k_e_init<<<grid_for(n, 256, dev), 256, 0, s>>>(g->in_deg.as<int32_t>(), n, left.as<int32_t>(),
                                                 g->e_mask.as<uint8_t>(), g->e_level.as<int32_t>(), eo, cnt_a);
    DI_CHECK_CUDA(cudaGetLastError());
    int32_t *hcount = nullptr;
    DI_CHECK_CUDA(cudaMallocHost(&hcount, sizeof(int32_t)));
    int64_t e_total = 0;
    int32_t level = 0;
    try {
        for (;;) {
            DI_CHECK_CUDA(cudaMemcpyAsync(hcount, cnt_a, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            DI_CHECK_CUDA(cudaStreamSynchronize(s));
            int32_t c = *hcount;
            if (c == 0) break;
            const int64_t at = e_total;   // this level's frontier: e_order[at, at + c)
            e_total += c;
            g->e_level_off.push_back(e_total);
            level++;
            DI_CHECK_CUDA(cudaMemsetAsync(cnt_b, 0, sizeof(int32_t), s));
            int blocks = grid_for((int64_t)c * 32, 256, dev);
            k_e_peel<<<blocks, 256, 0, s>>>(eo + at, cnt_a, g->rp_out.as<int64_t>(), g->col_out.as<int32_t>(),
                                            left.as<int32_t>(), g->e_mask.as<uint8_t>(), g->e_level.as<int32_t>(),
                                            level, eo + e_total, cnt_b);
            DI_CHECK_CUDA(cudaGetLastError());
            std::swap(cnt_a, cnt_b);
        }
    } catch (...) {
        cudaFreeHost(hcount);
        throw;
    }
    cudaFreeHost(hcount);
    // each level's nodes in ascending id order (a stable sort of (level, id) keys): the
    // pre-diffusion selects a level's nodes by id chunks, so the windowed push sees id-sorted
    // segments
    if (e_total > 1) {
        DevBuf keys, alt, hist2, scan2;
        keys.ensure(sizeof(uint64_t) * (size_t)e_total);
        k_e_keys<<<grid_for(e_total, 256, dev), 256, 0, s>>>(eo, e_total, g->e_level.as<int32_t>(), bits,
                                                             keys.as<uint64_t>());
        int lbits = 1;
        while ((1 << lbits) < level + 1) lbits++;
        radix_sort(keys, alt, e_total, 0, bits + lbits, hist2, scan2, s);
        k_e_unkey<<<grid_for(e_total, 256, dev), 256, 0, s>>>(keys.as<uint64_t>(), e_total, bits, eo);
        DI_CHECK_CUDA(cudaGetLastError());
        DI_CHECK_CUDA(cudaStreamSynchronize(s));
    }
    // the id span of each level (its first and last id, now that levels are sorted)
    g->e_level_span.assign(g->e_level_off.size() > 0 ? g->e_level_off.size() - 1 : 0, 0);
    for (size_t lv = 0; lv + 1 < g->e_level_off.size(); lv++) {
        int32_t ends[2] = {0, 0};
        DI_CHECK_CUDA(cudaMemcpyAsync(&ends[0], eo + g->e_level_off[lv], sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        DI_CHECK_CUDA(cudaMemcpyAsync(&ends[1], eo + g->e_level_off[lv + 1] - 1, sizeof(int32_t),
                                      cudaMemcpyDeviceToHost, s));
        DI_CHECK_CUDA(cudaStreamSynchronize(s));
        g->e_level_span[lv] = (int64_t)ends[1] - ends[0] + 1;
    }

    // heavy in-CSR rows for the pull kernels
    {
        DevBuf flag, fpos, nch, cpos;
        flag.ensure(sizeof(uint32_t) * (size_t)n);
        nch.ensure(sizeof(uint32_t) * (size_t)n);
        fpos.ensure(sizeof(uint32_t) * ((size_t)n + 1));
        cpos.ensure(sizeof(uint32_t) * ((size_t)n + 1));
        k_heavy_in_flags<<<grid_for(n, 256, dev), 256, 0, s>>>(g->in_deg.as<int32_t>(), n, flag.as<uint32_t>(),
                                                             nch.as<uint32_t>());
        exclusive_scan_u32(flag.as<uint32_t>(), fpos.as<uint32_t>(), n, scan_tmp, s);
        exclusive_scan_u32(nch.as<uint32_t>(), cpos.as<uint32_t>(), n, scan_tmp, s);
        uint32_t tot[2] = {0, 0};
        DI_CHECK_CUDA(cudaMemcpyAsync(&tot[0], fpos.as<uint32_t>() + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        DI_CHECK_CUDA(cudaMemcpyAsync(&tot[1], cpos.as<uint32_t>() + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
        DI_CHECK_CUDA(cudaStreamSynchronize(s));
        g->n_heavy_in = (int32_t)tot[0];
        g->n_heavy_in_chunks = (int32_t)tot[1];
        g->heavy_in_rows.ensure(sizeof(int32_t) * (size_t)(tot[0] + 1));
        g->heavy_in_chunk_off.ensure(sizeof(int32_t) * (size_t)(tot[0] + 1));
        g->heavy_in_chunk_row.ensure(sizeof(int32_t) * (size_t)(tot[1] + 1));
        g->heavy_in_partial.ensure(sizeof(float) * 2 * (size_t)(tot[1] + 1));
        if (tot[0] > 0) {
            k_heavy_in_lists<<<grid_for(n, 256, dev), 256, 0, s>>>(
                flag.as<uint32_t>(), fpos.as<uint32_t>(), cpos.as<uint32_t>(), n, g->heavy_in_rows.as<int32_t>(),
                g->heavy_in_chunk_off.as<int32_t>(), g->heavy_in_chunk_row.as<int32_t>(), g->in_deg.as<int32_t>());
            int32_t last = (int32_t)tot[1];
            DI_CHECK_CUDA(cudaMemcpyAsync(g->heavy_in_chunk_off.as<int32_t>() + tot[0], &last, sizeof(int32_t),
                                          cudaMemcpyHostToDevice, s));
            DI_CHECK_CUDA(cudaGetLastError());
        }
        // the pull's link prefix, sampled, so a pull launch can judge whether contiguous stripes
        // of rows carry even work (the links of the light rows stay below 2^32)
        DevBuf smp;
        smp.ensure(sizeof(int64_t) * (size_t)(kPullSamples + 1));
        k_pull_links<<<grid_for(n, 256, dev), 256, 0, s>>>(g->in_deg.as<int32_t>(), n, flag.as<uint32_t>());
        exclusive_scan_u32(flag.as<uint32_t>(), fpos.as<uint32_t>(), n, scan_tmp, s);
        k_sample_prefix<<<(kPullSamples + 256) / 256, 256, 0, s>>>(fpos.as<uint32_t>(), n, kPullSamples,
                                                                   smp.as<int64_t>());
        g->pull_sample.assign((size_t)kPullSamples + 1, 0);
        DI_CHECK_CUDA(cudaMemcpyAsync(g->pull_sample.data(), smp.p, sizeof(int64_t) * (size_t)(kPullSamples + 1),
                                      cudaMemcpyDeviceToHost, s));
        DI_CHECK_CUDA(cudaStreamSynchronize(s));
        DI_CHECK_CUDA(cudaGetLastError());
    }

    BuildStats hst{};
    unsigned long long hout = 0;
    DI_CHECK_CUDA(cudaMemcpyAsync(&hst, bst, sizeof(hst), cudaMemcpyDeviceToHost, s));
    DI_CHECK_CUDA(cudaMemcpyAsync(&hout, heavy_out_cnt, sizeof(hout), cudaMemcpyDeviceToHost, s));
    DI_CHECK_CUDA(cudaStreamSynchronize(s));
    g->n_heavy_out = (int64_t)hout;
    g->stats.n_nodes = n;
    g->stats.L = L;
    g->stats.D = (int64_t)hst.D;
    g->stats.O = (int64_t)hst.O;
    g->stats.E = e_total;
    g->stats.max_in = hst.max_in;
    g->stats.max_out = hst.max_out;
    g->stats.e_levels = level;
}

extern "C" {

di_status di_graph_create(int32_t n_nodes, const int32_t *src, const int32_t *dst, int64_t n_edges, void *stream,
                          di_graph **out) {
    return guarded([&] {
        DI_REQUIRE(out != nullptr, DI_ERR_INVALID_ARG, "out is NULL");
        *out = nullptr;
        DI_REQUIRE(n_nodes >= 1, DI_ERR_INVALID_ARG, "n_nodes must be >= 1 (got %d)", n_nodes);
        DI_REQUIRE(n_edges >= 0 && n_edges <= INT32_MAX, DI_ERR_INVALID_ARG,
                   "n_edges must be in [0, 2^31-1] (got %lld)", (long long)n_edges);
        DI_REQUIRE(n_edges == 0 || (src && dst), DI_ERR_INVALID_ARG, "src/dst is NULL");
        di_graph *g = new di_graph();
        g->n = n_nodes;
        try {
            build_graph(g, src, dst, n_edges, (cudaStream_t)stream);
            // the solves' pinned control-block mirror, so a solve with an attached workspace
            // allocates nothing
            DI_CHECK_CUDA(cudaMallocHost(&g->ws.ctl_host, sizeof(SolveCtl)));
        } catch (...) {
            delete g;
            throw;
        }
        *out = g;
    });
}

void di_graph_destroy(di_graph *g) { delete g; }

di_status di_graph_stats_get(const di_graph *g, di_graph_stats *out) {
    return guarded([&] {
        DI_REQUIRE(g && out, DI_ERR_INVALID_ARG, "graph or out is NULL");
        *out = g->stats;
    });
}

di_status di_graph_export(const di_graph *g, int32_t which, void *dst, int64_t capacity_bytes, void *stream) {
    return guarded([&] {
        DI_REQUIRE(g && dst, DI_ERR_INVALID_ARG, "graph or dst is NULL");
        const DevBuf *b = nullptr;
        size_t bytes = 0;
        const size_t n = (size_t)g->n, L = (size_t)g->L;
        switch (which) {
            case DI_ARR_ROWPTR_OUT: b = &g->rp_out; bytes = 8 * (n + 1); break;
            case DI_ARR_COL_OUT: b = &g->col_out; bytes = 4 * L; break;
            case DI_ARR_ROWPTR_IN: b = &g->rp_in; bytes = 8 * (n + 1); break;
            case DI_ARR_COL_IN: b = &g->col_in; bytes = 4 * L; break;
            case DI_ARR_OUT_DEG: b = &g->out_deg; bytes = 4 * n; break;
            case DI_ARR_IN_DEG: b = &g->in_deg; bytes = 4 * n; break;
            case DI_ARR_LOOP: b = &g->loop; bytes = n; break;
            case DI_ARR_E_MASK: b = &g->e_mask; bytes = n; break;
            case DI_ARR_E_LEVEL: b = &g->e_level; bytes = 4 * n; break;
            default: DI_REQUIRE(false, DI_ERR_INVALID_ARG, "unknown array id %d", which);
        }
        DI_REQUIRE(capacity_bytes >= (int64_t)bytes, DI_ERR_INVALID_ARG, "buffer holds %lld bytes, need %zu",
                   (long long)capacity_bytes, bytes);
        cudaStream_t s = (cudaStream_t)stream;
        from_device(dst, b->p, bytes, s);
        DI_CHECK_CUDA(cudaStreamSynchronize(s));
    });
}

const char *di_last_error(void) { return di::last_error(); }

const char *di_version(void) { return "di-gb300 0.1 (sm_103a)"; }

}  // extern "C"
