// Exact residual of a history without any allocation.
//
// Some callers cannot call cudaMalloc: hosts that own all device memory through their own pool
// and forbid the runtime's allocator, and code that must not add a device-wide synchronisation
// between two stream-ordered steps (cudaMalloc may synchronise the device). di_residual_noalloc
// serves them: the caller passes every input and output, and the only scratch the kernels need
// lives in the file-scope array below, which every GPU that loads this library holds until the
// process exits.
//
// It is a variant of the refinement kernel of the single-RHS solve: F* = B + P.H - H with the
// link sums in double-float, and ||F*||_1 by a last-block-done FP64 reduction. It walks every row
// with one warp (no split of long rows), so it suits the bounded sizes it accepts.
#include <cstring>
#include <mutex>

#include "di_internal.cuh"

namespace {

constexpr int32_t kNoAllocMaxNodes = 1 << 20;   // largest n accepted
constexpr int kNoAllocBlocks = 512;             // reduction partials
constexpr size_t kYBytes = sizeof(float2) * (size_t)kNoAllocMaxNodes;
constexpr size_t kPartialOffset = kYBytes;
constexpr size_t kTicketOffset = kPartialOffset + sizeof(double) * kNoAllocBlocks;
constexpr size_t kScratchBytes = kTicketOffset + 256;

// y table (d * H_j / out_j as double-float), block partials, and the last-block ticket.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
void *g_scratch_ptr[64] = {};   // device address of g_noalloc_scratch, per device

__device__ __forceinline__ float2 na_add(float2 a, float2 b) {
    const float s = a.x + b.x;
    const float bb = s - a.x;
    float e = (a.x - (s - bb)) + (b.x - bb);
    e += a.y + b.y;
    const float hi = s + e;
    return make_float2(hi, e - (hi - s));
}

__global__ void k_na_scale(const double *H, const int32_t *out_deg, int32_t n, double d, float2 *y) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t o = out_deg[i];
        const double v = o ? d * H[i] / (double)o : 0.0;
        const float hi = (float)v;
        y[i] = make_float2(hi, (float)(v - (double)hi));
    }
}

__global__ void __launch_bounds__(256) k_na_resid(const int64_t *rp_in, const int32_t *col_in, int32_t n,
                                                  const double *B, const double *H, const float2 *y, double *Fstar,
                                                  double *partials, unsigned int *ticket, double *norm_out) {
    __shared__ double wsum[8];
    __shared__ bool is_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double sum = 0.0;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n; i += nwarps) {
        float2 acc = make_float2(0.f, 0.f);
        for (int64_t k = rp_in[i] + lane; k < rp_in[i + 1]; k += 32) acc = na_add(acc, y[col_in[k]]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            float2 t;
            t.x = __shfl_xor_sync(0xffffffffu, acc.x, o);
            t.y = __shfl_xor_sync(0xffffffffu, acc.y, o);
            acc = na_add(acc, t);
        }
        if (lane == 0) {
            const double fs = B[i] + ((double)acc.x + (double)acc.y) - H[i];
            if (Fstar) Fstar[i] = fs;
            sum += fabs(fs);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) wsum[warp] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < 8; w++) b += wsum[w];
        partials[blockIdx.x] = b;
        __threadfence();
        is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (is_last && threadIdx.x == 0) {
        __threadfence();
        double tot = 0.0;
        for (unsigned b = 0; b < gridDim.x; b++) tot += __ldcg(&partials[b]);
        *norm_out = tot;
        *ticket = 0u;   // leaves the shared scratch ready for the next call
    }
}

// Device address of the scratch array on the current device; set up once per device.
void *scratch_for(int dev) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    DI_REQUIRE(dev >= 0 && dev < 64, DI_ERR_INVALID_ARG, "device %d out of range", dev);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        DI_CHECK_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        g_scratch_ptr[dev] = ptr;
    }
    return g_scratch_ptr[dev];
}

// True when p is device (or managed) memory of device `dev`, the one the kernels run on.
bool on_device(const void *p, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" di_status di_residual_noalloc(int32_t n, const int64_t *rp_in, const int32_t *col_in,
                                         const int32_t *out_deg, const double *B, double d, const double *H,
                                         double *Fstar_out, double *norm_out, void *stream) {
    return di::guarded([&] {
        DI_REQUIRE(n >= 1 && n <= kNoAllocMaxNodes, DI_ERR_INVALID_ARG,
                   "n = %d is outside [1, %d], the size the no-allocation scratch holds", n, kNoAllocMaxNodes);
        DI_REQUIRE(d >= 0.0 && d < 1.0, DI_ERR_INVALID_ARG, "d must be in [0, 1) (got %g)", d);
        DI_REQUIRE(rp_in && col_in && out_deg && B && H && norm_out, DI_ERR_INVALID_ARG, "NULL argument");
        int dev = 0;
        DI_CHECK_CUDA(cudaGetDevice(&dev));
        const void *ptrs[7] = {rp_in, col_in, out_deg, B, H, norm_out, Fstar_out ? Fstar_out : (const void *)H};
        for (const void *p : ptrs)
            DI_REQUIRE(on_device(p, dev), DI_ERR_INVALID_ARG, "every array must be device memory of the current device (%d)",
                       dev);
        unsigned char *scratch = static_cast<unsigned char *>(scratch_for(dev));
        float2 *y = reinterpret_cast<float2 *>(scratch);
        double *partials = reinterpret_cast<double *>(scratch + kPartialOffset);
        unsigned int *ticket = reinterpret_cast<unsigned int *>(scratch + kTicketOffset);
        cudaStream_t s = (cudaStream_t)stream;
        DI_CHECK_CUDA(cudaMemsetAsync(ticket, 0, sizeof(unsigned int), s));
        int sms = 0;
        DI_CHECK_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const int ew = (int)((n + 255) / 256 < sms * 8 ? (n + 255) / 256 : sms * 8);
        k_na_scale<<<ew, 256, 0, s>>>(H, out_deg, n, d, y);
        const int rb = (int)(((int64_t)n + 7) / 8 < kNoAllocBlocks ? ((int64_t)n + 7) / 8 : kNoAllocBlocks);
        k_na_resid<<<rb, 256, 0, s>>>(rp_in, col_in, n, B, H, y, Fstar_out, partials, ticket, norm_out);
        DI_CHECK_CUDA(cudaGetLastError());
    });
}
