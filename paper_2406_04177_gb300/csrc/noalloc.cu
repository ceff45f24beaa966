// FP64 compartment totals of a caller-held state without any device allocation.
//
// Some callers cannot let a library allocate device memory: a host application that owns the
// whole GPU memory pool (or runs under a hard memory cap) and hands its plugins only the buffers
// they work on; a latency-critical loop in which cudaMalloc/cudaFree would stall on an implicit
// device synchronisation.  vga_state_totals_noalloc serves them: its only scratch is the
// file-scope array below, which every GPU that loads this library holds until the process exits.
//
// The scratch holds one FP64 partial sum per block and compartment.  Each call writes every slot
// it later reads, so nothing has to start at zero; all calls share the array, so calls that
// overlap on the GPU (on different streams, or from several threads) race and must be serialised
// by the caller.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "stencil.cuh"
#include "vga_internal.cuh"

namespace vga {

namespace {

constexpr int kThreads = 256;
constexpr int kNodesPerBlock = 8192;
constexpr int kMaxBlocks = 4096;  // 4096 x 8192 = 33,554,432 nodes at most
constexpr int kSlots = 5;

// 4096 blocks x 5 compartments x 8 bytes = 160 KiB per device.
static __device__ __align__(256) double g_partials[kMaxBlocks * kSlots];

__global__ void __launch_bounds__(kThreads) k_totals_blocks(const float *__restrict__ values,
                                                            const uint16_t *__restrict__ residuals, int64_t n,
                                                            int64_t stride, double *__restrict__ partials) {
    const int64_t base = (int64_t)blockIdx.x * kNodesPerBlock;
    const int64_t end = min(base + (int64_t)kNodesPerBlock, n);
    double s[kSlots] = {0, 0, 0, 0, 0};
    for (int64_t i = base + threadIdx.x; i < end; i += blockDim.x) {
#pragma unroll
        for (int c = 0; c < kSlots; ++c) {
            double v = (double)values[c * stride + i];
            if (residuals) v += (double)bf16_bits_to_float(residuals[c * stride + i]);
            s[c] += v;
        }
    }
    __shared__ double out[kSlots];
    block_sum_store<kSlots>(s, out);
    if (threadIdx.x < kSlots) partials[(int64_t)blockIdx.x * kSlots + threadIdx.x] = out[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) k_totals_blocks_final(const double *__restrict__ partials, int nblocks,
                                                                  double *__restrict__ totals) {
    double s[kSlots] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int c = 0; c < kSlots; ++c) s[c] += partials[(int64_t)b * kSlots + c];
    __shared__ double out[kSlots];
    block_sum_store<kSlots>(s, out);
    if (threadIdx.x < kSlots) totals[threadIdx.x] = out[threadIdx.x];
}

// Device address of g_partials, looked up once per device with that device current.
constexpr int kMaxDevices = 64;
std::mutex g_addr_mutex;
double *g_addr[kMaxDevices] = {};

vga_status partials_address(double **out) {
    int dev = 0;
    VGA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(VGA_ERR_UNSUPPORTED, "device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_partials);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_partials)", __FILE__, __LINE__);
        g_addr[dev] = static_cast<double *>(p);
    }
    *out = g_addr[dev];
    return VGA_OK;
}

}  // namespace

}  // namespace vga

using namespace vga;

extern "C" vga_status vga_state_totals_noalloc(const float *values, const uint16_t *residuals, int64_t n,
                                               int64_t row_stride, double *totals, void *stream) {
    if (!values || !totals) return fail(VGA_ERR_INVALID_ARG, "values or totals is NULL");
    if (n < 0 || row_stride < n) return fail(VGA_ERR_INVALID_ARG, "need n >= 0 and row_stride >= n");
    if (n > (int64_t)kMaxBlocks * kNodesPerBlock) {
        char buf[160];
        std::snprintf(buf, sizeof(buf), "n = %lld exceeds the no-allocation limit of %lld nodes", (long long)n,
                      (long long)kMaxBlocks * kNodesPerBlock);
        return fail(VGA_ERR_INVALID_ARG, buf);
    }
    double *scratch = nullptr;
    VGA_TRY(partials_address(&scratch));
    cudaStream_t st = (cudaStream_t)stream;
    const int nblocks = (int)((n + kNodesPerBlock - 1) / kNodesPerBlock);
    if (nblocks > 0)
        k_totals_blocks<<<nblocks, kThreads, 0, st>>>(values, residuals, n, row_stride, scratch);
    k_totals_blocks_final<<<1, kThreads, 0, st>>>(scratch, nblocks, totals);
    VGA_CHECK_LAUNCH();
    return VGA_OK;
}
