// Temporal blocking of the explicit time loop (Sec. III, Scheme 1 fused with the transformation):
// several fused passes run inside one persistent kernel as a wavefront over chunks of nodes, so
// that the state one pass writes is read back by the next pass from L2 instead of HBM.
//
// Dependencies are tracked per chunk of C consecutive nodes; work is done per warp item, 32
// consecutive nodes.  Item (s, j, w) = fused pass s over warp item w of chunk j.  Pass s reads
// buffer set s & 1 and writes the other set.  An item may run once pass s - 1 has completed every
// chunk in [dep_lo[j], dep_hi[j]], the chunks that neighbours of chunk j's nodes lie in: that
// covers the transformed DOM it reads (read after write) and every reader of the values it
// overwrites (write after read: chunk j's values are read only by chunks whose neighbours reach
// j, and adjacency is symmetric).  count[j] counts the warp items of chunk j completed in this
// launch over all passes; pass s is complete for chunk j exactly when count[j] >= (s + 1) nw_j
// (nw_j = warp items of chunk j), because no item of pass s + 1 in chunk j can start before pass
// s of chunk j is complete (j lies in its own dependency range).
//
// Items are numbered (tickets) in a skewed order: passes are grouped in blocks of T; inside a
// block, diagonal d holds the chunks (t, d - t L) for t = 0..T-1, each contributing its warp items
// consecutively, with L larger than any dependency reach (max dep_hi[j] - j) plus the chunks the
// grid works on at once.  Every item depends only on items with smaller tickets.  Warp g of the
// grid takes tickets g, g + W, g + 2W, ... in order, so the lowest unfinished ticket always has
// its dependencies complete and the launch makes progress; the waits are bounded nonetheless (a
// spin limit sets the device error flag and the warps return).  Warps never wait for one another
// inside a CTA, so a warp's dependency check or memory latency overlaps the other warps' work.
//
// The arithmetic per node is table_node (bit-identical to the one-pass-per-launch table kernel);
// state loads go through L2 (ld.global.cg) because other warps of the launch wrote them.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "stencil.cuh"
#include "vga_internal.cuh"

namespace vga {
namespace {

constexpr int kWaveSpin = 1 << 21;  // dependency polls before a wait gives up (>= 0.25 s with the sleeps)
constexpr int kWaveThreads = 256;   // 8 independent warps per CTA

struct WaveArgs {
    int64_t n;
    int32_t C;     // nodes per chunk (a power of two >= 256): dependency granularity
    int32_t T;     // passes per block of the skewed order
    int32_t P;     // fused passes in this launch
    int32_t nord;  // entries of order (T x chunks)
    const int32_t *order;  // (t << 24) | j in ticket order within one block of T passes
    const int32_t *dep;    // per chunk: dep_lo at 2j, dep_hi at 2j + 1
    uint32_t *count;       // per chunk: warp items completed in this launch (zero at launch)
    int32_t *err;
};

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t *p) { return *(const volatile uint32_t *)p; }
__device__ __forceinline__ int32_t ld_volatile_i32(const int32_t *p) { return *(const volatile int32_t *)p; }

template <int WM, int TR, int PREC>
__global__ void __launch_bounds__(kWaveThreads) k_wave(WaveArgs a, NbrTable tb, BlockTable bt, StepParams p,
                                                       StateIO io0, StateIO io1) {
    const int lane = threadIdx.x & 31;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * (kWaveThreads / 32);
    const unsigned long long gw = (unsigned long long)blockIdx.x * (kWaveThreads / 32) + (threadIdx.x >> 5);
    const int32_t wpc = a.C >> 5;  // warp items per full chunk
    const int32_t J = a.nord / a.T;
    const uint32_t w_last = (uint32_t)(((a.n - (int64_t)(J - 1) * a.C) + 31) >> 5);  // warp items of the last chunk
    const unsigned long long per_blk = (unsigned long long)a.nord * wpc;
    const unsigned long long total = (unsigned long long)((a.P + a.T - 1) / a.T) * per_blk;
    for (unsigned long long t = gw; t < total; t += nwarps) {
        const int32_t blk = (int32_t)(t / per_blk);
        const unsigned long long r = t - (unsigned long long)blk * per_blk;
        const int32_t e = __ldg(a.order + (int32_t)(r / (unsigned)wpc));
        const int32_t w = (int32_t)(r % (unsigned)wpc);
        const int32_t s = blk * a.T + (e >> 24);
        const int32_t j = e & 0xffffff;
        const int64_t i0 = (int64_t)j * a.C + (int64_t)w * 32;
        if (s >= a.P || i0 >= a.n) continue;  // warp-uniform
        if (s > 0) {
            const int32_t lo = __ldg(a.dep + 2 * j), hi = __ldg(a.dep + 2 * j + 1);
            for (int it = 0;; ++it) {
                bool ok = true;
                for (int32_t q = lo + lane; q <= hi; q += 32) {
                    const uint32_t need = (uint32_t)s * (q == J - 1 ? w_last : (uint32_t)wpc);
                    if (ld_volatile_u32(a.count + q) < need) {
                        ok = false;
                        break;
                    }
                }
                if (__all_sync(0xffffffffu, ok)) break;
                int stop = 0;
                if (lane == 0 && (it > kWaveSpin || ld_volatile_i32(a.err))) {
                    atomicExch(a.err, 2);
                    stop = 1;
                }
                if (__shfl_sync(0xffffffffu, stop, 0)) return;
                __nanosleep(64);
            }
            __threadfence();  // order the observed counts before the state loads
        }
        const int64_t i = i0 + lane;
        if (s & 1) table_node<1, WM, TR, PREC, LD_CG>((uint32_t)i, i < a.n, tb, bt, p, io1);
        else table_node<1, WM, TR, PREC, LD_CG>((uint32_t)i, i < a.n, tb, bt, p, io0);
        __syncwarp();
        if (lane == 0) {
            __threadfence();
            atomicAdd(a.count + j, 1u);
        }
    }
}

// dep[2j], dep[2j+1] = chunks of the lowest- and highest-index neighbours of chunk j's nodes
// (chunk j itself included).
constexpr int kDepThreads = 256;

__global__ void __launch_bounds__(kDepThreads) k_wave_deps(int64_t n, NbrTable tb, int32_t C, int32_t *dep) {
    const int32_t j = blockIdx.x;
    const int64_t base = (int64_t)j * C;
    int64_t hi = base, lo = base;
    for (int32_t k = threadIdx.x; k < C; k += blockDim.x) {
        const int64_t i = base + k;
        if (i >= n) break;
        const uint32_t ty = __ldg(tb.ty + i);
        int64_t h = i, l = i;
        if (ty >> 31) h = i + 1;
        if ((ty >> 15) & 1u) l = i - 1;
        const uint32_t dym = ty & 0x7fffu, dyp = (ty >> 16) & 0x7fffu;
        if (dyp) h = max(h, i + (int64_t)dyp);
        if (dym) l = min(l, i - (int64_t)dym);
        const uint32_t dzp = __ldg(tb.tzp + i), dzm = __ldg(tb.tzm + i);
        if (dzp) h = max(h, i + (int64_t)dzp);
        if (dzm) l = min(l, i - (int64_t)dzm);
        hi = max(hi, h);
        lo = min(lo, l);
    }
    __shared__ long long sh[2][kDepThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        hi = max(hi, (int64_t)__shfl_down_sync(0xffffffffu, (long long)hi, o));
        lo = min(lo, (int64_t)__shfl_down_sync(0xffffffffu, (long long)lo, o));
    }
    if ((threadIdx.x & 31) == 0) {
        sh[0][threadIdx.x >> 5] = lo;
        sh[1][threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t ml = sh[0][0], mh = sh[1][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            ml = min(ml, (int64_t)sh[0][w]);
            mh = max(mh, (int64_t)sh[1][w]);
        }
        dep[2 * j] = (int32_t)(ml / C);
        dep[2 * j + 1] = (int32_t)(mh / C);
    }
}

void *wave_kernel_for(int wm, int prec, int tr) {
    if (wm == W_UNIT) {
        if (prec == P_COMP) return tr ? (void *)k_wave<W_UNIT, 1, P_COMP> : (void *)k_wave<W_UNIT, 0, P_COMP>;
        return tr ? (void *)k_wave<W_UNIT, 1, P_F32> : (void *)k_wave<W_UNIT, 0, P_F32>;
    }
    if (prec == P_COMP) return tr ? (void *)k_wave<W_BLOCK, 1, P_COMP> : (void *)k_wave<W_BLOCK, 0, P_COMP>;
    return tr ? (void *)k_wave<W_BLOCK, 1, P_F32> : (void *)k_wave<W_BLOCK, 0, P_F32>;
}

}  // namespace

bool wave_params_valid(int chunk, int depth, int ctas_per_sm) {
    const bool pow2 = chunk > 0 && (chunk & (chunk - 1)) == 0;
    return pow2 && chunk >= 256 && chunk <= 8192 && depth >= 1 && depth <= 64 && ctas_per_sm >= 0 && ctas_per_sm <= 32;
}

// Runs P fused passes (the passes 1..P of a step(P + 1) call) as one wavefront launch.  On return
// the compartments' current buffers are flipped when P is odd.
vga_status sim_wave_fused(vga_sim *s, int64_t P) {
    if (P <= 0) return VGA_OK;
    if (P > (int64_t)(1 << 30)) return fail(VGA_ERR_INVALID_ARG, "too many passes for one wavefront launch");
    NbrTable tb;
    BlockTable bt;
    bool block_ok = true;
    VGA_TRY(sim_nbr_table(s, &tb));
    if (s->wmode == W_BLOCK) VGA_TRY(sim_block_table(s, &bt, &block_ok));
    if (!block_ok) return fail(VGA_ERR_UNSUPPORTED, "block grid too large for the block table");
    const int C = s->wave_chunk, T = s->wave_depth;
    const int64_t J64 = (s->n + C - 1) / C;
    if (J64 >= (1 << 24)) return fail(VGA_ERR_UNSUPPORTED, "too many chunks for the wavefront order");
    if (P * (C / 32) >= ((int64_t)1 << 31)) return fail(VGA_ERR_INVALID_ARG, "too many passes for one wavefront launch");
    const int32_t J = (int32_t)J64;
    int dev = 0, nsm = 0;
    VGA_CUDA(cudaGetDevice(&dev));
    VGA_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    void *kern = wave_kernel_for(s->wmode, s->precision(), s->sp.transform);
    int occ = 0;
    VGA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kWaveThreads, 0));
    if (occ < 1) return fail(VGA_ERR_CUDA, "wavefront kernel does not fit on an SM");
    const int per_sm = s->wave_ctas > 0 ? std::min(s->wave_ctas, occ) : occ;
    const int64_t witems = (s->n + 31) / 32;
    const int grid = (int)std::min<int64_t>((int64_t)per_sm * nsm, std::max<int64_t>((witems + 7) / 8, 1));
    // dependency ranges per chunk (once per chunk size), then one completion flag per chunk
    if (s->wave_built_chunk != C) {
        dfree(s->wave_dep);
        s->wave_dep = nullptr;
        s->wave_built_chunk = 0;
        VGA_TRY(dmalloc((void **)&s->wave_dep, sizeof(int32_t) * 3 * (size_t)J, "wavefront dependencies"));
        k_wave_deps<<<J, kDepThreads, 0, s->stream>>>(s->n, tb, C, s->wave_dep);
        VGA_CHECK_LAUNCH();
        std::vector<int32_t> h(2 * (size_t)J);
        VGA_CUDA(cudaMemcpyAsync(h.data(), s->wave_dep, sizeof(int32_t) * 2 * (size_t)J, cudaMemcpyDeviceToHost,
                                 s->stream));
        VGA_CUDA(cudaStreamSynchronize(s->stream));
        int32_t reach = 0;
        for (int32_t j = 0; j < J; ++j) reach = std::max(reach, h[2 * (size_t)j + 1] - j);
        s->wave_reach = reach;
        s->wave_built_chunk = C;
        s->wave_built_lag = -1;
    }
    // skewed order: lag = reach + 1 + 1.5 times the chunk diagonals the grid's warps work on at
    // once (+ margin), so an item's dependencies were issued well before it
    const int64_t chunks_in_flight = ((int64_t)grid * (kWaveThreads / 32) + (C / 32) - 1) / (C / 32);
    const int32_t lag = s->wave_reach + 1 + (int32_t)((3 * chunks_in_flight + 2 * T - 1) / (2 * T)) + 4;
    if (s->wave_built_lag != lag || s->wave_built_depth != T) {
        std::vector<int32_t> ord;
        ord.reserve((size_t)T * J);
        const int64_t ndiag = (int64_t)J + (int64_t)(T - 1) * lag;
        for (int64_t d = 0; d < ndiag; ++d)
            for (int t = 0; t < T; ++t) {
                const int64_t j = d - (int64_t)t * lag;
                if (j >= 0 && j < J) ord.push_back((t << 24) | (int32_t)j);
            }
        dfree(s->wave_order);
        s->wave_order = nullptr;
        s->wave_built_lag = -1;
        VGA_TRY(dmalloc((void **)&s->wave_order, sizeof(int32_t) * ord.size(), "wavefront order"));
        VGA_CUDA(cudaMemcpyAsync(s->wave_order, ord.data(), sizeof(int32_t) * ord.size(), cudaMemcpyHostToDevice,
                                 s->stream));
        VGA_CUDA(cudaStreamSynchronize(s->stream));
        s->wave_built_lag = lag;
        s->wave_built_depth = T;
    }
    uint32_t *count = reinterpret_cast<uint32_t *>(s->wave_dep + 2 * (size_t)J);
    VGA_CUDA(cudaMemsetAsync(count, 0, sizeof(uint32_t) * (size_t)J, s->stream));
    WaveArgs a;
    a.n = s->n;
    a.C = C;
    a.T = T;
    a.P = (int32_t)P;
    a.nord = T * J;
    a.order = s->wave_order;
    a.dep = s->wave_dep;
    a.count = count;
    a.err = s->d_err;
    StateIO io0, io1;
    for (int c = 0; c < 5; ++c) {
        io0.in[c] = s->comp(c);
        io0.out[c] = s->spare(c);
        io0.lin[c] = s->lcomp(c);
        io0.lout[c] = s->lspare(c);
        io1.in[c] = s->spare(c);
        io1.out[c] = s->comp(c);
        io1.lin[c] = s->lspare(c);
        io1.lout[c] = s->lcomp(c);
    }
    StepParams sp = s->sp;
    void *args[] = {&a, &tb, &bt, &sp, &io0, &io1};
    timing_begin(s, VGA_KERNEL_FUSED_STEP);
    const cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(kWaveThreads), args, 0, s->stream);
    timing_end_weighted(s, P);
    if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchCooperativeKernel(k_wave)", __FILE__, __LINE__);
    ++s->launches;
    if (P & 1)
        for (int c = 0; c < 5; ++c) s->cur[c] ^= 1;
    return VGA_OK;
}

}  // namespace vga
