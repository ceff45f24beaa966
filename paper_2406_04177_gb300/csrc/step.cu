// Explicit time stepping (Sec. III with Scheme 1, Sec. II.B.3a) fused with the transformation
// (Sec. II.C), FP64 compartment totals, and state conversions.
//
// One time step is "transform every voxel, then diffuse the transformed DOM" (Sec. III).  The
// diffusion of voxel i needs the transformed DOM y2 of its neighbours, so the time loop is
// re-associated around the stored state:
//     pass 0           Y^k     = T(X^k)                            (transform only)
//     pass 1..N-1      Y^{j+1} = T(Diffuse(Y^j))                   (fused: one read, one write)
//     pass N           X^{k+N} = Diffuse(Y^{k+N-1})                (DOM only)
// Every intermediate Y already holds the transformed DOM that the neighbours read, so each fused
// pass reads and writes the 5-compartment state once, and N steps cost N+1 passes.
//
// The stencil kernel works on chunks of `cap` consecutive nodes.  A block first decodes, from the
// row bitmask, the (x, row) position of each of its nodes into shared memory; a neighbour's index
// is then found from one mask word and one prefix entry (see Topo), so no per-node neighbour table
// is read from memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "physics.cuh"
#include "stencil.cuh"
#include "vga_internal.cuh"

namespace vga {

namespace {

constexpr int kThreads = 256;
constexpr int kTotBlocks = 1024;


template <int TR>
__global__ void __launch_bounds__(kThreads) k_transform(int64_t n, StepParams p, StateIO io) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x1 = io.in[0][i], x2 = io.in[1][i], x3 = io.in[2][i], x4 = io.in[3][i], x5 = io.in[4][i];
    transform<TR>(x1, x2, x3, x4, x5, p);
    io.out[0][i] = x1;
    io.out[1][i] = x2;
    io.out[2][i] = x3;
    io.out[3][i] = x4;
    io.out[4][i] = x5;
}

// MODE 1: fused (diffuse the stored transformed DOM, then transform the result).
// MODE 2: diffusion only (writes DOM).
template <int MODE, int WM, int TR>
__global__ void __launch_bounds__(kThreads) k_stencil(Topo t, const int32_t *__restrict__ chunk_row, int32_t cap,
                                                      StepParams p, BlockWeights bw, StateIO io) {
    extern __shared__ uint32_t smem[];
    uint32_t *s_x = smem;             // x | boundary flags << 16
    uint32_t *s_row = smem + cap;     // image row
    uint32_t *s_yz = smem + 2 * cap;  // y | z << 16 (block weights only)
    int64_t v0;
    const int32_t nv = decode_chunk<WM == W_BLOCK>(t, chunk_row, cap, s_x, s_row, s_yz, v0);

    const float *__restrict__ Y2 = io.in[1];
    for (int32_t k = threadIdx.x; k < nv; k += blockDim.x) {
        const int64_t i = v0 + k;
        const uint32_t sx = s_x[k];
        const int32_t x = (int32_t)(sx & 0xffffu);
        const uint32_t fl = sx >> 16;
        const int32_t r = (int32_t)s_row[k];
        int32_t y = 0, z = 0;
        if (WM == W_BLOCK) {
            y = (int32_t)(s_yz[k] & 0xffffu);
            z = (int32_t)(s_yz[k] >> 16);
        }
        const float yi = __ldg(Y2 + i);
        float acc = 0.0f;  // sum_j g_ij (y_i - y_j) in slot order; absent neighbours add nothing
        for_each_neighbour(t, i, x, r, fl, [&](int slot, int64_t j) {
            const float d = __fsub_rn(yi, __ldg(Y2 + j));
            if (WM == W_UNIT) acc = __fadd_rn(acc, d);
            else acc = __fmaf_rn(block_theta(bw, slot, x, y, z), d, acc);
        });
        float x2 = __fmaf_rn(-p.c, acc, yi);  // Scheme 1: y_i - D dt sum_j g_ij (y_i - y_j)
        if (MODE == 1) {
            float x1 = __ldg(io.in[0] + i), x3 = __ldg(io.in[2] + i), x4 = __ldg(io.in[3] + i),
                  x5 = __ldg(io.in[4] + i);
            transform<TR>(x1, x2, x3, x4, x5, p);
            io.out[0][i] = x1;
            io.out[1][i] = x2;
            io.out[2][i] = x3;
            io.out[3][i] = x4;
            io.out[4][i] = x5;
        } else {
            io.out[1][i] = x2;
        }
    }
}

// ---- FP64 totals ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kThreads) k_totals(int64_t n, const float *__restrict__ c0,
                                                     const float *__restrict__ c1, const float *__restrict__ c2,
                                                     const float *__restrict__ c3, const float *__restrict__ c4,
                                                     double *__restrict__ partials) {
    __shared__ double sh[5][kThreads / 32];
    double s[5] = {0, 0, 0, 0, 0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        s[0] += c0[i];
        s[1] += c1[i];
        s[2] += c2[i];
        s[3] += c3[i];
        s[4] += c4[i];
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const double w = warp_sum(s[c]);
        if (lane == 0) sh[c][wid] = w;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double b = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) b += sh[threadIdx.x][w];
        partials[(int64_t)blockIdx.x * 5 + threadIdx.x] = b;
    }
}

__global__ void __launch_bounds__(kThreads) k_totals_final(const double *__restrict__ partials, int nblocks,
                                                           double *__restrict__ out) {
    __shared__ double sh[5][kThreads / 32];
    double s[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int c = 0; c < 5; ++c) s[c] += partials[(int64_t)b * 5 + c];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const double w = warp_sum(s[c]);
        if (lane == 0) sh[c][wid] = w;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double b = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) b += sh[threadIdx.x][w];
        out[threadIdx.x] = b;
    }
}

// ---- conversions ---------------------------------------------------------------------------
__global__ void k_convert_in(int64_t n, const double *__restrict__ x, float *c0, float *c1, float *c2, float *c3,
                             float *c4) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    c0[i] = (float)x[i];
    c1[i] = (float)x[n + i];
    c2[i] = (float)x[2 * n + i];
    c3[i] = (float)x[3 * n + i];
    c4[i] = (float)x[4 * n + i];
}

__global__ void k_convert_out(int64_t n, double *__restrict__ x, const float *c0, const float *c1, const float *c2,
                              const float *c3, const float *c4) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    x[i] = c0[i];
    x[n + i] = c1[i];
    x[2 * n + i] = c2[i];
    x[3 * n + i] = c3[i];
    x[4 * n + i] = c4[i];
}

__global__ void k_pack(int64_t n, float *__restrict__ x, float *c0, float *c1, float *c2, float *c3, float *c4,
                       int to_state) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float *c[5] = {c0, c1, c2, c3, c4};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        if (to_state) c[k][i] = x[k * n + i];
        else x[k * n + i] = c[k][i];
    }
}

inline unsigned grid_for(int64_t count, int threads) { return (unsigned)((count + threads - 1) / threads); }

template <int MODE, int WM>
vga_status launch_stencil_tr(vga_sim *s, const StateIO &io) {
    const Topo t = s->g->topo();
    const size_t smem = sizeof(uint32_t) * (size_t)s->chunks.cap * (WM == W_BLOCK ? 3 : 2);
    if (s->sp.transform == 0)
        k_stencil<MODE, WM, 0><<<s->chunks.count, kThreads, smem, s->stream>>>(t, s->chunks.row, s->chunks.cap, s->sp,
                                                                             s->bw, io);
    else
        k_stencil<MODE, WM, 1><<<s->chunks.count, kThreads, smem, s->stream>>>(t, s->chunks.row, s->chunks.cap, s->sp,
                                                                             s->bw, io);
    VGA_CHECK_LAUNCH();
    ++s->launches;
    return VGA_OK;
}

template <int MODE>
vga_status launch_stencil(vga_sim *s, const StateIO &io) {
    if (s->wmode == W_BLOCK) return launch_stencil_tr<MODE, W_BLOCK>(s, io);
    return launch_stencil_tr<MODE, W_UNIT>(s, io);
}

StateIO full_io(vga_sim *s) {
    StateIO io;
    for (int c = 0; c < 5; ++c) {
        io.in[c] = s->comp(c);
        io.out[c] = s->spare(c);
    }
    return io;
}

}  // namespace

vga_status sim_prepare_params(vga_sim *s, const vga_params *p) {
    StepParams sp;
    sp.a = (float)(p->v_dom * p->dt);
    sp.K = (float)p->K_dom;
    sp.r = (float)(p->rho * p->dt);
    sp.m = (float)(p->mu * p->dt);
    sp.beta = (float)p->beta;
    sp.omb = (float)(1.0 - p->beta);
    sp.f = (float)(p->v_fom * p->dt);
    sp.s = (float)(p->v_som * p->dt);
    sp.c = (float)(p->D * p->dt);
    sp.transform = p->transform;
    s->sp = sp;
    s->params = *p;
    return VGA_OK;
}

vga_status sim_transform_pass(vga_sim *s) {
    StateIO io = full_io(s);
    if (s->sp.transform == 0) k_transform<0><<<grid_for(s->n, kThreads), kThreads, 0, s->stream>>>(s->n, s->sp, io);
    else k_transform<1><<<grid_for(s->n, kThreads), kThreads, 0, s->stream>>>(s->n, s->sp, io);
    VGA_CHECK_LAUNCH();
    ++s->launches;
    for (int c = 0; c < 5; ++c) s->cur[c] ^= 1;
    return VGA_OK;
}

vga_status sim_step_explicit(vga_sim *s, int64_t n_steps) {
    if (n_steps <= 0 || s->n == 0) {
        s->steps_done += std::max<int64_t>(n_steps, 0);
        return VGA_OK;
    }
    VGA_TRY(sim_transform_pass(s));
    for (int64_t k = 1; k < n_steps; ++k) {
        VGA_TRY(launch_stencil<1>(s, full_io(s)));
        for (int c = 0; c < 5; ++c) s->cur[c] ^= 1;
    }
    StateIO io = full_io(s);
    VGA_TRY(launch_stencil<2>(s, io));
    s->cur[1] ^= 1;
    s->steps_done += n_steps;
    return VGA_OK;
}

vga_status sim_totals(vga_sim *s, double *h_out) {
    if (s->n == 0) {
        for (int c = 0; c < 5; ++c) h_out[c] = 0.0;
        return VGA_OK;
    }
    const int nb = (int)std::min<int64_t>(kTotBlocks, (int64_t)grid_for(s->n, kThreads));
    k_totals<<<nb, kThreads, 0, s->stream>>>(s->n, s->comp(0), s->comp(1), s->comp(2), s->comp(3), s->comp(4),
                                           s->partials);
    VGA_CHECK_LAUNCH();
    k_totals_final<<<1, kThreads, 0, s->stream>>>(s->partials, nb, s->d_totals);
    VGA_CHECK_LAUNCH();
    s->launches += 2;
    VGA_CUDA(cudaMemcpyAsync(s->h_totals, s->d_totals, 5 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    for (int c = 0; c < 5; ++c) h_out[c] = s->h_totals[c];
    return VGA_OK;
}

vga_status sim_convert_in(vga_sim *s, const double *d_x) {
    if (s->n == 0) return VGA_OK;
    k_convert_in<<<grid_for(s->n, kThreads), kThreads, 0, s->stream>>>(s->n, d_x, s->comp(0), s->comp(1), s->comp(2),
                                                                     s->comp(3), s->comp(4));
    VGA_CHECK_LAUNCH();
    ++s->launches;
    return VGA_OK;
}

vga_status sim_convert_out(vga_sim *s, double *d_x) {
    if (s->n == 0) return VGA_OK;
    k_convert_out<<<grid_for(s->n, kThreads), kThreads, 0, s->stream>>>(s->n, d_x, s->comp(0), s->comp(1), s->comp(2),
                                                                      s->comp(3), s->comp(4));
    VGA_CHECK_LAUNCH();
    ++s->launches;
    return VGA_OK;
}

vga_status sim_pack_f32(vga_sim *s, float *d_x, bool to_state) {
    if (s->n == 0) return VGA_OK;
    k_pack<<<grid_for(s->n, kThreads), kThreads, 0, s->stream>>>(s->n, d_x, s->comp(0), s->comp(1), s->comp(2),
                                                               s->comp(3), s->comp(4), to_state ? 1 : 0);
    VGA_CHECK_LAUNCH();
    ++s->launches;
    return VGA_OK;
}

int totals_blocks() { return kTotBlocks; }

}  // namespace vga
