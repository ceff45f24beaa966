// Implicit time stepping: Scheme 2 (Sec. II.B.3b), (I + D dt L_g) m^{k+1} = y, solved matrix-free
// by the Jacobi-preconditioned conjugate gradient of Sec. III (t_ii = 1 / b_ii), after the
// transformation of every voxel (Sec. III).
//
// The solve runs in FP64 (a relative residual of 1e-8 is below FP32 resolution); the initial
// guess is the right-hand side y and the stopping test is ||r||_2 <= rtol ||y||_2 on the recurrence
// residual.  Every reduction is a fixed-order block-partial sum, so results are run-to-run
// deterministic.  The recurrence scalars live on the device; the host only polls a "done" flag
// every kBatch iterations, and kernels launched after convergence return at once.
//
// Kernels of one iteration (matrix B = I + c L_g, c = D dt):
//   k_update_p   p = T r + beta p           (elementwise; beta = 0 on the first iteration)
//   k_spmv       q = B p, partial p.q       (stencil over the chunk decode)
//   k_scalar_a   alpha = (r.Tr) / (p.q)     (one block)
//   k_update_xr  x += alpha p, r -= alpha q, partial r.Tr and r.r
//   k_scalar_b   convergence test, beta     (one block)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "stencil.cuh"
#include "vga_internal.cuh"

namespace vga {

namespace {

constexpr int kThreads = 256;
constexpr int kEwBlocks = 1024;  // grid of the elementwise kernels (grid-stride loops)
constexpr int kBatch = 8;        // iterations enqueued between two polls of the done flag

struct CgScalars {
    double rz, rr, bb, alpha, beta, relres, rtol2;
    int32_t done, iters, notconv, maxit;
};

struct CgVecs {
    double *x, *r, *p, *q, *t;
};

// b = y2, x = b, r = b - B x = -c L_g b, t = 1 / (1 + c sum_j g_ij); partials (r.Tr, r.r, b.b)
template <int WM, int PREC>
__global__ void __launch_bounds__(kThreads) k_cg_init(Topo t, const int32_t *__restrict__ chunk_row, int32_t cap,
                                                      double c, BlockWeights bw, const float *__restrict__ y2,
                                                      const uint16_t *__restrict__ y2l, CgVecs v,
                                                      double *__restrict__ part) {
    extern __shared__ uint32_t smem[];
    int32_t *s_nb = reinterpret_cast<int32_t *>(smem + cap);
    int64_t v0;
    const int32_t nv = decode_chunk<WM == W_BLOCK>(t, chunk_row, cap, smem, s_nb, smem + 5 * cap, v0);
    double acc[3] = {0.0, 0.0, 0.0};
    for (int32_t k = threadIdx.x; k < nv; k += blockDim.x) {
        const int64_t i = v0 + k;
        const uint32_t info = smem[k];
        const uint32_t fl = info >> 16;
        int32_t x = 0, y = 0, z = 0;
        if (WM == W_BLOCK) {
            x = (int32_t)(info & 0xffffu);
            y = (int32_t)(smem[5 * cap + k] & 0xffffu);
            z = (int32_t)(smem[5 * cap + k] >> 16);
        }
        const double bi = (double)__ldg(y2 + i) + (PREC == P_COMP ? (double)bf16_bits_to_float(__ldg(y2l + i)) : 0.0);
        double lb = 0.0, deg = 0.0;
        for_each_neighbour(i, k, fl, s_nb, cap, [&](int slot, int64_t j) {
            const double g = (WM == W_UNIT) ? 1.0 : (double)block_theta(bw, slot, x, y, z);
            const double bj =
                (double)__ldg(y2 + j) + (PREC == P_COMP ? (double)bf16_bits_to_float(__ldg(y2l + j)) : 0.0);
            lb += g * (bi - bj);
            deg += g;
        });
        const double ri = -c * lb;
        const double ti = 1.0 / (1.0 + c * deg);
        v.x[i] = bi;
        v.r[i] = ri;
        v.t[i] = ti;
        acc[0] += ri * ti * ri;
        acc[1] += ri * ri;
        acc[2] += bi * bi;
    }
    __shared__ double out[3];
    block_sum_store<3>(acc, out);
    if (threadIdx.x < 3) part[(int64_t)blockIdx.x * 3 + threadIdx.x] = out[threadIdx.x];
}

// q = B p = p + c L_g p; partial p.q
template <int WM>
__global__ void __launch_bounds__(kThreads) k_spmv(Topo t, const int32_t *__restrict__ chunk_row, int32_t cap,
                                                   double c, BlockWeights bw, const double *__restrict__ p,
                                                   double *__restrict__ q, double *__restrict__ part,
                                                   const CgScalars *__restrict__ sc) {
    if (sc->done) return;
    extern __shared__ uint32_t smem[];
    int32_t *s_nb = reinterpret_cast<int32_t *>(smem + cap);
    int64_t v0;
    const int32_t nv = decode_chunk<WM == W_BLOCK>(t, chunk_row, cap, smem, s_nb, smem + 5 * cap, v0);
    double acc[1] = {0.0};
    for (int32_t k = threadIdx.x; k < nv; k += blockDim.x) {
        const int64_t i = v0 + k;
        const uint32_t info = smem[k];
        const uint32_t fl = info >> 16;
        int32_t x = 0, y = 0, z = 0;
        if (WM == W_BLOCK) {
            x = (int32_t)(info & 0xffffu);
            y = (int32_t)(smem[5 * cap + k] & 0xffffu);
            z = (int32_t)(smem[5 * cap + k] >> 16);
        }
        const double pi = p[i];
        double lp = 0.0;
        for_each_neighbour(i, k, fl, s_nb, cap, [&](int slot, int64_t j) {
            const double g = (WM == W_UNIT) ? 1.0 : (double)block_theta(bw, slot, x, y, z);
            lp += g * (pi - p[j]);
        });
        const double qi = pi + c * lp;
        q[i] = qi;
        acc[0] += pi * qi;
    }
    __shared__ double out[1];
    block_sum_store<1>(acc, out);
    if (threadIdx.x == 0) part[blockIdx.x] = out[0];
}

// Table-driven versions of the two stencil kernels (unit conductances): one node per thread,
// neighbours from the offset table, +-x values by warp shuffles.  Same arithmetic and slot order.
__device__ __forceinline__ double nbr_sum_table(NbrTable tb, uint32_t i, bool live, double vi,
                                                const double *__restrict__ v, double &deg) {
    const uint32_t ty = live ? __ldg(tb.ty + i) : 0u;
    const uint32_t dzm = live ? __ldg(tb.tzm + i) : 0u;
    const uint32_t dzp = live ? __ldg(tb.tzp + i) : 0u;
    const int lane = threadIdx.x & 31;
    double vl = __shfl_up_sync(0xffffffffu, vi, 1);
    double vr = __shfl_down_sync(0xffffffffu, vi, 1);
    const uint32_t dym = ty & 0x7fffu, dyp = (ty >> 16) & 0x7fffu;
    const bool hxm = (ty >> 15) & 1u, hxp = ty >> 31;
    if (lane == 0 && hxm) vl = v[i - 1];
    if (lane == 31 && hxp) vr = v[i + 1];
    double s = 0.0;
    deg = 0.0;
    if (hxm) { s += vi - vl; deg += 1.0; }
    if (hxp) { s += vi - vr; deg += 1.0; }
    if (dym) { s += vi - v[i - dym]; deg += 1.0; }
    if (dyp) { s += vi - v[i + dyp]; deg += 1.0; }
    if (dzm) { s += vi - v[i - dzm]; deg += 1.0; }
    if (dzp) { s += vi - v[i + dzp]; deg += 1.0; }
    return s;
}

// x = b (the right-hand side y2 as FP64)
template <int PREC>
__global__ void __launch_bounds__(kThreads) k_cg_rhs(int64_t n, const float *__restrict__ y2,
                                                     const uint16_t *__restrict__ y2l, double *__restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = (double)__ldg(y2 + i) + (PREC == P_COMP ? (double)bf16_bits_to_float(__ldg(y2l + i)) : 0.0);
}

// Grid-stride loops over 256-node tiles (lanes = consecutive nodes) on a fixed grid, so the block
// partials stay few and the single-block scalar kernels stay short.
template <int PREC>
__global__ void __launch_bounds__(kThreads) k_cg_init_table_b(int64_t n, NbrTable tb, double c, CgVecs v,
                                                              double *__restrict__ part) {
    double acc[3] = {0.0, 0.0, 0.0};
    const int64_t ntile = (n + kThreads - 1) / kThreads;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const uint32_t i = (uint32_t)(tile * kThreads + threadIdx.x);
        const bool live = i < (uint64_t)n;
        const double bi = live ? v.x[i] : 0.0;
        double deg = 0.0;
        const double lb = nbr_sum_table(tb, i, live, bi, v.x, deg);
        if (live) {
            const double ri = -c * lb;
            const double ti = 1.0 / (1.0 + c * deg);
            v.r[i] = ri;
            v.t[i] = ti;
            acc[0] += ri * ti * ri;
            acc[1] += ri * ri;
            acc[2] += bi * bi;
        }
    }
    __shared__ double out[3];
    block_sum_store<3>(acc, out);
    if (threadIdx.x < 3) part[(int64_t)blockIdx.x * 3 + threadIdx.x] = out[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) k_spmv_table(int64_t n, NbrTable tb, double c, const double *__restrict__ p,
                                                         double *__restrict__ q, double *__restrict__ part,
                                                         const CgScalars *__restrict__ sc) {
    if (sc->done) return;
    double acc[1] = {0.0};
    const int64_t ntile = (n + kThreads - 1) / kThreads;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const uint32_t i = (uint32_t)(tile * kThreads + threadIdx.x);
        const bool live = i < (uint64_t)n;
        const double pi = live ? p[i] : 0.0;
        double deg;
        const double lp = nbr_sum_table(tb, i, live, pi, p, deg);
        if (live) {
            const double qi = pi + c * lp;
            q[i] = qi;
            acc[0] += pi * qi;
        }
    }
    __shared__ double out[1];
    block_sum_store<1>(acc, out);
    if (threadIdx.x == 0) part[blockIdx.x] = out[0];
}

__global__ void __launch_bounds__(kThreads) k_update_p(int64_t n, CgVecs v, const CgScalars *__restrict__ sc,
                                                       int first) {
    if (sc->done) return;
    const double beta = first ? 0.0 : sc->beta;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v.p[i] = v.t[i] * v.r[i] + beta * (first ? 0.0 : v.p[i]);
}

__global__ void __launch_bounds__(kThreads) k_update_xr(int64_t n, CgVecs v, const CgScalars *__restrict__ sc,
                                                        double *__restrict__ part) {
    if (sc->done) return;
    const double alpha = sc->alpha;
    double acc[2] = {0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        v.x[i] += alpha * v.p[i];
        const double ri = v.r[i] - alpha * v.q[i];
        v.r[i] = ri;
        acc[0] += ri * v.t[i] * ri;
        acc[1] += ri * ri;
    }
    __shared__ double out[2];
    block_sum_store<2>(acc, out);
    if (threadIdx.x < 2) part[(int64_t)blockIdx.x * 2 + threadIdx.x] = out[threadIdx.x];
}

// Deterministic sum of part[k*stride + comp] over k < count by one block.
__device__ double block_reduce_partials(const double *part, int64_t count, int stride, int comp) {
    double acc[1] = {0.0};
    for (int64_t k = threadIdx.x; k < count; k += blockDim.x) acc[0] += part[k * stride + comp];
    __shared__ double out[1];
    block_sum_store<1>(acc, out);
    return out[0];
}

__global__ void __launch_bounds__(kThreads) k_scalar_init(const double *__restrict__ part, int64_t count,
                                                          CgScalars *sc, double rtol, int maxit) {
    const double rz = block_reduce_partials(part, count, 3, 0);
    const double rr = block_reduce_partials(part, count, 3, 1);
    const double bb = block_reduce_partials(part, count, 3, 2);
    if (threadIdx.x == 0) {
        sc->rz = rz;
        sc->rr = rr;
        sc->bb = bb;
        sc->rtol2 = rtol * rtol;
        sc->iters = 0;
        sc->notconv = 0;
        sc->maxit = maxit;
        sc->alpha = 0.0;
        sc->beta = 0.0;
        sc->relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        sc->done = (bb == 0.0 || rr <= sc->rtol2 * bb) ? 1 : 0;
    }
}

__global__ void __launch_bounds__(kThreads) k_scalar_a(const double *__restrict__ part, int64_t count,
                                                       CgScalars *sc) {
    if (sc->done) return;
    const double pq = block_reduce_partials(part, count, 1, 0);
    if (threadIdx.x == 0) sc->alpha = sc->rz / pq;
}

__global__ void __launch_bounds__(kThreads) k_scalar_b(const double *__restrict__ part, int64_t count,
                                                       CgScalars *sc) {
    if (sc->done) return;
    const double rz = block_reduce_partials(part, count, 2, 0);
    const double rr = block_reduce_partials(part, count, 2, 1);
    if (threadIdx.x == 0) {
        sc->iters += 1;
        sc->rr = rr;
        sc->relres = sqrt(rr / sc->bb);
        if (rr <= sc->rtol2 * sc->bb) {
            sc->done = 1;
        } else if (sc->iters >= sc->maxit) {
            sc->done = 1;
            sc->notconv = 1;
        } else {
            sc->beta = rz / sc->rz;
            sc->rz = rz;
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_cg_out(int64_t n, const double *__restrict__ x, float *__restrict__ out,
                                                     uint16_t *__restrict__ outl, int comp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    const float h = (float)v;
    out[i] = h;
    if (comp) outl[i] = float_to_bf16_bits((float)(v - (double)h));
}

inline unsigned grid_for(int64_t count, int threads) { return (unsigned)((count + threads - 1) / threads); }

template <int WM, int PREC>
vga_status solve(vga_sim *s, CgVecs v, double *part_chunk, double *part_ew, CgScalars *sc) {
    const Topo t = s->g->topo();
    const double c = s->params.D * s->params.dt;
    const size_t smem = sizeof(uint32_t) * (size_t)s->chunks.cap * decode_words(WM == W_BLOCK);
    const int G = s->chunks.count;
    const int ew = (int)std::min<int64_t>(kEwBlocks, (int64_t)grid_for(s->n, kThreads));
    cudaStream_t st = s->stream;
    const bool table = (WM == W_UNIT) && s->g->nx <= 32767;
    NbrTable tb;
    if (table) VGA_TRY(sim_nbr_table(s, &tb));
    const int Gs = table ? (int)std::min<int64_t>(kEwBlocks, grid_for(s->n, kThreads)) : G;  // stencil grid
    timing_begin(s, VGA_KERNEL_PCG_STENCIL);
    if (table) {
        k_cg_rhs<PREC><<<grid_for(s->n, kThreads), kThreads, 0, st>>>(s->n, s->comp(1), s->lcomp(1), v.x);
        k_cg_init_table_b<PREC><<<Gs, kThreads, 0, st>>>(s->n, tb, c, v, part_chunk);
    } else {
        k_cg_init<WM, PREC><<<G, kThreads, smem, st>>>(t, s->chunks.row, s->chunks.cap, c, s->bw, s->comp(1),
                                                       s->lcomp(1), v, part_chunk);
    }
    timing_end(s);
    k_scalar_init<<<1, kThreads, 0, st>>>(part_chunk, Gs, sc, s->params.cg_rtol, s->params.cg_maxit);
    VGA_CHECK_LAUNCH();
    s->launches += 2;
    CgScalars *h = reinterpret_cast<CgScalars *>(s->h_cg);
    bool first = true;
    for (;;) {
        for (int b = 0; b < kBatch; ++b) {
            timing_begin(s, VGA_KERNEL_PCG_VECTOR);
            k_update_p<<<ew, kThreads, 0, st>>>(s->n, v, sc, first ? 1 : 0);
            timing_end(s);
            timing_begin(s, VGA_KERNEL_PCG_STENCIL);
            if (table) k_spmv_table<<<Gs, kThreads, 0, st>>>(s->n, tb, c, v.p, v.q, part_chunk, sc);
            else k_spmv<WM><<<G, kThreads, smem, st>>>(t, s->chunks.row, s->chunks.cap, c, s->bw, v.p, v.q, part_chunk, sc);
            timing_end(s);
            timing_begin(s, VGA_KERNEL_PCG_VECTOR);
            k_scalar_a<<<1, kThreads, 0, st>>>(part_chunk, Gs, sc);
            k_update_xr<<<ew, kThreads, 0, st>>>(s->n, v, sc, part_ew);
            k_scalar_b<<<1, kThreads, 0, st>>>(part_ew, ew, sc);
            timing_end(s);
            first = false;
        }
        VGA_CHECK_LAUNCH();
        s->launches += 5 * kBatch;
        VGA_CUDA(cudaMemcpyAsync(h, sc, sizeof(CgScalars), cudaMemcpyDeviceToHost, st));
        VGA_CUDA(cudaStreamSynchronize(st));
        if (h->done) break;
    }
    k_cg_out<<<grid_for(s->n, kThreads), kThreads, 0, st>>>(s->n, v.x, s->spare(1), s->lspare(1), PREC == P_COMP);
    VGA_CHECK_LAUNCH();
    ++s->launches;
    s->cur[1] ^= 1;
    s->cg_iterations += h->iters;
    s->cg_last_relres = h->relres;
    return h->notconv ? VGA_ERR_NOT_CONVERGED : VGA_OK;
}

}  // namespace

vga_status sim_step_implicit(vga_sim *s, int64_t n_steps) {
    if (n_steps <= 0 || s->n == 0) {
        s->steps_done += std::max<int64_t>(n_steps, 0);
        return VGA_OK;
    }
    const int64_t G = std::max<int64_t>(s->chunks.count, (s->n + kThreads - 1) / kThreads);
    const int64_t need = 5 * s->npad + 3 * std::max<int64_t>(G, 1) + 2 * kEwBlocks;
    if (s->cg_count < need) {
        dfree(s->cg);
        s->cg = nullptr;
        s->cg_count = 0;
        VGA_TRY(dmalloc((void **)&s->cg, sizeof(double) * (size_t)need, "PCG vectors"));
        s->cg_count = need;
    }
    if (!s->cg_scalars) VGA_TRY(dmalloc((void **)&s->cg_scalars, sizeof(CgScalars) + 64, "PCG scalars"));
    if (!s->h_cg) VGA_CUDA(cudaMallocHost((void **)&s->h_cg, sizeof(CgScalars) + 64));
    CgVecs v;
    v.x = s->cg;
    v.r = v.x + s->npad;
    v.p = v.r + s->npad;
    v.q = v.p + s->npad;
    v.t = v.q + s->npad;
    double *part_chunk = v.t + s->npad;
    double *part_ew = part_chunk + 3 * std::max<int64_t>(G, 1);
    CgScalars *sc = reinterpret_cast<CgScalars *>(s->cg_scalars);
    vga_status worst = VGA_OK;
    for (int64_t k = 0; k < n_steps; ++k) {
        if (s->subcycled()) {
            s->sp.ntrans = sim_ticks_of_step(s, s->steps_done);
            const vga_status ts = sim_transform_pass(s);
            s->sp.ntrans = 1;
            VGA_TRY(ts);
        } else {
            VGA_TRY(sim_transform_pass(s));
        }
        const bool comp = s->precision() == P_COMP;
        vga_status st;
        if (s->wmode == W_BLOCK)
            st = comp ? solve<W_BLOCK, P_COMP>(s, v, part_chunk, part_ew, sc) : solve<W_BLOCK, P_F32>(s, v, part_chunk, part_ew, sc);
        else
            st = comp ? solve<W_UNIT, P_COMP>(s, v, part_chunk, part_ew, sc) : solve<W_UNIT, P_F32>(s, v, part_chunk, part_ew, sc);
        if (st == VGA_ERR_NOT_CONVERGED) {
            worst = st;
        } else if (st != VGA_OK) {
            return st;
        }
        s->steps_done += 1;
    }
    if (worst != VGA_OK) return fail(worst, "implicit solve reached cg_maxit before cg_rtol");
    return VGA_OK;
}

}  // namespace vga
