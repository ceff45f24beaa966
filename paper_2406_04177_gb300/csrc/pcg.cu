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
#include <cstring>
#include <new>
#include <tuple>
#include <utility>

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
                                                      const res_t *__restrict__ y2l, CgVecs v,
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
        const double bi = ld_value_d<PREC>(y2, y2l, i);
        double lb = 0.0, deg = 0.0;
        for_each_neighbour(i, k, fl, s_nb, cap, [&](int slot, int64_t j) {
            const double g = (WM == W_UNIT) ? 1.0 : (double)edge_g(bw, i, slot, x, y, z);
            const double bj =
                ld_value_d<PREC>(y2, y2l, j);
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
            const double g = (WM == W_UNIT) ? 1.0 : (double)edge_g(bw, i, slot, x, y, z);
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
                                                     const res_t *__restrict__ y2l, double *__restrict__ x) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = ld_value_d<PREC>(y2, y2l, i);
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
                                                     res_t *__restrict__ outl, int comp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double v = x[i];
    const float h = (float)v;
    out[i] = h;
    if (comp) outl[i] = res_encode((float)(v - (double)h), h);
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


// ---- mixed precision: float-float iterative refinement around an FP32 Jacobi-PCG (unit conductances) ----
//
// GB300 executes FP64 at a small fraction of its FP32 rate, and the FP64 PCG above is bound by that
// arithmetic.  Here the outer loop keeps x and b as unevaluated sums of two FP32 numbers (hi + lo,
// about 48 significant bits) and forms the true residual r = b - B x in that arithmetic with FP32
// instructions (error-free TwoSum and FMA products); the correction B d = r is solved by the same
// Jacobi-PCG in FP32 to a relative reduction tol_in; x += d; the loop stops when
// ||b - B x||_2 <= rtol ||b||_2 (the true residual, not the recurrence; ||r||^2 and ||b||^2 are
// accumulated in FP64).  Every reduction is a fixed-order block-partial sum.
//
// Kernels of one inner iteration (three launches; no single-block scalar kernels):
//   k_mx_spmv   q = B p (four nodes per thread), partial p.q; the last block to finish forms alpha
//   k_mx_upd    d += alpha p, r -= alpha q, partials r.Tr and r.r; the last block tests the inner
//               stop and forms beta
//   k_mx_p      p = T r + beta p
// The Jacobi scaling T = diag(1 / (1 + c deg_i)) is not stored: each node keeps its degree in one
// byte and the kernels look t up in a 7-entry table computed by the same expression everywhere.
// "Last block": each block stores its partials, fences, and takes a ticket from a counter; the
// block that draws the final ticket sums all partials in block order (so the result does not
// depend on which block that is) and resets the counter.  No block waits for another.

constexpr double kInnerTol = 1e-4;  // reduction asked of one FP32 inner solve
constexpr int kMxBlocks = 2432;     // grid of the mixed-solver kernels: 152 SMs x 16 (grid-stride)
constexpr int kMaxOuter = 64;

struct MxScalars {
    double bb, rr_out, rz, alpha, beta, rr_in, stop_in, relres, rtol2;
    int32_t done, inner_done, iters, in_iters, notconv, maxit, outer;
    uint32_t ticket_a, ticket_b;  // arrival counters of the last-block reductions (0 between launches)
    int32_t fresh;                // set by the first residual pass: the next k_mx_scal_out starts a solve
    int32_t guard;                // inner iterations of this solve (a bound on the device-side loops)
    float scale, unscale;         // powers of two: the solve runs on b * scale; x leaves as x * unscale
};

// Device-side loops (the solve as one CUDA graph): the kernels that decide whether a loop goes on
// set the while-node conditions.  cond = 0 outside a graph (host-driven loop).
struct MxLoop {
    cudaGraphConditionalHandle outer, inner;
    int cond;
};

// Deterministic sum of part[k*stride + comp] over k < count by one block, read at L2 (the partials
// were written by other blocks of the same launch).
__device__ double block_reduce_partials_cg(const double *part, int64_t count, int stride, int comp) {
    double acc[1] = {0.0};
    for (int64_t k = threadIdx.x; k < count; k += blockDim.x) acc[0] += __ldcg(part + k * stride + comp);
    __shared__ double out[1];
    block_sum_store<1>(acc, out);
    return out[0];
}

// Called by every thread once the block's partials are stored: true in the block that arrives
// last, which then sees every block's partials.  The counter is reset for the next launch.  No
// block waits for another.
__device__ __forceinline__ bool last_block(uint32_t *ticket) {
    __shared__ int last;
    __threadfence();  // the partials stored by this thread are visible before the arrival
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t t = atomicAdd(ticket, 1u);
        last = (t == gridDim.x - 1) ? 1 : 0;
        if (last) *ticket = 0u;
    }
    __syncthreads();
    if (last) __threadfence();
    return last != 0;
}

// x and b: hi and lo parts; r, p, q, d: the FP32 inner solve; deg: node degree (0..6).
struct MxVecs {
    float *xh, *xl, *bh, *bl;
    float *r, *p, *q, *d;
    uint8_t *deg;
};

// Jacobi scaling t = 1 / (1 + c deg) (Sec. III: t_ii = 1 / b_ii), one expression for every kernel.
__device__ __forceinline__ float jacobi_t(float c, int deg) {
    return __fdiv_rn(1.0f, __fmaf_rn(c, (float)deg, 1.0f));
}

// Float-float values h + l and their error-free building blocks: TwoSum (Knuth) and the product
// error of a fused multiply-add.  Round-to-nearest intrinsics keep the compiler from contracting
// or reordering them.
struct FF {
    float h, l;
};

__device__ __forceinline__ FF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ FF ff_sub(FF a, FF b) {
    const FF s = two_sum(a.h, -b.h);
    return two_sum(s.h, __fadd_rn(s.l, __fsub_rn(a.l, b.l)));
}

__device__ __forceinline__ FF ff_mul(FF a, FF b) {
    const float p = __fmul_rn(a.h, b.h);
    const float e = __fmaf_rn(a.h, b.h, -p);
    return two_sum(p, __fadd_rn(e, __fadd_rn(__fmul_rn(a.h, b.l), __fmul_rn(a.l, b.h))));
}

// Sum over the neighbours of node i of x_j in float-float (TwoSum chain of the high parts; low parts
// and the chain's errors added in FP32), and their number.
template <int TF>
__device__ __forceinline__ FF nbr_sum_ff(const NbrTable &tb, uint32_t i, bool live, FF xi,
                                         const float *__restrict__ xh, const float *__restrict__ xl, int &deg) {
    const uint32_t ty = live ? __ldg(tb.ty + i) : 0u;
    uint32_t dzm, dzp;
    if (TF == 1) {
        const uint32_t tz = live ? __ldg(tb.tz + i) : 0u;
        dzm = tz & 0xffffu;
        dzp = tz >> 16;
    } else {
        dzm = live ? __ldg(tb.tzm + i) : 0u;
        dzp = live ? __ldg(tb.tzp + i) : 0u;
    }
    const int lane = threadIdx.x & 31;
    float hl = __shfl_up_sync(0xffffffffu, xi.h, 1), ll = __shfl_up_sync(0xffffffffu, xi.l, 1);
    float hr = __shfl_down_sync(0xffffffffu, xi.h, 1), lr = __shfl_down_sync(0xffffffffu, xi.l, 1);
    const uint32_t dym = ty & 0x7fffu, dyp = (ty >> 16) & 0x7fffu;
    const bool hxm = (ty >> 15) & 1u, hxp = ty >> 31;
    if (lane == 0 && hxm) {
        hl = __ldg(xh + (i - 1));
        ll = __ldg(xl + (i - 1));
    }
    if (lane == 31 && hxp) {
        hr = __ldg(xh + (i + 1));
        lr = __ldg(xl + (i + 1));
    }
    FF s = {0.0f, 0.0f};
    auto add = [&](float h, float l) {
        const FF t = two_sum(s.h, h);
        s.h = t.h;
        s.l = __fadd_rn(s.l, __fadd_rn(t.l, l));
    };
    if (hxm) add(hl, ll);
    if (hxp) add(hr, lr);
    if (dym) add(__ldg(xh + (i - dym)), __ldg(xl + (i - dym)));
    if (dyp) add(__ldg(xh + (i + dyp)), __ldg(xl + (i + dyp)));
    if (dzm) add(__ldg(xh + (i - dzm)), __ldg(xl + (i - dzm)));
    if (dzp) add(__ldg(xh + (i + dzp)), __ldg(xl + (i + dzp)));
    deg = (int)hxm + (int)hxp + (dym != 0) + (dyp != 0) + (dzm != 0) + (dzp != 0);
    return s;
}

// Outer residual r = b - B x = b - x - c (deg x_i - sum_j x_j) in float-float (FIRST: x = b, so
// r = -c L b), rounded to FP32 for the inner solve; deg, p = T r, d = 0; partials (r.r and b.b
// (FIRST) in FP64, r.Tr).  FP32 instructions only per node, apart from the two FP64 squares.
template <bool FIRST, int TF>
__global__ void __launch_bounds__(kThreads) k_mx_res(int64_t n, NbrTable tb, FF c, MxVecs v,
                                                     double *__restrict__ part, MxScalars *sc) {
    if (!FIRST && sc->done) return;
    if (FIRST && blockIdx.x == 0 && threadIdx.x == 0) sc->fresh = 1;
    FF rr = {0.0f, 0.0f};  // |r|^2 per thread in float-float (no FP64 arithmetic per node)
    double bb = 0.0;       // |b|^2, once per solve
    float rz = 0.0f;
    const int64_t ntile = (n + kThreads - 1) / kThreads;
    const float *__restrict__ sh = FIRST ? v.bh : v.xh;  // FIRST: x = b, neighbours read from b
    const float *__restrict__ sl = FIRST ? v.bl : v.xl;
    for (int64_t tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const uint32_t i = (uint32_t)(tile * kThreads + threadIdx.x);
        const bool live = i < (uint64_t)n;
        FF xi = {0.0f, 0.0f}, bi = {0.0f, 0.0f};
        if (live) {
            bi = {__ldg(v.bh + i), __ldg(v.bl + i)};
            xi = FIRST ? bi : FF{__ldg(v.xh + i), __ldg(v.xl + i)};
        }
        int deg = 0;
        const FF sx = nbr_sum_ff<TF>(tb, i, live, xi, sh, sl, deg);
        if (live) {
            const float fd = (float)deg;
            const float ph = __fmul_rn(fd, xi.h);
            const FF dx = two_sum(ph, __fadd_rn(__fmaf_rn(fd, xi.h, -ph), __fmul_rn(fd, xi.l)));  // deg x_i
            const FF cl = ff_mul(c, ff_sub(dx, sx));                                             // c (L x)_i
            const FF r = FIRST ? FF{-cl.h, -cl.l} : ff_sub(ff_sub(bi, xi), cl);
            const float r32 = __fadd_rn(r.h, r.l);
            const float ti = jacobi_t(c.h, deg);
            if (FIRST) {
                v.xh[i] = bi.h;
                v.xl[i] = bi.l;
            }
            v.deg[i] = (uint8_t)deg;
            v.r[i] = r32;
            v.p[i] = __fmul_rn(ti, r32);
            v.d[i] = 0.0f;
            const float q = __fmul_rn(r32, r32);
            const FF t = two_sum(rr.h, q);
            rr = {t.h, __fadd_rn(rr.l, __fadd_rn(t.l, __fmaf_rn(r32, r32, -q)))};
            if (FIRST) {
                const double b = (double)bi.h + (double)bi.l;
                bb = fma(b, b, bb);
            }
            rz = __fmaf_rn(r32, __fmul_rn(ti, r32), rz);
        }
    }
    double acc[3] = {(double)rr.h + (double)rr.l, bb, (double)rz};
    __shared__ double out[3];
    block_sum_store<3>(acc, out);
    if (threadIdx.x < 3) part[(int64_t)blockIdx.x * 3 + threadIdx.x] = out[threadIdx.x];
}

// Scale of the solve.  The system (I + c L) x = b is linear, so it may be solved for b * 2^-e and
// the solution multiplied by 2^e.  With 2^e the binade of max |b| every vector of the solve is at
// most about 1 in magnitude, whatever unit the caller stores masses in: the FP32 squares of the
// residual and the inner dot products stay far from underflow (they would vanish below |r| ~ 1e-19,
// and with them the stop test and alpha).  Scaling by a power of two is exact, so the iterations and
// the result are the same bits as an unscaled solve wherever that one neither underflows nor
// overflows.  k_mx_bmax stores the maximum of each block, k_mx_bscale turns them into the scale.
__global__ void __launch_bounds__(kThreads) k_mx_bmax(int64_t n, const float *__restrict__ y2,
                                                      double *__restrict__ part) {
    float m = 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(__ldg(y2 + i)));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    __shared__ float wm[kThreads / 32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kThreads / 32; ++w) m = fmaxf(m, wm[w]);
        part[blockIdx.x] = (double)m;
    }
}

__global__ void __launch_bounds__(kThreads) k_mx_bscale(const double *__restrict__ part, int count, MxScalars *sc) {
    double m = 0.0;
    for (int b = threadIdx.x; b < count; b += blockDim.x) m = fmax(m, part[b]);
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
    __shared__ double wm[kThreads / 32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kThreads / 32; ++w) m = fmax(m, wm[w]);
        int e = 0;
        if (m > 0.0 && m <= 3.0e38) frexp(m, &e);  // m = f 2^e, f in [0.5, 1)
        e = max(-120, min(120, e));
        sc->scale = ldexpf(1.0f, -e);
        sc->unscale = ldexpf(1.0f, e);
    }
}

// b = the stored DOM after the transformation, times the scale: FP32 value and its residual as hi
// and lo.
template <int PREC>
__global__ void __launch_bounds__(kThreads) k_mx_rhs(int64_t n, const float *__restrict__ y2,
                                                     const res_t *__restrict__ y2l, float *__restrict__ bh,
                                                     float *__restrict__ bl, const MxScalars *__restrict__ sc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float s = sc->scale;
    const float h = __ldg(y2 + i);
    bh[i] = __fmul_rn(h, s);
    bl[i] = (PREC == P_COMP) ? __fmul_rn(res_decode(__ldg(y2l + i), h), s) : 0.0f;
}

// Start of an outer iteration: the residual norms, the outer stop test, the next inner solve's
// tolerance; sets both loop conditions to "not done".
__global__ void __launch_bounds__(kThreads) k_mx_scal_out(const double *__restrict__ part, int64_t count, MxScalars *sc,
                                                          double rtol, int maxit, MxLoop loop) {
    const int first = sc->fresh;
    if (!first && sc->done) {
        if (loop.cond && threadIdx.x == 0) {
            cudaGraphSetConditional(loop.inner, 0u);
            cudaGraphSetConditional(loop.outer, 0u);
        }
        return;
    }
    const double rr = block_reduce_partials(part, count, 3, 0);
    const double bb = first ? block_reduce_partials(part, count, 3, 1) : 0.0;
    const double rz = block_reduce_partials(part, count, 3, 2);
    if (threadIdx.x == 0) {
        if (first) {
            sc->bb = bb;
            sc->rtol2 = rtol * rtol;
            sc->iters = 0;
            sc->outer = 0;
            sc->notconv = 0;
            sc->maxit = maxit;
            sc->done = 0;
            sc->guard = 0;
            sc->fresh = 0;
        }
        sc->rr_out = rr;
        sc->relres = sc->bb > 0.0 ? sqrt(rr / sc->bb) : 0.0;
        sc->outer += 1;
        if (sc->bb == 0.0 || rr <= sc->rtol2 * sc->bb) {
            sc->done = 1;
        } else if (sc->iters >= sc->maxit || sc->outer > kMaxOuter) {
            sc->done = 1;
            sc->notconv = 1;
        }
        // reduce the residual by kInnerTol, or just below the target if that asks less
        const double want = 0.25 * sc->rtol2 * sc->bb / (rr > 0.0 ? rr : 1.0);
        const double tol2 = want > kInnerTol * kInnerTol ? want : kInnerTol * kInnerTol;
        sc->stop_in = tol2 * rr;
        sc->rz = rz;
        sc->rr_in = rr;
        sc->in_iters = 0;
        sc->inner_done = sc->done;
        sc->ticket_a = 0u;
        sc->ticket_b = 0u;
        if (loop.cond) {
            cudaGraphSetConditional(loop.inner, sc->done ? 0u : 1u);
            cudaGraphSetConditional(loop.outer, sc->done ? 0u : 1u);
        }
    }
}

// q = B p in FP32 with four consecutive nodes per thread (16-byte accesses of p, q and the offset
// table; the -x neighbour of the first node and the +x neighbour of the last come from the adjacent
// lanes), partial p.q; the block that finishes last forms alpha = r.Tr / p.q.
template <int TF>
__global__ void __launch_bounds__(kThreads) k_mx_spmv(int64_t n, NbrTable tb, float c, MxVecs v,
                                                      double *__restrict__ part, MxScalars *sc) {
    if (sc->inner_done) return;
    constexpr int K = 4;
    float acc = 0.0f;
    const float *__restrict__ p = v.p;
    float *__restrict__ q = v.q;
    const uint32_t nn = (uint32_t)n;
    const int lane = threadIdx.x & 31;
    const int64_t nsup = (n + (int64_t)kThreads * K - 1) / ((int64_t)kThreads * K);
    for (int64_t sup = blockIdx.x; sup < nsup; sup += gridDim.x) {
        const uint32_t i0 = (uint32_t)(sup * kThreads * K + (int64_t)threadIdx.x * K);
        const bool full = i0 + K <= nn;
        float pv[K];
        uint32_t ty[K], zm[K], zp[K];
        if (full) {
            ldg_floats<K>(p + i0, pv);
            ldg_words_k<K, true>(tb.ty, i0, nn, ty);
            if (TF == 1) {
                ldg_words_k<K, true>(tb.tz, i0, nn, zm);
            } else {
                ldg_words_k<K, true>(tb.tzm, i0, nn, zm);
                ldg_words_k<K, true>(tb.tzp, i0, nn, zp);
            }
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k) pv[k] = i0 + k < nn ? __ldg(p + i0 + k) : 0.0f;
            ldg_words_k<K, false>(tb.ty, i0, nn, ty);
            if (TF == 1) {
                ldg_words_k<K, false>(tb.tz, i0, nn, zm);
            } else {
                ldg_words_k<K, false>(tb.tzm, i0, nn, zm);
                ldg_words_k<K, false>(tb.tzp, i0, nn, zp);
            }
        }
        if (TF == 1) {
#pragma unroll
            for (int k = 0; k < K; ++k) {
                zp[k] = zm[k] >> 16;
                zm[k] &= 0xffffu;
            }
        }
        float pl = __shfl_up_sync(0xffffffffu, pv[K - 1], 1);
        float pr = __shfl_down_sync(0xffffffffu, pv[0], 1);
        if (lane == 0 && ((ty[0] >> 15) & 1u)) pl = __ldg(p + (i0 - 1));
        if (lane == 31 && (ty[K - 1] >> 31)) pr = __ldg(p + (i0 + K));
        float qv[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const uint32_t dym = ty[k] & 0x7fffu, dyp = (ty[k] >> 16) & 0x7fffu;
            const float vi = pv[k];
            float sum = 0.0f;
            if ((ty[k] >> 15) & 1u) sum += vi - (k == 0 ? pl : pv[k > 0 ? k - 1 : 0]);
            if (ty[k] >> 31) sum += vi - (k == K - 1 ? pr : pv[k < K - 1 ? k + 1 : 0]);
            if (dym) sum += vi - __ldg(p + (i0 + k - dym));
            if (dyp) sum += vi - __ldg(p + (i0 + k + dyp));
            if (zm[k]) sum += vi - __ldg(p + (i0 + k - zm[k]));
            if (zp[k]) sum += vi - __ldg(p + (i0 + k + zp[k]));
            qv[k] = vi + c * sum;
            if (i0 + k < nn) acc += vi * qv[k];
        }
        if (full) {
            st_floats<K>(q + i0, qv);
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (i0 + k < nn) q[i0 + k] = qv[k];
        }
    }
    double a[1] = {(double)acc};
    __shared__ double out[1];
    block_sum_store<1>(a, out);
    if (threadIdx.x == 0) part[blockIdx.x] = out[0];
    if (last_block(&sc->ticket_a)) {
        const double pq = block_reduce_partials_cg(part, gridDim.x, 1, 0);
        if (threadIdx.x == 0) sc->alpha = pq > 0.0 ? sc->rz / pq : 0.0;
    }
}

// The streaming kernels below move four nodes per thread and access (16-byte vectors: every FP32
// array starts on a 16-byte boundary, the degrees on a 4-byte one); the n % 4 last nodes go through
// a scalar tail, so the padding after node n never enters a sum.  c is the FP32 c of the inner
// solve (the Jacobi table is built from it).
__global__ void __launch_bounds__(kThreads) k_mx_upd(int64_t n, float c, MxVecs v, MxScalars *sc,
                                                     double *__restrict__ part, int in_maxit, MxLoop loop) {
    if (sc->inner_done) {
        if (loop.cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(loop.inner, 0u);
        return;
    }
    __shared__ float tdeg[8];
    if (threadIdx.x < 8) tdeg[threadIdx.x] = jacobi_t(c, (int)threadIdx.x);
    __syncthreads();
    const float alpha = (float)sc->alpha;
    float a0 = 0.0f, a1 = 0.0f;
    const int64_t n4 = n >> 2;
    const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
    float4 *__restrict__ d4 = reinterpret_cast<float4 *>(v.d);
    float4 *__restrict__ r4 = reinterpret_cast<float4 *>(v.r);
    const float4 *__restrict__ p4 = reinterpret_cast<const float4 *>(v.p);
    const float4 *__restrict__ q4 = reinterpret_cast<const float4 *>(v.q);
    const uchar4 *__restrict__ g4 = reinterpret_cast<const uchar4 *>(v.deg);
    for (int64_t k = g0; k < n4; k += gs) {
        float4 d = d4[k], r = r4[k];
        const float4 p = p4[k], q = q4[k];
        const uchar4 g = g4[k];
        d.x += alpha * p.x;
        d.y += alpha * p.y;
        d.z += alpha * p.z;
        d.w += alpha * p.w;
        r.x -= alpha * q.x;
        r.y -= alpha * q.y;
        r.z -= alpha * q.z;
        r.w -= alpha * q.w;
        d4[k] = d;
        r4[k] = r;
        a0 += r.x * (tdeg[g.x] * r.x) + r.y * (tdeg[g.y] * r.y) + r.z * (tdeg[g.z] * r.z) + r.w * (tdeg[g.w] * r.w);
        a1 += r.x * r.x + r.y * r.y + r.z * r.z + r.w * r.w;
    }
    for (int64_t i = 4 * n4 + g0; i < n; i += gs) {
        v.d[i] += alpha * v.p[i];
        const float ri = v.r[i] - alpha * v.q[i];
        v.r[i] = ri;
        a0 += ri * (tdeg[v.deg[i]] * ri);
        a1 += ri * ri;
    }
    double a[2] = {(double)a0, (double)a1};
    __shared__ double out[2];
    block_sum_store<2>(a, out);
    if (threadIdx.x < 2) part[(int64_t)blockIdx.x * 2 + threadIdx.x] = out[threadIdx.x];
    // the last block: inner convergence test and beta (every block has passed its inner_done test
    // before the last one arrives, so none of this launch sees the update)
    if (last_block(&sc->ticket_b)) {
        const double rz = block_reduce_partials_cg(part, gridDim.x, 2, 0);
        const double rr = block_reduce_partials_cg(part, gridDim.x, 2, 1);
        if (threadIdx.x == 0) {
            sc->iters += 1;
            sc->in_iters += 1;
            sc->rr_in = rr;
            if (rr <= sc->stop_in || sc->in_iters >= in_maxit || sc->iters >= sc->maxit || !(sc->rz > 0.0)) {
                sc->inner_done = 1;
            } else {
                sc->beta = rz / sc->rz;
                sc->rz = rz;
            }
            // the iteration limits above end every loop; this bound holds even if they did not
            if (++sc->guard > (kMaxOuter + 2) * (in_maxit + 1)) {
                sc->inner_done = 1;
                sc->done = 1;
                sc->notconv = 1;
            }
            if (loop.cond) cudaGraphSetConditional(loop.inner, sc->inner_done ? 0u : 1u);
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_mx_p(int64_t n, float c, MxVecs v, const MxScalars *__restrict__ sc) {
    if (sc->inner_done) return;
    __shared__ float tdeg[8];
    if (threadIdx.x < 8) tdeg[threadIdx.x] = jacobi_t(c, (int)threadIdx.x);
    __syncthreads();
    const float beta = (float)sc->beta;
    const int64_t n4 = n >> 2;
    const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
    float4 *__restrict__ p4 = reinterpret_cast<float4 *>(v.p);
    const float4 *__restrict__ r4 = reinterpret_cast<const float4 *>(v.r);
    const uchar4 *__restrict__ g4 = reinterpret_cast<const uchar4 *>(v.deg);
    for (int64_t k = g0; k < n4; k += gs) {
        float4 p = p4[k];
        const float4 r = r4[k];
        const uchar4 g = g4[k];
        p.x = tdeg[g.x] * r.x + beta * p.x;
        p.y = tdeg[g.y] * r.y + beta * p.y;
        p.z = tdeg[g.z] * r.z + beta * p.z;
        p.w = tdeg[g.w] * r.w + beta * p.w;
        p4[k] = p;
    }
    for (int64_t i = 4 * n4 + g0; i < n; i += gs) v.p[i] = tdeg[v.deg[i]] * v.r[i] + beta * v.p[i];
}

// x += d in float-float (TwoSum of the high part and d, then renormalised).
__device__ __forceinline__ void ff_add_f(float &xh, float &xl, float d) {
    const FF s = two_sum(xh, d);
    const FF t = two_sum(s.h, __fadd_rn(s.l, xl));
    xh = t.h;
    xl = t.l;
}

__global__ void __launch_bounds__(kThreads) k_mx_x(int64_t n, MxVecs v, const MxScalars *__restrict__ sc) {
    if (sc->done) return;
    const int64_t n4 = n >> 2;
    const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, gs = (int64_t)gridDim.x * blockDim.x;
    float4 *__restrict__ h4 = reinterpret_cast<float4 *>(v.xh);
    float4 *__restrict__ l4 = reinterpret_cast<float4 *>(v.xl);
    const float4 *__restrict__ d4 = reinterpret_cast<const float4 *>(v.d);
    for (int64_t k = g0; k < n4; k += gs) {
        float4 h = h4[k], l = l4[k];
        const float4 d = d4[k];
        ff_add_f(h.x, l.x, d.x);
        ff_add_f(h.y, l.y, d.y);
        ff_add_f(h.z, l.z, d.z);
        ff_add_f(h.w, l.w, d.w);
        h4[k] = h;
        l4[k] = l;
    }
    for (int64_t i = 4 * n4 + g0; i < n; i += gs) ff_add_f(v.xh[i], v.xl[i], v.d[i]);
}

// The solution as the new stored DOM: h = RN(xh + xl) and the exact remainder as residual.
template <int PREC>
__global__ void __launch_bounds__(kThreads) k_mx_out(int64_t n, MxVecs v, float *__restrict__ out,
                                                     res_t *__restrict__ outl, const MxScalars *__restrict__ sc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float u = sc->unscale;  // back to the caller's units (exact: a power of two)
    const FF s = two_sum(__fmul_rn(v.xh[i], u), __fmul_rn(v.xl[i], u));
    out[i] = s.h;
    if (PREC == P_COMP) outl[i] = res_encode(s.l, s.h);
}

// ---- the mixed solve as one CUDA graph -------------------------------------------------------
//
//   k_mx_bmax -> k_mx_bscale -> k_mx_rhs -> k_mx_res<first> -> WHILE(outer) { k_mx_scal_out ->
//   WHILE(inner) { k_mx_spmv -> k_mx_upd -> k_mx_p } -> k_mx_x -> k_mx_res } -> k_mx_out
//
// k_mx_scal_out sets both conditions to "not done" at the start of every outer iteration and
// k_mx_upd clears the inner one when the inner solve stops, so the host launches the graph and
// synchronises once per time step instead of polling every kBatch iterations.  Each loop is
// bounded by the iteration limits (in_maxit, cg_maxit, kMaxOuter) and by the guard counter.  The
// state buffers alternate between steps, so one graph is kept per parity of the DOM buffer.

template <typename Tuple, size_t... I>
void kernel_arg_ptrs(Tuple &t, void **a, std::index_sequence<I...>) {
    ((a[I] = (void *)&std::get<I>(t)), ...);
}

// Adds a kernel node (kThreads threads per block) that depends on *dep (if not NULL).  The node
// copies the argument values.
template <typename... P, typename... A>
cudaError_t add_kernel(cudaGraphNode_t *node, cudaGraph_t g, const cudaGraphNode_t *dep, void (*fn)(P...),
                       unsigned grid, A... a) {
    static_assert(sizeof...(P) == sizeof...(A), "kernel argument count");
    std::tuple<P...> vals(static_cast<P>(a)...);
    void *args[sizeof...(P) > 0 ? sizeof...(P) : 1];
    kernel_arg_ptrs(vals, args, std::index_sequence_for<P...>{});
    cudaKernelNodeParams kp = {};
    kp.func = (void *)fn;
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(kThreads);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    kp.extra = nullptr;
    return cudaGraphAddKernelNode(node, g, dep, dep ? 1 : 0, &kp);
}

// Adds a while node after *dep; its body graph is returned in *body.
cudaError_t add_while(cudaGraphNode_t *node, cudaGraph_t g, const cudaGraphNode_t *dep,
                      cudaGraphConditionalHandle h, cudaGraph_t *body) {
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    const cudaError_t e = cudaGraphAddNode(node, g, dep, nullptr, dep ? 1 : 0, &cp);
    if (e == cudaSuccess) *body = cp.conditional.phGraph_out[0];
    return e;
}

struct MxGraphKey {
    const void *ptr[12];
    int64_t n;
    double c, rtol;
    int32_t maxit, G, prec, tf;
};

struct MxGraphCache {
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    MxGraphKey key[2];
};

void mx_graph_drop(MxGraphCache *gc, int slot) {
    if (gc->exec[slot]) cudaGraphExecDestroy(gc->exec[slot]);
    if (gc->graph[slot]) cudaGraphDestroy(gc->graph[slot]);
    gc->exec[slot] = nullptr;
    gc->graph[slot] = nullptr;
}

template <int PREC, int TF>
cudaError_t mx_graph_build(vga_sim *s, const MxVecs &v, const NbrTable &tb, FF cff, int G, int in_maxit,
                           double *part_a, double *part_b, MxScalars *sc, cudaGraph_t *gout) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    MxLoop loop = {0, 0, 1};
    cudaGraphNode_t n_bm, n_bs, n_rhs, n_res0, n_outer, n_out, n_scal, n_inner, n_x, n_res, n_spmv, n_upd, n_p;
    cudaGraph_t body_o = nullptr, body_i = nullptr;
    const unsigned ge = grid_for(s->n, kThreads);
    const double rtol = s->params.cg_rtol;
    const int maxit = s->params.cg_maxit;
    const float ch = cff.h;
#define MX_TRY(x)                        \
    do {                                 \
        e = (x);                         \
        if (e != cudaSuccess) goto fail; \
    } while (0)
    MX_TRY(cudaGraphConditionalHandleCreate(&loop.outer, g, 1u, cudaGraphCondAssignDefault));
    MX_TRY(add_kernel(&n_bm, g, nullptr, k_mx_bmax, G, s->n, s->comp(1), part_a));
    MX_TRY(add_kernel(&n_bs, g, &n_bm, k_mx_bscale, 1u, part_a, G, sc));
    MX_TRY(add_kernel(&n_rhs, g, &n_bs, k_mx_rhs<PREC>, ge, s->n, s->comp(1), s->lcomp(1), v.bh, v.bl, sc));
    MX_TRY(add_kernel(&n_res0, g, &n_rhs, k_mx_res<true, TF>, G, s->n, tb, cff, v, part_a, sc));
    MX_TRY(add_while(&n_outer, g, &n_res0, loop.outer, &body_o));
    MX_TRY(add_kernel(&n_out, g, &n_outer, k_mx_out<PREC>, ge, s->n, v, s->spare(1), s->lspare(1), sc));
    MX_TRY(cudaGraphConditionalHandleCreate(&loop.inner, body_o, 0u, 0u));
    MX_TRY(add_kernel(&n_scal, body_o, nullptr, k_mx_scal_out, 1u, part_a, (int64_t)G, sc, rtol, maxit, loop));
    MX_TRY(add_while(&n_inner, body_o, &n_scal, loop.inner, &body_i));
    MX_TRY(add_kernel(&n_x, body_o, &n_inner, k_mx_x, G, s->n, v, sc));
    MX_TRY(add_kernel(&n_res, body_o, &n_x, k_mx_res<false, TF>, G, s->n, tb, cff, v, part_a, sc));
    MX_TRY(add_kernel(&n_spmv, body_i, nullptr, k_mx_spmv<TF>, G, s->n, tb, ch, v, part_a, sc));
    MX_TRY(add_kernel(&n_upd, body_i, &n_spmv, k_mx_upd, G, s->n, ch, v, sc, part_b, in_maxit, loop));
    MX_TRY(add_kernel(&n_p, body_i, &n_upd, k_mx_p, G, s->n, ch, v, sc));
#undef MX_TRY
    *gout = g;
    return cudaSuccess;
fail:
    cudaGraphDestroy(g);
    return e;
}

template <int PREC>
vga_status solve_mixed(vga_sim *s, double *base, double *part_a, double *part_b, MxScalars *sc) {
    const double c = s->params.D * s->params.dt;
    const float ch = (float)c;
    const FF cff = {ch, (float)(c - (double)ch)};
    cudaStream_t st = s->stream;
    NbrTable tb;
    VGA_TRY(sim_nbr_table(s, &tb));
    // 8.25 npad FP32 words inside the 5 npad doubles of the vector buffer
    MxVecs v;
    float *f = reinterpret_cast<float *>(base);
    v.xh = f;
    v.xl = f + s->npad;
    v.bh = f + 2 * s->npad;
    v.bl = f + 3 * s->npad;
    v.r = f + 4 * s->npad;
    v.p = f + 5 * s->npad;
    v.q = f + 6 * s->npad;
    v.d = f + 7 * s->npad;
    v.deg = reinterpret_cast<uint8_t *>(f + 8 * s->npad);
    const int G = (int)std::min<int64_t>(kMxBlocks, grid_for(s->n, kThreads));
    const int in_maxit = 200;
    MxScalars *h = reinterpret_cast<MxScalars *>(s->h_cg);

    if (!s->cg_host_loop && !s->mx_graph_failed) {
        if (!s->mx_graph) s->mx_graph = new (std::nothrow) MxGraphCache();
        MxGraphCache *gc = static_cast<MxGraphCache *>(s->mx_graph);
        if (gc) {
            const int slot = s->cur[1] & 1;
            MxGraphKey key;
            std::memset(&key, 0, sizeof(key));
            const void *ptrs[12] = {base, part_a, part_b, sc, s->comp(1), s->lcomp(1), s->spare(1), s->lspare(1),
                                    tb.ty, tb.tz, tb.tzm, tb.tzp};
            std::memcpy(key.ptr, ptrs, sizeof(ptrs));
            key.n = s->n;
            key.c = c;
            key.rtol = s->params.cg_rtol;
            key.maxit = s->params.cg_maxit;
            key.G = G;
            key.prec = PREC;
            key.tf = tb.tz ? 1 : 0;
            if (!gc->exec[slot] || std::memcmp(&key, &gc->key[slot], sizeof(key)) != 0) {
                mx_graph_drop(gc, slot);
                cudaError_t e = tb.tz ? mx_graph_build<PREC, 1>(s, v, tb, cff, G, in_maxit, part_a, part_b, sc, &gc->graph[slot])
                                      : mx_graph_build<PREC, 0>(s, v, tb, cff, G, in_maxit, part_a, part_b, sc, &gc->graph[slot]);
                if (e == cudaSuccess) e = cudaGraphInstantiate(&gc->exec[slot], gc->graph[slot], 0);
                if (e == cudaSuccess) {
                    gc->key[slot] = key;
                } else {
                    // no conditional graph nodes here: keep the host-driven loop from now on
                    mx_graph_drop(gc, slot);
                    (void)cudaGetLastError();
                    s->mx_graph_failed = true;
                }
            }
            if (gc->exec[slot]) {
                timing_begin(s, VGA_KERNEL_PCG_STENCIL);
                VGA_CUDA(cudaGraphLaunch(gc->exec[slot], st));
                timing_end(s);
                VGA_CUDA(cudaMemcpyAsync(h, sc, sizeof(MxScalars), cudaMemcpyDeviceToHost, st));
                VGA_CUDA(cudaStreamSynchronize(st));
                s->graph_launches += 1;
                s->launches += 5 + 3 * (int64_t)h->outer + 3 * (int64_t)h->iters;  // kernels the graph ran
                s->cur[1] ^= 1;
                s->cg_iterations += h->iters;
                s->cg_last_relres = h->relres;
                return h->notconv ? VGA_ERR_NOT_CONVERGED : VGA_OK;
            }
        }
    }

    // host-driven loop: the same kernels, the done flags polled every kBatch inner iterations
    const MxLoop noloop = {0, 0, 0};
    timing_begin(s, VGA_KERNEL_PCG_STENCIL);
    k_mx_bmax<<<G, kThreads, 0, st>>>(s->n, s->comp(1), part_a);
    k_mx_bscale<<<1, kThreads, 0, st>>>(part_a, G, sc);
    k_mx_rhs<PREC><<<grid_for(s->n, kThreads), kThreads, 0, st>>>(s->n, s->comp(1), s->lcomp(1), v.bh, v.bl, sc);
    if (tb.tz) k_mx_res<true, 1><<<G, kThreads, 0, st>>>(s->n, tb, cff, v, part_a, sc);
    else k_mx_res<true, 0><<<G, kThreads, 0, st>>>(s->n, tb, cff, v, part_a, sc);
    timing_end(s);
    k_mx_scal_out<<<1, kThreads, 0, st>>>(part_a, G, sc, s->params.cg_rtol, s->params.cg_maxit, noloop);
    VGA_CHECK_LAUNCH();
    s->launches += 5;
    for (int guard = 0; guard < 100000; ++guard) {
        for (int k = 0; k < kBatch; ++k) {
            timing_begin(s, VGA_KERNEL_PCG_STENCIL);
            if (tb.tz) k_mx_spmv<1><<<G, kThreads, 0, st>>>(s->n, tb, ch, v, part_a, sc);
            else k_mx_spmv<0><<<G, kThreads, 0, st>>>(s->n, tb, ch, v, part_a, sc);
            timing_end(s);
            timing_begin(s, VGA_KERNEL_PCG_VECTOR);
            k_mx_upd<<<G, kThreads, 0, st>>>(s->n, ch, v, sc, part_b, in_maxit, noloop);
            k_mx_p<<<G, kThreads, 0, st>>>(s->n, ch, v, sc);
            timing_end(s);
        }
        VGA_CHECK_LAUNCH();
        s->launches += 3 * kBatch;
        VGA_CUDA(cudaMemcpyAsync(h, sc, sizeof(MxScalars), cudaMemcpyDeviceToHost, st));
        VGA_CUDA(cudaStreamSynchronize(st));
        if (h->done) break;
        if (h->inner_done) {
            // x += d, then the true residual of the new x and the next inner solve's start
            timing_begin(s, VGA_KERNEL_PCG_STENCIL);
            k_mx_x<<<G, kThreads, 0, st>>>(s->n, v, sc);
            if (tb.tz) k_mx_res<false, 1><<<G, kThreads, 0, st>>>(s->n, tb, cff, v, part_a, sc);
            else k_mx_res<false, 0><<<G, kThreads, 0, st>>>(s->n, tb, cff, v, part_a, sc);
            timing_end(s);
            k_mx_scal_out<<<1, kThreads, 0, st>>>(part_a, G, sc, s->params.cg_rtol, s->params.cg_maxit, noloop);
            VGA_CHECK_LAUNCH();
            s->launches += 3;
        }
    }
    k_mx_out<PREC><<<grid_for(s->n, kThreads), kThreads, 0, st>>>(s->n, v, s->spare(1), s->lspare(1), sc);
    VGA_CHECK_LAUNCH();
    ++s->launches;
    s->cur[1] ^= 1;
    s->cg_iterations += h->iters;
    s->cg_last_relres = h->relres;
    return h->notconv ? VGA_ERR_NOT_CONVERGED : VGA_OK;
}

}  // namespace

void sim_mx_graph_release(vga_sim *s) {
    MxGraphCache *gc = static_cast<MxGraphCache *>(s->mx_graph);
    if (!gc) return;
    mx_graph_drop(gc, 0);
    mx_graph_drop(gc, 1);
    delete gc;
    s->mx_graph = nullptr;
}

vga_status sim_step_implicit(vga_sim *s, int64_t n_steps) {
    if (n_steps <= 0 || s->n == 0) {
        s->steps_done += std::max<int64_t>(n_steps, 0);
        return VGA_OK;
    }
    const int64_t G = std::max<int64_t>(s->chunks.count, (s->n + kThreads - 1) / kThreads);
    // partials: 3 per block of the stencil grids, 2 per block of the elementwise grids
    const int64_t pa = 3 * std::max<int64_t>(std::max<int64_t>(G, kMxBlocks), 1);
    const int64_t pb = 2 * (int64_t)std::max(kEwBlocks, kMxBlocks);
    const int64_t need = 5 * s->npad + pa + pb;
    if (s->cg_count < need) {
        dfree(s->cg);
        s->cg = nullptr;
        s->cg_count = 0;
        VGA_TRY(dmalloc((void **)&s->cg, sizeof(double) * (size_t)need, "PCG vectors"));
        s->cg_count = need;
    }
    constexpr size_t kScal = sizeof(CgScalars) > sizeof(MxScalars) ? sizeof(CgScalars) : sizeof(MxScalars);
    if (!s->cg_scalars) VGA_TRY(dmalloc((void **)&s->cg_scalars, kScal + 64, "PCG scalars"));
    if (!s->h_cg) VGA_CUDA(cudaMallocHost((void **)&s->h_cg, kScal + 64));
    CgVecs v;
    v.x = s->cg;
    v.r = v.x + s->npad;
    v.p = v.r + s->npad;
    v.q = v.p + s->npad;
    v.t = v.q + s->npad;
    double *part_chunk = v.t + s->npad;
    double *part_ew = part_chunk + pa;
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
        else if (s->g->nx <= 32767 && s->cg_mixed)
            st = comp ? solve_mixed<P_COMP>(s, s->cg, part_chunk, part_ew, reinterpret_cast<MxScalars *>(sc))
                      : solve_mixed<P_F32>(s, s->cg, part_chunk, part_ew, reinterpret_cast<MxScalars *>(sc));
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
