// Discrete adjoint of the explicit synchronous time step, with checkpointing, and the block-mass
// objective used to fit block conductances.
//
// Forward step k: Y = T(X^k) voxel by voxel, X^{k+1} = (y1, Q_g y2, y3, y4, y5) with
// Q_g = I - D dt L_g (Scheme 1 with edge conductances, Sec. II.B.3a and the weighted flux of
// Sec. V.A).  Q_g is symmetric, so the reverse of step k is
//     mu = (lam1, Q_g lam2, lam3, lam4, lam5)             (lam = dL/dX^{k+1})
//     dL/dX^k = J_T(X^k)^T mu                              (transform_sync_reverse)
// with parameter gradients
//     dL/dD        += -dt sum_i lam2_i (L_g y2)_i
//     dL/dtheta_f  += -D dt sum_{edges e crossing face f} (y2_i - y2_j)(lam2_i - lam2_j)
//     dL/drates    += w . df/drate                         (transform_sync_reverse)
// This is the multi-step, transformation-coupled form of the closed-form gradients of Sec. V.A.
//
// Memory: the forward stores the state every `ckpt` steps; each segment is recomputed once from
// its checkpoint, recording X^k (FP32) and the transformed DOM y2^k, and then reversed step by
// step.  The adjoint state is carried like the forward state (FP32 value + BF16 residual) and every
// parameter gradient is accumulated in FP64 (per-block partials, FP64 atomics for the faces).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "physics.cuh"
#include "stencil.cuh"
#include "vga_internal.cuh"

namespace vga {

namespace {

constexpr int kThreads = 256;
#ifndef VGA_ADJ_MIN_BLOCKS
#define VGA_ADJ_MIN_BLOCKS 4  // resident blocks per SM the reverse step is compiled for
#endif
#ifndef VGA_ADJ_K
#define VGA_ADJ_K 2  // consecutive nodes per thread in the reverse step (2 or 4)
#endif
constexpr int kAdjK = VGA_ADJ_K;
// The reverse steps keep their partial sums in per-thread slots across a sweep when a thread takes
// at most this many groups of nodes per launch (small graphs), else reduce them per launch.
constexpr int64_t kSlotGroups = 8;
static_assert(kAdjK == 2 || kAdjK == 4, "the reverse step takes 2 or 4 nodes per thread");
constexpr int kPar = GR_COUNT + 1;  // per-block partial slots: 7 rate slots + D

struct Rec {
    float *x;   // 5 x npad FP32 values of X^k (recording target, or NULL)
    float *y2;  // npad transformed DOM of step k (recording target)
};

// Transformation-only pass that also records y2 = T(X)_2.
template <int PREC>
__global__ void __launch_bounds__(kThreads) k_transform_rec(int64_t n, StepParams p, StateIO io, float *rec_y2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    V x[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) x[c] = vload<PREC>(io.in[c], io.lin[c], i);
    transform_sync<PREC>(x[0], x[1], x[2], x[3], x[4], p);
#pragma unroll
    for (int c = 0; c < 5; ++c) vstore<PREC>(io.out[c], io.lout[c], i, x[c]);
    rec_y2[i] = __fadd_rn(x[1].h, x[1].l);
}

// Fused pass (diffuse, transform) that records X^{k} (after diffusion, before the transformation)
// and y2^k.  Same arithmetic as the forward fused pass, so the recomputed trajectory is identical.
template <int WM, int PREC>
__global__ void __launch_bounds__(kThreads) k_fused_rec(Topo t, const int32_t *__restrict__ chunk_row, int32_t cap,
                                                        StepParams p, BlockWeights bw, StateIO io, int64_t npad,
                                                        Rec rec) {
    extern __shared__ uint32_t smem[];
    int32_t *s_nb = reinterpret_cast<int32_t *>(smem + cap);
    int64_t v0;
    const int32_t nv = decode_chunk<WM == W_BLOCK>(t, chunk_row, cap, smem, s_nb, smem + 5 * cap, v0);
    const float *__restrict__ Y2 = io.in[1];
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
        V x2 = vload<PREC>(Y2, io.lin[1], i);
        const float yi = x2.h;
        float acc = 0.0f;
        for_each_neighbour(i, k, fl, s_nb, cap, [&](int slot, int64_t j) {
            const float d = __fsub_rn(yi, __ldg(Y2 + j));
            if (WM == W_UNIT) acc = __fadd_rn(acc, d);
            else acc = __fmaf_rn(edge_g(bw, i, slot, x, y, z), d, acc);
        });
        vadd<PREC>(x2, __fmul_rn(-p.c, acc));
        vround<PREC>(x2);
        V x1 = vload<PREC>(io.in[0], io.lin[0], i), x3 = vload<PREC>(io.in[2], io.lin[2], i),
          x4 = vload<PREC>(io.in[3], io.lin[3], i), x5 = vload<PREC>(io.in[4], io.lin[4], i);
        rec.x[i] = __fadd_rn(x1.h, x1.l);
        rec.x[npad + i] = __fadd_rn(x2.h, x2.l);
        rec.x[2 * npad + i] = __fadd_rn(x3.h, x3.l);
        rec.x[3 * npad + i] = __fadd_rn(x4.h, x4.l);
        rec.x[4 * npad + i] = __fadd_rn(x5.h, x5.l);
        transform_sync<PREC>(x1, x2, x3, x4, x5, p);
        vstore<PREC>(io.out[0], io.lout[0], i, x1);
        vstore<PREC>(io.out[1], io.lout[1], i, x2);
        vstore<PREC>(io.out[2], io.lout[2], i, x3);
        vstore<PREC>(io.out[3], io.lout[3], i, x4);
        vstore<PREC>(io.out[4], io.lout[4], i, x5);
        rec.y2[i] = __fadd_rn(x2.h, x2.l);
    }
}

// One reverse step.  lam (io.in) = dL/dX^{k+1}; writes dL/dX^k (io.out).  xk: recorded X^k values,
// y2k: recorded transformed DOM of step k.
template <int WM, int PREC>
__global__ void __launch_bounds__(kThreads) k_adjoint_step(Topo t, const int32_t *__restrict__ chunk_row, int32_t cap,
                                                           StepParams p, BlockWeights bw, StateIO io, int64_t npad,
                                                           const float *__restrict__ xk, const float *__restrict__ y2k,
                                                           double *__restrict__ gpart, double *__restrict__ gtheta) {
    extern __shared__ uint32_t smem[];
    int32_t *s_nb = reinterpret_cast<int32_t *>(smem + cap);
    int64_t v0;
    const int32_t nv = decode_chunk<WM == W_BLOCK>(t, chunk_row, cap, smem, s_nb, smem + 5 * cap, v0);
    const float *__restrict__ L2 = io.in[1];
    double acc[kPar];
#pragma unroll
    for (int q = 0; q < kPar; ++q) acc[q] = 0.0;
    const double mc = -(double)p.c;
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
        V mu[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) mu[c] = vload<PREC>(io.in[c], io.lin[c], i);
        const float li = mu[1].h;
        const float yi = __ldg(y2k + i);
        float lsum = 0.0f, ysum = 0.0f;
        for_each_neighbour(i, k, fl, s_nb, cap, [&](int slot, int64_t j) {
            const float g = (WM == W_UNIT) ? 1.0f : edge_g(bw, i, slot, x, y, z);
            const float dl = __fsub_rn(li, __ldg(L2 + j));
            const float dy = __fsub_rn(yi, __ldg(y2k + j));
            lsum = __fmaf_rn(g, dl, lsum);
            ysum = __fmaf_rn(g, dy, ysum);
            if (WM == W_BLOCK && (slot & 1)) {  // +x, +y, +z: each edge once
                const int64_t f = edge_face(bw, i, slot, x, y, z);
                if (f >= 0) atomicAdd(gtheta + f, mc * (double)dy * (double)dl);
            }
        });
        acc[GR_COUNT] -= (double)li * (double)ysum;  // times dt on the host: dL/dD
        vadd<PREC>(mu[1], __fmul_rn(-p.c, lsum));    // mu2 = Q_g lam2
        float xs[5];
#pragma unroll
        for (int c = 0; c < 5; ++c) xs[c] = __ldg(xk + c * npad + i);
        float gr[GR_COUNT];
#pragma unroll
        for (int q = 0; q < GR_COUNT; ++q) gr[q] = 0.0f;
        V lam[5];
        transform_sync_reverse<PREC>(xs, mu, lam, gr, p);
#pragma unroll
        for (int q = 0; q < GR_COUNT; ++q) acc[q] += (double)gr[q];
#pragma unroll
        for (int c = 0; c < 5; ++c) vstore<PREC>(io.out[c], io.lout[c], i, lam[c]);
    }
    __shared__ double out[kPar];
    block_sum_store<kPar>(acc, out);
    if (threadIdx.x < kPar) gpart[(int64_t)blockIdx.x * kPar + threadIdx.x] += out[threadIdx.x];
}

// Table-driven fused pass with recording: four nodes per thread (table_vec, the forward's own body, so the recomputed
// trajectory is the forward's bit for bit), recording X^k and y2^k as vectors.
template <int WM, int PREC, int TF>
__global__ void __launch_bounds__(kThreads) k_fused_rec_vec(int64_t n, NbrTable tb, BlockTable bt, StepParams p,
                                                            StateIO io, PassRecord rec) {
    const uint32_t i0 = 4u * ((uint32_t)blockIdx.x * blockDim.x + threadIdx.x);
    table_vec<1, WM, 0, PREC, TF, 4, true>(i0, (uint32_t)n, tb, bt, p, io, rec);
}

// Sparse fused pass with recording, first half: the forward's MODE 4 body (every node's DOM diffused,
// marked nodes left for the second half), writing h + l of every node's diffused DOM to rec.y2.  At
// an unmarked node the transformation is the identity, so that value is both X^k_2 and y2^k.
template <int WM, int PREC, int TF>
__global__ void __launch_bounds__(kThreads) k_dom_rec_vec(int64_t n, NbrTable tb, BlockTable bt, StepParams p,
                                                          StateIO io, PassRecord rec, SparseState ss) {
    const uint32_t i0 = 4u * ((uint32_t)blockIdx.x * blockDim.x + threadIdx.x);
    table_vec<4, WM, 0, PREC, TF, 4, true>(i0, (uint32_t)n, tb, bt, p, io, rec, ss);
}

// Second half: the marked nodes in rank order (k_transform_compact's arithmetic), recording their
// X^k (MB, DOM, SOM, FOM, FP32 h + l; xc row q at q * xcap) and overwriting y2^k with the
// transformed DOM.
template <int PREC>
__global__ void __launch_bounds__(kThreads) k_transform_compact_rec(int64_t m, SparseState ss, StepParams p,
                                                                    StateIO io, float *__restrict__ y2,
                                                                    float *__restrict__ xc, int64_t xcap) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    const uint32_t i = __ldg(ss.list + r);
    V x2;
    x2.h = io.out[1][i];
    x2.l = PREC == P_COMP ? res_decode(io.lout[1][i], x2.h) : 0.0f;
    V v[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[q].h = ss.h[q][r];
        v[q].l = PREC == P_COMP ? res_decode(ss.l[q][r], v[q].h) : 0.0f;
    }
    xc[r] = __fadd_rn(v[0].h, v[0].l);
    xc[xcap + r] = __fadd_rn(x2.h, x2.l);
    xc[2 * xcap + r] = __fadd_rn(v[1].h, v[1].l);
    xc[3 * xcap + r] = __fadd_rn(v[2].h, v[2].l);
    transform_sync<PREC>(v[0], x2, v[1], v[2], v[3], p);
#pragma unroll
    for (int q = 0; q < 4; ++q) vstore<PREC>(ss.h[q], ss.l[q], r, v[q]);
    vstore<PREC>(io.out[1], io.lout[1], i, x2);
    y2[i] = __fadd_rn(x2.h, x2.l);
}

// Compensated FP32 accumulator (TwoSum into a second float): GB300 issues FP64 at a small fraction of
// its FP32 rate, and a per-thread sum of ~100 terms carried this way keeps ~45 significant bits.
struct CAcc {
    float s = 0.0f, c = 0.0f;
};

__device__ __forceinline__ void cacc_add(CAcc &a, float x) {
    const float t = __fadd_rn(a.s, x);
    const float bp = __fsub_rn(t, a.s);
    const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
    a.s = t;
    a.c = __fadd_rn(a.c, err);
}

// x * y added exactly (TwoProd by FMA: the product's rounding error is a second float).
__device__ __forceinline__ void cacc_add_prod(CAcc &a, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float e = __fmaf_rn(x, y, -p);
    cacc_add(a, p);
    a.c = __fadd_rn(a.c, e);
}

// FP32 value as FP64, built with integer operations: exact for normal values, infinities and NaN;
// subnormal values (below 2^-126 in magnitude) become zeros of their sign.  The conversion
// instruction would issue on the FP64 pipe, which GB300 runs at a small fraction of its FP32 rate.
__device__ __forceinline__ double f32_to_f64_alu(float f) {
    const uint32_t u = __float_as_uint(f);
    const uint32_t e = (u >> 23) & 0xffu;
    const uint32_t sign = u & 0x80000000u;
    uint32_t hi = sign, lo = 0u;
    if (e != 0u) {
        const uint32_t ed = e == 0xffu ? 0x7ffu : e + 896u;  // rebias 127 -> 1023
        hi = sign | (ed << 20) | ((u & 0x7fffffu) >> 3);
        lo = u << 29;
    }
    return __hiloint2double((int)hi, (int)lo);
}

// Block sums of K compensated per-thread accumulators into out[0..K) (FP64, by thread 0 .. K-1): a
// warp butterfly of the (sum, error) pairs in FP32, merged by TwoSum at each level, then one FP64
// conversion per value and warp and the warps' sums in FP64.  The FP64 work is a few instructions
// per warp instead of five FP64 shuffle-adds per value and thread, which at one warp-group of nodes
// per thread (small graphs) cost more than the step itself.
template <int K>
__device__ __forceinline__ void block_sum_cacc(const CAcc (&a)[K], double *out) {
    __shared__ double sh[K][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    double mine = 0.0;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float s = a[k].s, c = a[k].c;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
            const float t = __fadd_rn(s, s2);
            const float bp = __fsub_rn(t, s);
            const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(s2, bp));
            s = t;
            c = __fadd_rn(__fadd_rn(c, c2), err);
        }
        if (lane == k) mine = (double)s + (double)c;  // every lane holds the warp's pair
    }
    if (lane < K) sh[lane][wid] = mine;
    __syncthreads();
    if (threadIdx.x < K) {
        double b = 0.0;
        for (int w = 0; w < nw; ++w) b += sh[threadIdx.x][w];
        out[threadIdx.x] = b;
    }
    __syncthreads();
}

// Adds v to gtheta[f] when f >= 0: one FP64 atomic per crossing edge.  At the porosities of the
// workloads a block face carries a few edges per step, spread over rows far apart in node order, so
// lanes of one warp rarely share a face and a warp-level pre-reduction would cost more instructions
// than it saves atomics.  The FP64 sums of FP32 terms are exact while the terms of a face span fewer
// than 29 binary orders, so the result does not depend on the atomics' order there.
__device__ __forceinline__ void face_atomic_add_f(double *gtheta, int32_t f, float v) {
    if (f >= 0) atomicAdd(gtheta + f, f32_to_f64_alu(v));
}

// Reverse step with four consecutive nodes per thread: the per-node streams (offset table, block
// ids, the five adjoint compartments, the recorded X^k and y2^k) move as 16-byte FP32 / table vectors
// and 8-byte residual vectors, so a warp issues a quarter of the memory instructions and address
// computations of the one-node kernel; the -x / +x neighbours of a group's end nodes come from the
// adjacent lanes.  Per node the arithmetic is k_adjoint_step's (same slot order, same operations),
// so dL/dX^k is the same bits; the per-thread gradient sums take the nodes in another order.
// The CO2 adjoint is read (respiration's weight) but not stored: no flux depends on CO2, so a step
// leaves it unchanged and the caller passes one buffer as its input and output.
// SP 0: X^k of every node from xk (rows of npad values).  SP 1 (sparse): X^k of the marked nodes of
// the activity mask `ss` from the compact record xk (rows of xcap values, in rank order); at an
// unmarked node MB, SOM and FOM are +0 and the DOM is y2^k (the transformation there is the
// identity), and the reverse transformation runs with those values and without the rate-gradient
// sums, whose terms are all products with MB, SOM, FOM or the mortality (zero there).  dL/dX^k and
// the gradients are the bits of SP 0.
template <int WM, int PREC, int TF, int SP, int SL>
__global__ void __launch_bounds__(kThreads, VGA_ADJ_MIN_BLOCKS) k_adjoint_vec(int64_t n, NbrTable tb, BlockTable bt, StepParams p,
                                                          StateIO io, int64_t npad, const float *__restrict__ xk,
                                                          const float *__restrict__ y2k, SparseState ss, int64_t xcap,
                                                          float *__restrict__ tacc, double *__restrict__ gpart,
                                                          double *__restrict__ gtheta) {
    constexpr int K = kAdjK;
    const float *__restrict__ L2 = io.in[1];
    // The thread's compensated partial sums.  SL 1 (graphs where a thread takes few groups per
    // launch): carried from launch to launch of one backward sweep in the thread's own slots of
    // tacc (value q: rows 2q, 2q + 1 of T = grid threads), reduced once after the sweep; otherwise
    // summed per block at the end of every launch into gpart.  The grid and the thread of each node
    // are fixed for a sweep, so either way the sums are the same bits on every run.
    const int64_t T = (int64_t)gridDim.x * blockDim.x, t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    CAcc acc[kPar];
    if (SL) {
#pragma unroll
        for (int q = 0; q < kPar; ++q) {
            acc[q].s = tacc[(2 * q) * T + t];
            acc[q].c = tacc[(2 * q + 1) * T + t];
        }
    }
    const float mc = -p.c;
    const uint32_t nn = (uint32_t)n;
    const int lane = threadIdx.x & 31;
    const int64_t nsup = (n + (int64_t)kThreads * K - 1) / ((int64_t)kThreads * K);
    for (int64_t sup = blockIdx.x; sup < nsup; sup += gridDim.x) {
        const uint32_t i0 = (uint32_t)(sup * kThreads * K + (int64_t)threadIdx.x * K);
        const bool full = i0 + K <= nn;
        uint32_t ty[K], zm[K], zp[K], bn[K];
        V l2[K], yv[K];
        if (full) {
            group_load<WM, PREC, TF, K, true>(i0, nn, tb, bt, io, ty, zm, zp, bn, l2);
            vload_k<P_F32, K, true>(y2k, nullptr, i0, nn, yv);
        } else {
            group_load<WM, PREC, TF, K, false>(i0, nn, tb, bt, io, ty, zm, zp, bn, l2);
            vload_k<P_F32, K, false>(y2k, nullptr, i0, nn, yv);
        }
        float li[K], yi[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            li[k] = l2[k].h;
            yi[k] = yv[k].h;
        }
        float ll = __shfl_up_sync(0xffffffffu, li[K - 1], 1), lr = __shfl_down_sync(0xffffffffu, li[0], 1);
        float yl = __shfl_up_sync(0xffffffffu, yi[K - 1], 1), yr = __shfl_down_sync(0xffffffffu, yi[0], 1);
        if (lane == 0 && ((ty[0] >> 15) & 1u)) {
            ll = __ldg(L2 + (i0 - 1));
            yl = __ldg(y2k + (i0 - 1));
        }
        if (lane == 31 && (ty[K - 1] >> 31)) {
            lr = __ldg(L2 + (i0 + K));
            yr = __ldg(y2k + (i0 + K));
        }
        float lsum[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const bool live = i0 + k < nn;
            const uint32_t dym = ty[k] & 0x7fffu, dyp = (ty[k] >> 16) & 0x7fffu;
            const uint32_t mask = live ? (((ty[k] >> 15) & 1u) | ((ty[k] >> 31) << 1) | ((uint32_t)(dym != 0) << 2) |
                                          ((uint32_t)(dyp != 0) << 3) | ((uint32_t)(zm[k] != 0) << 4) |
                                          ((uint32_t)(zp[k] != 0) << 5))
                                       : 0u;
            // an absent neighbour carries the node's own values: its terms are g * (+0), which leave
            // a sum that started at +0 unchanged (under round-to-nearest such a sum is never -0), so
            // every slot is visited without a branch and the sums are those of the existing edges
            float lv[6], yw[6];
            lv[0] = (mask & 1u) ? (k == 0 ? ll : li[k > 0 ? k - 1 : 0]) : li[k];
            yw[0] = (mask & 1u) ? (k == 0 ? yl : yi[k > 0 ? k - 1 : 0]) : yi[k];
            lv[1] = (mask & 2u) ? (k == K - 1 ? lr : li[k < K - 1 ? k + 1 : 0]) : li[k];
            yw[1] = (mask & 2u) ? (k == K - 1 ? yr : yi[k < K - 1 ? k + 1 : 0]) : yi[k];
            const uint32_t off[4] = {i0 + k - dym, i0 + k + dyp, i0 + k - zm[k], i0 + k + zp[k]};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const bool ex = (mask >> (q + 2)) & 1u;
                lv[q + 2] = ex ? __ldg(L2 + off[q]) : li[k];
                yw[q + 2] = ex ? __ldg(y2k + off[q]) : yi[k];
            }
            float ls = 0.0f, ys = 0.0f;
#pragma unroll
            for (int d = 0; d < 6; ++d) {
                const float g = (WM == W_UNIT) ? 1.0f : table_theta_sel(bt, bn[k], d);
                const float dl = __fsub_rn(li[k], lv[d]);
                const float dy = __fsub_rn(yi[k], yw[d]);
                ls = __fmaf_rn(g, dl, ls);
                ys = __fmaf_rn(g, dy, ys);
                if (WM == W_BLOCK && (d & 1))  // +x, +y, +z: each edge once
                    face_atomic_add_f(gtheta, table_face_sel(bt, bn[k], d, (mask >> d) & 1u),
                                      __fmul_rn(__fmul_rn(mc, dy), dl));
            }
            lsum[k] = ls;
            if (live) cacc_add_prod(acc[GR_COUNT], -li[k], ys);
        }
        if (i0 >= nn) continue;
        // the other compartments and the recorded X^k (MB, DOM, SOM, FOM: the reverse transformation
        // reads no CO2); the reverse transformation per node
        V m0[K], m2[K], m3[K], m4[K], x0[K], x1[K], x2v[K], x3[K];
        if (full) {
            vload_k<PREC, K, true>(io.in[0], io.lin[0], i0, nn, m0);
            vload_k<PREC, K, true>(io.in[2], io.lin[2], i0, nn, m2);
            vload_k<PREC, K, true>(io.in[3], io.lin[3], i0, nn, m3);
            vload_k<PREC, K, true>(io.in[4], io.lin[4], i0, nn, m4);
            if (SP == 0) {
                vload_k<P_F32, K, true>(xk, nullptr, i0, nn, x0);
                vload_k<P_F32, K, true>(xk + npad, nullptr, i0, nn, x1);
                vload_k<P_F32, K, true>(xk + 2 * npad, nullptr, i0, nn, x2v);
                vload_k<P_F32, K, true>(xk + 3 * npad, nullptr, i0, nn, x3);
            }
        } else {
            vload_k<PREC, K, false>(io.in[0], io.lin[0], i0, nn, m0);
            vload_k<PREC, K, false>(io.in[2], io.lin[2], i0, nn, m2);
            vload_k<PREC, K, false>(io.in[3], io.lin[3], i0, nn, m3);
            vload_k<PREC, K, false>(io.in[4], io.lin[4], i0, nn, m4);
            if (SP == 0) {
                vload_k<P_F32, K, false>(xk, nullptr, i0, nn, x0);
                vload_k<P_F32, K, false>(xk + npad, nullptr, i0, nn, x1);
                vload_k<P_F32, K, false>(xk + 2 * npad, nullptr, i0, nn, x2v);
                vload_k<P_F32, K, false>(xk + 3 * npad, nullptr, i0, nn, x3);
            }
        }
        uint32_t act = 0u, r0 = 0u;  // SP 1: activity bits of the group, rank of its first node
        if (SP == 1) {
            const uint32_t w = __ldg(ss.mask + (i0 >> 5));
            act = (w >> (i0 & 31u)) & ((1u << K) - 1u);
            if (act) r0 = __ldg(ss.prefix + (i0 >> 5)) + __popc(w & ((1u << (i0 & 31u)) - 1u));
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (i0 + k >= nn) continue;
            vadd<PREC>(l2[k], __fmul_rn(-p.c, lsum[k]));
            const V mu[5] = {m0[k], l2[k], m2[k], m3[k], m4[k]};
            V lam[5];
            if (SP == 0 || ((act >> k) & 1u)) {
                float xs[5];
                if (SP == 0) {
                    xs[0] = x0[k].h;
                    xs[1] = x1[k].h;
                    xs[2] = x2v[k].h;
                    xs[3] = x3[k].h;
                } else {
                    const uint32_t r = r0 + __popc(act & ((1u << k) - 1u));
                    xs[0] = __ldg(xk + r);
                    xs[1] = __ldg(xk + xcap + r);
                    xs[2] = __ldg(xk + 2 * xcap + r);
                    xs[3] = __ldg(xk + 3 * xcap + r);
                }
                xs[4] = 0.0f;
                float gr[GR_COUNT];
#pragma unroll
                for (int q = 0; q < GR_COUNT; ++q) gr[q] = 0.0f;
                transform_sync_reverse<PREC>(xs, mu, lam, gr, p);
#pragma unroll
                for (int q = 0; q < GR_COUNT; ++q) cacc_add(acc[q], gr[q]);
            } else {
                const float xs[5] = {0.0f, yi[k], 0.0f, 0.0f, 0.0f};
                float gr[GR_COUNT];  // every term is +-0 here; not accumulated
#pragma unroll
                for (int q = 0; q < GR_COUNT; ++q) gr[q] = 0.0f;
                transform_sync_reverse<PREC>(xs, mu, lam, gr, p);
            }
            m0[k] = lam[0];
            l2[k] = lam[1];
            m2[k] = lam[2];
            m3[k] = lam[3];
        }
        if (full) {
            vstore_k<PREC, K, true>(io.out[0], io.lout[0], i0, nn, m0);
            vstore_k<PREC, K, true>(io.out[1], io.lout[1], i0, nn, l2);
            vstore_k<PREC, K, true>(io.out[2], io.lout[2], i0, nn, m2);
            vstore_k<PREC, K, true>(io.out[3], io.lout[3], i0, nn, m3);
        } else {
            vstore_k<PREC, K, false>(io.out[0], io.lout[0], i0, nn, m0);
            vstore_k<PREC, K, false>(io.out[1], io.lout[1], i0, nn, l2);
            vstore_k<PREC, K, false>(io.out[2], io.lout[2], i0, nn, m2);
            vstore_k<PREC, K, false>(io.out[3], io.lout[3], i0, nn, m3);
        }
    }
    if (SL) {
#pragma unroll
        for (int q = 0; q < kPar; ++q) {
            tacc[(2 * q) * T + t] = acc[q].s;
            tacc[(2 * q + 1) * T + t] = acc[q].c;
        }
        return;
    }
    __shared__ double out[kPar];
    block_sum_cacc<kPar>(acc, out);
    if (threadIdx.x < kPar) gpart[(int64_t)blockIdx.x * kPar + threadIdx.x] += out[threadIdx.x];
}

// One reverse step on the offset table: compact z offsets or not, per-thread slots or per-launch
// block sums for the partials.
template <int WM, int PREC, int SP>
void launch_reverse(int G, cudaStream_t st, bool tz, bool slots, int64_t n, const NbrTable &tb, const BlockTable &bt,
                    const StepParams &p, const StateIO &io, int64_t npad, const float *xk, const float *y2k,
                    const SparseState &ss, int64_t xcap, float *tacc, double *gpart, double *gtheta) {
    if (tz) {
        if (slots) k_adjoint_vec<WM, PREC, 1, SP, 1><<<G, kThreads, 0, st>>>(n, tb, bt, p, io, npad, xk, y2k, ss, xcap, tacc, gpart, gtheta);
        else k_adjoint_vec<WM, PREC, 1, SP, 0><<<G, kThreads, 0, st>>>(n, tb, bt, p, io, npad, xk, y2k, ss, xcap, tacc, gpart, gtheta);
    } else {
        if (slots) k_adjoint_vec<WM, PREC, 0, SP, 1><<<G, kThreads, 0, st>>>(n, tb, bt, p, io, npad, xk, y2k, ss, xcap, tacc, gpart, gtheta);
        else k_adjoint_vec<WM, PREC, 0, SP, 0><<<G, kThreads, 0, st>>>(n, tb, bt, p, io, npad, xk, y2k, ss, xcap, tacc, gpart, gtheta);
    }
}

// After a backward sweep: the per-thread slots of the reverse steps' partial sums (grid G x kThreads)
// into per-block FP64 partials gpart[G x kPar] (the block sums of block_sum_cacc).
__global__ void __launch_bounds__(kThreads) k_reduce_tacc(const float *__restrict__ tacc, double *__restrict__ gpart) {
    const int64_t T = (int64_t)gridDim.x * blockDim.x, t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    CAcc acc[kPar];
#pragma unroll
    for (int q = 0; q < kPar; ++q) {
        acc[q].s = tacc[(2 * q) * T + t];
        acc[q].c = tacc[(2 * q + 1) * T + t];
    }
    __shared__ double out[kPar];
    block_sum_cacc<kPar>(acc, out);
    if (threadIdx.x < kPar) gpart[(int64_t)blockIdx.x * kPar + threadIdx.x] = out[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) k_reduce_gpart(const double *__restrict__ gpart, int G,
                                                           double *__restrict__ out) {
    double s[kPar];
#pragma unroll
    for (int q = 0; q < kPar; ++q) s[q] = 0.0;
    for (int b = threadIdx.x; b < G; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < kPar; ++q) s[q] += gpart[(int64_t)b * kPar + q];
    __shared__ double o[kPar];
    block_sum_store<kPar>(s, o);
    if (threadIdx.x < kPar) out[threadIdx.x] = o[threadIdx.x];
}

// ---- block-mass objective ----------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_block_mass(Topo t, const int32_t *__restrict__ chunk_row, int32_t cap,
                                                         BlockWeights bw, StateIO io, int comp_mask,
                                                         double *__restrict__ mass, int64_t nblocks) {
    extern __shared__ uint32_t smem[];
    int32_t *s_nb = reinterpret_cast<int32_t *>(smem + cap);
    int64_t v0;
    const int32_t nv = decode_chunk<true>(t, chunk_row, cap, smem, s_nb, smem + 5 * cap, v0);
    for (int32_t k = threadIdx.x; k < nv; k += blockDim.x) {
        const int64_t i = v0 + k;
        const int32_t x = (int32_t)(smem[k] & 0xffffu);
        const int32_t y = (int32_t)(smem[5 * cap + k] & 0xffffu), z = (int32_t)(smem[5 * cap + k] >> 16);
        const int64_t b = ((int64_t)(z / bw.bs) * bw.nby + y / bw.bs) * bw.nbx + x / bw.bs;
        int slot = 0;
        for (int c = 0; c < 5; ++c) {
            if (!((comp_mask >> c) & 1)) continue;
            const double v = (double)io.in[c][i] + (double)res_decode(io.lin[c][i], io.in[c][i]);
            atomicAdd(mass + slot * nblocks + b, v);
            ++slot;
        }
    }
}

// r = mass - target over all selected blocks; block partial sums of r^2
__global__ void __launch_bounds__(kThreads) k_block_resid(const double *__restrict__ mass, const double *__restrict__ target,
                                                          int64_t count, double *__restrict__ resid,
                                                          double *__restrict__ part) {
    double acc[1] = {0.0};
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += (int64_t)gridDim.x * blockDim.x) {
        const double r = mass[q] - target[q];
        resid[q] = r;
        acc[0] += r * r;
    }
    __shared__ double o[1];
    block_sum_store<1>(acc, o);
    if (threadIdx.x == 0) part[blockIdx.x] = o[0];
}

__global__ void __launch_bounds__(kThreads) k_sum_parts(const double *__restrict__ part, int count, double *out) {
    double acc[1] = {0.0};
    for (int q = threadIdx.x; q < count; q += blockDim.x) acc[0] += part[q];
    __shared__ double o[1];
    block_sum_store<1>(acc, o);
    if (threadIdx.x == 0) out[0] = o[0];
}

// dL/dX_c,i = 2 r_c,b(i) for the selected compartments, 0 for the others.
__global__ void __launch_bounds__(kThreads) k_block_mass_grad(Topo t, const int32_t *__restrict__ chunk_row,
                                                              int32_t cap, BlockWeights bw, int comp_mask,
                                                              const double *__restrict__ resid, int64_t nblocks,
                                                              double *__restrict__ dldx) {
    extern __shared__ uint32_t smem[];
    int32_t *s_nb = reinterpret_cast<int32_t *>(smem + cap);
    int64_t v0;
    const int32_t nv = decode_chunk<true>(t, chunk_row, cap, smem, s_nb, smem + 5 * cap, v0);
    const int64_t n = t.n;
    for (int32_t k = threadIdx.x; k < nv; k += blockDim.x) {
        const int64_t i = v0 + k;
        const int32_t x = (int32_t)(smem[k] & 0xffffu);
        const int32_t y = (int32_t)(smem[5 * cap + k] & 0xffffu), z = (int32_t)(smem[5 * cap + k] >> 16);
        const int64_t b = ((int64_t)(z / bw.bs) * bw.nby + y / bw.bs) * bw.nbx + x / bw.bs;
        int slot = 0;
        for (int c = 0; c < 5; ++c) {
            double g = 0.0;
            if ((comp_mask >> c) & 1) {
                g = 2.0 * resid[slot * nblocks + b];
                ++slot;
            }
            dldx[c * n + i] = g;
        }
    }
}

// FP64 (5 x n) -> compensated buffers with row stride npad.  The CO2 adjoint, which the reverse
// steps read but never store (no flux depends on CO2), is stored in the form that a load, a zero
// increment and a store leave unchanged: that cycle, applied until it changes nothing.  A cycle
// moves h only on a residual tie, after which h is even and the residual exact, so two cycles suffice
// and the third is a check.
__global__ void k_lam_in(int64_t n, const double *__restrict__ x, StateIO io) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const double v = x[c * n + i];
        float h = (float)v;
        res_t q = res_encode((float)(v - (double)h), h);
        if (c == 4) {
#pragma unroll 1
            for (int t = 0; t < 3; ++t) {
                V u = {h, res_decode(q, h)};
                vadd<P_COMP>(u, 0.0f);
                const float s = __fadd_rn(u.h, u.l);
                const float r = __fadd_rn(__fsub_rn(u.h, s), u.l);
                h = s;
                q = res_encode(r, s);
            }
        }
        io.out[c][i] = h;
        io.lout[c][i] = q;
    }
}

__global__ void k_lam_out(int64_t n, double *__restrict__ x, StateIO io) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int c = 0; c < 5; ++c) x[c * n + i] = (double)io.in[c][i] + (double)res_decode(io.lin[c][i], io.in[c][i]);
}

inline unsigned grid_for(int64_t count, int threads) { return (unsigned)((count + threads - 1) / threads); }

// Pair of FP32 + residual buffers for 5 compartments with row stride npad.
struct PairBuf {
    float *h = nullptr;
    res_t *l = nullptr;
};

StateIO io_from(PairBuf in, PairBuf out, int64_t npad) {
    StateIO io;
    for (int c = 0; c < 5; ++c) {
        io.in[c] = in.h + (size_t)c * npad;
        io.lin[c] = in.l + (size_t)c * npad;
        io.out[c] = out.h + (size_t)c * npad;
        io.lout[c] = out.l + (size_t)c * npad;
    }
    return io;
}

// The adjoint state lam[lb] -> lam[1 - lb], with the CO2 row of lam[0] as both input and output
// (the reverse steps leave it unchanged).
StateIO lam_io(const PairBuf *lam, int lb, int64_t npad) {
    StateIO io = io_from(lam[lb], lam[1 - lb], npad);
    io.in[4] = io.out[4] = lam[0].h + 4 * (size_t)npad;
    io.lin[4] = io.lout[4] = lam[0].l + 4 * (size_t)npad;
    return io;
}

}  // namespace

// Adjoint work buffers, owned by the simulation and kept between calls.
struct AdjointBuffers {
    int64_t npad = 0, nseg = 0, ckpt = 0, G = 0, ntheta = 0;
    // the forward pass the checkpoints belong to
    bool valid = false;
    bool last_recorded = false;  // the records hold the last segment (written by the forward sweep)
    bool grad_ready = false;     // gtheta holds the conductance gradient of a completed backward sweep
    int64_t N = 0, cur_ckpt = 0, param_gen = -1;
    char *ck = nullptr;    // nseg checkpoints, each 5*npad floats + 5*npad u16
    float *rec_x = nullptr;   // ckpt x 5 x npad (dense records, allocated when first used)
    int64_t rec_x_ckpt = 0;
    float *rec_y2 = nullptr;  // ckpt x npad
    // Sparse records: the activity mask of X^0 (the marked set never grows, so it covers every
    // step), and X^k of its marked nodes, ckpt x 4 x xcap (MB, DOM, SOM, FOM in rank order).
    bool sparse = false;
    Activity act;
    float *rec_xc = nullptr;
    int64_t rec_xc_count = 0, xcap = 1;
    PairBuf work[2];
    PairBuf lam[2];
    double *gpart = nullptr;  // G x kPar
    float *tacc = nullptr;    // per-thread partial sums of the table reverse steps: 2 kPar x (grid threads)
    int64_t tacc_count = 0;
    cudaStream_t cap_stream = nullptr;  // private stream the backward sweep's loops are captured on
    double *gtheta = nullptr; // ntheta
    double *gsum = nullptr;   // kPar
    double *lamstage = nullptr;  // 5 n FP64 (host-pointer staging)
};

void adjoint_free(AdjointBuffers *a) {
    if (!a) return;
    dfree(a->ck);
    dfree(a->rec_x);
    dfree(a->rec_y2);
    dfree(a->rec_xc);
    activity_free(&a->act);
    for (int b = 0; b < 2; ++b) {
        dfree(a->work[b].h);
        dfree(a->work[b].l);
        dfree(a->lam[b].h);
        dfree(a->lam[b].l);
    }
    dfree(a->gpart);
    dfree(a->tacc);
    if (a->cap_stream) cudaStreamDestroy(a->cap_stream);
    dfree(a->gtheta);
    dfree(a->gsum);
    dfree(a->lamstage);
    delete a;
}

static vga_status ensure_adjoint(vga_sim *s, int64_t nseg, int64_t ckpt) {
    AdjointBuffers *a = s->adj;
    const int64_t npad = s->npad, ntheta = std::max<int64_t>(s->n_theta, 1);
    const int64_t G = std::max<int64_t>(s->chunks.count, (s->n + kThreads - 1) / kThreads);
    if (a && a->npad == npad && a->nseg >= nseg && a->ckpt >= ckpt && a->G == G && a->ntheta >= ntheta) return VGA_OK;
    adjoint_free(a);
    s->adj = nullptr;
    a = new (std::nothrow) AdjointBuffers();
    if (!a) return fail(VGA_ERR_OOM, "host allocation of the adjoint buffers failed");
    s->adj = a;
    a->npad = npad;
    a->nseg = nseg;
    a->ckpt = ckpt;
    a->G = G;
    a->ntheta = ntheta;
    const size_t pairb = 5 * (size_t)npad * (sizeof(float) + sizeof(res_t));
    VGA_TRY(dmalloc((void **)&a->ck, pairb * (size_t)nseg, "adjoint checkpoints"));
    VGA_TRY(dmalloc((void **)&a->rec_y2, sizeof(float) * (size_t)npad * (size_t)ckpt, "adjoint records"));
    for (int b = 0; b < 2; ++b) {
        VGA_TRY(dmalloc((void **)&a->work[b].h, sizeof(float) * 5 * (size_t)npad, "adjoint work"));
        VGA_TRY(dmalloc((void **)&a->work[b].l, sizeof(res_t) * 5 * (size_t)npad, "adjoint work"));
        VGA_TRY(dmalloc((void **)&a->lam[b].h, sizeof(float) * 5 * (size_t)npad, "adjoint state"));
        VGA_TRY(dmalloc((void **)&a->lam[b].l, sizeof(res_t) * 5 * (size_t)npad, "adjoint state"));
    }
    VGA_TRY(dmalloc((void **)&a->gpart, sizeof(double) * kPar * (size_t)std::max<int64_t>(G, 1), "gradient partials"));
    VGA_TRY(dmalloc((void **)&a->gtheta, sizeof(double) * (size_t)ntheta, "theta gradient"));
    VGA_TRY(dmalloc((void **)&a->gsum, sizeof(double) * kPar, "gradient sums"));
    return VGA_OK;
}

// Records of X^k for the current mode: every node (dense) or the marked nodes (sparse).
static vga_status ensure_records(AdjointBuffers *a) {
    if (a->sparse) {
        const int64_t count = 4 * a->xcap * a->ckpt;
        if (a->rec_xc && a->rec_xc_count >= count) return VGA_OK;
        dfree(a->rec_xc);
        a->rec_xc = nullptr;
        a->rec_xc_count = 0;
        VGA_TRY(dmalloc((void **)&a->rec_xc, sizeof(float) * (size_t)count, "adjoint records"));
        a->rec_xc_count = count;
        return VGA_OK;
    }
    if (a->rec_x && a->rec_x_ckpt >= a->ckpt) return VGA_OK;
    dfree(a->rec_x);
    a->rec_x = nullptr;
    a->rec_x_ckpt = 0;
    VGA_TRY(dmalloc((void **)&a->rec_x, sizeof(float) * 5 * (size_t)a->npad * (size_t)a->ckpt, "adjoint records"));
    a->rec_x_ckpt = a->ckpt;
    return VGA_OK;
}

static PairBuf ck_slot(AdjointBuffers *a, int64_t s) {
    const size_t pairb = 5 * (size_t)a->npad * (sizeof(float) + sizeof(res_t));
    PairBuf p;
    p.h = reinterpret_cast<float *>(a->ck + pairb * (size_t)s);
    p.l = reinterpret_cast<res_t *>(a->ck + pairb * (size_t)s + 5 * (size_t)a->npad * sizeof(float));
    return p;
}

// Copies the simulation's current state into a pair buffer (or back).
static vga_status copy_state(vga_sim *s, PairBuf p, bool to_sim) {
    for (int c = 0; c < 5; ++c) {
        float *h = p.h + (size_t)c * s->npad;
        res_t *l = p.l + (size_t)c * s->npad;
        if (to_sim) {
            VGA_CUDA(cudaMemcpyAsync(s->comp(c), h, sizeof(float) * (size_t)s->n, cudaMemcpyDeviceToDevice, s->stream));
            VGA_CUDA(cudaMemcpyAsync(s->lcomp(c), l, sizeof(res_t) * (size_t)s->n, cudaMemcpyDeviceToDevice,
                                     s->stream));
        } else {
            VGA_CUDA(cudaMemcpyAsync(h, s->comp(c), sizeof(float) * (size_t)s->n, cudaMemcpyDeviceToDevice, s->stream));
            VGA_CUDA(cudaMemcpyAsync(l, s->lcomp(c), sizeof(res_t) * (size_t)s->n, cudaMemcpyDeviceToDevice,
                                     s->stream));
        }
    }
    return VGA_OK;
}

// The steps of the last segment in the forward sweep, written as the backward sweep's
// recomputation would write them: the same passes as sim_step_explicit (transformation pass, fused
// passes on the four-node body, diffusion-only pass) with the records of X^k and y2^k, so the
// backward sweep need not recompute that segment.  Needs the neighbour-offset table.
template <int WM>
static vga_status forward_recording(vga_sim *s, AdjointBuffers *a, int64_t len) {
    constexpr int PREC = P_COMP;
    const int64_t npad = s->npad;
    NbrTable tb;
    BlockTable bt;
    bool ok = true;
    VGA_TRY(sim_nbr_table(s, &tb));
    if (WM == W_BLOCK) VGA_TRY(sim_block_table(s, &bt, &ok));
    if (!ok) return VGA_ERR_UNSUPPORTED;  // the caller falls back to the plain forward
    VGA_TRY(ensure_records(a));
    cudaStream_t st = s->stream;
    const int Gv = (int)(((s->n + 3) / 4 + kThreads - 1) / kThreads);
    timing_begin(s, VGA_KERNEL_TRANSFORM);
    k_transform_rec<PREC><<<grid_for(s->n, kThreads), kThreads, 0, st>>>(s->n, s->sp, state_io(s), a->rec_y2);
    timing_end(s);
    VGA_CHECK_LAUNCH();
    ++s->launches;
    for (int c = 0; c < 5; ++c) s->cur[c] ^= 1;
    if (a->sparse) {
        // the sparse fused passes: the marked nodes' MB, SOM, FOM, CO2 in the compact state, the
        // DOM rows alternating; MB, SOM, FOM, CO2 stay in the current rows (zero at the unmarked nodes)
        const SparseState ss = activity_state(a->act);
        const int64_t m = a->act.n_active;
        if (m > 0) VGA_TRY(activity_copy(a->act, s->n, state_io_inplace(s), true, true, st));
        for (int64_t j = 1; j < len; ++j) {
            const PassRecord pr = {nullptr, a->rec_y2 + (size_t)j * npad, npad};
            const StateIO io = state_io(s);
            timing_begin(s, VGA_KERNEL_FUSED_STEP);
            if (tb.tz) k_dom_rec_vec<WM, PREC, 1><<<Gv, kThreads, 0, st>>>(s->n, tb, bt, s->sp, io, pr, ss);
            else k_dom_rec_vec<WM, PREC, 0><<<Gv, kThreads, 0, st>>>(s->n, tb, bt, s->sp, io, pr, ss);
            if (m > 0)
                k_transform_compact_rec<PREC><<<grid_for(m, kThreads), kThreads, 0, st>>>(
                    m, ss, s->sp, io, pr.y2, a->rec_xc + (size_t)j * 4 * a->xcap, a->xcap);
            timing_end(s);
            VGA_CHECK_LAUNCH();
            s->launches += m > 0 ? 2 : 1;
            s->cur[1] ^= 1;
        }
        if (m > 0) VGA_TRY(activity_copy(a->act, s->n, state_io_inplace(s), false, true, st));
        s->launches += m > 0 ? 2 : 0;
    } else {
        for (int64_t j = 1; j < len; ++j) {
            const PassRecord pr = {a->rec_x + (size_t)j * 5 * npad, a->rec_y2 + (size_t)j * npad, npad};
            timing_begin(s, VGA_KERNEL_FUSED_STEP);
            if (tb.tz) k_fused_rec_vec<WM, PREC, 1><<<Gv, kThreads, 0, st>>>(s->n, tb, bt, s->sp, state_io(s), pr);
            else k_fused_rec_vec<WM, PREC, 0><<<Gv, kThreads, 0, st>>>(s->n, tb, bt, s->sp, state_io(s), pr);
            timing_end(s);
            VGA_CHECK_LAUNCH();
            ++s->launches;
            for (int c = 0; c < 5; ++c) s->cur[c] ^= 1;
        }
    }
    VGA_TRY(sim_diffuse_pass(s));
    s->steps_done += len;
    return VGA_OK;
}

vga_status sim_adjoint_forward(vga_sim *s, int64_t N, int64_t ckpt) {
    const int64_t nseg = N > 0 ? (N + ckpt - 1) / ckpt : 0;
    VGA_TRY(ensure_adjoint(s, std::max<int64_t>(nseg, 1), ckpt));
    AdjointBuffers *a = s->adj;
    a->valid = false;
    a->last_recorded = false;
    a->grad_ready = false;
    // sparse records and reverse steps: the activity mask of X^0 on the neighbour-offset table
    a->sparse = false;
    if (s->activity_skip && s->g->nx <= 32767 && s->n > 0) {
        bool ok = true;
        if (s->wmode == W_BLOCK) {
            BlockTable bt;
            VGA_TRY(sim_block_table(s, &bt, &ok));
        }
        if (ok) {
            // the current rows as the "spare" too: the zeros it writes at unmarked nodes are there already
            VGA_TRY(activity_build(&a->act, s->n, s->npad, state_io_inplace(s), state_io_inplace(s), true, s->stream));
            s->launches += 2;
            a->sparse = true;
            a->xcap = std::max<int64_t>(a->act.n_active, 1);
        }
    }
    for (int64_t sg = 0; sg < nseg; ++sg) {
        VGA_TRY(copy_state(s, ck_slot(a, sg), false));
        const int64_t len = std::min(ckpt, N - sg * ckpt);
        if (sg == nseg - 1 && s->g->nx <= 32767) {
            const vga_status r = s->wmode == W_BLOCK ? forward_recording<W_BLOCK>(s, a, len)
                                                     : forward_recording<W_UNIT>(s, a, len);
            if (r == VGA_OK) {
                a->last_recorded = true;
                continue;
            }
            if (r != VGA_ERR_UNSUPPORTED) return r;
        }
        VGA_TRY(sim_step_explicit(s, len));
    }
    a->N = N;
    a->cur_ckpt = ckpt;
    a->param_gen = s->param_gen;
    a->valid = true;
    return VGA_OK;
}

// The loops of a backward sweep (recording passes, reverse steps) repeat with the same kernels and
// arguments for every segment of one length: each is captured once per sweep as a CUDA graph, on a
// private stream (the simulation's may be the legacy default stream, which cannot be captured), and
// replayed on the simulation's stream.  Kernel timing and a failed capture run the loops directly.
struct SweepGraphs {
    cudaStream_t st = nullptr, cap = nullptr;
    bool on = false;
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    int64_t key[2] = {-1, -1};
    ~SweepGraphs() {
        for (auto &e : exec)
            if (e) cudaGraphExecDestroy(e);
    }
    template <class F>
    vga_status run(int slot, int64_t k, F &&issue) {
        if (!on) return issue(st);
        if (!exec[slot] || key[slot] != k) {
            if (exec[slot]) cudaGraphExecDestroy(exec[slot]);
            exec[slot] = nullptr;
            key[slot] = -1;
            VGA_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
            const vga_status r = issue(cap);
            cudaGraph_t g = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(cap, &g);
            cudaError_t ei = cudaErrorUnknown;
            if (r == VGA_OK && ec == cudaSuccess) ei = cudaGraphInstantiate(&exec[slot], g, 0);
            if (g) cudaGraphDestroy(g);
            if (r != VGA_OK) return r;
            if (ec != cudaSuccess || ei != cudaSuccess) {  // run the loops directly from now on
                cudaGetLastError();
                exec[slot] = nullptr;
                on = false;
                return issue(st);
            }
            key[slot] = k;
        }
        VGA_CUDA(cudaGraphLaunch(exec[slot], st));
        return VGA_OK;
    }
};

template <int WM>
static vga_status adjoint_backward_impl(vga_sim *s, const double *d_lamN, double *d_lam0, double *grad8,
                                        double *h_gtheta) {
    constexpr int PREC = P_COMP;
    AdjointBuffers *a = s->adj;
    const int64_t N = a->N, ckpt = a->cur_ckpt;
    const int64_t nseg = N > 0 ? (N + ckpt - 1) / ckpt : 0;
    const Topo t = s->g->topo();
    NbrTable tb;
    BlockTable bt;
    bool table = s->g->nx <= 32767;
    if (table) VGA_TRY(sim_nbr_table(s, &tb));
    if (table && WM == W_BLOCK) VGA_TRY(sim_block_table(s, &bt, &table));
    // grid of the table kernels: the blocks that fit on the GPU at once (grid-stride over groups of
    // kThreads x 4 nodes), so every thread's FP64 partial-sum tail is paid once per launch
    int Gt = 1;
    if (table) {
        int dev = 0, sms = 0, occ0 = 0, occ1 = 0;
        VGA_CUDA(cudaGetDevice(&dev));
        VGA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (tb.tz) {
            VGA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ0, k_adjoint_vec<WM, PREC, 1, 0, 0>, kThreads, 0));
            VGA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, k_adjoint_vec<WM, PREC, 1, 1, 0>, kThreads, 0));
        } else {
            VGA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ0, k_adjoint_vec<WM, PREC, 0, 0, 0>, kThreads, 0));
            VGA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, k_adjoint_vec<WM, PREC, 0, 1, 0>, kThreads, 0));
        }
        const int64_t groups = (s->n + kAdjK * kThreads - 1) / (kAdjK * kThreads);
        Gt = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::max(1, std::min(occ0, occ1)) * sms, groups));
    }
    const int Gv = (int)(((s->n + 3) / 4 + kThreads - 1) / kThreads);  // four nodes per thread
    const int G = table ? Gt : s->chunks.count;  // blocks writing gradient partials
    const size_t smem = sizeof(uint32_t) * (size_t)s->chunks.cap * decode_words(WM == W_BLOCK);
    const int64_t npad = s->npad;
    cudaStream_t st = s->stream;

    SweepGraphs graphs;
    graphs.st = st;
    graphs.on = table && !s->timing;
    if (graphs.on && !a->cap_stream && cudaStreamCreateWithFlags(&a->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        a->cap_stream = nullptr;
    }
    graphs.cap = a->cap_stream;
    graphs.on = graphs.on && graphs.cap;
    const bool sparse = a->sparse && table;
    const SparseState ss = sparse ? activity_state(a->act) : SparseState{};
    const int64_t m = sparse ? a->act.n_active : 0;
    if (a->sparse && !sparse) {  // (not reached: the forward sweep checked the same tables) dense form
        a->sparse = false;
        a->last_recorded = false;
    }
    VGA_TRY(ensure_records(a));
    k_lam_in<<<grid_for(s->n, kThreads), kThreads, 0, st>>>(s->n, d_lamN, io_from(a->lam[0], a->lam[0], npad));
    VGA_CHECK_LAUNCH();
    VGA_CUDA(cudaMemsetAsync(a->gpart, 0, sizeof(double) * kPar * (size_t)std::max(G, 1), st));
    // per-thread slots when a thread takes at most kSlotGroups groups of nodes per reverse launch
    const int64_t groups_per_thread = table ? ((s->n + kAdjK * kThreads - 1) / (kAdjK * kThreads) + Gt - 1) / Gt : 0;
    float *tacc = nullptr;
    if (table && groups_per_thread <= kSlotGroups) {  // zeroed for this sweep
        const int64_t count = 2 * kPar * (int64_t)Gt * kThreads;
        if (a->tacc_count < count) {
            dfree(a->tacc);
            a->tacc = nullptr;
            a->tacc_count = 0;
            VGA_TRY(dmalloc((void **)&a->tacc, sizeof(float) * (size_t)count, "gradient partials"));
            a->tacc_count = count;
        }
        VGA_CUDA(cudaMemsetAsync(a->tacc, 0, sizeof(float) * (size_t)count, st));
        tacc = a->tacc;
    }
    VGA_CUDA(cudaMemsetAsync(a->gtheta, 0, sizeof(double) * (size_t)a->ntheta, st));
    int lb = 0;
    for (int64_t sg = nseg - 1; sg >= 0; --sg) {
        const int64_t len = std::min(ckpt, N - sg * ckpt);
        // recompute the segment, recording X^k and y2^k for k = 0 .. len-1 (relative to its start),
        // unless the forward sweep recorded it (the last segment)
        PairBuf cks = ck_slot(a, sg);
        Rec rec;
        const bool recorded = sg == nseg - 1 && a->last_recorded;
        if (!recorded) {
            timing_begin(s, VGA_KERNEL_TRANSFORM);
            k_transform_rec<PREC><<<grid_for(s->n, kThreads), kThreads, 0, st>>>(s->n, s->sp, io_from(cks, a->work[0], npad),
                                                                                a->rec_y2);
            timing_end(s);
            VGA_CHECK_LAUNCH();
            ++s->launches;
            int wb = 0;
            if (sparse && m > 0) {
                VGA_TRY(activity_copy(a->act, s->n, io_from(a->work[0], a->work[0], npad), true, true, st));
                ++s->launches;
            }
            if (sparse) {  // the recording passes j = 1 .. len-1: one graph per sweep and segment length
                auto issue = [&](cudaStream_t cs) -> vga_status {
                    int w = 0;
                    for (int64_t j = 1; j < len; ++j) {
                        const PassRecord pr = {nullptr, a->rec_y2 + (size_t)j * npad, npad};
                        const StateIO io = io_from(a->work[w], a->work[1 - w], npad);
                        timing_begin(s, VGA_KERNEL_FUSED_STEP);
                        if (tb.tz) k_dom_rec_vec<WM, PREC, 1><<<Gv, kThreads, 0, cs>>>(s->n, tb, bt, s->sp, io, pr, ss);
                        else k_dom_rec_vec<WM, PREC, 0><<<Gv, kThreads, 0, cs>>>(s->n, tb, bt, s->sp, io, pr, ss);
                        if (m > 0)
                            k_transform_compact_rec<PREC><<<grid_for(m, kThreads), kThreads, 0, cs>>>(
                                m, ss, s->sp, io, pr.y2, a->rec_xc + (size_t)j * 4 * a->xcap, a->xcap);
                        timing_end(s);
                        VGA_CHECK_LAUNCH();
                        w = 1 - w;
                    }
                    return VGA_OK;
                };
                VGA_TRY(graphs.run(0, len, issue));
                s->launches += (len - 1) * (m > 0 ? 2 : 1);
            }
            for (int64_t j = 1; j < len && !sparse; ++j) {
                rec.x = a->rec_x + (size_t)j * 5 * npad;
                rec.y2 = a->rec_y2 + (size_t)j * npad;
                timing_begin(s, VGA_KERNEL_FUSED_STEP);
                if (table) {
                    const PassRecord pr = {rec.x, rec.y2, npad};
                    const StateIO io = io_from(a->work[wb], a->work[1 - wb], npad);
                    if (tb.tz) k_fused_rec_vec<WM, PREC, 1><<<Gv, kThreads, 0, st>>>(s->n, tb, bt, s->sp, io, pr);
                    else k_fused_rec_vec<WM, PREC, 0><<<Gv, kThreads, 0, st>>>(s->n, tb, bt, s->sp, io, pr);
                } else
                    k_fused_rec<WM, PREC><<<G, kThreads, smem, st>>>(t, s->chunks.row, s->chunks.cap, s->sp, s->bw,
                                                                    io_from(a->work[wb], a->work[1 - wb], npad), npad, rec);
                timing_end(s);
                VGA_CHECK_LAUNCH();
                ++s->launches;
                wb = 1 - wb;
            }
        }
        // reverse: steps len-1 .. 1 (on the table: one graph per sweep, segment length and parity of
        // the adjoint buffers), then step 0, whose X^0 is the segment's checkpoint
        if (table) {
            const int lb0 = lb;
            auto issue = [&](cudaStream_t cs) -> vga_status {
                int l = lb0;
                for (int64_t j = len - 1; j >= 1; --j) {
                    const float *xk = sparse ? a->rec_xc + (size_t)j * 4 * a->xcap : a->rec_x + (size_t)j * 5 * npad;
                    const float *y2k = a->rec_y2 + (size_t)j * npad;
                    const StateIO io = lam_io(a->lam, l, npad);
                    timing_begin(s, VGA_KERNEL_ADJOINT);
                    if (sparse)
                        launch_reverse<WM, PREC, 1>(G, cs, tb.tz != nullptr, tacc != nullptr, s->n, tb, bt, s->sp, io,
                                                    npad, xk, y2k, ss, a->xcap, tacc, a->gpart, a->gtheta);
                    else
                        launch_reverse<WM, PREC, 0>(G, cs, tb.tz != nullptr, tacc != nullptr, s->n, tb, bt, s->sp, io,
                                                    npad, xk, y2k, SparseState{}, 1, tacc, a->gpart, a->gtheta);
                    timing_end(s);
                    VGA_CHECK_LAUNCH();
                    l = 1 - l;
                }
                return VGA_OK;
            };
            VGA_TRY(graphs.run(1, 2 * len + lb0, issue));
            s->launches += len - 1;
            lb = (int)(lb0 ^ ((len - 1) & 1));
            const StateIO io = lam_io(a->lam, lb, npad);
            timing_begin(s, VGA_KERNEL_ADJOINT);
            launch_reverse<WM, PREC, 0>(G, st, tb.tz != nullptr, tacc != nullptr, s->n, tb, bt, s->sp, io, npad, cks.h,
                                        a->rec_y2, SparseState{}, 1, tacc, a->gpart, a->gtheta);
            timing_end(s);
            VGA_CHECK_LAUNCH();
            ++s->launches;
            lb = 1 - lb;
        } else {
            for (int64_t j = len - 1; j >= 0; --j) {
                const float *xk = (j == 0) ? cks.h : a->rec_x + (size_t)j * 5 * npad;
                const float *y2k = a->rec_y2 + (size_t)j * npad;
                const StateIO io = lam_io(a->lam, lb, npad);
                timing_begin(s, VGA_KERNEL_ADJOINT);
                k_adjoint_step<WM, PREC><<<G, kThreads, smem, st>>>(t, s->chunks.row, s->chunks.cap, s->sp, s->bw, io,
                                                                   npad, xk, y2k, a->gpart, a->gtheta);
                timing_end(s);
                VGA_CHECK_LAUNCH();
                ++s->launches;
                lb = 1 - lb;
            }
        }
    }
    if (nseg > 1) a->last_recorded = false;  // the records now hold the first segment
    if (d_lam0) {
        StateIO io = io_from(a->lam[lb], a->lam[lb], npad);  // CO2 from lam[0]
        io.in[4] = a->lam[0].h + 4 * (size_t)npad;
        io.lin[4] = a->lam[0].l + 4 * (size_t)npad;
        k_lam_out<<<grid_for(s->n, kThreads), kThreads, 0, st>>>(s->n, d_lam0, io);
        VGA_CHECK_LAUNCH();
    }
    if (tacc) {
        k_reduce_tacc<<<Gt, kThreads, 0, st>>>(tacc, a->gpart);
        ++s->launches;
    }
    k_reduce_gpart<<<1, kThreads, 0, st>>>(a->gpart, G, a->gsum);
    VGA_CHECK_LAUNCH();
    s->launches += 2;
    double h[kPar];
    VGA_CUDA(cudaMemcpyAsync(h, a->gsum, sizeof(double) * kPar, cudaMemcpyDeviceToHost, st));
    if (s->face_mode) VGA_TRY(sim_face_mirror(s, a->gtheta));  // both slots of every edge
    if (h_gtheta && s->n_theta > 0 && s->wmode == W_BLOCK)
        VGA_CUDA(cudaMemcpyAsync(h_gtheta, a->gtheta, sizeof(double) * (size_t)s->n_theta, cudaMemcpyDeviceToHost, st));
    VGA_CUDA(cudaStreamSynchronize(st));
    a->grad_ready = s->wmode == W_BLOCK && s->n_theta > 0;
    const double dt = s->params.dt;
    // order: D, rho, mu, beta, v_som, v_fom, v_dom, K_dom
    grad8[0] = h[GR_COUNT] * dt;
    grad8[1] = h[GR_R] * dt;
    grad8[2] = h[GR_M] * dt;
    grad8[3] = h[GR_BETA];
    grad8[4] = h[GR_S] * dt;
    grad8[5] = h[GR_F] * dt;
    grad8[6] = h[GR_A] * dt;
    grad8[7] = h[GR_K];
    return VGA_OK;
}

vga_status sim_adjoint_grad_theta(vga_sim *s, double *out, bool on_device, int64_t n) {
    AdjointBuffers *a = s->adj;
    if (!a || !a->valid || !a->grad_ready)
        return fail(VGA_ERR_INVALID_ARG, "no conductance gradient: run vga_adjoint_backward with conductances set");
    if (n != s->n_theta) return fail(VGA_ERR_INVALID_ARG, "n must be the number of conductances");
    VGA_CUDA(cudaMemcpyAsync(out, a->gtheta, sizeof(double) * (size_t)n,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->stream));
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    return VGA_OK;
}

vga_status sim_adjoint_backward(vga_sim *s, const double *d_lamN, double *d_lam0, double *grad8, double *h_gtheta) {
    if (!s->adj || !s->adj->valid) return fail(VGA_ERR_INVALID_ARG, "no adjoint forward pass to reverse");
    if (s->adj->param_gen != s->param_gen)
        return fail(VGA_ERR_INVALID_ARG, "parameters or conductances changed since the adjoint forward pass");
    if (s->wmode == W_BLOCK) return adjoint_backward_impl<W_BLOCK>(s, d_lamN, d_lam0, grad8, h_gtheta);
    return adjoint_backward_impl<W_UNIT>(s, d_lamN, d_lam0, grad8, h_gtheta);
}

// Block masses of the selected compartments, the objective L = sum (mass - target)^2 and, if
// d_dldx != NULL, dL/dX (5 x n FP64, device).  d_work: 2*count + 64 doubles of device scratch.
vga_status sim_block_mass_loss(vga_sim *s, int32_t bs, uint32_t comp_mask, const double *d_target, double *d_work,
                               double *h_loss, double *h_mass, double *d_dldx) {
    const vga_graph *g = s->g;
    BlockWeights bw;
    bw.bs = bs;
    bw.nbx = (g->nx + bs - 1) / bs;
    bw.nby = (g->ny + bs - 1) / bs;
    bw.nbz = (g->nz + bs - 1) / bs;
    const int64_t nblocks = (int64_t)bw.nbx * bw.nby * bw.nbz;
    int nsel = 0;
    for (int c = 0; c < 5; ++c) nsel += (comp_mask >> c) & 1;
    const int64_t count = nsel * nblocks;
    double *mass = d_work, *resid = d_work + count, *part = d_work + 2 * count;
    const Topo t = g->topo();
    const size_t smem = sizeof(uint32_t) * (size_t)s->chunks.cap * decode_words(true);
    cudaStream_t st = s->stream;
    VGA_CUDA(cudaMemsetAsync(mass, 0, sizeof(double) * (size_t)count, st));
    if (s->n > 0) {
        k_block_mass<<<s->chunks.count, kThreads, smem, st>>>(t, s->chunks.row, s->chunks.cap, bw, state_io_inplace(s),
                                                            (int)comp_mask, mass, nblocks);
        VGA_CHECK_LAUNCH();
    }
    const int rb = (int)std::min<int64_t>(32, std::max<int64_t>(1, (count + kThreads - 1) / kThreads));
    k_block_resid<<<rb, kThreads, 0, st>>>(mass, d_target, count, resid, part);
    k_sum_parts<<<1, kThreads, 0, st>>>(part, rb, part + 32);
    VGA_CHECK_LAUNCH();
    s->launches += 3;
    if (d_dldx && s->n > 0) {
        k_block_mass_grad<<<s->chunks.count, kThreads, smem, st>>>(t, s->chunks.row, s->chunks.cap, bw, (int)comp_mask,
                                                                 resid, nblocks, d_dldx);
        VGA_CHECK_LAUNCH();
        ++s->launches;
    }
    VGA_CUDA(cudaMemcpyAsync(h_loss, part + 32, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (h_mass) VGA_CUDA(cudaMemcpyAsync(h_mass, mass, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, st));
    VGA_CUDA(cudaStreamSynchronize(st));
    return VGA_OK;
}

// Normalised (element-wise sign) gradient step on the block conductances, Sec. V.A:
// theta <- clamp(theta - lr * g / |g|, lo, hi), with g / |g| = 0 where g = 0.
__global__ void k_sgd_sign(int64_t n, float *__restrict__ theta, const double *__restrict__ g, double lr, double lo,
                           double hi) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double gk = g[k];
    const double sgn = gk > 0.0 ? 1.0 : (gk < 0.0 ? -1.0 : 0.0);
    double t = (double)theta[k] - lr * sgn;
    t = t < lo ? lo : (t > hi ? hi : t);
    theta[k] = (float)t;
}

vga_status sim_sgd_theta(vga_sim *s, double lr, double lo, double hi) {
    if (!s->adj || !s->adj->valid) return fail(VGA_ERR_INVALID_ARG, "no adjoint gradient to step along");
    if (s->wmode != W_BLOCK || s->n_theta == 0) return fail(VGA_ERR_INVALID_ARG, "no block conductances set");
    if (s->face_mode) return fail(VGA_ERR_UNSUPPORTED, "the sign-SGD update covers block conductances");
    k_sgd_sign<<<(unsigned)((s->n_theta + 255) / 256), 256, 0, s->stream>>>(s->n_theta, s->theta, s->adj->gtheta, lr, lo,
                                                                          hi);
    VGA_CHECK_LAUNCH();
    ++s->launches;
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    return VGA_OK;
}

}  // namespace vga
