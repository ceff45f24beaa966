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
// The stencil kernel works on chunks of `cap` consecutive nodes; decode_chunk() (stencil.cuh)
// turns the row bitmask into per-node neighbour indices in shared memory, so no per-node
// neighbour table is read from memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>

#include "physics.cuh"
#include "stencil.cuh"
#include "tma.cuh"
#include "vga_internal.cuh"

namespace vga {

namespace {

constexpr int kThreads = 256;
constexpr int kTotBlocks = 1024;

template <int TR, int PREC>
__global__ void __launch_bounds__(kThreads) k_transform(int64_t n, StepParams p, StateIO io) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    V x[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) x[c] = vload<PREC>(io.in[c], io.lin[c], i);
    transform_n<TR, PREC>(x[0], x[1], x[2], x[3], x[4], p);
#pragma unroll
    for (int c = 0; c < 5; ++c) vstore<PREC>(io.out[c], io.lout[c], i, x[c]);
}

// MODE 1: fused (diffuse the stored transformed DOM, then transform the result).
// MODE 2: diffusion only (writes DOM).
template <int MODE, int WM, int TR, int PREC>
__global__ void __launch_bounds__(kThreads) k_stencil(Topo t, const int32_t *__restrict__ chunk_row, int32_t cap,
                                                      StepParams p, BlockWeights bw, StateIO io) {
    extern __shared__ uint32_t smem[];
    uint32_t *s_info = smem;
    int32_t *s_nb = reinterpret_cast<int32_t *>(smem + cap);
    uint32_t *s_yz = smem + 5 * cap;
    int64_t v0;
    const int32_t nv = decode_chunk<WM == W_BLOCK>(t, chunk_row, cap, s_info, s_nb, s_yz, v0);

    const float *__restrict__ Y2 = io.in[1];
    for (int32_t k = threadIdx.x; k < nv; k += blockDim.x) {
        const int64_t i = v0 + k;
        const uint32_t info = s_info[k];
        const uint32_t fl = info >> 16;
        int32_t x = 0, y = 0, z = 0;
        if (WM == W_BLOCK) {
            x = (int32_t)(info & 0xffffu);
            y = (int32_t)(s_yz[k] & 0xffffu);
            z = (int32_t)(s_yz[k] >> 16);
        }
        V x2 = vload<PREC>(Y2, io.lin[1], i);
        const float yi = x2.h;
        float acc = 0.0f;  // sum_j g_ij (y_i - y_j) in slot order; absent neighbours add nothing
        for_each_neighbour(i, k, fl, s_nb, cap, [&](int slot, int64_t j) {
            const float d = __fsub_rn(yi, __ldg(Y2 + j));
            if (WM == W_UNIT) acc = __fadd_rn(acc, d);
            else acc = __fmaf_rn(edge_g(bw, i, slot, x, y, z), d, acc);
        });
        vadd<PREC>(x2, __fmul_rn(-p.c, acc));  // Scheme 1: y_i - D dt sum_j g_ij (y_i - y_j)
        if (MODE == 1) {
            vround<PREC>(x2);  // as if X^{k+1} had been stored (split runs stay bit-identical)
            V x1 = vload<PREC>(io.in[0], io.lin[0], i), x3 = vload<PREC>(io.in[2], io.lin[2], i),
              x4 = vload<PREC>(io.in[3], io.lin[3], i), x5 = vload<PREC>(io.in[4], io.lin[4], i);
            transform_n<TR, PREC>(x1, x2, x3, x4, x5, p);
            vstore<PREC>(io.out[0], io.lout[0], i, x1);
            vstore<PREC>(io.out[1], io.lout[1], i, x2);
            vstore<PREC>(io.out[2], io.lout[2], i, x3);
            vstore<PREC>(io.out[3], io.lout[3], i, x4);
            vstore<PREC>(io.out[4], io.lout[4], i, x5);
        } else {
            vstore<PREC>(io.out[1], io.lout[1], i, x2);
        }
    }
}

// Staged variant of k_stencil.  One thread issues bulk asynchronous copies (cp.async.bulk) of the
// chunk's own contiguous state into shared memory while all threads decode the topology; then
// every node reads its own values and its in-chunk neighbours (+-x always, +-y mostly) from shared
// memory and only the remaining neighbours (+-z, chunk edges) from L2.  The results overwrite the
// staged inputs in shared memory and leave with bulk stores, so the node loop issues no global
// load or store of its own state.  Arithmetic is identical to k_stencil.
template <int CAP, int NT>
struct StagedLayout {
    static constexpr int kPer = CAP / NT;
    static constexpr size_t bar = 0;
    static constexpr size_t h = 16;                                 // 5 x CAP floats
    static constexpr size_t l = h + sizeof(float) * 5 * CAP;        // 5 x CAP residuals
    static constexpr size_t dec = l + sizeof(res_t) * 5 * CAP;      // decode words
    static constexpr size_t bytes(bool need_yz) { return dec + sizeof(uint32_t) * CAP * decode_words(need_yz); }
};

template <int MODE, int WM, int TR, int PREC, int CAP, int NT>
__global__ void __launch_bounds__(NT) k_stencil_staged(Topo t, const int32_t *__restrict__ chunk_row, StepParams p,
                                                        BlockWeights bw, StateIO io, int32_t *__restrict__ err) {
    using Ly = StagedLayout<CAP, NT>;
    extern __shared__ __align__(16) unsigned char sbuf[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(sbuf + Ly::bar);
    float *sh = reinterpret_cast<float *>(sbuf + Ly::h);
    res_t *sl = reinterpret_cast<res_t *>(sbuf + Ly::l);
    uint32_t *s_info = reinterpret_cast<uint32_t *>(sbuf + Ly::dec);
    int32_t *s_nb = reinterpret_cast<int32_t *>(s_info + CAP);
    uint32_t *s_yz = s_info + 5 * CAP;
    constexpr int c0 = (MODE == 1) ? 0 : 1, c1 = (MODE == 1) ? 5 : 2;

    const int64_t v0 = (int64_t)blockIdx.x * CAP;
    const int32_t nv = (int32_t)min((int64_t)CAP, t.n - v0);
    const uint32_t nvp = (uint32_t)((nv + 15) & ~15);  // 16-byte multiples; the extra entries are padding
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t per = nvp * 4u + (PREC == P_COMP ? nvp * (uint32_t)sizeof(res_t) : 0u);
        mbar_arrive_expect_tx(bar, per * (uint32_t)(c1 - c0));
        for (int c = c0; c < c1; ++c) {
            bulk_g2s(sh + c * CAP, io.in[c] + v0, nvp * 4u, bar);
            if (PREC == P_COMP) bulk_g2s(sl + c * CAP, io.lin[c] + v0, nvp * (uint32_t)sizeof(res_t), bar);
        }
    }
    int64_t v0d;
    decode_chunk<WM == W_BLOCK>(t, chunk_row, CAP, s_info, s_nb, s_yz, v0d);
    const bool ok = mbar_wait_bounded(bar, 0, err, 1);

    const float *__restrict__ Y2 = io.in[1];
    float *__restrict__ sh2 = sh + CAP;
    float acc[Ly::kPer];
#pragma unroll
    for (int u = 0; u < Ly::kPer; ++u) {
        const int32_t k = threadIdx.x + u * NT;
        acc[u] = 0.0f;
        if (!ok || k >= nv) continue;
        const uint32_t info = s_info[k];
        const uint32_t fl = info >> 16;
        int32_t x = 0, y = 0, z = 0;
        if (WM == W_BLOCK) {
            x = (int32_t)(info & 0xffffu);
            y = (int32_t)(s_yz[k] & 0xffffu);
            z = (int32_t)(s_yz[k] >> 16);
        }
        const int64_t i = v0 + k;
        const float yi = sh2[k];
        float a = 0.0f;
        for_each_neighbour(i, k, fl, s_nb, CAP, [&](int slot, int64_t j) {
            const int64_t jj = j - v0;
            const float yj = (jj >= 0 && jj < nv) ? sh2[jj] : __ldg(Y2 + j);
            const float d = __fsub_rn(yi, yj);
            if (WM == W_UNIT) a = __fadd_rn(a, d);
            else a = __fmaf_rn(edge_g(bw, i, slot, x, y, z), d, a);
        });
        acc[u] = a;
    }
    __syncthreads();  // every neighbour read of the staged DOM is done: results may overwrite it
    if (ok) {
#pragma unroll
        for (int u = 0; u < Ly::kPer; ++u) {
            const int32_t k = threadIdx.x + u * NT;
            if (k >= nv) continue;
            V x2 = {sh2[k], PREC == P_COMP ? res_decode(sl[CAP + k], sh2[k]) : 0.0f};
            vadd<PREC>(x2, __fmul_rn(-p.c, acc[u]));
            V xs[5];
            if (MODE == 1) {
                vround<PREC>(x2);
#pragma unroll
                for (int c = 0; c < 5; ++c)
                    if (c != 1)
                        xs[c] = V{sh[c * CAP + k], PREC == P_COMP ? res_decode(sl[c * CAP + k], sh[c * CAP + k]) : 0.0f};
                xs[1] = x2;
                transform_n<TR, PREC>(xs[0], xs[1], xs[2], xs[3], xs[4], p);
            } else {
                xs[1] = x2;
            }
#pragma unroll
            for (int c = c0; c < c1; ++c) {
                if (PREC == P_COMP) {
                    const float s = __fadd_rn(xs[c].h, xs[c].l);  // renormalise as vstore does
                    const float r = __fadd_rn(__fsub_rn(xs[c].h, s), xs[c].l);
                    sh[c * CAP + k] = s;
                    sl[c * CAP + k] = res_encode(r, s);
                } else {
                    sh[c * CAP + k] = xs[c].h;
                }
            }
        }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0 && ok) {
        for (int c = c0; c < c1; ++c) {
            bulk_s2g(io.out[c] + v0, sh + c * CAP, nvp * 4u);
            if (PREC == P_COMP) bulk_s2g(io.lout[c] + v0, sl + c * CAP, nvp * (uint32_t)sizeof(res_t));
        }
        bulk_commit();
        bulk_wait_read_all();
    }
}

// ---- neighbour-offset table ---------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_build_table(Topo t, const int32_t *__restrict__ chunk_row, int32_t cap,
                                                          uint32_t *__restrict__ ty, uint32_t *__restrict__ tzm,
                                                          uint32_t *__restrict__ tzp) {
    extern __shared__ uint32_t smem[];
    int32_t *s_nb = reinterpret_cast<int32_t *>(smem + cap);
    int64_t v0;
    const int32_t nv = decode_chunk<false>(t, chunk_row, cap, smem, s_nb, nullptr, v0);
    for (int32_t k = threadIdx.x; k < nv; k += blockDim.x) {
        const int64_t i = v0 + k;
        const uint32_t fl = smem[k] >> 16;
        const uint32_t dym = (fl & 4u) ? (uint32_t)(i - s_nb[k]) : 0u;
        const uint32_t dyp = (fl & 8u) ? (uint32_t)(s_nb[cap + k] - i) : 0u;
        ty[i] = dym | ((fl & 1u) << 15) | (dyp << 16) | ((fl & 2u) << 30);
        tzm[i] = (fl & 16u) ? (uint32_t)(i - s_nb[2 * cap + k]) : 0u;
        tzp[i] = (fl & 32u) ? (uint32_t)(s_nb[3 * cap + k] - i) : 0u;
    }
}

__global__ void __launch_bounds__(kThreads) k_build_bnode(Topo t, const int32_t *__restrict__ chunk_row, int32_t cap,
                                                          int32_t bs, int32_t nbx, int32_t nby,
                                                          uint32_t *__restrict__ bnode) {
    extern __shared__ uint32_t smem[];
    int32_t *s_nb = reinterpret_cast<int32_t *>(smem + cap);
    int64_t v0;
    const int32_t nv = decode_chunk<true>(t, chunk_row, cap, smem, s_nb, smem + 5 * cap, v0);
    for (int32_t k = threadIdx.x; k < nv; k += blockDim.x) {
        const int32_t x = (int32_t)(smem[k] & 0xffffu);
        const int32_t y = (int32_t)(smem[5 * cap + k] & 0xffffu), z = (int32_t)(smem[5 * cap + k] >> 16);
        const uint32_t b = (uint32_t)(((int64_t)(z / bs) * nby + y / bs) * nbx + x / bs);
        const uint32_t fb = (uint32_t)(x % bs == 0) | ((uint32_t)((x + 1) % bs == 0) << 1) |
                            ((uint32_t)(y % bs == 0) << 2) | ((uint32_t)((y + 1) % bs == 0) << 3) |
                            ((uint32_t)(z % bs == 0) << 4) | ((uint32_t)((z + 1) % bs == 0) << 5);
        bnode[v0 + k] = b | (fb << 26);
    }
}

__global__ void k_build_bface(BlockWeights bw, int32_t *__restrict__ face) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nb = (int64_t)bw.nbx * bw.nby * bw.nbz;
    if (b >= nb) return;
    const int32_t bx = (int32_t)(b % bw.nbx), by = (int32_t)((b / bw.nbx) % bw.nby), bz = (int32_t)(b / ((int64_t)bw.nbx * bw.nby));
    int32_t *f = face + 6 * b;
    f[0] = bx > 0 ? (int32_t)(((int64_t)bz * bw.nby + by) * (bw.nbx - 1) + bx - 1) : -1;
    f[1] = bx < bw.nbx - 1 ? (int32_t)(((int64_t)bz * bw.nby + by) * (bw.nbx - 1) + bx) : -1;
    f[2] = by > 0 ? (int32_t)(bw.off_y + ((int64_t)bz * (bw.nby - 1) + by - 1) * bw.nbx + bx) : -1;
    f[3] = by < bw.nby - 1 ? (int32_t)(bw.off_y + ((int64_t)bz * (bw.nby - 1) + by) * bw.nbx + bx) : -1;
    f[4] = bz > 0 ? (int32_t)(bw.off_z + ((int64_t)(bz - 1) * bw.nby + by) * bw.nbx + bx) : -1;
    f[5] = bz < bw.nbz - 1 ? (int32_t)(bw.off_z + ((int64_t)bz * bw.nby + by) * bw.nbx + bx) : -1;
}

// theta6[k] = theta[face[k]] for the 6 slots of every block (1 where the face lies on the border).
__global__ void k_build_theta6(int64_t m, const int32_t *__restrict__ face, const float *__restrict__ theta,
                               float *__restrict__ theta6) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    const int32_t f = face[k];
    theta6[k] = f >= 0 ? theta[f] : 1.0f;
}

// One node per thread, neighbours from the offset table (table_node).
template <int MODE, int WM, int TR, int PREC, int TF>
__global__ void __launch_bounds__(kThreads) k_stencil_table(int64_t n, NbrTable tb, BlockTable bt, StepParams p,
                                                            StateIO io) {
    const uint32_t i = (uint32_t)blockIdx.x * blockDim.x + threadIdx.x;
    table_node<MODE, WM, TR, PREC, LD_NC, TF>(i, i < (uint64_t)n, tb, bt, p, io);
}

// Programmatic dependent launch (PTX griddepcontrol, sm_90 and later). A grid launched with
// programmatic stream serialisation may be scheduled while the kernel before it on the stream is
// still running; pdl_wait, before the grid's first global access, holds it until that kernel has
// completed and its writes are visible. For a grid launched without the attribute it returns at
// once. pdl_trigger lets the next grid on the stream be scheduled once every block of this one has
// issued it (its blocks then sit in their own pdl_wait).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Resident blocks per SM the compiler must fit: the DOM half of the sparse pass (MODE 4) is bound
// by the latency of its gathers and fits 40 registers (6 blocks) without spills, except with block
// conductances (5).
template <int MODE, int WM>
constexpr int tablev_min_blocks() {
    return MODE == 4 ? (WM == W_UNIT ? 6 : 5) : 4;
}

// K consecutive nodes per thread (table_vec); n < 2^31, so K * thread index fits 32 bits.
template <int MODE, int WM, int TR, int PREC, int TF, int K>
__global__ void __launch_bounds__(kThreads, tablev_min_blocks<MODE, WM>()) k_stencil_tablev(int64_t n, NbrTable tb, BlockTable bt, StepParams p,
                                                             StateIO io, SparseState ss) {
    if constexpr (MODE == 1 || MODE == 4) {
        pdl_wait();
        pdl_trigger();
    }
    const uint32_t i0 = (uint32_t)K * ((uint32_t)blockIdx.x * blockDim.x + threadIdx.x);
    table_vec<MODE, WM, TR, PREC, TF, K>(i0, (uint32_t)n, tb, bt, p, io, PassRecord{}, ss);
}

// Second half of the two-kernel sparse pass: one thread per marked node, in rank order, with its
// MB, SOM, FOM, CO2 from the compact state (updated in place) and its DOM as the first half stored it
// (the rounded pair); stores the DOM as MODE 1 does.
template <int TR, int PREC>
__global__ void __launch_bounds__(kThreads) k_transform_compact(int64_t m, SparseState ss, StepParams p, StateIO io) {
    pdl_wait();
    pdl_trigger();
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
    transform_n<TR, PREC>(v[0], x2, v[1], v[2], v[3], p);
#pragma unroll
    for (int q = 0; q < 4; ++q) vstore<PREC>(ss.h[q], ss.l[q], r, v[q]);
    vstore<PREC>(io.out[1], io.lout[1], i, x2);
}

// Node of each rank (once per state upload, after the prefix).
__global__ void k_build_list(int64_t n, SparseState ss, uint32_t *__restrict__ list) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t w = (uint32_t)(i >> 5), bit = 1u << (i & 31);
    const uint32_t m = __ldg(ss.mask + w);
    if (m & bit) list[__ldg(ss.prefix + w) + __popc(m & (bit - 1u))] = (uint32_t)i;
}

// Exclusive prefix of the marked nodes per mask word (once per state upload), in three coalesced
// phases over tiles of kScanTile words: the popcount of every tile, the exclusive scan of those
// counts, then each tile's words scanned from its tile's offset.  Thread t of a tile holds its
// words 8 t .. 8 t + 7 (32 contiguous bytes).
constexpr int kScanWords = 8;
constexpr int kScanTile = kThreads * kScanWords;

inline int64_t mask_tiles(int64_t words) { return (words + kScanTile - 1) / kScanTile; }

// Exclusive scan over the block of one value per thread; *total gets the block's sum.
__device__ __forceinline__ uint32_t block_excl_scan_u32(uint32_t v, uint32_t *total) {
    __shared__ uint32_t ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = (blockDim.x + 31) >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t y = lane < nwarp ? ws[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += t;
        }
        ws[lane] = y;
    }
    __syncthreads();
    const uint32_t before = (wid > 0 ? ws[wid - 1] : 0u) + x - v;
    *total = ws[nwarp - 1];
    __syncthreads();
    return before;
}

__device__ __forceinline__ void mask_words(int64_t words, const uint32_t *__restrict__ mask, int64_t w0,
                                           uint32_t (&m)[kScanWords]) {
#pragma unroll
    for (int j = 0; j < kScanWords; ++j) m[j] = w0 + j < words ? __ldg(mask + w0 + j) : 0u;
}

__global__ void __launch_bounds__(kThreads) k_mask_tile_count(int64_t words, const uint32_t *__restrict__ mask,
                                                              uint32_t *__restrict__ tile_sum) {
    uint32_t m[kScanWords];
    mask_words(words, mask, (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanWords, m);
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < kScanWords; ++j) c += __popc(m[j]);
    uint32_t total;
    block_excl_scan_u32(c, &total);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

// In place: tile_sum[t] <- the sum of the tiles before t (one block).
__global__ void __launch_bounds__(kThreads) k_mask_tile_scan(int64_t tiles, uint32_t *__restrict__ tile_sum) {
    uint32_t run = 0;
    for (int64_t t0 = 0; t0 < tiles; t0 += kThreads) {
        const int64_t t = t0 + threadIdx.x;
        const uint32_t v = t < tiles ? tile_sum[t] : 0u;
        uint32_t total;
        const uint32_t before = block_excl_scan_u32(v, &total);
        if (t < tiles) tile_sum[t] = run + before;
        run += total;
    }
}

__global__ void __launch_bounds__(kThreads) k_mask_prefix(int64_t words, const uint32_t *__restrict__ mask,
                                                          const uint32_t *__restrict__ tile_sum,
                                                          uint32_t *__restrict__ prefix) {
    const int64_t w0 = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanWords;
    uint32_t m[kScanWords];
    mask_words(words, mask, w0, m);
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < kScanWords; ++j) c += __popc(m[j]);
    uint32_t total;
    uint32_t run = __ldg(tile_sum + blockIdx.x) + block_excl_scan_u32(c, &total);
#pragma unroll
    for (int j = 0; j < kScanWords; ++j) {
        if (w0 + j < words) prefix[w0 + j] = run;
        run += __popc(m[j]);
    }
}

// Marked nodes' MB, SOM, FOM, CO2 between the state arrays (io.in read, io.out written) and the
// compact state: to_compact copies state -> compact, otherwise compact -> state.
__global__ void k_active_copy(int64_t m, SparseState ss, StateIO io, int to_compact, int comp) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // rank: one thread per marked node
    if (r >= m) return;
    const uint32_t i = __ldg(ss.list + r);
    const int cs[4] = {0, 2, 3, 4};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (to_compact) {
            ss.h[q][r] = io.in[cs[q]][i];
            if (comp) ss.l[q][r] = io.lin[cs[q]][i];
        } else {
            io.out[cs[q]][i] = ss.h[q][r];
            if (comp) io.lout[cs[q]][i] = ss.l[q][r];
        }
    }
}

// Activity mask of the sparse fused pass (vga_sim.active): bit i set when node i may change under
// the transformation: any bit of MB, SOM, FOM or CO2 (value or residual) nonzero, or a
// negative-zero DOM (the transformation's zero increment would turn it into +0).  Every flux of
// both transformations is proportional to MB, SOM or FOM, so at the other nodes the
// transformation is the identity and stays so.  Those nodes also get zeros in the spare buffers
// of MB, SOM, FOM and CO2 (their current values are zero), so that a pass may skip them.
template <int PREC>
__global__ void k_build_active(int64_t n, StateIO cur, StateIO spare, uint32_t *__restrict__ mask,
                               unsigned long long *__restrict__ count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool act = false;
    if (i < n) {
        const int cs[4] = {0, 2, 3, 4};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            act |= __float_as_uint(cur.in[cs[q]][i]) != 0u;
            if (PREC == P_COMP) act |= cur.lin[cs[q]][i] != 0;
        }
        act |= __float_as_uint(cur.in[1][i]) == 0x80000000u;
        if (PREC == P_COMP) act |= cur.lin[1][i] == (res_t)0x8000u;
        if (!act) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                spare.out[cs[q]][i] = 0.0f;
                if (PREC == P_COMP) spare.lout[cs[q]][i] = 0;
            }
        }
    }
    const unsigned b = __ballot_sync(0xffffffffu, act);
    if ((threadIdx.x & 31) == 0 && i < n) {
        mask[i >> 5] = b;
        if (b) atomicAdd(count, (unsigned long long)__popc(b));
    }
}

// Largest z offset of the table (for the compact form).
__global__ void k_table_zmax(int64_t n, const uint32_t *__restrict__ tzm, const uint32_t *__restrict__ tzp,
                             unsigned int *__restrict__ out) {
    uint32_t m = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = max(m, max(__ldg(tzm + i), __ldg(tzp + i)));
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void k_table_pack_z(int64_t n, const uint32_t *__restrict__ tzm, const uint32_t *__restrict__ tzp,
                               uint32_t *__restrict__ tz) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) tz[i] = tzm[i] | (tzp[i] << 16);
}

// ---- FP64 totals ---------------------------------------------------------------------------
template <int PREC>
// Each thread sums its nodes in float-float (TwoSum of the high parts; the low parts and the sum
// errors added in FP32), about 2^-48 relative for the tens of terms a thread takes; threads and
// blocks are summed in FP64.  No FP64 arithmetic per node: the FP64 rate of this part is a small
// fraction of its FP32 rate, and the FP64 form took 0.8 ms for 21 M nodes.
// The same pass scans the state: flags bit 0 is set when a value is not finite, bit 1 when one is
// negative (the schemes keep every compartment >= 0 within the stability bound).
__global__ void __launch_bounds__(kThreads) k_totals(int64_t n, StateIO io, double *__restrict__ partials,
                                                     int32_t *__restrict__ flags) {
    float sh[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f}, sl[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    uint32_t f = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            const V v = vload<PREC>(io.in[c], io.lin[c], i);
            f |= ((__float_as_uint(v.h) & 0x7f800000u) == 0x7f800000u ? 1u : 0u) | (v.h < 0.0f ? 2u : 0u);
            const float t = __fadd_rn(sh[c], v.h);
            const float bb = __fsub_rn(t, sh[c]);
            const float e = __fadd_rn(__fsub_rn(sh[c], __fsub_rn(t, bb)), __fsub_rn(v.h, bb));
            sh[c] = t;
            sl[c] = __fadd_rn(sl[c], __fadd_rn(e, v.l));
        }
    }
    f = __reduce_or_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0 && f) atomicOr(flags, (int32_t)f);
    double s[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) s[c] = (double)sh[c] + (double)sl[c];
    __shared__ double out[5];
    block_sum_store<5>(s, out);
    if (threadIdx.x < 5) partials[(int64_t)blockIdx.x * 5 + threadIdx.x] = out[threadIdx.x];
}

__global__ void __launch_bounds__(kThreads) k_totals_final(const double *__restrict__ partials, int nblocks,
                                                           double *__restrict__ out) {
    double s[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
        for (int c = 0; c < 5; ++c) s[c] += partials[(int64_t)b * 5 + c];
    __shared__ double o[5];
    block_sum_store<5>(s, o);
    if (threadIdx.x < 5) out[threadIdx.x] = o[threadIdx.x];
}

// ---- conversions ---------------------------------------------------------------------------
// FP64 (5 x n) -> state: h = RN(x), l = the rounding error (quantised residual)
__global__ void k_convert_in(int64_t n, const double *__restrict__ x, StateIO io, int comp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const double v = x[c * n + i];
        const float h = (float)v;
        io.out[c][i] = h;
        if (comp) io.lout[c][i] = res_encode((float)(v - (double)h), h);
    }
}

__global__ void k_convert_out(int64_t n, double *__restrict__ x, StateIO io, int comp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        const float h = io.in[c][i];
        double v = (double)h;
        if (comp) v += (double)res_decode(io.lin[c][i], h);
        x[c * n + i] = v;
    }
}

// FP32 (5 x n) <-> state; to the state the residual is zero, from the state h + l is rounded.
__global__ void k_pack(int64_t n, float *__restrict__ x, StateIO io, int to_state, int comp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        if (to_state) {
            io.out[c][i] = x[c * n + i];
            if (comp) io.lout[c][i] = 0;
        } else {
            const float h = io.in[c][i];
            double v = (double)h;
            if (comp) v += (double)res_decode(io.lin[c][i], h);
            x[c * n + i] = (float)v;
        }
    }
}

// Checkpoint residuals: stored residual <-> the BF16 bits of its value (the identity for the
// current BF16 storage, kept so that the checkpoint format does not depend on it).
__global__ void k_res_export(int64_t n, StateIO io, uint16_t *__restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int c = 0; c < 5; ++c) out[c * n + i] = float_to_bf16_bits(res_decode(io.lin[c][i], io.in[c][i]));
}

__global__ void k_res_import(int64_t n, const uint16_t *__restrict__ in, StateIO io) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int c = 0; c < 5; ++c) io.lout[c][i] = res_encode(bf16_bits_to_float(in[c * n + i]), io.out[c][i]);
}

inline unsigned grid_for(int64_t count, int threads) { return (unsigned)((count + threads - 1) / threads); }

constexpr int kStagedThreads = 256;

template <int MODE, int WM, int TR, int PREC, int CAP>
void launch_staged(vga_sim *s, const StateIO &io) {
    using Ly = StagedLayout<CAP, kStagedThreads>;
    constexpr size_t smem = Ly::bytes(WM == W_BLOCK);
    auto kern = k_stencil_staged<MODE, WM, TR, PREC, CAP, kStagedThreads>;
    static uint64_t configured = 0;  // one attribute call per instantiation and device (ordinals < 64)
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !((configured >> dev) & 1ull)) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        configured |= 1ull << dev;
    }
    kern<<<s->chunks.count, kStagedThreads, smem, s->stream>>>(s->g->topo(), s->chunks.row, s->sp, s->bw, io, s->d_err);
}

// Chunk sizes with a staged instantiation.
bool staged_cap_supported(int cap) { return cap == 512 || cap == 1024 || cap == 2048; }

template <int MODE, int WM, int TR, int PREC>
void launch_staged_any(vga_sim *s, const StateIO &io) {
    switch (s->chunks.cap) {
        case 512: launch_staged<MODE, WM, TR, PREC, 512>(s, io); break;
        case 2048: launch_staged<MODE, WM, TR, PREC, 2048>(s, io); break;
        default: launch_staged<MODE, WM, TR, PREC, 1024>(s, io); break;
    }
}

// The compact state of the running step call.
SparseState sparse_state(vga_sim *s) { return activity_state(s->act); }

// Launch with programmatic stream serialisation: the grid may be scheduled during the tail of the
// kernel before it on the stream and waits for it in pdl_wait (the kernel must call it first).
template <typename... KArgs, typename... Args>
void launch_pdl(void (*kernel)(KArgs...), unsigned grid, cudaStream_t stream, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

template <int MODE, int WM, int PREC, int K>
void launch_tablev_m(vga_sim *s, const StateIO &io, const NbrTable &tb, const BlockTable &bt) {
    const unsigned grid = grid_for((s->n + K - 1) / K, kThreads);
    const SparseState act = sparse_state(s);
    if constexpr (MODE == 1 || MODE == 4) {
        if (tb.tz) {
            if (s->sp.transform == 0) launch_pdl(k_stencil_tablev<MODE, WM, 0, PREC, 1, K>, grid, s->stream, s->n, tb, bt, s->sp, io, act);
            else launch_pdl(k_stencil_tablev<MODE, WM, 1, PREC, 1, K>, grid, s->stream, s->n, tb, bt, s->sp, io, act);
        } else {
            if (s->sp.transform == 0) launch_pdl(k_stencil_tablev<MODE, WM, 0, PREC, 0, K>, grid, s->stream, s->n, tb, bt, s->sp, io, act);
            else launch_pdl(k_stencil_tablev<MODE, WM, 1, PREC, 0, K>, grid, s->stream, s->n, tb, bt, s->sp, io, act);
        }
        return;
    }
    if (tb.tz) {
        if (s->sp.transform == 0) k_stencil_tablev<MODE, WM, 0, PREC, 1, K><<<grid, kThreads, 0, s->stream>>>(s->n, tb, bt, s->sp, io, act);
        else k_stencil_tablev<MODE, WM, 1, PREC, 1, K><<<grid, kThreads, 0, s->stream>>>(s->n, tb, bt, s->sp, io, act);
    } else {
        if (s->sp.transform == 0) k_stencil_tablev<MODE, WM, 0, PREC, 0, K><<<grid, kThreads, 0, s->stream>>>(s->n, tb, bt, s->sp, io, act);
        else k_stencil_tablev<MODE, WM, 1, PREC, 0, K><<<grid, kThreads, 0, s->stream>>>(s->n, tb, bt, s->sp, io, act);
    }
}

// Fused passes of the four-node kernel run sparse inside a sparse step call: the DOM of every node
// (MODE 4), then the transformation of the marked nodes in rank order.
template <int MODE, int WM, int PREC, int K>
void launch_tablev(vga_sim *s, const StateIO &io, const NbrTable &tb, const BlockTable &bt) {
    if (MODE == 1 && K == 4 && s->sparse_call) {
        launch_tablev_m<4, WM, PREC, K>(s, io, tb, bt);
        const int64_t m = s->act.n_active;
        if (m > 0) {
            const unsigned g = grid_for(m, kThreads);
            const SparseState ss = activity_state(s->act);
            if (s->sp.transform == 0) launch_pdl(k_transform_compact<0, PREC>, g, s->stream, m, ss, s->sp, io);
            else launch_pdl(k_transform_compact<1, PREC>, g, s->stream, m, ss, s->sp, io);
            ++s->launches;
        }
        return;
    }
    launch_tablev_m<MODE, WM, PREC, K>(s, io, tb, bt);
}

template <int MODE, int WM, int PREC>
vga_status launch_table(vga_sim *s, const StateIO &io, const NbrTable &tb, const BlockTable &bt) {
    if (s->kernel_variant == 4) {
        launch_tablev<MODE, WM, PREC, 2>(s, io, tb, bt);
        return VGA_OK;
    }
    if (s->kernel_variant == 5 || s->kernel_variant == 6) {  // 6: its unblocked passes are variant 5's
        launch_tablev<MODE, WM, PREC, 4>(s, io, tb, bt);
        return VGA_OK;
    }
    const unsigned grid = grid_for(s->n, kThreads);
    if (tb.tz) {
        if (s->sp.transform == 0) k_stencil_table<MODE, WM, 0, PREC, 1><<<grid, kThreads, 0, s->stream>>>(s->n, tb, bt, s->sp, io);
        else k_stencil_table<MODE, WM, 1, PREC, 1><<<grid, kThreads, 0, s->stream>>>(s->n, tb, bt, s->sp, io);
    } else {
        if (s->sp.transform == 0) k_stencil_table<MODE, WM, 0, PREC, 0><<<grid, kThreads, 0, s->stream>>>(s->n, tb, bt, s->sp, io);
        else k_stencil_table<MODE, WM, 1, PREC, 0><<<grid, kThreads, 0, s->stream>>>(s->n, tb, bt, s->sp, io);
    }
    return VGA_OK;
}

template <int MODE, int WM, int PREC>
void launch_stencil_tr(vga_sim *s, const StateIO &io) {
    const Topo t = s->g->topo();
    const size_t smem = sizeof(uint32_t) * (size_t)s->chunks.cap * decode_words(WM == W_BLOCK);
    if (s->kernel_variant == 1 && staged_cap_supported(s->chunks.cap)) {
        if (s->sp.transform == 0) launch_staged_any<MODE, WM, 0, PREC>(s, io);
        else launch_staged_any<MODE, WM, 1, PREC>(s, io);
        return;
    }
    if (s->sp.transform == 0)
        k_stencil<MODE, WM, 0, PREC><<<s->chunks.count, kThreads, smem, s->stream>>>(t, s->chunks.row, s->chunks.cap,
                                                                                   s->sp, s->bw, io);
    else
        k_stencil<MODE, WM, 1, PREC><<<s->chunks.count, kThreads, smem, s->stream>>>(t, s->chunks.row, s->chunks.cap,
                                                                                   s->sp, s->bw, io);
}

template <int MODE>
vga_status launch_stencil(vga_sim *s, const StateIO &io) {
    const bool comp = s->precision() == P_COMP;
    if (s->kernel_variant >= 2 && s->g->nx <= 32767) {
        // table kernels: build the tables (first use) before the timed launch
        NbrTable tb;
        BlockTable bt;
        bool block_ok = true;
        VGA_TRY(sim_nbr_table(s, &tb));
        if (s->wmode == W_BLOCK) VGA_TRY(sim_block_table(s, &bt, &block_ok));
        if (block_ok) {
            timing_begin(s, MODE == 1 ? VGA_KERNEL_FUSED_STEP : VGA_KERNEL_DIFFUSE);
            vga_status st;
            if (s->wmode == W_BLOCK)
                st = comp ? launch_table<MODE, W_BLOCK, P_COMP>(s, io, tb, bt) : launch_table<MODE, W_BLOCK, P_F32>(s, io, tb, bt);
            else
                st = comp ? launch_table<MODE, W_UNIT, P_COMP>(s, io, tb, bt) : launch_table<MODE, W_UNIT, P_F32>(s, io, tb, bt);
            timing_end(s);
            VGA_TRY(st);
            VGA_CHECK_LAUNCH();
            ++s->launches;
            return VGA_OK;
        }
    }
    timing_begin(s, MODE == 1 ? VGA_KERNEL_FUSED_STEP : VGA_KERNEL_DIFFUSE);
    if (s->wmode == W_BLOCK) {
        if (comp) launch_stencil_tr<MODE, W_BLOCK, P_COMP>(s, io);
        else launch_stencil_tr<MODE, W_BLOCK, P_F32>(s, io);
    } else {
        if (comp) launch_stencil_tr<MODE, W_UNIT, P_COMP>(s, io);
        else launch_stencil_tr<MODE, W_UNIT, P_F32>(s, io);
    }
    timing_end(s);
    VGA_CHECK_LAUNCH();
    ++s->launches;
    return VGA_OK;
}

}  // namespace

StateIO state_io(vga_sim *s) {
    StateIO io;
    for (int c = 0; c < 5; ++c) {
        io.in[c] = s->comp(c);
        io.out[c] = s->spare(c);
        io.lin[c] = s->lcomp(c);
        io.lout[c] = s->lspare(c);
    }
    return io;
}

StateIO state_io_inplace(vga_sim *s) {
    StateIO io;
    for (int c = 0; c < 5; ++c) {
        io.in[c] = s->comp(c);
        io.out[c] = s->comp(c);
        io.lin[c] = s->lcomp(c);
        io.lout[c] = s->lcomp(c);
    }
    return io;
}

vga_status sim_prepare_params(vga_sim *s, const vga_params *p) {
    StepParams sp;
    const double dtt = p->dt_transform > 0.0 ? p->dt_transform : p->dt;
    sp.a = (float)(p->v_dom * dtt);
    sp.K = (float)p->K_dom;
    sp.r = (float)(p->rho * dtt);
    sp.m = (float)(p->mu * dtt);
    sp.beta = (float)p->beta;
    sp.omb = (float)(1.0 - p->beta);
    sp.f = (float)(p->v_fom * dtt);
    sp.s = (float)(p->v_som * dtt);
    sp.c = (float)(p->D * p->dt);
    sp.transform = p->transform;
    sp.ntrans = 1;
    s->sp = sp;
    s->params = *p;
    return VGA_OK;
}

int64_t sim_ticks_before(const vga_sim *s, int64_t k) {
    if (!s->subcycled()) return k;
    if (k <= 0) return 0;
    const double r = s->params.dt / s->params.dt_transform;
    const double kr = (double)k * r;
    return (int64_t)std::ceil(kr - 1e-9);
}

int sim_ticks_of_step(const vga_sim *s, int64_t k) {
    return (int)(sim_ticks_before(s, k + 1) - sim_ticks_before(s, k));
}

vga_status sim_transform_pass(vga_sim *s) {
    if (s->sp.ntrans == 0) return VGA_OK;  // identity: leave the state where it is
    StateIO io = state_io(s);
    const unsigned grid = grid_for(s->n, kThreads);
    const bool comp = s->precision() == P_COMP;
    timing_begin(s, VGA_KERNEL_TRANSFORM);
    if (s->sp.transform == 0) {
        if (comp) k_transform<0, P_COMP><<<grid, kThreads, 0, s->stream>>>(s->n, s->sp, io);
        else k_transform<0, P_F32><<<grid, kThreads, 0, s->stream>>>(s->n, s->sp, io);
    } else {
        if (comp) k_transform<1, P_COMP><<<grid, kThreads, 0, s->stream>>>(s->n, s->sp, io);
        else k_transform<1, P_F32><<<grid, kThreads, 0, s->stream>>>(s->n, s->sp, io);
    }
    timing_end(s);
    VGA_CHECK_LAUNCH();
    ++s->launches;
    for (int c = 0; c < 5; ++c) s->cur[c] ^= 1;
    return VGA_OK;
}

// The last pass of a step call: diffusion of the stored transformed DOM only.
vga_status sim_diffuse_pass(vga_sim *s) {
    VGA_TRY(launch_stencil<2>(s, state_io(s)));
    s->cur[1] ^= 1;
    return VGA_OK;
}

SparseState activity_state(const Activity &a) {
    SparseState ss;
    ss.mask = a.words;
    ss.prefix = a.words ? a.words + a.nw : nullptr;
    const size_t cap = (size_t)std::max<int64_t>(a.cap, 1);
    float *h = reinterpret_cast<float *>(a.state);
    res_t *l = reinterpret_cast<res_t *>(h + 4 * cap);
    for (int q = 0; q < 4; ++q) {
        ss.h[q] = a.state ? h + q * cap : nullptr;
        ss.l[q] = a.state ? l + q * cap : nullptr;
    }
    ss.list = a.state ? reinterpret_cast<const uint32_t *>(l + 4 * cap) : nullptr;
    return ss;
}

vga_status activity_build(Activity *a, int64_t n, int64_t npad, const StateIO &cur, const StateIO &spare, bool comp,
                          cudaStream_t st) {
    const int64_t nw = (std::max<int64_t>(npad, 64) + 31) / 32 + 8;
    if (!a->words || a->nw < nw) {  // mask words, their prefix, a counter, the tile sums of the prefix
        dfree(a->words);
        a->words = nullptr;
        VGA_TRY(dmalloc((void **)&a->words,
                        sizeof(uint32_t) * (2 * (size_t)nw + (size_t)mask_tiles(nw)) + sizeof(unsigned long long),
                        "activity mask"));
        a->nw = nw;
        VGA_CUDA(cudaMemsetAsync(a->words, 0, sizeof(uint32_t) * 2 * (size_t)nw, st));
    }
    unsigned long long *count = reinterpret_cast<unsigned long long *>(a->words + 2 * a->nw);
    VGA_CUDA(cudaMemsetAsync(count, 0, sizeof(unsigned long long), st));
    if (n > 0) {
        if (comp) k_build_active<P_COMP><<<grid_for(n, kThreads), kThreads, 0, st>>>(n, cur, spare, a->words, count);
        else k_build_active<P_F32><<<grid_for(n, kThreads), kThreads, 0, st>>>(n, cur, spare, a->words, count);
        VGA_CHECK_LAUNCH();
    }
    {
        const int64_t tiles = mask_tiles(a->nw);
        uint32_t *tile_sum = a->words + 2 * a->nw + 2;  // after the 64-bit counter
        k_mask_tile_count<<<(unsigned)tiles, kThreads, 0, st>>>(a->nw, a->words, tile_sum);
        k_mask_tile_scan<<<1, kThreads, 0, st>>>(tiles, tile_sum);
        k_mask_prefix<<<(unsigned)tiles, kThreads, 0, st>>>(a->nw, a->words, tile_sum, a->words + a->nw);
        VGA_CHECK_LAUNCH();
    }
    unsigned long long h = 0;
    VGA_CUDA(cudaMemcpyAsync(&h, count, sizeof(h), cudaMemcpyDeviceToHost, st));
    VGA_CUDA(cudaStreamSynchronize(st));
    a->n_active = (int64_t)h;
    if (a->cap < a->n_active) {  // compact MB, SOM, FOM, CO2 (values and residuals)
        dfree(a->state);
        a->state = nullptr;
        a->cap = 0;
        VGA_TRY(dmalloc((void **)&a->state,
                        ((sizeof(float) + sizeof(res_t)) * 4 + sizeof(uint32_t)) * (size_t)a->n_active + 16,
                        "compact active state"));
        a->cap = a->n_active;
    }
    if (n > 0 && a->n_active > 0) {
        const SparseState ss = activity_state(*a);
        k_build_list<<<grid_for(n, kThreads), kThreads, 0, st>>>(n, ss, const_cast<uint32_t *>(ss.list));
        VGA_CHECK_LAUNCH();
    }
    a->valid = true;
    static std::atomic<int64_t> next_build{0};  // unique over the process, so a freed mask never matches
    a->builds = ++next_build;
    return VGA_OK;
}

vga_status activity_copy(const Activity &a, int64_t n, const StateIO &io, bool to_compact, bool comp, cudaStream_t st) {
    if (n <= 0 || a.n_active <= 0) return VGA_OK;
    k_active_copy<<<grid_for(a.n_active, kThreads), kThreads, 0, st>>>(a.n_active, activity_state(a), io,
                                                                     to_compact ? 1 : 0, comp ? 1 : 0);
    VGA_CHECK_LAUNCH();
    return VGA_OK;
}

void activity_free(Activity *a) {
    dfree(a->words);
    dfree(a->state);
    *a = Activity{};
}

// Builds the activity mask for the current state (once per state upload; stepping keeps it valid).
vga_status sim_build_active(vga_sim *s) {
    StateIO spare;
    for (int c = 0; c < 5; ++c) {
        spare.in[c] = s->spare(c);
        spare.out[c] = s->spare(c);
        spare.lin[c] = s->lspare(c);
        spare.lout[c] = s->lspare(c);
    }
    VGA_TRY(activity_build(&s->act, s->n, s->npad, state_io(s), spare, s->precision() == P_COMP, s->stream));
    s->launches += 2;
    return VGA_OK;
}

static vga_status step_body(vga_sim *s, int64_t n_steps, bool sparse);

// ---- CUDA graphs of whole step calls on small graphs ----------------------------------------------
// Below kStepGraphNodes a pass takes a few microseconds on the GPU and the call is bound by the host's
// launch rate.  A call whose shape was seen before (step count, state-buffer parity, parameters and
// conductances, activity mask, variant) is captured as a graph (on a private stream: the simulation's
// may be the legacy default stream) and later replayed; a replay reapplies the call's host-side
// changes (buffer parity, step count, launch count).  Timing, sub-cycling, the wavefront and blocked
// variants and a failed capture run the launches directly.
constexpr int64_t kStepGraphNodes = (int64_t)1 << 21;

static bool step_graph_eligible(const vga_sim *s, int64_t n_steps) {
    return s->n < kStepGraphNodes && n_steps > 1 && !s->timing && !s->subcycled() && s->step_graphs_ok &&
           s->kernel_variant != 3 && s->kernel_variant != 6;
}

static uint32_t cur_mask(const vga_sim *s) {
    uint32_t m = 0;
    for (int c = 0; c < 5; ++c) m |= (uint32_t)(s->cur[c] & 1) << c;
    return m;
}

void step_graphs_free(vga_sim *s) {
    for (auto &g : s->step_graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = StepGraph{};
    }
    if (s->step_cap) cudaStreamDestroy(s->step_cap);
    s->step_cap = nullptr;
}

static vga_status step_graphed(vga_sim *s, int64_t n_steps, bool sparse) {
    StepGraph key;
    key.n_steps = n_steps;
    key.cur_in = cur_mask(s);
    key.param_gen = s->param_gen;
    key.builds = sparse ? s->act.builds : -1;
    key.variant = s->kernel_variant;
    key.sparse = sparse;
    StepGraph *hit = nullptr, *lru = &s->step_graphs[0];
    for (auto &g : s->step_graphs) {
        if (g.n_steps == key.n_steps && g.cur_in == key.cur_in && g.param_gen == key.param_gen &&
            g.builds == key.builds && g.variant == key.variant && g.sparse == key.sparse) {
            hit = &g;
            break;
        }
        if (g.use < lru->use) lru = &g;
    }
    ++s->step_graph_clock;
    if (!hit) {  // first time: remember the shape, run directly
        if (lru->exec) cudaGraphExecDestroy(lru->exec);
        *lru = key;
        lru->use = s->step_graph_clock;
        return step_body(s, n_steps, sparse);
    }
    hit->use = s->step_graph_clock;
    if (!hit->exec) {  // seen before: capture this call and keep the graph
        if (!s->step_cap && cudaStreamCreateWithFlags(&s->step_cap, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            s->step_cap = nullptr;
            s->step_graphs_ok = false;
            return step_body(s, n_steps, sparse);
        }
        int cur0[5];
        for (int c = 0; c < 5; ++c) cur0[c] = s->cur[c];
        const int64_t done0 = s->steps_done, launches0 = s->launches;
        cudaStream_t real = s->stream;
        VGA_CUDA(cudaStreamBeginCapture(s->step_cap, cudaStreamCaptureModeThreadLocal));
        s->stream = s->step_cap;
        const vga_status r = step_body(s, n_steps, sparse);
        s->stream = real;
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(s->step_cap, &graph);
        cudaError_t ei = cudaErrorUnknown;
        if (r == VGA_OK && ec == cudaSuccess) ei = cudaGraphInstantiate(&hit->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (r != VGA_OK || ec != cudaSuccess || ei != cudaSuccess) {  // nothing ran: undo the host changes
            cudaGetLastError();
            hit->exec = nullptr;
            for (int c = 0; c < 5; ++c) s->cur[c] = cur0[c];
            s->steps_done = done0;
            s->launches = launches0;
            if (r != VGA_OK) return r;
            s->step_graphs_ok = false;
            return step_body(s, n_steps, sparse);
        }
        hit->cur_xor = cur_mask(s) ^ key.cur_in;
        hit->launches = s->launches - launches0;
        VGA_CUDA(cudaGraphLaunch(hit->exec, s->stream));
        return VGA_OK;
    }
    VGA_CUDA(cudaGraphLaunch(hit->exec, s->stream));
    for (int c = 0; c < 5; ++c) s->cur[c] ^= (int)((hit->cur_xor >> c) & 1u);
    s->steps_done += n_steps;
    s->launches += hit->launches;
    return VGA_OK;
}

vga_status sim_step_explicit(vga_sim *s, int64_t n_steps) {
    if (n_steps <= 0 || s->n == 0) {
        s->steps_done += std::max<int64_t>(n_steps, 0);
        return VGA_OK;
    }
    // sparse fused passes: variant 5 on the neighbour-offset table (and the block table, if used)
    bool sparse = s->activity_skip && (s->kernel_variant == 5 || s->kernel_variant == 6) && s->g->nx <= 32767 &&
                  n_steps > 1;
    if (sparse && s->wmode == W_BLOCK) {
        BlockTable bt;
        bool ok = false;
        VGA_TRY(sim_block_table(s, &bt, &ok));
        sparse = ok;
    }
    if (sparse && !s->act.valid) VGA_TRY(sim_build_active(s));
    if (step_graph_eligible(s, n_steps)) return step_graphed(s, n_steps, sparse);
    return step_body(s, n_steps, sparse);
}

// The passes of one explicit step call (the host logic and the launches; no host synchronisation).
static vga_status step_body(vga_sim *s, int64_t n_steps, bool sparse) {
    const bool sub = s->subcycled();
    const int64_t k0 = s->steps_done;
    // ntrans is reset on every exit so that no other path sees a sub-cycled count
    struct Reset {
        StepParams &sp;
        ~Reset() { sp.ntrans = 1; }
    } reset{s->sp};
    if (sub) s->sp.ntrans = sim_ticks_of_step(s, k0);
    VGA_TRY(sim_transform_pass(s));
    if (s->kernel_variant == 3 && !sub && s->g->nx <= 32767 && n_steps > 1) {
        VGA_TRY(sim_wave_fused(s, n_steps - 1));
    } else {
        // sparse call: the marked nodes' MB, SOM, FOM, CO2 live in the compact state during the
        // fused passes and go back to the state arrays after them
        struct SparseEnd {
            vga_sim *s;
            ~SparseEnd() { s->sparse_call = false; }
        } sparse_end{s};
        const bool copy = sparse && s->act.n_active > 0;
        const bool comp = s->precision() == P_COMP;
        if (copy) {
            VGA_TRY(activity_copy(s->act, s->n, state_io(s), true, comp, s->stream));
            ++s->launches;
        }
        s->sparse_call = sparse;
        // with timing on, the fused passes of the call are timed as one span (credited as n_steps - 1
        // passes): an event pair around every launch would stop each grid from being scheduled in the
        // tail of the one before it (programmatic dependent launch)
        struct Span {
            vga_sim *s;
            bool on;
            ~Span() { s->timing_hold = false; }
        } span{s, s->timing && n_steps > 1};
        if (span.on) {
            timing_begin(s, VGA_KERNEL_FUSED_STEP);
            s->timing_hold = true;
        }
        bool blocked = false;  // variant 6: the fused passes as temporally blocked launches
        if (sparse && s->kernel_variant == 6 && !sub) VGA_TRY(sim_block_fused(s, n_steps - 1, &blocked));
        for (int64_t k = 1; k < n_steps && !blocked; ++k) {
            if (sub) s->sp.ntrans = sim_ticks_of_step(s, k0 + k);
            VGA_TRY(launch_stencil<1>(s, state_io(s)));
            for (int c = 0; c < 5; ++c) s->cur[c] ^= 1;
        }
        if (span.on) {
            s->timing_hold = false;
            timing_end_weighted(s, n_steps - 1);
        }
        s->sparse_call = false;
        if (copy) {
            VGA_TRY(activity_copy(s->act, s->n, state_io_inplace(s), false, comp, s->stream));
            ++s->launches;
        }
    }
    VGA_TRY(launch_stencil<2>(s, state_io(s)));
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
    StateIO io = state_io(s);
    timing_begin(s, VGA_KERNEL_TOTALS);
    int32_t *flags = s->d_err + 1;  // state scan of the totals pass
    if (s->precision() == P_COMP) k_totals<P_COMP><<<nb, kThreads, 0, s->stream>>>(s->n, io, s->partials, flags);
    else k_totals<P_F32><<<nb, kThreads, 0, s->stream>>>(s->n, io, s->partials, flags);
    k_totals_final<<<1, kThreads, 0, s->stream>>>(s->partials, nb, s->d_totals);
    timing_end(s);
    VGA_CHECK_LAUNCH();
    s->launches += 2;
    int32_t *h_flags = reinterpret_cast<int32_t *>(s->h_totals + 6);
    VGA_CUDA(cudaMemcpyAsync(s->h_totals, s->d_totals, 5 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    VGA_CUDA(cudaMemcpyAsync(h_flags, flags, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    for (int c = 0; c < 5; ++c) h_out[c] = s->h_totals[c];
    if (*h_flags) {
        const int32_t fl = *h_flags;
        VGA_CUDA(cudaMemsetAsync(flags, 0, sizeof(int32_t), s->stream));
        VGA_CUDA(cudaStreamSynchronize(s->stream));
        if (fl & 2) ++s->negative_reports;
        if (fl & 1) return fail(VGA_ERR_NONFINITE, "the state holds a non-finite mass (found by the totals pass)");
    }
    return VGA_OK;
}

vga_status sim_convert_in(vga_sim *s, const double *d_x) {
    s->act.valid = false;
    if (s->n == 0) return VGA_OK;
    k_convert_in<<<grid_for(s->n, kThreads), kThreads, 0, s->stream>>>(s->n, d_x, state_io_inplace(s),
                                                                     s->precision() == P_COMP);
    VGA_CHECK_LAUNCH();
    ++s->launches;
    return VGA_OK;
}

vga_status sim_convert_out(vga_sim *s, double *d_x) {
    if (s->n == 0) return VGA_OK;
    k_convert_out<<<grid_for(s->n, kThreads), kThreads, 0, s->stream>>>(s->n, d_x, state_io_inplace(s),
                                                                      s->precision() == P_COMP);
    VGA_CHECK_LAUNCH();
    ++s->launches;
    return VGA_OK;
}

vga_status sim_pack_f32(vga_sim *s, float *d_x, bool to_state) {
    if (to_state) s->act.valid = false;
    if (s->n == 0) return VGA_OK;
    k_pack<<<grid_for(s->n, kThreads), kThreads, 0, s->stream>>>(s->n, d_x, state_io_inplace(s), to_state ? 1 : 0,
                                                               s->precision() == P_COMP);
    VGA_CHECK_LAUNCH();
    ++s->launches;
    return VGA_OK;
}

int totals_blocks() { return kTotBlocks; }

vga_status sim_res_export(vga_sim *s, uint16_t *d_out) {
    if (s->n == 0) return VGA_OK;
    k_res_export<<<grid_for(s->n, kThreads), kThreads, 0, s->stream>>>(s->n, state_io_inplace(s), d_out);
    VGA_CHECK_LAUNCH();
    ++s->launches;
    return VGA_OK;
}

vga_status sim_res_import(vga_sim *s, const uint16_t *d_in) {
    s->act.valid = false;
    if (s->n == 0) return VGA_OK;
    k_res_import<<<grid_for(s->n, kThreads), kThreads, 0, s->stream>>>(s->n, d_in, state_io_inplace(s));
    VGA_CHECK_LAUNCH();
    ++s->launches;
    return VGA_OK;
}

vga_status build_nbr_table(const Topo &t, uint32_t *ty, uint32_t *tzm, uint32_t *tzp, cudaStream_t st) {
    if (t.n == 0) return VGA_OK;
    Chunks ch;
    VGA_TRY(build_chunks(t, 1024, &ch, st));
    const size_t smem = sizeof(uint32_t) * 1024 * decode_words(false);
    k_build_table<<<ch.count, kThreads, smem, st>>>(t, ch.row, 1024, ty, tzm, tzp);
    const cudaError_t e = cudaGetLastError();
    const cudaError_t e2 = cudaStreamSynchronize(st);
    free_chunks(&ch);
    if (e != cudaSuccess) return cuda_fail(e, "k_build_table", __FILE__, __LINE__);
    if (e2 != cudaSuccess) return cuda_fail(e2, "k_build_table", __FILE__, __LINE__);
    return VGA_OK;
}

// The per-face table: node i is its own block with every slot crossing (table_theta reads g6[6 i + d],
// table_face gives 6 i + d).
__global__ void k_face_nodes(int64_t n, uint32_t *__restrict__ node) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) node[i] = (uint32_t)i | 0xfc000000u;
}

vga_status sim_block_table(vga_sim *s, BlockTable *out, bool *ok) {
    *ok = false;
    if (s->wmode != W_BLOCK) return VGA_OK;
    if (s->face_mode) {
        if (s->n >= kMaxTableBlocks) return VGA_OK;
        if (!s->fnode) {
            VGA_TRY(dmalloc((void **)&s->fnode, sizeof(uint32_t) * (size_t)std::max<int64_t>(s->npad, 64), "face table"));
            if (s->n > 0) k_face_nodes<<<grid_for(s->n, kThreads), kThreads, 0, s->stream>>>(s->n, s->fnode);
            VGA_CHECK_LAUNCH();
            ++s->launches;
        }
        out->node = s->fnode;
        out->face = nullptr;
        out->theta = nullptr;
        out->theta6 = s->g6;
        *ok = true;
        return VGA_OK;
    }
    const int64_t nb = (int64_t)s->bw.nbx * s->bw.nby * s->bw.nbz;
    if (nb >= kMaxTableBlocks) return VGA_OK;
    if (s->btable_bs != s->bw.bs) {
        dfree(s->bnode);
        dfree(s->bface);
        s->bnode = nullptr;
        s->bface = nullptr;
        s->btable_bs = 0;
        VGA_TRY(dmalloc((void **)&s->bnode, sizeof(uint32_t) * (size_t)std::max<int64_t>(s->npad, 64), "block table"));
        VGA_TRY(dmalloc((void **)&s->bface, sizeof(int32_t) * 6 * (size_t)std::max<int64_t>(nb, 1), "block faces"));
        k_build_bface<<<(unsigned)((nb + kThreads - 1) / kThreads), kThreads, 0, s->stream>>>(s->bw, s->bface);
        VGA_CHECK_LAUNCH();
        if (s->n > 0) {
            Chunks ch;
            VGA_TRY(build_chunks(s->g->topo(), 1024, &ch, s->stream));
            const size_t smem = sizeof(uint32_t) * 1024 * decode_words(true);
            k_build_bnode<<<ch.count, kThreads, smem, s->stream>>>(s->g->topo(), ch.row, 1024, s->bw.bs, s->bw.nbx,
                                                                 s->bw.nby, s->bnode);
            const cudaError_t e = cudaGetLastError();
            const cudaError_t e2 = cudaStreamSynchronize(s->stream);
            free_chunks(&ch);
            if (e != cudaSuccess) return cuda_fail(e, "k_build_bnode", __FILE__, __LINE__);
            if (e2 != cudaSuccess) return cuda_fail(e2, "k_build_bnode", __FILE__, __LINE__);
        }
        s->launches += 2;
        s->btable_bs = s->bw.bs;
        dfree(s->btheta6);
        s->btheta6 = nullptr;
        VGA_TRY(dmalloc((void **)&s->btheta6, sizeof(float) * 6 * (size_t)std::max<int64_t>(nb, 1), "block conductances"));
        s->btheta6_gen = -1;
    }
    if (s->btheta6_gen != s->param_gen) {
        k_build_theta6<<<(unsigned)((6 * nb + kThreads - 1) / kThreads), kThreads, 0, s->stream>>>(6 * nb, s->bface,
                                                                                              s->bw.theta, s->btheta6);
        VGA_CHECK_LAUNCH();
        ++s->launches;
        s->btheta6_gen = s->param_gen;
    }
    out->node = s->bnode;
    out->face = s->bface;
    out->theta = s->bw.theta;
    out->theta6 = s->btheta6;
    *ok = true;
    return VGA_OK;
}

// Per-face conductances: flags |= 1 where g6[6 i + d] differs from the opposite slot of the
// neighbour (the flux of Sec. V.A is symmetric), and the largest sum over a node's edges.
__global__ void k_face_check(int64_t n, NbrTable tb, const float *__restrict__ g6, int32_t *__restrict__ flags,
                             unsigned int *__restrict__ rowmax) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float sum = 0.0f;
    bool bad = false;
    if (i < n) {
        const uint32_t ty = __ldg(tb.ty + i), dzm = __ldg(tb.tzm + i), dzp = __ldg(tb.tzp + i);
        const int64_t j[6] = {(ty >> 15) & 1u ? i - 1 : -1, (ty >> 31) ? i + 1 : -1,
                              (ty & 0x7fffu) ? i - (int64_t)(ty & 0x7fffu) : -1,
                              ((ty >> 16) & 0x7fffu) ? i + (int64_t)((ty >> 16) & 0x7fffu) : -1,
                              dzm ? i - (int64_t)dzm : -1, dzp ? i + (int64_t)dzp : -1};
#pragma unroll
        for (int d = 0; d < 6; ++d) {
            if (j[d] < 0) continue;
            const float g = __ldg(g6 + 6 * i + d);
            sum += g;
            bad |= __float_as_uint(g) != __float_as_uint(__ldg(g6 + 6 * j[d] + (d ^ 1)));
        }
    }
    if (bad) atomicOr(flags, 1);
    unsigned int m = __float_as_uint(sum);  // sums are >= 0: their bits order like the values
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(rowmax, m);
}

// Gradients of per-face conductances are accumulated in the +x, +y, +z slot of each edge; this copies
// each into the opposite slot of the neighbour, so both slots of an edge hold its derivative.
__global__ void k_face_mirror(int64_t n, NbrTable tb, double *__restrict__ g) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t ty = __ldg(tb.ty + i), dzp = __ldg(tb.tzp + i);
    if (ty >> 31) g[6 * (i + 1) + 0] = g[6 * i + 1];
    if ((ty >> 16) & 0x7fffu) g[6 * (i + (int64_t)((ty >> 16) & 0x7fffu)) + 2] = g[6 * i + 3];
    if (dzp) g[6 * (i + (int64_t)dzp) + 4] = g[6 * i + 5];
}

vga_status sim_face_check(vga_sim *s, const float *d_g6, bool *symmetric, float *rowmax) {
    *symmetric = true;
    *rowmax = 0.0f;
    if (s->n == 0) return VGA_OK;
    NbrTable tb;
    VGA_TRY(sim_nbr_table(s, &tb));
    unsigned int *d = nullptr;
    VGA_TRY(dmalloc((void **)&d, 2 * sizeof(unsigned int), "face check"));
    unsigned int h[2] = {0u, 0u};
    cudaError_t e = cudaMemsetAsync(d, 0, 2 * sizeof(unsigned int), s->stream);
    if (e == cudaSuccess) {
        k_face_check<<<grid_for(s->n, kThreads), kThreads, 0, s->stream>>>(s->n, tb, d_g6, reinterpret_cast<int32_t *>(d),
                                                                        d + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    dfree(d);
    if (e != cudaSuccess) return cuda_fail(e, "k_face_check", __FILE__, __LINE__);
    ++s->launches;
    *symmetric = h[0] == 0u;
    std::memcpy(rowmax, &h[1], sizeof(float));
    return VGA_OK;
}

// Block conductances in device memory: flags |= 1 for a value that is not finite or is negative; the
// largest value (as the bits of a non-negative float, which order like the values) into *mx.
__global__ void k_theta_check(int64_t n, const float *__restrict__ theta, unsigned int *__restrict__ flags,
                              unsigned int *__restrict__ mx) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    unsigned int bits = 0u;
    if (k < n) {
        const float t = theta[k];
        bad = !(isfinite(t) && t >= 0.0f);
        bits = bad ? 0u : __float_as_uint(t + 0.0f);  // +0 for -0
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, 1u);
    for (int o = 16; o > 0; o >>= 1) bits = max(bits, __shfl_down_sync(0xffffffffu, bits, o));
    if ((threadIdx.x & 31) == 0 && bits) atomicMax(mx, bits);
}

vga_status sim_theta_check(vga_sim *s, const float *d_theta, int64_t n, bool *valid, float *maxv) {
    *valid = true;
    *maxv = 0.0f;
    if (n <= 0) return VGA_OK;
    unsigned int *d = nullptr;
    VGA_TRY(dmalloc((void **)&d, 2 * sizeof(unsigned int), "conductance check"));
    unsigned int h[2] = {0u, 0u};
    cudaError_t e = cudaMemsetAsync(d, 0, 2 * sizeof(unsigned int), s->stream);
    if (e == cudaSuccess) {
        k_theta_check<<<grid_for(n, kThreads), kThreads, 0, s->stream>>>(n, d_theta, d, d + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    dfree(d);
    if (e != cudaSuccess) return cuda_fail(e, "k_theta_check", __FILE__, __LINE__);
    ++s->launches;
    *valid = h[0] == 0u;
    std::memcpy(maxv, &h[1], sizeof(float));
    return VGA_OK;
}

vga_status sim_face_mirror(vga_sim *s, double *d_g) {
    if (s->n == 0) return VGA_OK;
    NbrTable tb;
    VGA_TRY(sim_nbr_table(s, &tb));
    k_face_mirror<<<grid_for(s->n, kThreads), kThreads, 0, s->stream>>>(s->n, tb, d_g);
    VGA_CHECK_LAUNCH();
    ++s->launches;
    return VGA_OK;
}

vga_status sim_nbr_table(vga_sim *s, NbrTable *out) {
    if (!s->nbr_table) {
        VGA_TRY(dmalloc((void **)&s->nbr_table, sizeof(uint32_t) * 3 * (size_t)std::max<int64_t>(s->npad, 64),
                        "neighbour table"));
        VGA_TRY(build_nbr_table(s->g->topo(), s->nbr_table, s->nbr_table + s->npad, s->nbr_table + 2 * s->npad,
                                s->stream));
        ++s->launches;
    }
    out->ty = s->nbr_table;
    out->tzm = s->nbr_table + s->npad;
    out->tzp = s->nbr_table + 2 * s->npad;
    if (s->nbr_tz_state == 0 && s->n > 0) {
        VGA_TRY(build_compact_z(s->n, std::max<int64_t>(s->npad, 64), out->tzm, out->tzp, &s->nbr_tz, s->stream));
        s->nbr_tz_state = s->nbr_tz ? 1 : 2;
        s->launches += 2;
    }
    out->tz = s->nbr_tz_state == 1 ? s->nbr_tz : nullptr;
    return VGA_OK;
}

vga_status build_compact_z(int64_t n, int64_t cap, const uint32_t *tzm, const uint32_t *tzp, uint32_t **out,
                           cudaStream_t st) {
    *out = nullptr;
    if (n <= 0) return VGA_OK;
    unsigned int *d_max = nullptr;
    VGA_TRY(dmalloc((void **)&d_max, sizeof(unsigned int), "table maximum"));
    unsigned int h_max = 0;
    cudaError_t e = cudaMemsetAsync(d_max, 0, sizeof(unsigned int), st);
    if (e == cudaSuccess) {
        const unsigned g = (unsigned)std::min<int64_t>(grid_for(n, kThreads), 4096);
        k_table_zmax<<<g, kThreads, 0, st>>>(n, tzm, tzp, d_max);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_max, d_max, sizeof(h_max), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(d_max);
    if (e != cudaSuccess) return cuda_fail(e, "table z offsets", __FILE__, __LINE__);
    if (h_max >= 65536u) return VGA_OK;
    VGA_TRY(dmalloc((void **)out, sizeof(uint32_t) * (size_t)cap, "compact neighbour table"));
    k_table_pack_z<<<grid_for(n, kThreads), kThreads, 0, st>>>(n, tzm, tzp, *out);
    VGA_CHECK_LAUNCH();
    return VGA_OK;
}

bool stencil_variant_supported(int variant, int cap) {
    return variant == 0 || variant == 2 || variant == 4 || variant == 5 || variant == 6 || staged_cap_supported(cap);
}

}  // namespace vga
