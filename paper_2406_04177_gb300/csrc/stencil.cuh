// Chunk decoding and neighbour walk shared by every stencil kernel.
//
// A block owns the chunk of nodes [v0, v0 + nv).  decode_chunk() visits the row-bitmask words of
// the image rows the chunk spans.  For one word (32 voxels of one row) it loads the words at the
// same x in the rows above/below (y +- 1) and in the neighbouring planes (z +- 1) together with
// their prefix entries; the index of every neighbour of every node in the word then follows from a
// popcount.  Per node it writes to shared memory:
//   s_info[k]        x | (neighbour-existence bits << 16), bit order -x, +x, -y, +y, -z, +z
//   s_nb[d*cap + k]  node index of the -y, +y, -z, +z neighbour (d = 0..3) when it exists
//   s_yz[k]          y | z << 16 (only when the caller needs block coordinates)
// so the stencil loop itself issues only independent loads of neighbour values.
#pragma once

#include "physics.cuh"
#include "vga_internal.cuh"

namespace vga {

// Shared-memory words per node used by decode_chunk.
__host__ __device__ constexpr int decode_words(bool need_yz) { return need_yz ? 6 : 5; }

template <bool NEED_YZ>
__device__ __forceinline__ int32_t decode_chunk(const Topo &t, const int32_t *__restrict__ chunk_row, int32_t cap,
                                                uint32_t *s_info, int32_t *s_nb, uint32_t *s_yz, int64_t &v0_out) {
    const int64_t v0 = (int64_t)blockIdx.x * cap;
    const int64_t v1 = min(v0 + (int64_t)cap, t.n);
    const int32_t nv = (int32_t)(v1 - v0);
    const int32_t r0 = chunk_row[blockIdx.x], r1 = chunk_row[blockIdx.x + 1];
    const int32_t W = t.W;
    const int32_t nw = (r1 - r0 + 1) * W;
    for (int32_t q = threadIdx.x; q < nw; q += blockDim.x) {
        const int32_t rr = q / W;
        const int32_t w = q - rr * W;
        const int32_t r = r0 + rr;
        const int32_t wq = r * W + w;
        const uint32_t m = __ldg(t.mask + wq);
        if (!m) continue;
        const int64_t p0 = __ldg(t.pre + wq);
        if (p0 >= v1 || p0 + __popc(m) <= v0) continue;
        const int32_t z = r / t.ny, y = r - z * t.ny;
        // neighbour words and their prefix entries (0 where the row does not exist)
        uint32_t mn[4] = {0u, 0u, 0u, 0u};
        int32_t pn[4] = {0, 0, 0, 0};
        if (y > 0) { mn[0] = __ldg(t.mask + wq - W); pn[0] = __ldg(t.pre + wq - W); }
        if (y < t.ny - 1) { mn[1] = __ldg(t.mask + wq + W); pn[1] = __ldg(t.pre + wq + W); }
        const int32_t plane = t.ny * W;
        if (z > 0) { mn[2] = __ldg(t.mask + wq - plane); pn[2] = __ldg(t.pre + wq - plane); }
        if (z < t.nz - 1) { mn[3] = __ldg(t.mask + wq + plane); pn[3] = __ldg(t.pre + wq + plane); }
        // x neighbours: bit b of mleft/mright tells whether voxel x-1 / x+1 is a node
        const uint32_t prev31 = (w > 0) ? (__ldg(t.mask + wq - 1) >> 31) : 0u;
        const uint32_t next0 = (w < W - 1) ? (__ldg(t.mask + wq + 1) & 1u) : 0u;
        const uint32_t mleft = (m << 1) | prev31;
        const uint32_t mright = (m >> 1) | (next0 << 31);
        int64_t idx = p0 - v0;
        uint32_t mm = m;
        while (mm) {
            const int b = __ffs(mm) - 1;
            mm &= mm - 1;
            if (idx >= 0 && idx < nv) {
                const uint32_t bit = 1u << b, below = bit - 1u;
                uint32_t fl = ((mleft >> b) & 1u) | (((mright >> b) & 1u) << 1);
#pragma unroll
                for (int d = 0; d < 4; ++d) {
                    if (mn[d] & bit) {
                        fl |= 4u << d;
                        s_nb[d * cap + idx] = pn[d] + __popc(mn[d] & below);
                    }
                }
                s_info[idx] = (uint32_t)(32 * w + b) | (fl << 16);
                if (NEED_YZ) s_yz[idx] = (uint32_t)y | ((uint32_t)z << 16);
            }
            ++idx;
        }
    }
    __syncthreads();
    v0_out = v0;
    return nv;
}

// Calls f(slot, j) for every existing neighbour j of the k-th node of the chunk (global index i),
// in slot order -x, +x, -y, +y, -z, +z.
template <class F>
__device__ __forceinline__ void for_each_neighbour(int64_t i, int32_t k, uint32_t fl, const int32_t *s_nb, int32_t cap,
                                                   F &&f) {
    if (fl & 1u) f(0, i - 1);
    if (fl & 2u) f(1, i + 1);
    if (fl & 4u) f(2, (int64_t)s_nb[k]);
    if (fl & 8u) f(3, (int64_t)s_nb[cap + k]);
    if (fl & 16u) f(4, (int64_t)s_nb[2 * cap + k]);
    if (fl & 32u) f(5, (int64_t)s_nb[3 * cap + k]);
}

// Conductance of the edge leaving a node at (x, y, z) through `slot` under block weights: theta of
// the block face it crosses, 1 inside a block.
__device__ __forceinline__ float block_theta(const BlockWeights &bw, int slot, int x, int y, int z) {
    const int bs = bw.bs;
    const int bx = x / bs, by = y / bs, bz = z / bs;
    switch (slot) {
        case 0:
            return (x % bs == 0) ? __ldg(bw.theta + ((int64_t)bz * bw.nby + by) * (bw.nbx - 1) + (bx - 1)) : 1.0f;
        case 1:
            return ((x + 1) % bs == 0) ? __ldg(bw.theta + ((int64_t)bz * bw.nby + by) * (bw.nbx - 1) + bx) : 1.0f;
        case 2:
            return (y % bs == 0) ? __ldg(bw.theta + bw.off_y + ((int64_t)bz * (bw.nby - 1) + (by - 1)) * bw.nbx + bx)
                                 : 1.0f;
        case 3:
            return ((y + 1) % bs == 0) ? __ldg(bw.theta + bw.off_y + ((int64_t)bz * (bw.nby - 1) + by) * bw.nbx + bx)
                                       : 1.0f;
        case 4:
            return (z % bs == 0) ? __ldg(bw.theta + bw.off_z + ((int64_t)(bz - 1) * bw.nby + by) * bw.nbx + bx) : 1.0f;
        default:
            return ((z + 1) % bs == 0) ? __ldg(bw.theta + bw.off_z + ((int64_t)bz * bw.nby + by) * bw.nbx + bx) : 1.0f;
    }
}

// Index of the block face crossed by the edge leaving (x, y, z) through `slot`, or -1.
__device__ __forceinline__ int64_t block_face(const BlockWeights &bw, int slot, int x, int y, int z) {
    const int bs = bw.bs;
    const int bx = x / bs, by = y / bs, bz = z / bs;
    switch (slot) {
        case 0: return (x % bs == 0) ? ((int64_t)bz * bw.nby + by) * (bw.nbx - 1) + (bx - 1) : -1;
        case 1: return ((x + 1) % bs == 0) ? ((int64_t)bz * bw.nby + by) * (bw.nbx - 1) + bx : -1;
        case 2: return (y % bs == 0) ? bw.off_y + ((int64_t)bz * (bw.nby - 1) + (by - 1)) * bw.nbx + bx : -1;
        case 3: return ((y + 1) % bs == 0) ? bw.off_y + ((int64_t)bz * (bw.nby - 1) + by) * bw.nbx + bx : -1;
        case 4: return (z % bs == 0) ? bw.off_z + ((int64_t)(bz - 1) * bw.nby + by) * bw.nbx + bx : -1;
        default: return ((z + 1) % bs == 0) ? bw.off_z + ((int64_t)bz * bw.nby + by) * bw.nbx + bx : -1;
    }
}

// Conductance of the edge leaving a node through `slot` under the block table (see BlockTable).
// Per-face conductances use the same table with one "block" per node (every slot crossing) and
// theta6 = the 6 x n conductances.
__device__ __forceinline__ float table_theta(const BlockTable &bt, uint32_t bn, int slot) {
    if (!((bn >> (26 + slot)) & 1u)) return 1.0f;
    return __ldg(bt.theta6 + 6 * (size_t)(bn & 0x3ffffffu) + slot);
}

// Gradient index of that edge: the block face, or (per-face table: face == NULL) 6 node + slot.
__device__ __forceinline__ int32_t table_face(const BlockTable &bt, uint32_t bn, int slot) {
    if (!((bn >> (26 + slot)) & 1u)) return -1;
    if (!bt.face) return (int32_t)(6 * (bn & 0x3ffffffu)) + slot;
    return __ldg(bt.face + 6 * (size_t)(bn & 0x3ffffffu) + slot);
}

// Forms for loops that visit every slot without branching: the lookups are selects (the addresses
// are valid for any block id, including the 0 of a lane past the end).
__device__ __forceinline__ float table_theta_sel(const BlockTable &bt, uint32_t bn, int slot) {
    return ((bn >> (26 + slot)) & 1u) ? __ldg(bt.theta6 + 6 * (size_t)(bn & 0x3ffffffu) + slot) : 1.0f;
}

// table_face for an edge that exists, -1 otherwise (the face table is read only for a crossing edge).
__device__ __forceinline__ int32_t table_face_sel(const BlockTable &bt, uint32_t bn, int slot, bool exists) {
    const uint32_t b = bn & 0x3ffffffu;
    const bool cross = exists && ((bn >> (26 + slot)) & 1u);
    if (!bt.face) return cross ? (int32_t)(6 * b) + slot : -1;
    return cross ? __ldg(bt.face + 6 * (size_t)b + slot) : -1;
}

// Conductance of the edge leaving node i (at x, y, z) through `slot`: per-face, else per block face.
__device__ __forceinline__ float edge_g(const BlockWeights &bw, int64_t i, int slot, int x, int y, int z) {
    return bw.g6 ? __ldg(bw.g6 + 6 * i + slot) : block_theta(bw, slot, x, y, z);
}

// Gradient index of that edge (see table_face), or -1 when it lies inside a block.
__device__ __forceinline__ int64_t edge_face(const BlockWeights &bw, int64_t i, int slot, int x, int y, int z) {
    return bw.g6 ? 6 * i + slot : block_face(bw, slot, x, y, z);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum of K doubles per thread; thread 0 writes the K results to out[0..K).
template <int K>
__device__ __forceinline__ void block_sum_store(const double (&v)[K], double *out) {
    __shared__ double sh[K][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const double w = warp_sum_d(v[k]);
        if (lane == 0) sh[k][wid] = w;
    }
    __syncthreads();
    if (threadIdx.x < K) {
        double b = 0.0;
        for (int w = 0; w < nw; ++w) b += sh[threadIdx.x][w];
        out[threadIdx.x] = b;
    }
    __syncthreads();
}

// Load path of state arrays: LD_NC reads through the read-only (non-coherent) data cache; LD_CG
// reads at L2, as a kernel must for values that other blocks of the same launch have written.
enum LoadPath { LD_NC = 0, LD_CG = 1 };

template <int LP>
__device__ __forceinline__ float ld_state(const float *p) {
    if (LP == LD_NC) return __ldg(p);
    return __ldcg(p);
}

template <int PREC, int LP>
__device__ __forceinline__ V vload_path(const float *__restrict__ H, const res_t *__restrict__ L, int64_t i) {
    if (LP == LD_NC) return vload<PREC>(H, L, i);
    V v;
    v.h = __ldcg(H + i);
    v.l = (PREC == P_COMP) ? res_decode(__ldcg(L + i), v.h) : 0.0f;
    return v;
}

// One node of a table-driven pass: MODE 1 diffuses the stored transformed DOM (Scheme 1) and
// transforms the result; MODE 2 only diffuses.  TF 1 reads the compact z offsets (NbrTable.tz).
// Neighbours come from the offset table; the +-x
// neighbours' values from the adjacent lanes (consecutive nodes) by warp shuffles.  Arithmetic and
// slot order as k_stencil.  Must be called by all 32 lanes of a warp (live = node exists).
template <int MODE, int WM, int TR, int PREC, int LP, int TF = 0>
__device__ __forceinline__ void table_node(uint32_t i, bool live, const NbrTable &tb, const BlockTable &bt,
                                           const StepParams &p, const StateIO &io) {
    const uint32_t bn = (WM == W_BLOCK && live) ? __ldg(bt.node + i) : 0u;
    const float *__restrict__ Y2 = io.in[1];
    const uint32_t ty = live ? __ldg(tb.ty + i) : 0u;
    uint32_t dzm, dzp;
    if (TF == 1) {  // compact z offsets
        const uint32_t tz = live ? __ldg(tb.tz + i) : 0u;
        dzm = tz & 0xffffu;
        dzp = tz >> 16;
    } else {
        dzm = live ? __ldg(tb.tzm + i) : 0u;
        dzp = live ? __ldg(tb.tzp + i) : 0u;
    }
    V x2 = live ? vload_path<PREC, LP>(Y2, io.lin[1], i) : V{0.0f, 0.0f};
    const float yi = x2.h;
    const int lane = threadIdx.x & 31;
    float yl = __shfl_up_sync(0xffffffffu, yi, 1);
    float yr = __shfl_down_sync(0xffffffffu, yi, 1);
    const uint32_t dym = ty & 0x7fffu, dyp = (ty >> 16) & 0x7fffu;
    const bool hxm = (ty >> 15) & 1u, hxp = ty >> 31;
    if (lane == 0 && hxm) yl = ld_state<LP>(Y2 + (i - 1));
    if (lane == 31 && hxp) yr = ld_state<LP>(Y2 + (i + 1));
    float ym = 0.0f, yp = 0.0f, zm = 0.0f, zp = 0.0f;
    if (dym) ym = ld_state<LP>(Y2 + (i - dym));
    if (dyp) yp = ld_state<LP>(Y2 + (i + dyp));
    if (dzm) zm = ld_state<LP>(Y2 + (i - dzm));
    if (dzp) zp = ld_state<LP>(Y2 + (i + dzp));
    if (!live) return;
    float acc = 0.0f;
    auto add = [&](int slot, float yj) {
        const float d = __fsub_rn(yi, yj);
        if (WM == W_UNIT) acc = __fadd_rn(acc, d);
        else acc = __fmaf_rn(table_theta(bt, bn, slot), d, acc);
    };
    if (hxm) add(0, yl);
    if (hxp) add(1, yr);
    if (dym) add(2, ym);
    if (dyp) add(3, yp);
    if (dzm) add(4, zm);
    if (dzp) add(5, zp);
    vadd<PREC>(x2, __fmul_rn(-p.c, acc));  // Scheme 1
    if (MODE == 1) {
        vround<PREC>(x2);
        V x1 = vload_path<PREC, LP>(io.in[0], io.lin[0], i), x3 = vload_path<PREC, LP>(io.in[2], io.lin[2], i),
          x4 = vload_path<PREC, LP>(io.in[3], io.lin[3], i), x5 = vload_path<PREC, LP>(io.in[4], io.lin[4], i);
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

// Vector access to K consecutive 32-bit words (K = 2: 8 bytes, K = 4: 16 bytes) and K consecutive
// residuals; p must be aligned to the vector size.
template <int K>
__device__ __forceinline__ void ldg_words(const uint32_t *p, uint32_t (&o)[K]) {
    if (K == 2) {
        const uint2 w = __ldg(reinterpret_cast<const uint2 *>(p));
        o[0] = w.x;
        o[1] = w.y;
    } else {
        const uint4 w = __ldg(reinterpret_cast<const uint4 *>(p));
        o[0] = w.x;
        o[1] = w.y;
        o[K > 2 ? 2 : 0] = w.z;
        o[K > 3 ? 3 : 0] = w.w;
    }
}

template <int K>
__device__ __forceinline__ void ldg_floats(const float *p, float (&o)[K]) {
    uint32_t w[K];
    ldg_words<K>(reinterpret_cast<const uint32_t *>(p), w);
#pragma unroll
    for (int k = 0; k < K; ++k) o[k] = __uint_as_float(w[k]);
}

template <int K>
__device__ __forceinline__ void st_floats(float *p, const float (&v)[K]) {
    if (K == 2) *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
    else *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[K > 2 ? 2 : 0], v[K > 3 ? 3 : 0]);
}

template <int K>
__device__ __forceinline__ void ldg_res(const res_t *p, res_t (&o)[K]) {
    if (K == 2) {
        const uint32_t w = __ldg(reinterpret_cast<const unsigned int *>(p));
        o[0] = (res_t)(w & 0xffffu);
        o[1] = (res_t)(w >> 16);
    } else {
        const uint2 w = __ldg(reinterpret_cast<const uint2 *>(p));
        o[0] = (res_t)(w.x & 0xffffu);
        o[1] = (res_t)(w.x >> 16);
        o[K > 2 ? 2 : 0] = (res_t)(w.y & 0xffffu);
        o[K > 3 ? 3 : 0] = (res_t)(w.y >> 16);
    }
}

template <int K>
__device__ __forceinline__ void st_res(res_t *p, const res_t (&v)[K]) {
    if (K == 2) {
        *reinterpret_cast<unsigned int *>(p) = (uint32_t)v[0] | ((uint32_t)v[1] << 16);
    } else {
        *reinterpret_cast<uint2 *>(p) = make_uint2((uint32_t)v[0] | ((uint32_t)v[1] << 16),
                                                   (uint32_t)v[K > 2 ? 2 : 0] | ((uint32_t)v[K > 3 ? 3 : 0] << 16));
    }
}

// K stored values i0 .. i0 + K - 1.  FULL: all K exist, one vector access per array; otherwise one
// access per live value (i0 + k < n).  Arithmetic as vload / vstore.
template <int PREC, int K, bool FULL>
__device__ __forceinline__ void vload_k(const float *__restrict__ H, const res_t *__restrict__ L, uint32_t i0,
                                        uint32_t n, V (&v)[K]) {
    if (FULL) {
        float h[K];
        ldg_floats<K>(H + i0, h);
        res_t q[K];
        if (PREC == P_COMP) ldg_res<K>(L + i0, q);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            v[k].h = h[k];
            v[k].l = (PREC == P_COMP) ? res_decode(q[k], h[k]) : 0.0f;
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = i0 + k < n ? vload<PREC>(H, L, i0 + k) : V{0.0f, 0.0f};
    }
}

template <int PREC, int K, bool FULL>
__device__ __forceinline__ void vstore_k(float *__restrict__ H, res_t *__restrict__ L, uint32_t i0, uint32_t n,
                                         const V (&v)[K]) {
    if (FULL) {
        float h[K];
        res_t q[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (PREC == P_COMP) {  // renormalise as vstore
                h[k] = __fadd_rn(v[k].h, v[k].l);
                q[k] = res_encode(__fadd_rn(__fsub_rn(v[k].h, h[k]), v[k].l), h[k]);
            } else {
                h[k] = v[k].h;
            }
        }
        st_floats<K>(H + i0, h);
        if (PREC == P_COMP) st_res<K>(L + i0, q);
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (i0 + k < n) vstore<PREC>(H, L, i0 + k, v[k]);
    }
}

template <int K, bool FULL>
__device__ __forceinline__ void ldg_words_k(const uint32_t *__restrict__ p, uint32_t i0, uint32_t n,
                                            uint32_t (&o)[K]) {
    if (FULL) {
        ldg_words<K>(p + i0, o);
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) o[k] = i0 + k < n ? __ldg(p + i0 + k) : 0u;
    }
}

// Per-node streams of a group of K nodes: offset table, block ids and the stored DOM.
template <int WM, int PREC, int TF, int K, bool FULL>
__device__ __forceinline__ void group_load(uint32_t i0, uint32_t n, const NbrTable &tb, const BlockTable &bt,
                                           const StateIO &io, uint32_t (&ty)[K], uint32_t (&zm)[K],
                                           uint32_t (&zp)[K], uint32_t (&bn)[K], V (&x2)[K]) {
    ldg_words_k<K, FULL>(tb.ty, i0, n, ty);
    if (TF == 1) {
        ldg_words_k<K, FULL>(tb.tz, i0, n, zm);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            zp[k] = zm[k] >> 16;
            zm[k] &= 0xffffu;
        }
    } else {
        ldg_words_k<K, FULL>(tb.tzm, i0, n, zm);
        ldg_words_k<K, FULL>(tb.tzp, i0, n, zp);
    }
    if (WM == W_BLOCK) ldg_words_k<K, FULL>(bt.node, i0, n, bn);
    vload_k<PREC, K, FULL>(io.in[1], io.lin[1], i0, n, x2);
}

// Transformation and stores of a group (MODE 1), or the DOM store alone (MODE 2).
// Record of one fused pass for the discrete adjoint: X (after the diffusion, before the
// transformation; 5 rows of npad FP32 values h + l) and the transformed DOM.
struct PassRecord {
    float *x;
    float *y2;
    int64_t npad;
};

// h + l of K values into dst[i0 ..] (vector store when FULL).
template <int K, bool FULL>
__device__ __forceinline__ void record_k(float *dst, uint32_t i0, uint32_t n, const V (&v)[K]) {
    float h[K];
#pragma unroll
    for (int k = 0; k < K; ++k) h[k] = __fadd_rn(v[k].h, v[k].l);
    if (FULL) {
        st_floats<K>(dst + i0, h);
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k)
            if (i0 + k < n) dst[i0 + k] = h[k];
    }
}

template <int MODE, int TR, int PREC, int K, bool FULL, bool REC = false>
__device__ __forceinline__ void group_finish(uint32_t i0, uint32_t n, const StepParams &p, const StateIO &io,
                                             V (&x2)[K], const PassRecord &rec = PassRecord{}) {
    if (MODE == 1) {
        V x1[K], x3[K], x4[K], x5[K];
        vload_k<PREC, K, FULL>(io.in[0], io.lin[0], i0, n, x1);
        vload_k<PREC, K, FULL>(io.in[2], io.lin[2], i0, n, x3);
        vload_k<PREC, K, FULL>(io.in[3], io.lin[3], i0, n, x4);
        vload_k<PREC, K, FULL>(io.in[4], io.lin[4], i0, n, x5);
#pragma unroll
        for (int k = 0; k < K; ++k) vround<PREC>(x2[k]);
        if (REC) {
            record_k<K, FULL>(rec.x, i0, n, x1);
            record_k<K, FULL>(rec.x + rec.npad, i0, n, x2);
            record_k<K, FULL>(rec.x + 2 * rec.npad, i0, n, x3);
            record_k<K, FULL>(rec.x + 3 * rec.npad, i0, n, x4);
            record_k<K, FULL>(rec.x + 4 * rec.npad, i0, n, x5);
        }
#pragma unroll
        for (int k = 0; k < K; ++k) transform_n<TR, PREC>(x1[k], x2[k], x3[k], x4[k], x5[k], p);
        if (REC) record_k<K, FULL>(rec.y2, i0, n, x2);
        vstore_k<PREC, K, FULL>(io.out[0], io.lout[0], i0, n, x1);
        vstore_k<PREC, K, FULL>(io.out[1], io.lout[1], i0, n, x2);
        vstore_k<PREC, K, FULL>(io.out[2], io.lout[2], i0, n, x3);
        vstore_k<PREC, K, FULL>(io.out[3], io.lout[3], i0, n, x4);
        vstore_k<PREC, K, FULL>(io.out[4], io.lout[4], i0, n, x5);
    } else {
        vstore_k<PREC, K, FULL>(io.out[1], io.lout[1], i0, n, x2);
    }
}

// First half of the sparse fused pass (MODE 4, unit conductances, compensated state) for a full
// group of four nodes, in packed pairs (0, 1) and (2, 3): the flux sum in slot order -x, +x, -y, +y,
// -z, +z (an absent neighbour carries the node's own value, adding +0), Scheme 1's increment by
// TwoSum, the rounding of vround, and the store of MODE 4 (a marked node's rounded pair itself, the
// others renormalised as vstore).  Every lane does the scalar path's operations in its order, so the
// results are the same bits.  REC: also writes h + l of the rounded pairs to rec_y2 (the adjoint's
// record of the diffused DOM; at an unmarked node it is also the transformed DOM).
template <bool REC = false>
__device__ __forceinline__ void dom4_packed(uint32_t i0, const uint32_t (&ty)[4], const float (&y)[4], float yl,
                                            float yr, const float (&ym)[4], const float (&yp)[4], const float (&zv)[4],
                                            const float (&zw)[4], const V (&x2)[4], uint32_t act_bits,
                                            const StepParams &p, const StateIO &io, float *rec_y2 = nullptr) {
    float xm[4], xp[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        xm[k] = ((ty[k] >> 15) & 1u) ? (k == 0 ? yl : y[k > 0 ? k - 1 : 0]) : y[k];
        xp[k] = (ty[k] >> 31) ? (k == 3 ? yr : y[k < 3 ? k + 1 : 0]) : y[k];
    }
    float hw[4], hr[4];
    uint32_t qw[2];
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
        const int a = 2 * h2, b = a + 1;
        const float2 Y = make_float2(y[a], y[b]);
        float2 acc = make_float2(0.0f, 0.0f);
        acc = add2_rn(acc, sub2_rn(Y, make_float2(xm[a], xm[b])));
        acc = add2_rn(acc, sub2_rn(Y, make_float2(xp[a], xp[b])));
        acc = add2_rn(acc, sub2_rn(Y, make_float2(ym[a], ym[b])));
        acc = add2_rn(acc, sub2_rn(Y, make_float2(yp[a], yp[b])));
        acc = add2_rn(acc, sub2_rn(Y, make_float2(zv[a], zv[b])));
        acc = add2_rn(acc, sub2_rn(Y, make_float2(zw[a], zw[b])));
        // Scheme 1: -D dt sum_j (y_i - y_j), in scalar (see add2_rn: a packed product would be fused)
        const float2 d = make_float2(__fmul_rn(-p.c, acc.x), __fmul_rn(-p.c, acc.y));
        float2 H = Y, L = make_float2(x2[a].l, x2[b].l);
        // vadd: TwoSum, the rounding error into the residual
        float2 s = add2_rn(H, d);
        const float2 bp = sub2_rn(s, H);
        const float2 e = add2_rn(sub2_rn(H, sub2_rn(s, bp)), sub2_rn(d, bp));
        L = add2_rn(L, e);
        H = s;
        // vround: as if stored and loaded
        s = add2_rn(H, L);
        const float2 r = add2_rn(sub2_rn(H, s), L);
        const uint32_t rq = bf16x2_bits(r.x, r.y);
        L = make_float2(__uint_as_float(rq << 16), __uint_as_float(rq & 0xffff0000u));
        H = s;
        // store: renormalised (unmarked) or the rounded pair itself (marked)
        const float2 hn = add2_rn(H, L);
        const float2 rn = add2_rn(sub2_rn(H, hn), L);
        const uint32_t qn = bf16x2_bits(rn.x, rn.y);
        const bool ma = (act_bits >> a) & 1u, mb = (act_bits >> b) & 1u;
        hw[a] = ma ? H.x : hn.x;
        hw[b] = mb ? H.y : hn.y;
        hr[a] = hn.x;
        hr[b] = hn.y;
        qw[h2] = ((ma ? rq : qn) & 0xffffu) | ((mb ? rq : qn) & 0xffff0000u);
    }
    st_floats<4>(io.out[1] + i0, hw);
    *reinterpret_cast<uint2 *>(io.lout[1] + i0) = make_uint2(qw[0], qw[1]);
    if (REC) st_floats<4>(rec_y2 + i0, hr);
}

// K consecutive nodes per thread (i0 a multiple of K, K = 2 or 4): table_node for nodes i0 ..
// i0 + K - 1, the per-node streams (offset table, block ids, the five compartments) read and
// written as 8- or 16-byte FP32 / table vectors and 4- or 8-byte residual vectors, so a warp moves
// 32 K nodes per memory instruction.  Groups with all K nodes take a branch-free vector path; only
// the last group of the range takes the per-node path.  The -x neighbour of the first node is the
// previous lane's last node and the +x neighbour of the last node the next lane's first node.
// Arithmetic and slot order per node are those of table_node, so the results are the same bits.
// Rows and tables start on 16-byte boundaries (row strides are multiples of 64 values).  REC: also
// writes the pass record of the discrete adjoint (MODE 1: X and the transformed DOM; MODE 4: h + l of
// every node's rounded DOM pair into rec.y2, which the second half overwrites at the marked nodes
// with their transformed DOM).  MODE 4 is the first half of
// the sparse fused pass: the DOM of every node is diffused and rounded as in MODE 1; a node whose
// bit in the activity mask is clear has its DOM stored as MODE 1 stores a DOM that the (identity)
// transformation left unchanged, a marked node the rounded pair itself (the second half, over the
// marked nodes in rank order, reads it back exactly as MODE 1 holds it in registers).  Must be
// called by all 32 lanes of a warp.
template <int MODE, int WM, int TR, int PREC, int TF, int K, bool REC = false>
__device__ __forceinline__ void table_vec(uint32_t i0, uint32_t n, const NbrTable &tb, const BlockTable &bt,
                                          const StepParams &p, const StateIO &io,
                                          const PassRecord &rec = PassRecord{}, const SparseState &ss = SparseState{}) {
    const bool full = i0 + K <= n;
    const float *__restrict__ Y2 = io.in[1];
    uint32_t ty[K], zm[K], zp[K], bn[K];
    V x2[K];
    if (full) group_load<WM, PREC, TF, K, true>(i0, n, tb, bt, io, ty, zm, zp, bn, x2);
    else group_load<WM, PREC, TF, K, false>(i0, n, tb, bt, io, ty, zm, zp, bn, x2);
    uint32_t act_bits = 0u;  // MODE 4: activity bits of the group
    if (MODE == 4 && i0 < n) act_bits = (__ldg(ss.mask + (i0 >> 5)) >> (i0 & 31)) & ((1u << K) - 1u);
    float y[K];
#pragma unroll
    for (int k = 0; k < K; ++k) y[k] = x2[k].h;
    const int lane = threadIdx.x & 31;
    float yl = __shfl_up_sync(0xffffffffu, y[K - 1], 1);  // node i0 - 1
    float yr = __shfl_down_sync(0xffffffffu, y[0], 1);    // node i0 + K
    if (lane == 0 && ((ty[0] >> 15) & 1u)) yl = __ldg(Y2 + (i0 - 1));
    if (lane == 31 && (ty[K - 1] >> 31)) yr = __ldg(Y2 + (i0 + K));
    // an absent neighbour reads the node's own value: the scalar path below skips it, the packed
    // path adds y - y = +0, which leaves a sum that starts at +0 unchanged (it is never -0)
    float ym[K], yp[K], zv[K], zw[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const uint32_t dym = ty[k] & 0x7fffu, dyp = (ty[k] >> 16) & 0x7fffu;
        ym[k] = dym ? __ldg(Y2 + (i0 + k - dym)) : y[k];
        yp[k] = dyp ? __ldg(Y2 + (i0 + k + dyp)) : y[k];
        zv[k] = zm[k] ? __ldg(Y2 + (i0 + k - zm[k])) : y[k];
        zw[k] = zp[k] ? __ldg(Y2 + (i0 + k + zp[k])) : y[k];
    }
    if (i0 >= n) return;
    if constexpr (MODE == 4 && WM == W_UNIT && PREC == P_COMP && K == 4) {
        if (full) {
            dom4_packed<REC>(i0, ty, y, yl, yr, ym, yp, zv, zw, x2, act_bits, p, io, rec.y2);
            return;
        }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float acc = 0.0f;
        if (WM == W_BLOCK) {  // every slot, branch-free: an absent one adds g * (+0), which changes nothing
            const float nb[6] = {((ty[k] >> 15) & 1u) ? (k == 0 ? yl : y[k > 0 ? k - 1 : 0]) : y[k],
                                 (ty[k] >> 31) ? (k == K - 1 ? yr : y[k < K - 1 ? k + 1 : 0]) : y[k],
                                 ym[k], yp[k], zv[k], zw[k]};
#pragma unroll
            for (int d = 0; d < 6; ++d) acc = __fmaf_rn(table_theta_sel(bt, bn[k], d), __fsub_rn(y[k], nb[d]), acc);
        } else {
            auto add = [&](float yj) { acc = __fadd_rn(acc, __fsub_rn(y[k], yj)); };
            if ((ty[k] >> 15) & 1u) add(k == 0 ? yl : y[k > 0 ? k - 1 : 0]);
            if (ty[k] >> 31) add(k == K - 1 ? yr : y[k < K - 1 ? k + 1 : 0]);
            if (ty[k] & 0x7fffu) add(ym[k]);
            if ((ty[k] >> 16) & 0x7fffu) add(yp[k]);
            if (zm[k]) add(zv[k]);
            if (zp[k]) add(zw[k]);
        }
        vadd<PREC>(x2[k], __fmul_rn(-p.c, acc));  // Scheme 1
    }
    if (MODE == 4) {
        float h[K], hr[K];
        res_t q[K];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            vround<PREC>(x2[k]);
            hr[k] = __fadd_rn(x2[k].h, x2[k].l);  // REC: the adjoint's record of the rounded pair
            if ((act_bits >> k) & 1u) {  // the rounded pair itself
                h[k] = x2[k].h;
                q[k] = PREC == P_COMP ? res_encode(x2[k].l, h[k]) : (res_t)0;
            } else if (PREC == P_COMP) {  // renormalised as vstore does
                h[k] = __fadd_rn(x2[k].h, x2[k].l);
                q[k] = res_encode(__fadd_rn(__fsub_rn(x2[k].h, h[k]), x2[k].l), h[k]);
            } else {
                h[k] = x2[k].h;
            }
        }
        if (full) {
            st_floats<K>(io.out[1] + i0, h);
            if (PREC == P_COMP) st_res<K>(io.lout[1] + i0, q);
            if (REC) st_floats<K>(rec.y2 + i0, hr);
        } else {
#pragma unroll
            for (int k = 0; k < K; ++k)
                if (i0 + k < n) {
                    io.out[1][i0 + k] = h[k];
                    if (PREC == P_COMP) io.lout[1][i0 + k] = q[k];
                    if (REC) rec.y2[i0 + k] = hr[k];
                }
        }
        return;
    }
    if (full) group_finish<MODE, TR, PREC, K, true, REC>(i0, n, p, io, x2, rec);
    else group_finish<MODE, TR, PREC, K, false, REC>(i0, n, p, io, x2, rec);
}

}  // namespace vga
