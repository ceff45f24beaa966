// Chunk decoding and neighbour walk shared by every stencil kernel.
//
// A block owns the chunk of nodes [v0, v0 + nv).  decode_chunk() scans the row-bitmask words of the
// rows the chunk spans and writes, for each of its nodes, x | (boundary flags << 16) and the image
// row into shared memory (and y | z << 16 when the caller needs block coordinates).  Boundary flag
// bits: 1 = y > 0, 2 = y < ny-1, 4 = z > 0, 8 = z < nz-1.
#pragma once

#include "physics.cuh"
#include "vga_internal.cuh"

namespace vga {

template <bool NEED_YZ>
__device__ __forceinline__ int32_t decode_chunk(const Topo &t, const int32_t *__restrict__ chunk_row, int32_t cap,
                                                uint32_t *s_x, uint32_t *s_row, uint32_t *s_yz, int64_t &v0_out) {
    const int64_t v0 = (int64_t)blockIdx.x * cap;
    const int64_t v1 = min(v0 + (int64_t)cap, t.n);
    const int32_t nv = (int32_t)(v1 - v0);
    const int32_t r0 = chunk_row[blockIdx.x], r1 = chunk_row[blockIdx.x + 1];
    const int32_t nw = (r1 - r0 + 1) * t.W;
    for (int32_t q = threadIdx.x; q < nw; q += blockDim.x) {
        const int32_t rr = q / t.W;
        const int32_t w = q - rr * t.W;
        const int32_t r = r0 + rr;
        const int32_t wq = r * t.W + w;
        uint32_t m = __ldg(t.mask + wq);
        if (!m) continue;
        const int64_t p0 = __ldg(t.pre + wq);
        if (p0 >= v1 || p0 + __popc(m) <= v0) continue;
        const int32_t z = r / t.ny, y = r - z * t.ny;
        const uint32_t fl = (uint32_t)(y > 0) | ((uint32_t)(y < t.ny - 1) << 1) | ((uint32_t)(z > 0) << 2) |
                            ((uint32_t)(z < t.nz - 1) << 3);
        int64_t idx = p0 - v0;
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            if (idx >= 0 && idx < nv) {
                s_x[idx] = (uint32_t)(32 * w + b) | (fl << 16);
                s_row[idx] = (uint32_t)r;
                if (NEED_YZ) s_yz[idx] = (uint32_t)y | ((uint32_t)z << 16);
            }
            ++idx;
        }
    }
    __syncthreads();
    v0_out = v0;
    return nv;
}

// Calls f(slot, j) for every existing neighbour j of node i (at x in image row r, boundary flags
// fl), in slot order -x, +x, -y, +y, -z, +z.
template <class F>
__device__ __forceinline__ void for_each_neighbour(const Topo &t, int64_t i, int32_t x, int32_t r, uint32_t fl, F &&f) {
    if (x > 0 && is_node(t, r, x - 1)) f(0, i - 1);
    if (x < t.nx - 1 && is_node(t, r, x + 1)) f(1, i + 1);
    if (fl & 1u) {
        const int64_t j = node_in_row(t, r - 1, x);
        if (j >= 0) f(2, j);
    }
    if (fl & 2u) {
        const int64_t j = node_in_row(t, r + 1, x);
        if (j >= 0) f(3, j);
    }
    if (fl & 4u) {
        const int64_t j = node_in_row(t, r - t.ny, x);
        if (j >= 0) f(4, j);
    }
    if (fl & 8u) {
        const int64_t j = node_in_row(t, r + t.ny, x);
        if (j >= 0) f(5, j);
    }
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

}  // namespace vga
