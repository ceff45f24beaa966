// Temporally blocked sparse fused passes: up to K time steps of Scheme 1 (Sec. II.B.3a) fused
// with the transformation (Sec. II.C eq. 3) per launch, over tiles of the image staged in shared
// memory with a K-voxel halo.
//
// Layout.  The image is cut into tiles of 32 x TY x TZ voxels (32 = one row-bitmask word in x).
// During a step call the DOM (value and residual) is held in *tile order*: the nodes of tile T are
// contiguous, in raster order inside the tile, starting at tstart[T] (a multiple of 8 nodes, so a
// tile's range is a 16-byte aligned block for the bulk copies).  tpos[q] is the tile-order position
// of the first node of mask word q; the permutation between raster order and tile order copies
// whole words' runs (k_perm_in / k_perm_out), once per step call.
//
// One CTA advances one tile by up to K passes.  Shared memory holds the DOM of the tile and of its
// halo (the voxels within K of the tile in each coordinate), compacted: the tile's own nodes first
// (one bulk copy, tile order), then the halo rows grouped by their distance rho from the tile, each
// row as its parts L (the K voxels left of the tile), M (the 32 voxels of the tile's column) and R
// (the K voxels to its right).  Every node gets the shared-memory slots of its six neighbours once
// per launch; an absent neighbour points at the node itself (y - y = +0 leaves the flux sum
// unchanged: the sum starts at +0 and round-to-nearest addition never makes it -0).  Pass s of a
// launch of S passes recomputes the nodes of rows within distance S - s of the tile (the halo
// shrinks by one voxel per pass, so every value it reads is exact), and the marked nodes of the
// sparse pass (MB, SOM, FOM or CO2 nonzero) are transformed from a list in shared memory.  Per node
// the arithmetic is that of the two-kernel sparse pass (stencil.cuh MODE 4, then
// k_transform_compact), so the results are the same bits for finite states.
//
// Tiles whose tile-plus-halo node count exceeds the capacity of the two-blocks-per-SM instance run
// in a second launch with twice the capacity (one block per SM).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "physics.cuh"
#include "stencil.cuh"
#include "tma.cuh"
#include "vga_internal.cuh"

namespace vga {

namespace {

constexpr int kPT = 256;  // threads of the layout kernels

// Tile geometry of the current layout (shared by every kernel here).
struct TileGrid {
    int32_t W, ny, nz, TY, TZ, NTY, NTZ;
    __host__ __device__ int64_t ntiles() const { return (int64_t)W * NTY * NTZ; }
    __device__ void coords(int64_t T, int32_t &tx, int32_t &ty, int32_t &tz) const {
        tx = (int32_t)(T % W);
        ty = (int32_t)((T / W) % NTY);
        tz = (int32_t)(T / ((int64_t)W * NTY));
    }
};

// Bits of a region row's part p: L = bits [32 - K, 32) of the word left of the tile column, M = the
// tile column's word, R = bits [0, K) of the word to its right.
__host__ __device__ __forceinline__ uint32_t part_bits(int p, int K) {
    return p == 0 ? (0xffffffffu << (32 - K)) : (p == 1 ? 0xffffffffu : ((1u << K) - 1u));
}
// First bit of part p, and the bits of a word below bit b (b in [0, 31]).
__host__ __device__ __forceinline__ int part_first(int p, int K) { return p == 0 ? 32 - K : 0; }
__device__ __forceinline__ uint32_t below(int b) { return (1u << b) - 1u; }

__device__ __forceinline__ int32_t block_sum_i32(int32_t s) {
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ int32_t ws[32];
    __syncthreads();
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    int32_t t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += ws[w];
    return t;  // valid in thread 0
}

// Node count of every tile (popcounts of its words), and the same rounded up to a multiple of 8.
__global__ void __launch_bounds__(kPT) k_tile_count(TileGrid g, const uint32_t *__restrict__ mask,
                                                    int32_t *__restrict__ cnt, int32_t *__restrict__ cnt8) {
    int32_t tx, ty, tz;
    g.coords(blockIdx.x, tx, ty, tz);
    int32_t s = 0;
    for (int32_t lr = threadIdx.x; lr < g.TY * g.TZ; lr += blockDim.x) {
        const int32_t y = ty * g.TY + lr % g.TY, z = tz * g.TZ + lr / g.TY;
        if (y < g.ny && z < g.nz) s += __popc(__ldg(mask + ((int64_t)z * g.ny + y) * g.W + tx));
    }
    const int32_t t = block_sum_i32(s);
    if (threadIdx.x == 0) {
        cnt[blockIdx.x] = t;
        cnt8[blockIdx.x] = (t + 7) & ~7;
    }
}

// Exclusive prefix of v[0 .. m) into out[0 .. m] (out[m] = total), one block.
__global__ void __launch_bounds__(1024) k_scan_i32(int64_t m, const int32_t *__restrict__ v, int32_t *__restrict__ out) {
    __shared__ int32_t part[1024];
    const int64_t per = (m + 1023) / 1024, a = threadIdx.x * per, b = min(m, a + per);
    int32_t sum = 0;
    for (int64_t i = a; i < b; ++i) sum += v[i];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int32_t t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    int32_t run = part[threadIdx.x] - sum;
    for (int64_t i = a; i < b; ++i) {
        out[i] = run;
        run += v[i];
    }
    if (threadIdx.x == 1023) out[m] = part[1023];
}

// tpos of every word of tile T: tstart[T] plus the nodes of the tile's earlier rows (raster order
// inside the tile).
__global__ void __launch_bounds__(kPT) k_tile_pos(TileGrid g, const uint32_t *__restrict__ mask,
                                                  const int32_t *__restrict__ tstart, int32_t *__restrict__ tpos) {
    int32_t tx, ty, tz;
    g.coords(blockIdx.x, tx, ty, tz);
    const int32_t rows = g.TY * g.TZ;
    const int32_t per = (rows + kPT - 1) / kPT, a = threadIdx.x * per, b = min(rows, a + per);
    int32_t sum = 0;
    for (int32_t lr = a; lr < b; ++lr) {
        const int32_t y = ty * g.TY + lr % g.TY, z = tz * g.TZ + lr / g.TY;
        if (y < g.ny && z < g.nz) sum += __popc(__ldg(mask + ((int64_t)z * g.ny + y) * g.W + tx));
    }
    __shared__ int32_t part[kPT];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (int off = 1; off < kPT; off <<= 1) {
        const int32_t t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += t;
        __syncthreads();
    }
    int32_t run = tstart[blockIdx.x] + part[threadIdx.x] - sum;
    for (int32_t lr = a; lr < b; ++lr) {
        const int32_t y = ty * g.TY + lr % g.TY, z = tz * g.TZ + lr / g.TY;
        if (y < g.ny && z < g.nz) {
            const int64_t q = ((int64_t)z * g.ny + y) * g.W + tx;
            tpos[q] = run;
            run += __popc(__ldg(mask + q));
        }
    }
}

// Node count of the tile-plus-halo region of every tile (halo K), and with amask (the activity
// mask over raster node indices) its marked nodes.
__global__ void __launch_bounds__(kPT) k_tile_region(TileGrid g, int32_t K, const uint32_t *__restrict__ mask,
                                                     const int32_t *__restrict__ pre, const uint32_t *__restrict__ amask,
                                                     int32_t *__restrict__ rcnt, int32_t *__restrict__ rmarked) {
    int32_t tx, ty, tz;
    g.coords(blockIdx.x, tx, ty, tz);
    const int32_t RY = g.TY + 2 * K, RZ = g.TZ + 2 * K;
    int32_t s = 0, sm = 0;
    for (int32_t rr = threadIdx.x; rr < RY * RZ; rr += blockDim.x) {
        const int32_t y = ty * g.TY - K + rr % RY, z = tz * g.TZ - K + rr / RY;
        if (y < 0 || y >= g.ny || z < 0 || z >= g.nz) continue;
        for (int p = 0; p < 3; ++p) {
            const int32_t w = tx + p - 1;
            if (w < 0 || w >= g.W) continue;
            const int64_t q = ((int64_t)z * g.ny + y) * g.W + w;
            const uint32_t mf = __ldg(mask + q);
            const int32_t cnt = __popc(mf & part_bits(p, K));
            s += cnt;
            if (amask && cnt) {
                const int64_t r0 = (int64_t)__ldg(pre + q) + __popc(mf & below(part_first(p, K)));
                for (int t = 0; t < cnt; ++t) {
                    const int64_t i = r0 + t;
                    sm += (int32_t)((__ldg(amask + (i >> 5)) >> (i & 31)) & 1u);
                }
            }
        }
    }
    const int32_t t = block_sum_i32(s);
    const int32_t tm = block_sum_i32(sm);
    if (threadIdx.x == 0) {
        if (rcnt) rcnt[blockIdx.x] = t;
        if (rmarked) rmarked[blockIdx.x] = tm;
    }
}

// ---- permutation between raster order and tile order (DOM value and residual) ---------------

// Tile order <- raster order, one thread per tile row (consecutive threads write consecutive runs).
template <int PREC>
__global__ void __launch_bounds__(kPT) k_perm_in(TileGrid g, const uint32_t *__restrict__ mask,
                                                 const int32_t *__restrict__ pre, const int32_t *__restrict__ tpos,
                                                 const float *__restrict__ h, const res_t *__restrict__ l,
                                                 float *__restrict__ th, res_t *__restrict__ tl) {
    const int64_t rows = (int64_t)g.TY * g.TZ;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= g.ntiles() * rows) return;
    const int64_t T = k / rows;
    const int32_t lr = (int32_t)(k - T * rows);
    int32_t tx, ty, tz;
    g.coords(T, tx, ty, tz);
    const int32_t y = ty * g.TY + lr % g.TY, z = tz * g.TZ + lr / g.TY;
    if (y >= g.ny || z >= g.nz) return;
    const int64_t q = ((int64_t)z * g.ny + y) * g.W + tx;
    const int32_t cnt = __popc(__ldg(mask + q));
    const int64_t s = __ldg(pre + q), d = __ldg(tpos + q);
    for (int32_t t = 0; t < cnt; ++t) {
        th[d + t] = __ldg(h + s + t);
        if (PREC == P_COMP) tl[d + t] = __ldg(l + s + t);
    }
}

// Raster order <- tile order, one thread per mask word in raster order.
template <int PREC>
__global__ void __launch_bounds__(kPT) k_perm_out(int64_t nwords, const uint32_t *__restrict__ mask,
                                                  const int32_t *__restrict__ pre, const int32_t *__restrict__ tpos,
                                                  const float *__restrict__ th, const res_t *__restrict__ tl,
                                                  float *__restrict__ h, res_t *__restrict__ l) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nwords) return;
    const int32_t cnt = __popc(__ldg(mask + q));
    if (!cnt) return;
    const int64_t s = __ldg(tpos + q), d = __ldg(pre + q);
    for (int32_t t = 0; t < cnt; ++t) {
        h[d + t] = __ldg(th + s + t);
        if (PREC == P_COMP) l[d + t] = __ldg(tl + s + t);
    }
}

// ---- the blocked pass ------------------------------------------------------------------------

struct BlockArgs {
    TileGrid g;
    const uint32_t *mask;    // row bitmask
    const int32_t *pre;      // raster index of each word's first node
    const int32_t *tpos;     // tile-order position of each word's first node
    const int32_t *tstart;   // ntiles + 1 (multiples of 8)
    const int32_t *tcnt;     // node count of each tile
    const int32_t *tiles;    // the tiles of this launch
    const uint16_t *rorder;  // region rows sorted by rho (stable in raster order)
    const float *hin;
    const res_t *lin;
    float *hout;
    res_t *lout;
    SparseState ss;          // activity mask and prefix; compact state read (h, l)
    float *cout_h[4];        // compact state written (own marked nodes)
    res_t *cout_l[4];
    StepParams p;
    int32_t steps;           // passes of this launch, 1 .. K
    int32_t *err;
};

template <int TY, int TZ, int K, int CAP, int MCAP, int NT>
struct BlockSmem {
    static constexpr int RY = TY + 2 * K, RZ = TZ + 2 * K, NR = RY * RZ;
    static constexpr size_t h0 = 0;
    static constexpr size_t h1 = h0 + 4 * (size_t)CAP;
    static constexpr size_t l = h1 + 4 * (size_t)CAP;
    static constexpr size_t nb = l + 2 * (size_t)CAP;                  // 6 x CAP uint16 (byte offsets)
    static constexpr size_t rmask = nb + 12 * (size_t)CAP;             // 3 x NR uint32
    static constexpr size_t rbase = rmask + 12 * (size_t)NR;           // 3 x NR uint16
    static constexpr size_t mh = (rbase + 6 * (size_t)NR + 15) & ~(size_t)15;  // 4 x MCAP float
    static constexpr size_t ml = mh + 16 * (size_t)MCAP;               // 4 x MCAP res_t
    static constexpr size_t mrank = ml + 8 * (size_t)MCAP;             // MCAP uint32
    static constexpr size_t mslot = mrank + 4 * (size_t)MCAP;          // MCAP uint16
    static constexpr size_t scan = (mslot + 2 * (size_t)MCAP + 15) & ~(size_t)15;  // NT/32 int32
    static constexpr size_t misc = scan + 4 * (size_t)(NT / 32);       // group ends (K+1), mcount
    static constexpr size_t bar = (misc + 4 * (size_t)(K + 4) + 7) & ~(size_t)7;
    static constexpr size_t bytes = bar + 8;
    static_assert(4 * (CAP - 1) <= 32767, "slot byte offsets must fit 15 bits");
    static_assert(NR <= NT, "one region row per thread");
    static_assert(K >= 1 && K <= 8, "halo width");
};

// rho of a region row coordinate d (0 .. T + 2K - 1): distance to the tile's range [K, K + T).
__device__ __forceinline__ int ring_of(int d, int T, int K) { return d < K ? K - d : (d >= K + T ? d - K - T + 1 : 0); }

// Compensated renormalisation as vstore does: h = RN(h + l) and the remainder as stored residual.
template <int PREC>
__device__ __forceinline__ void renorm(const V &v, float &h, res_t &q) {
    if (PREC == P_COMP) {
        h = __fadd_rn(v.h, v.l);
        q = res_encode(__fadd_rn(__fsub_rn(v.h, h), v.l), h);
    } else {
        h = v.h;
        q = 0;
    }
}

template <int PREC>
__device__ __forceinline__ float lsm_decode(res_t q) {
    return PREC == P_COMP ? res_decode(q, 0.0f) : 0.0f;
}

// Phase A of one pass over slots [0, end): diffuse (Scheme 1) the DOM held in hc into hn.
template <int PREC, int CAP>
__device__ __forceinline__ void pass_diffuse(const unsigned char *sb, size_t hc_off, size_t hn_off, res_t *lsm,
                                             const uint16_t *nb, int end, float c, int NT) {
    const float *hc = reinterpret_cast<const float *>(sb + hc_off);
    float *hn = reinterpret_cast<float *>(const_cast<unsigned char *>(sb) + hn_off);
    for (int slot = threadIdx.x; slot < end; slot += NT) {
        uint32_t o0 = nb[slot];
        const bool marked = (o0 >> 15) & 1u;
        o0 &= 0x7fffu;
        const uint32_t o1 = nb[CAP + slot], o2 = nb[2 * CAP + slot], o3 = nb[3 * CAP + slot],
                       o4 = nb[4 * CAP + slot], o5 = nb[5 * CAP + slot];
        const float y = hc[slot];
        const unsigned char *hb = sb + hc_off;
        float acc = 0.0f;  // slot order -x, +x, -y, +y, -z, +z; absent neighbours are the node itself
        acc = __fadd_rn(acc, __fsub_rn(y, *reinterpret_cast<const float *>(hb + o0)));
        acc = __fadd_rn(acc, __fsub_rn(y, *reinterpret_cast<const float *>(hb + o1)));
        acc = __fadd_rn(acc, __fsub_rn(y, *reinterpret_cast<const float *>(hb + o2)));
        acc = __fadd_rn(acc, __fsub_rn(y, *reinterpret_cast<const float *>(hb + o3)));
        acc = __fadd_rn(acc, __fsub_rn(y, *reinterpret_cast<const float *>(hb + o4)));
        acc = __fadd_rn(acc, __fsub_rn(y, *reinterpret_cast<const float *>(hb + o5)));
        V x2 = {y, lsm_decode<PREC>(lsm[slot])};
        vadd<PREC>(x2, __fmul_rn(-c, acc));  // Scheme 1
        vround<PREC>(x2);
        float hw;
        res_t qw = 0;
        if (marked) {  // the rounded pair itself: the transformation reads it back
            hw = x2.h;
            if (PREC == P_COMP) qw = res_encode(x2.l, hw);
        } else {
            renorm<PREC>(x2, hw, qw);
        }
        hn[slot] = hw;
        if (PREC == P_COMP) lsm[slot] = qw;
    }
}

template <int TY, int TZ, int K, int CAP, int MCAP, int NT, int TR, int PREC>
__global__ void __launch_bounds__(NT, (NT <= 512 ? 2 : 1)) k_dom_block(BlockArgs a) {
    using L = BlockSmem<TY, TZ, K, CAP, MCAP, NT>;
    constexpr int RY = L::RY, RZ = L::RZ, NR = L::NR;
    extern __shared__ __align__(128) unsigned char sb[];
    float *h0 = reinterpret_cast<float *>(sb + L::h0);
    res_t *lsm = reinterpret_cast<res_t *>(sb + L::l);
    uint16_t *nb = reinterpret_cast<uint16_t *>(sb + L::nb);
    uint32_t *rmask = reinterpret_cast<uint32_t *>(sb + L::rmask);
    uint16_t *rbase = reinterpret_cast<uint16_t *>(sb + L::rbase);
    float *mh = reinterpret_cast<float *>(sb + L::mh);
    res_t *ml = reinterpret_cast<res_t *>(sb + L::ml);
    uint32_t *mrank = reinterpret_cast<uint32_t *>(sb + L::mrank);
    uint16_t *mslot = reinterpret_cast<uint16_t *>(sb + L::mslot);
    int32_t *wscan = reinterpret_cast<int32_t *>(sb + L::scan);
    int32_t *gend = reinterpret_cast<int32_t *>(sb + L::misc);  // K + 1 group ends, then mcount
    int32_t *mcount = gend + K + 1;
    uint64_t *bar = reinterpret_cast<uint64_t *>(sb + L::bar);

    const TileGrid &g = a.g;
    const int64_t T = a.tiles[blockIdx.x];
    int32_t tx, ty, tz;
    g.coords(T, tx, ty, tz);
    const int32_t ts = __ldg(a.tstart + T);
    const int32_t own_pad = __ldg(a.tstart + T + 1) - ts;
    const int32_t own_cnt = __ldg(a.tcnt + T);
    const int tid = threadIdx.x;

    // own nodes: one bulk copy of the value and residual ranges (16-byte multiples)
    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
        *mcount = 0;
    }
    __syncthreads();
    if (tid == 0 && own_pad > 0) {
        const uint32_t hb = (uint32_t)own_pad * 4u, lb = PREC == P_COMP ? (uint32_t)own_pad * 2u : 0u;
        mbar_arrive_expect_tx(bar, hb + lb);
        bulk_g2s(h0, a.hin + ts, hb, bar);
        if (PREC == P_COMP) bulk_g2s(lsm, a.lin + ts, lb, bar);
    }

    // ---- R1: one region row per thread, in rho order: masks, positions, slot bases ----
    // During the decode the h1 buffer holds a descriptor per slot and the neighbour-slot area holds
    // the global start of every halo run (both are written for real only afterwards).
    uint32_t *desc = reinterpret_cast<uint32_t *>(sb + L::h1);
    uint32_t *gstart = reinterpret_cast<uint32_t *>(sb + L::nb);
    const int j = tid;
    int rr = 0, rho = K + 1;
    bool valid = false;
    uint32_t mf[3] = {0u, 0u, 0u}, am[3] = {0u, 0u, 0u};
    int32_t tp[3] = {0, 0, 0}, pr[3] = {0, 0, 0};
    int size = 0;
    if (j < NR) {
        rr = a.rorder[j];
        const int dz = rr / RY, dy = rr - dz * RY;
        rho = max(ring_of(dy, TY, K), ring_of(dz, TZ, K));
        const int32_t y = ty * TY - K + dy, z = tz * TZ - K + dz;
        valid = y >= 0 && y < g.ny && z >= 0 && z < g.nz;
        if (valid) {
            // every load of the row at once: mask words, tile-order and raster positions
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                const int32_t w = tx + p - 1;
                if (w < 0 || w >= g.W) continue;
                const int64_t q = ((int64_t)z * g.ny + y) * g.W + w;
                mf[p] = __ldg(a.mask + q);
                tp[p] = __ldg(a.tpos + q);
                if (a.ss.mask) pr[p] = __ldg(a.pre + q);
            }
#pragma unroll
            for (int p = 0; p < 3; ++p) am[p] = mf[p] & part_bits(p, K);
        }
        size = __popc(am[0]) + __popc(am[2]) + (rho == 0 ? 0 : __popc(am[1]));
    }
    // exclusive scan of the halo sizes in rho order
    int incl = size;
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wscan[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int v = lane < NT / 32 ? wscan[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, v, o);
            if (lane >= o) v += u;
        }
        if (lane < NT / 32) wscan[lane] = v;  // inclusive warp totals
    }
    __syncthreads();
    const int excl = incl - size + (wid > 0 ? wscan[wid - 1] : 0);
    int base[3] = {0, 0, 0};
    if (j < NR) {
        const int hb0 = own_pad + excl;
        base[0] = hb0;
        if (rho == 0) {
            base[1] = valid ? tp[1] - ts : 0;  // the tile's own row: its place in the own range
            base[2] = hb0 + __popc(am[0]);
        } else {
            base[1] = hb0 + __popc(am[0]);
            base[2] = base[1] + __popc(am[1]);
        }
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            rmask[p * NR + rr] = am[p];
            rbase[p * NR + rr] = (uint16_t)base[p];
            gstart[p * NR + rr] = (uint32_t)(tp[p] + __popc(mf[p] & below(part_first(p, K))));
        }
        // the last row of each rho group closes it: slots [0, gend[rho]) are the groups <= rho
        const int last = (TY + 2 * rho) * (TZ + 2 * rho) - 1;
        if (rho <= K && j == last) gend[rho] = own_pad + excl + size;
    }

    // ---- R2: per row, the descriptor of each node's slot (row, part, bit, rank in the part) and
    // the marked nodes (their ranks follow from the row's first one: marked nodes in raster order
    // have consecutive ranks) ----
    if (j < NR && valid) {
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            uint32_t m = am[p];
            int t = 0;
            while (m) {
                const int b = __ffs(m) - 1;
                m &= m - 1u;
                desc[base[p] + t] = (uint32_t)rr | ((uint32_t)p << 10) | ((uint32_t)b << 12);
                ++t;
            }
        }
        if (a.ss.mask) {
            int before = 0;  // marked nodes of the row's earlier parts
            uint32_t rank0 = 0u;
            bool have_rank = false;
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                if (!am[p]) continue;
                const int cnt = __popc(am[p]);
                const int64_t r0 = (int64_t)pr[p] + __popc(mf[p] & below(part_first(p, K)));
                const int64_t w0 = r0 >> 5, w1 = (r0 + cnt - 1) >> 5;
                const uint32_t m0 = __ldg(a.ss.mask + w0);
                const uint64_t two = (uint64_t)m0 | (w1 != w0 ? (uint64_t)__ldg(a.ss.mask + w1) << 32 : 0ull);
                uint32_t act = (uint32_t)(two >> (r0 & 31)) & (cnt == 32 ? 0xffffffffu : ((1u << cnt) - 1u));
                if (!act) continue;
                if (!have_rank) {  // rank of the first marked node of the row
                    const int64_t i = r0 + (__ffs(act) - 1);
                    const uint32_t wm = (i >> 5) == w0 ? m0 : __ldg(a.ss.mask + (i >> 5));
                    rank0 = __ldg(a.ss.prefix + (i >> 5)) + __popc(wm & below((int)(i & 31)));
                    have_rank = true;
                }
                while (act) {
                    const int t = __ffs(act) - 1;
                    act &= act - 1u;
                    const int slot = base[p] + t;
                    const uint32_t rank = rank0 + (uint32_t)before;
                    ++before;
                    desc[slot] |= 1u << 31;
                    const int e = atomicAdd(mcount, 1);
                    if (e < MCAP) {
                        mslot[e] = (uint16_t)slot;
                        mrank[e] = rank;
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            mh[c * MCAP + e] = __ldg(a.ss.h[c] + rank);
                            ml[c * MCAP + e] = PREC == P_COMP ? __ldg(a.ss.l[c] + rank) : (res_t)0;
                        }
                    } else {
                        atomicExch(a.err, 3);
                    }
                }
            }
        }
    }
    // padding slots of the own range: inert (every neighbour is the slot itself)
    for (int s = own_cnt + tid; s < own_pad; s += NT) desc[s] = 1u << 30;
    __syncthreads();

    // ---- F1: halo values, four loads in flight per thread ----
    const int halo_end = gend[K];
    for (int s0 = own_pad + tid; s0 < halo_end; s0 += 4 * NT) {
        float hv[4];
        res_t lv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int s = s0 + u * NT;
            if (s < halo_end) {
                const uint32_t d = desc[s];
                const uint32_t rrr = d & 1023u, p = (d >> 10) & 3u;
                const int t = s - (int)rbase[p * NR + rrr];
                const uint32_t gi = gstart[p * NR + rrr] + (uint32_t)t;
                hv[u] = __ldg(a.hin + gi);
                lv[u] = PREC == P_COMP ? __ldg(a.lin + gi) : (res_t)0;
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int s = s0 + u * NT;
            if (s < halo_end) {
                h0[s] = hv[u];
                if (PREC == P_COMP) lsm[s] = lv[u];
            }
        }
    }
    __syncthreads();  // the run starts are read: the neighbour slots may overwrite them

    // ---- F2: the six neighbour slots of every node (byte offsets; absent = the node itself) ----
    for (int s = tid; s < halo_end; s += NT) {
        const uint32_t d = desc[s];
        int sx0 = s, sx1 = s, sn[4] = {s, s, s, s};
        if (!(d & (1u << 30))) {
            const int r = (int)(d & 1023u), p = (int)((d >> 10) & 3u), b = (int)((d >> 12) & 31u);
            const uint32_t m0 = rmask[r], m1 = rmask[NR + r], m2 = rmask[2 * NR + r];
            if (p == 1) {
                if (b > 0) { if ((m1 >> (b - 1)) & 1u) sx0 = s - 1; }
                else if (m0 >> 31) sx0 = (int)rbase[r] + __popc(m0) - 1;
                if (b < 31) { if ((m1 >> (b + 1)) & 1u) sx1 = s + 1; }
                else if (m2 & 1u) sx1 = (int)rbase[2 * NR + r];
            } else if (p == 0) {
                if (b > 32 - K && ((m0 >> (b - 1)) & 1u)) sx0 = s - 1;
                if (b < 31) { if ((m0 >> (b + 1)) & 1u) sx1 = s + 1; }
                else if (m1 & 1u) sx1 = (int)rbase[NR + r];
            } else {
                if (b > 0) { if ((m2 >> (b - 1)) & 1u) sx0 = s - 1; }
                else if (m1 >> 31) sx0 = (int)rbase[NR + r] + __popc(m1) - 1;
                if (b + 1 < K && ((m2 >> (b + 1)) & 1u)) sx1 = s + 1;
            }
            const int dz = r / RY, dy = r - dz * RY;
            const int nrr[4] = {dy > 0 ? r - 1 : -1, dy < RY - 1 ? r + 1 : -1, dz > 0 ? r - RY : -1,
                                dz < RZ - 1 ? r + RY : -1};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (nrr[q] < 0) continue;
                const uint32_t mm = rmask[p * NR + nrr[q]];
                if ((mm >> b) & 1u) sn[q] = (int)rbase[p * NR + nrr[q]] + __popc(mm & below(b));
            }
        }
        nb[s] = (uint16_t)(4 * sx0) | ((d >> 31) ? 0x8000u : 0u);
        nb[CAP + s] = (uint16_t)(4 * sx1);
        nb[2 * CAP + s] = (uint16_t)(4 * sn[0]);
        nb[3 * CAP + s] = (uint16_t)(4 * sn[1]);
        nb[4 * CAP + s] = (uint16_t)(4 * sn[2]);
        nb[5 * CAP + s] = (uint16_t)(4 * sn[3]);
    }
    // one thread waits for the bulk copy (bounded); the block barrier then publishes its data
    if (tid == 0) gend[K + 2] = (own_pad > 0) ? (int32_t)mbar_wait_bounded(bar, 0, a.err, 1) : 1;
    __syncthreads();
    if (!gend[K + 2]) return;  // timed out: the flag is set and the copies have drained
    const int nm = min(*mcount, MCAP);

    // ---- the passes ----
    const StepParams &p = a.p;
    const int steps = a.steps;
    for (int s = 1; s <= steps; ++s) {
        const int end = gend[steps - s];
        const bool odd = s & 1;  // pass s reads buffer (s - 1) & 1
        const size_t hc = odd ? L::h0 : L::h1, hn = odd ? L::h1 : L::h0;
        pass_diffuse<PREC, CAP>(sb, hc, hn, lsm, nb, end, p.c, NT);
        __syncthreads();
        if (nm > 0) {
            float *hnp = reinterpret_cast<float *>(sb + hn);
            for (int e = tid; e < nm; e += NT) {
                const int slot = mslot[e];
                if (slot >= end) continue;
                V x2 = {hnp[slot], lsm_decode<PREC>(lsm[slot])};
                V v[4];
#pragma unroll
                for (int c = 0; c < 4; ++c) v[c] = V{mh[c * MCAP + e], lsm_decode<PREC>(ml[c * MCAP + e])};
                transform_n<TR, PREC>(v[0], x2, v[1], v[2], v[3], p);
                float hw;
                res_t q;
                renorm<PREC>(x2, hw, q);
                hnp[slot] = hw;
                if (PREC == P_COMP) lsm[slot] = q;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    renorm<PREC>(v[c], hw, q);
                    mh[c * MCAP + e] = hw;
                    ml[c * MCAP + e] = q;
                }
            }
            __syncthreads();
        }
    }

    // ---- own nodes back: bulk stores of the final buffer; own marked nodes' compact state ----
    const float *hfin = reinterpret_cast<const float *>(sb + ((steps & 1) ? L::h1 : L::h0));
    for (int e = tid; e < nm; e += NT) {
        if (mslot[e] >= own_pad) continue;
        const uint32_t r = mrank[e];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            a.cout_h[c][r] = mh[c * MCAP + e];
            if (PREC == P_COMP) a.cout_l[c][r] = ml[c * MCAP + e];
        }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0 && own_pad > 0) {
        bulk_s2g(a.hout + ts, hfin, (uint32_t)own_pad * 4u);
        if (PREC == P_COMP) bulk_s2g(a.lout + ts, lsm, (uint32_t)own_pad * 2u);
        bulk_commit();
        bulk_wait_read_all();
    }
}

}  // namespace
}  // namespace vga

namespace vga {

namespace {

// Tile geometry and the two capacity classes.  Both classes share the geometry (and so the tile-order
// layout); a tile runs in class B when its tile-plus-halo region holds more than kCapA nodes.
constexpr int kTY = 16, kTZ = 16, kK = 3;
constexpr int kCapA = 4096, kMcapA = 256, kNtA = 512;
constexpr int kCapB = 8192, kMcapB = 512, kNtB = 1024;

struct BlockLayout {
    TileGrid g{};
    int64_t ntiles = 0;
    int32_t ntot = 0;  // tile-order length (padded tiles)
    int32_t *tstart = nullptr, *tcnt = nullptr, *tpos = nullptr, *tiles = nullptr;  // tiles: class A, then B
    int64_t nA = 0, nB = 0;
    uint16_t *rorder = nullptr;
    float *th[2] = {nullptr, nullptr};
    res_t *tl[2] = {nullptr, nullptr};
    char *cstate2 = nullptr;  // second compact state (the blocked launches alternate between the two)
    int64_t ccap = 0;
    int32_t *rmarked = nullptr;     // marked nodes per tile region (per activity build)
    std::vector<int32_t> h_class;   // 0: A, 1: B
    int64_t marked_build = -1;      // activity build the marked check was made for
    bool marked_ok = false;
    bool usable = false;            // every region fits a class
};

void layout_free(BlockLayout *b) {
    dfree(b->tstart);
    dfree(b->tcnt);
    dfree(b->tpos);
    dfree(b->tiles);
    dfree(b->rorder);
    dfree(b->th[0]);
    dfree(b->th[1]);
    dfree(b->tl[0]);
    dfree(b->tl[1]);
    dfree(b->cstate2);
    dfree(b->rmarked);
    delete b;
}

// Region rows (dz, dy) of the K-halo in order of rho = max(distance in y, distance in z) from the tile,
// raster order within one rho: the rows with rho <= r are the first (TY + 2r)(TZ + 2r).
std::vector<uint16_t> region_order(int TY, int TZ, int K) {
    const int RY = TY + 2 * K, RZ = TZ + 2 * K;
    auto ring = [&](int d, int T) { return d < K ? K - d : (d >= K + T ? d - K - T + 1 : 0); };
    std::vector<uint16_t> out;
    for (int r = 0; r <= K; ++r)
        for (int rr = 0; rr < RY * RZ; ++rr)
            if (std::max(ring(rr % RY, TY), ring(rr / RY, TZ)) == r) out.push_back((uint16_t)rr);
    return out;
}

inline unsigned blocks_for(int64_t count, int threads) { return (unsigned)((count + threads - 1) / threads); }

vga_status layout_build(vga_sim *s, BlockLayout *b) {
    const vga_graph *gr = s->g;
    const Topo t = gr->topo();
    TileGrid &g = b->g;
    g.W = t.W;
    g.ny = t.ny;
    g.nz = t.nz;
    g.TY = kTY;
    g.TZ = kTZ;
    g.NTY = (t.ny + kTY - 1) / kTY;
    g.NTZ = (t.nz + kTZ - 1) / kTZ;
    b->ntiles = g.ntiles();
    if (b->ntiles <= 0 || s->n + 8 * b->ntiles >= ((int64_t)1 << 31)) return VGA_OK;  // not usable
    cudaStream_t st = s->stream;
    int32_t *cnt8 = nullptr, *rcnt = nullptr;
    VGA_TRY(dmalloc((void **)&b->tcnt, sizeof(int32_t) * (size_t)b->ntiles, "tile counts"));
    VGA_TRY(dmalloc((void **)&b->tstart, sizeof(int32_t) * (size_t)(b->ntiles + 1), "tile starts"));
    VGA_TRY(dmalloc((void **)&b->tpos, sizeof(int32_t) * (size_t)t.nrows * t.W, "tile positions"));
    VGA_TRY(dmalloc((void **)&b->rmarked, sizeof(int32_t) * (size_t)b->ntiles, "tile marked counts"));
    VGA_TRY(dmalloc((void **)&cnt8, sizeof(int32_t) * 2 * (size_t)b->ntiles, "tile scratch"));
    rcnt = cnt8 + b->ntiles;
    k_tile_count<<<(unsigned)b->ntiles, kPT, 0, st>>>(g, t.mask, b->tcnt, cnt8);
    k_scan_i32<<<1, 1024, 0, st>>>(b->ntiles, cnt8, b->tstart);
    k_tile_pos<<<(unsigned)b->ntiles, kPT, 0, st>>>(g, t.mask, b->tstart, b->tpos);
    k_tile_region<<<(unsigned)b->ntiles, kPT, 0, st>>>(g, kK, t.mask, t.pre, nullptr, rcnt, nullptr);
    cudaError_t e = cudaGetLastError();
    std::vector<int32_t> h_r((size_t)b->ntiles), h_c((size_t)b->ntiles), h_c8((size_t)b->ntiles);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&b->ntot, b->tstart + b->ntiles, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_r.data(), rcnt, sizeof(int32_t) * h_r.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_c.data(), b->tcnt, sizeof(int32_t) * h_c.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_c8.data(), cnt8, sizeof(int32_t) * h_c8.size(), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dfree(cnt8);
    if (e != cudaSuccess) return cuda_fail(e, "tile layout", __FILE__, __LINE__);
    s->launches += 4;
    // slots a tile uses: its region's nodes plus the padding of its own range
    for (int64_t T = 0; T < b->ntiles; ++T) h_r[T] += h_c8[T] - h_c[T];
    // classes
    std::vector<int32_t> list;
    list.reserve((size_t)b->ntiles);
    b->h_class.assign((size_t)b->ntiles, 0);
    for (int64_t T = 0; T < b->ntiles; ++T) {
        if (h_r[T] > kCapB) return VGA_OK;  // a region too large for either class: not usable
        if (h_r[T] <= kCapA) list.push_back((int32_t)T);
    }
    b->nA = (int64_t)list.size();
    for (int64_t T = 0; T < b->ntiles; ++T)
        if (h_r[T] > kCapA) {
            list.push_back((int32_t)T);
            b->h_class[T] = 1;
        }
    b->nB = (int64_t)list.size() - b->nA;
    VGA_TRY(dmalloc((void **)&b->tiles, sizeof(int32_t) * list.size(), "tile lists"));
    VGA_CUDA(cudaMemcpyAsync(b->tiles, list.data(), sizeof(int32_t) * list.size(), cudaMemcpyHostToDevice, st));
    const std::vector<uint16_t> ro = region_order(kTY, kTZ, kK);
    VGA_TRY(dmalloc((void **)&b->rorder, sizeof(uint16_t) * ro.size(), "region order"));
    VGA_CUDA(cudaMemcpyAsync(b->rorder, ro.data(), sizeof(uint16_t) * ro.size(), cudaMemcpyHostToDevice, st));
    const size_t len = (size_t)b->ntot + 64;
    for (int k = 0; k < 2; ++k) {
        VGA_TRY(dmalloc((void **)&b->th[k], sizeof(float) * len, "tile-order DOM"));
        VGA_TRY(dmalloc((void **)&b->tl[k], sizeof(res_t) * len, "tile-order DOM residuals"));
        VGA_CUDA(cudaMemsetAsync(b->th[k], 0, sizeof(float) * len, st));  // padding stays zero
        VGA_CUDA(cudaMemsetAsync(b->tl[k], 0, sizeof(res_t) * len, st));
    }
    VGA_CUDA(cudaStreamSynchronize(st));
    b->usable = true;
    return VGA_OK;
}

// The marked nodes of every region fit their class's list (checked once per activity build).
vga_status marked_check(vga_sim *s, BlockLayout *b) {
    if (b->marked_build == s->act.builds) return VGA_OK;
    b->marked_ok = false;
    const Topo t = s->g->topo();
    cudaStream_t st = s->stream;
    k_tile_region<<<(unsigned)b->ntiles, kPT, 0, st>>>(b->g, kK, t.mask, t.pre, s->act.words, nullptr, b->rmarked);
    VGA_CHECK_LAUNCH();
    ++s->launches;
    std::vector<int32_t> h_m((size_t)b->ntiles);
    VGA_CUDA(cudaMemcpyAsync(h_m.data(), b->rmarked, sizeof(int32_t) * h_m.size(), cudaMemcpyDeviceToHost, st));
    VGA_CUDA(cudaStreamSynchronize(st));
    bool ok = true;
    for (int64_t T = 0; T < b->ntiles && ok; ++T) ok = h_m[T] <= (b->h_class[T] ? kMcapB : kMcapA);
    // second compact state of the same capacity
    if (ok && s->act.n_active > 0 && b->ccap < s->act.cap) {
        dfree(b->cstate2);
        b->cstate2 = nullptr;
        b->ccap = 0;
        VGA_TRY(dmalloc((void **)&b->cstate2, (sizeof(float) + sizeof(res_t)) * 4 * (size_t)s->act.cap + 16,
                        "second compact state"));
        b->ccap = s->act.cap;
    }
    b->marked_ok = ok;
    b->marked_build = s->act.builds;
    return VGA_OK;
}

template <int CAP, int MCAP, int NT, int TR, int PREC>
cudaError_t launch_class(const BlockArgs &args, int64_t count, int32_t tile_offset, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    using Ly = BlockSmem<kTY, kTZ, kK, CAP, MCAP, NT>;
    auto kern = k_dom_block<kTY, kTZ, kK, CAP, MCAP, NT, TR, PREC>;
    static uint64_t configured = 0;  // one attribute call per instantiation and device (ordinals < 64)
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !((configured >> dev) & 1ull)) {
        const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Ly::bytes);
        if (e != cudaSuccess) return e;
        configured |= 1ull << dev;
    }
    BlockArgs a = args;
    a.tiles = args.tiles + tile_offset;
    kern<<<(unsigned)count, NT, Ly::bytes, st>>>(a);
    return cudaGetLastError();
}

template <int TR, int PREC>
cudaError_t launch_both(const BlockArgs &a, const BlockLayout *b, cudaStream_t st) {
    cudaError_t e = launch_class<kCapB, kMcapB, kNtB, TR, PREC>(a, b->nB, (int32_t)b->nA, st);
    if (e == cudaSuccess) e = launch_class<kCapA, kMcapA, kNtA, TR, PREC>(a, b->nA, 0, st);
    return e;
}

SparseState compact_view(const Activity &act, char *blob) {
    Activity v = act;
    v.state = blob;
    return activity_state(v);
}

}  // namespace

void block_free(vga_sim *s) {
    if (s->blk) layout_free(static_cast<BlockLayout *>(s->blk));
    s->blk = nullptr;
}

bool block_supported(const vga_sim *s) {
    return s->wmode == W_UNIT && !s->subcycled() && s->sp.ntrans == 1 && s->n > 0 && s->g->nx <= 32767;
}

vga_status sim_block_fused(vga_sim *s, int64_t P, bool *done) {
    *done = false;
    if (P <= 0 || !block_supported(s) || !s->act.valid) return VGA_OK;
    if (!s->blk) {
        BlockLayout *b = new (std::nothrow) BlockLayout();
        if (!b) return fail(VGA_ERR_OOM, "tile layout");
        s->blk = b;
        const vga_status st = layout_build(s, b);
        if (st != VGA_OK) {
            block_free(s);
            return st;
        }
    }
    BlockLayout *b = static_cast<BlockLayout *>(s->blk);
    if (!b->usable) return VGA_OK;
    VGA_TRY(marked_check(s, b));
    if (!b->marked_ok) return VGA_OK;
    const bool comp = s->precision() == P_COMP;
    const Topo t = s->g->topo();
    cudaStream_t st = s->stream;
    const StateIO io = state_io(s);  // DOM in: io.in[1]; the pass parity decides where it lands
    timing_begin(s, VGA_KERNEL_FUSED_STEP);
    const int64_t nwords = (int64_t)t.nrows * t.W;
    const int64_t perm_threads = b->ntiles * kTY * kTZ;
    if (comp)
        k_perm_in<P_COMP><<<blocks_for(perm_threads, kPT), kPT, 0, st>>>(b->g, t.mask, t.pre, b->tpos, io.in[1], io.lin[1],
                                                                       b->th[0], b->tl[0]);
    else
        k_perm_in<P_F32><<<blocks_for(perm_threads, kPT), kPT, 0, st>>>(b->g, t.mask, t.pre, b->tpos, io.in[1], io.lin[1],
                                                                      b->th[0], b->tl[0]);
    VGA_CHECK_LAUNCH();
    BlockArgs a{};
    a.g = b->g;
    a.mask = t.mask;
    a.pre = t.pre;
    a.tpos = b->tpos;
    a.tstart = b->tstart;
    a.tcnt = b->tcnt;
    a.tiles = b->tiles;
    a.rorder = b->rorder;
    a.p = s->sp;
    a.err = s->d_err;
    const SparseState c0 = activity_state(s->act);
    const SparseState c1 = b->cstate2 ? compact_view(s->act, b->cstate2) : c0;
    int src = 0;
    int64_t launches = 1;
    for (int64_t done_passes = 0; done_passes < P;) {
        const int steps = (int)std::min<int64_t>(kK, P - done_passes);
        const SparseState &cin = (launches & 1) ? c0 : c1;  // launch 1 reads the state's compact copy
        const SparseState &cout = (launches & 1) ? c1 : c0;
        a.hin = b->th[src];
        a.lin = b->tl[src];
        a.hout = b->th[src ^ 1];
        a.lout = b->tl[src ^ 1];
        a.ss = cin;
        for (int c = 0; c < 4; ++c) {
            a.cout_h[c] = cout.h[c];
            a.cout_l[c] = cout.l[c];
        }
        a.steps = steps;
        cudaError_t e;
        if (s->sp.transform == 0) e = comp ? launch_both<0, P_COMP>(a, b, st) : launch_both<0, P_F32>(a, b, st);
        else e = comp ? launch_both<1, P_COMP>(a, b, st) : launch_both<1, P_F32>(a, b, st);
        if (e != cudaSuccess) return cuda_fail(e, "k_dom_block", __FILE__, __LINE__);
        s->launches += (b->nA > 0) + (b->nB > 0);
        src ^= 1;
        done_passes += steps;
        ++launches;
    }
    // the DOM lands where the unblocked passes would leave it (they swap the buffers every pass)
    float *dst = (P & 1) ? io.out[1] : const_cast<float *>(io.in[1]);
    res_t *dstl = (P & 1) ? io.lout[1] : const_cast<res_t *>(io.lin[1]);
    if (comp)
        k_perm_out<P_COMP><<<blocks_for(nwords, kPT), kPT, 0, st>>>(nwords, t.mask, t.pre, b->tpos, b->th[src], b->tl[src],
                                                                  dst, dstl);
    else
        k_perm_out<P_F32><<<blocks_for(nwords, kPT), kPT, 0, st>>>(nwords, t.mask, t.pre, b->tpos, b->th[src], b->tl[src],
                                                                 dst, dstl);
    VGA_CHECK_LAUNCH();
    s->launches += 2;
    // an odd number of blocked launches leaves the compact state in the second copy
    if (((launches - 1) & 1) == 1 && s->act.n_active > 0 && b->cstate2) {
        const size_t bytes = (sizeof(float) + sizeof(res_t)) * 4 * (size_t)s->act.cap;
        VGA_CUDA(cudaMemcpyAsync(s->act.state, b->cstate2, bytes, cudaMemcpyDeviceToDevice, st));
    }
    timing_end_weighted(s, P);
    s->blocked_passes += P;
    if (P & 1)
        for (int c = 0; c < 5; ++c) s->cur[c] ^= 1;
    *done = true;
    return VGA_OK;
}

}  // namespace vga
