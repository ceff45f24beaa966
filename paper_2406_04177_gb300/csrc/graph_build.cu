// Graph of pore voxels on the GPU (Sec. II.A: V = voxels with I == 0, edges between face-adjacent
// voxels, Fig. 2; Sec. III: the image is turned into the adjacency graph before the time loop).
//
// Pipeline (integer only, bit-exact):
//   1. union-find connected-component labelling over 6-connectivity.  Each union links the larger
//      root below the smaller one with atomicMin, so after compression every pore voxel holds the
//      smallest raster index of its component (a scheduling-independent result);
//   2. component id = rank of that root among all roots (bitmask + prefix popcount), i.e. the
//      components are numbered in raster order of their first voxel;
//   3. sizes, and the largest component (ties: lowest id) by a 64-bit atomicMax on (size, ~id);
//   4. the node set as a row-padded bitmask, and the node index of every mask word by an
//      exclusive prefix sum of popcounts.  Node i is the i-th kept voxel in raster order.
#include <cuda_runtime.h>

#include <algorithm>

#include "vga_internal.cuh"

namespace vga {

namespace {

constexpr int kThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kThreads * kScanItems;  // words per scan block
constexpr int kUnionCap = 1 << 26;                // bound on the retry loop of one union

__device__ __forceinline__ int32_t find_root_coherent(const int32_t *L, int32_t v) {
    // L2-coherent loads: other threads lower entries with atomics during the merge pass.
    for (int it = 0; it < kUnionCap; ++it) {
        const int32_t p = __ldcg(L + v);
        if (p == v) return v;
        v = p;
    }
    return v;
}

__device__ __forceinline__ void unite(int32_t *L, int32_t a, int32_t b, int32_t *err) {
    for (int it = 0; it < kUnionCap; ++it) {
        a = find_root_coherent(L, a);
        b = find_root_coherent(L, b);
        if (a == b) return;
        if (a < b) {
            const int32_t old = atomicMin(L + b, a);
            if (old == b) return;
            b = old;
        } else {
            const int32_t old = atomicMin(L + a, b);
            if (old == a) return;
            a = old;
        }
    }
    atomicExch(err, 1);
}

__global__ void k_init_labels(const uint8_t *__restrict__ img, int64_t nvox, int32_t *__restrict__ L) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nvox) L[v] = img[v] == 0 ? (int32_t)v : -1;
}

__global__ void k_merge(const uint8_t *__restrict__ img, int32_t nx, int32_t ny, int64_t nvox,
                        int32_t *L, int32_t *err) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox || img[v] != 0) return;
    const int64_t plane = (int64_t)nx * ny;
    const int32_t x = (int32_t)(v % nx);
    const int32_t y = (int32_t)((v / nx) % ny);
    const int64_t z = v / plane;
    if (x > 0 && img[v - 1] == 0) unite(L, (int32_t)v, (int32_t)(v - 1), err);
    if (y > 0 && img[v - nx] == 0) unite(L, (int32_t)v, (int32_t)(v - nx), err);
    if (z > 0 && img[v - plane] == 0) unite(L, (int32_t)v, (int32_t)(v - plane), err);
}

__global__ void k_compress(int64_t nvox, int32_t *L) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    int32_t p = L[v];
    if (p < 0) return;
    for (int it = 0; it < kUnionCap && L[p] != p; ++it) p = L[p];
    L[v] = p;
}

// bit (v & 31) of word (v >> 5) set iff v is a root (L[v] == v)
__global__ void k_root_bits(const int32_t *__restrict__ L, int64_t nvox, uint32_t *__restrict__ bits) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool root = v < nvox && L[v] == (int32_t)v;
    const uint32_t b = __ballot_sync(0xffffffffu, root);
    if ((threadIdx.x & 31) == 0 && (v >> 5) < (nvox + 31) / 32) bits[v >> 5] = b;
}

// label = rank of the component's root among all roots; component sizes
__global__ void k_label(int64_t nvox, int32_t *__restrict__ L, const uint32_t *__restrict__ bits,
                        const int32_t *__restrict__ rank, int32_t *__restrict__ size) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const int32_t r = L[v];
    if (r < 0) return;
    const uint32_t w = bits[r >> 5];
    const int32_t id = rank[r >> 5] + __popc(w & ((1u << (r & 31)) - 1u));
    L[v] = id;
    atomicAdd(size + id, 1);
}

__global__ void k_largest(const int32_t *__restrict__ size, int32_t ncomp, unsigned long long *best) {
    const int32_t c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncomp) return;
    const unsigned long long key =
        ((unsigned long long)(uint32_t)size[c] << 32) | (unsigned long long)(0xffffffffu - (uint32_t)c);
    atomicMax(best, key);
}

// one warp per row word: bit b of word (r, w) = voxel x = 32w + b of row r is a node
__global__ void k_kept_mask(const int32_t *__restrict__ L, int32_t nx, int64_t nrows, int32_t W,
                            int32_t keep_id, uint32_t *__restrict__ mask) {
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (gw >= nrows * W) return;  // whole warp exits together
    const int64_t r = gw / W;
    const int32_t w = (int32_t)(gw - r * W);
    const int32_t x = 32 * w + lane;
    bool kept = false;
    if (x < nx) {
        const int32_t lab = L[r * nx + x];
        kept = lab >= 0 && (keep_id < 0 || lab == keep_id);
    }
    const uint32_t b = __ballot_sync(0xffffffffu, kept);
    if (lane == 0) mask[gw] = b;
}

// ---- exclusive prefix sum of word popcounts ------------------------------------------------
__device__ __forceinline__ int32_t block_excl_scan(int32_t v, int32_t *total, int32_t *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) sh[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int32_t s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
        int32_t si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t t = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= o) si += t;
        }
        sh[lane] = si - s;  // exclusive warp offsets
        if (lane == 31) sh[32] = si;
    }
    __syncthreads();
    const int32_t out = sh[wid] + incl - v;
    *total = sh[32];
    __syncthreads();
    return out;
}

__global__ void k_scan_reduce(const uint32_t *__restrict__ words, int64_t nwords, int32_t *__restrict__ bsum) {
    __shared__ int32_t sh[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t q = base + (int64_t)k * kThreads + threadIdx.x;
        if (q < nwords) s += __popc(words[q]);
    }
    int32_t tot;
    block_excl_scan(s, &tot, sh);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// single block: exclusive scan of nb block sums in place; total into *total
__global__ void k_scan_blocks(int32_t *bsum, int64_t nb, int32_t *total) {
    __shared__ int32_t sh[33];
    int32_t carry = 0;
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        const int64_t q = base + threadIdx.x;
        const int32_t v = q < nb ? bsum[q] : 0;
        int32_t tot;
        const int32_t ex = block_excl_scan(v, &tot, sh);
        if (q < nb) bsum[q] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_down(const uint32_t *__restrict__ words, int64_t nwords, const int32_t *__restrict__ bsum,
                            int32_t *__restrict__ out) {
    __shared__ int32_t sh[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t c[kScanItems];
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t q = base + k;
        c[k] = q < nwords ? __popc(words[q]) : 0;
        s += c[k];
    }
    int32_t tot;
    int32_t run = bsum[blockIdx.x] + block_excl_scan(s, &tot, sh);
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t q = base + k;
        if (q < nwords) out[q] = run;
        run += c[k];
    }
}

// ---- chunk table -----------------------------------------------------------------------------
__global__ void k_chunk_rows(const int32_t *__restrict__ pre, int64_t nrows, int32_t W, int64_t n,
                             int32_t cap, int32_t G, int32_t *__restrict__ row) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const int64_t s = pre[r * W], e = pre[(r + 1) * W];
    if (s == e) return;
    for (int64_t g = (s + cap - 1) / cap; g * cap < e; ++g) row[g] = (int32_t)r;
    if (s <= n - 1 && n - 1 < e) row[G] = (int32_t)r;
}

// ---- exports -----------------------------------------------------------------------------------
__global__ void k_export_nodes(const uint32_t *__restrict__ mask, const int32_t *__restrict__ pre, int32_t nx,
                               int32_t ny, int32_t nz, int32_t W, int64_t *__restrict__ von,
                               int32_t *__restrict__ nbr) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nq = (int64_t)ny * nz * W;
    if (q >= nq) return;
    uint32_t m = mask[q];
    if (!m) return;
    const int64_t r = q / W;
    const int32_t w = (int32_t)(q - r * W);
    const int32_t z = (int32_t)(r / ny), y = (int32_t)(r - (int64_t)z * ny);
    int64_t i = pre[q];
    auto node_at = [&](int64_t row, int32_t x) -> int32_t {
        const int64_t qq = row * W + (x >> 5);
        const uint32_t mm = mask[qq];
        const uint32_t bit = 1u << (x & 31);
        return (mm & bit) ? (int32_t)(pre[qq] + __popc(mm & (bit - 1u))) : -1;
    };
    while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        const int32_t x = 32 * w + b;
        if (von) von[i] = r * nx + x;
        if (nbr) {
            int32_t *o = nbr + 6 * i;
            o[0] = x > 0 ? node_at(r, x - 1) : -1;
            o[1] = x < nx - 1 ? node_at(r, x + 1) : -1;
            o[2] = y > 0 ? node_at(r - 1, x) : -1;
            o[3] = y < ny - 1 ? node_at(r + 1, x) : -1;
            o[4] = z > 0 ? node_at(r - ny, x) : -1;
            o[5] = z < nz - 1 ? node_at(r + ny, x) : -1;
        }
        ++i;
    }
}

inline unsigned grid_for(int64_t count, int threads) { return (unsigned)((count + threads - 1) / threads); }

}  // namespace

size_t scan_scratch_ints(int64_t nwords) {
    const int64_t nb = (nwords + kScanTile - 1) / kScanTile;
    return (size_t)std::max<int64_t>(nb, 1) + 1;
}

vga_status scan_popc(const uint32_t *words, int64_t nwords, int32_t *out, int32_t *scratch, cudaStream_t st) {
    const int64_t nb = std::max<int64_t>((nwords + kScanTile - 1) / kScanTile, 1);
    int32_t *bsum = scratch;
    k_scan_reduce<<<(unsigned)nb, kThreads, 0, st>>>(words, nwords, bsum);
    VGA_CHECK_LAUNCH();
    k_scan_blocks<<<1, 1024, 0, st>>>(bsum, nb, out + nwords);
    VGA_CHECK_LAUNCH();
    k_scan_down<<<(unsigned)nb, kThreads, 0, st>>>(words, nwords, bsum, out);
    VGA_CHECK_LAUNCH();
    return VGA_OK;
}

vga_status build_chunks(const Topo &t, int32_t cap, Chunks *ch, cudaStream_t st) {
    free_chunks(ch);
    ch->cap = cap;
    ch->count = (int32_t)((t.n + cap - 1) / cap);
    VGA_TRY(dmalloc((void **)&ch->row, sizeof(int32_t) * (size_t)(ch->count + 1), "chunk table"));
    VGA_CUDA(cudaMemsetAsync(ch->row, 0, sizeof(int32_t) * (size_t)(ch->count + 1), st));
    if (t.n > 0) {
        k_chunk_rows<<<grid_for(t.nrows, kThreads), kThreads, 0, st>>>(t.pre, t.nrows, t.W, t.n, cap, ch->count,
                                                                    ch->row);
        VGA_CHECK_LAUNCH();
    }
    return VGA_OK;
}

void free_chunks(Chunks *ch) {
    dfree(ch->row);
    ch->row = nullptr;
    ch->count = 0;
}

// Builds the graph into g (fields nx, ny, nz, flags set by the caller).  d_img is a device image.
vga_status graph_build_device(vga_graph *g, const uint8_t *d_img, cudaStream_t st) {
    const int64_t nvox = g->nvox;
    const int64_t nrows = (int64_t)g->ny * g->nz;
    const int32_t W = (g->nx + 31) / 32;
    const int64_t nwords_lin = (nvox + 31) / 32;
    const int64_t nwords_row = nrows * W;

    int32_t *err = nullptr, *root_rank = nullptr, *scratch = nullptr, *size = nullptr;
    uint32_t *root_bits = nullptr;
    unsigned long long *best = nullptr;
    int32_t *h_small = nullptr;
    vga_status status = VGA_OK;
    auto cleanup = [&]() {
        dfree(err); dfree(root_rank); dfree(scratch); dfree(size); dfree(root_bits); dfree(best);
        if (h_small) cudaFreeHost(h_small);
    };
#define STEP(expr)                  \
    do {                            \
        status = (expr);            \
        if (status != VGA_OK) {     \
            cleanup();              \
            return status;          \
        }                           \
    } while (0)
#define STEPC(call)                                                   \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) {                                      \
            status = cuda_fail(e_, #call, __FILE__, __LINE__);        \
            cleanup();                                                \
            return status;                                            \
        }                                                             \
    } while (0)

    STEP(dmalloc((void **)&g->labels, sizeof(int32_t) * (size_t)nvox, "labels"));
    STEP(dmalloc((void **)&g->mask, sizeof(uint32_t) * (size_t)std::max<int64_t>(nwords_row, 1), "node mask"));
    STEP(dmalloc((void **)&g->pre, sizeof(int32_t) * (size_t)(nwords_row + 1), "node prefix"));
    STEP(dmalloc((void **)&err, sizeof(int32_t) * 4, "flags"));
    STEP(dmalloc((void **)&root_bits, sizeof(uint32_t) * (size_t)(nwords_lin + 1), "root bits"));
    STEP(dmalloc((void **)&root_rank, sizeof(int32_t) * (size_t)(nwords_lin + 1), "root ranks"));
    const size_t scr = std::max(scan_scratch_ints(nwords_lin), scan_scratch_ints(nwords_row));
    STEP(dmalloc((void **)&scratch, sizeof(int32_t) * scr, "scan scratch"));
    STEP(dmalloc((void **)&best, sizeof(unsigned long long), "largest"));
    STEPC(cudaMallocHost((void **)&h_small, sizeof(int32_t) * 8));
    STEPC(cudaMemsetAsync(err, 0, sizeof(int32_t) * 4, st));
    STEPC(cudaMemsetAsync(best, 0, sizeof(unsigned long long), st));

    const unsigned gv = grid_for(nvox, kThreads);
    k_init_labels<<<gv, kThreads, 0, st>>>(d_img, nvox, g->labels);
    STEPC(cudaGetLastError());
    k_merge<<<gv, kThreads, 0, st>>>(d_img, g->nx, g->ny, nvox, g->labels, err);
    k_compress<<<gv, kThreads, 0, st>>>(nvox, g->labels);
    // root bitmask needs whole warps: pad the grid to a multiple of 32 threads (it already is)
    k_root_bits<<<gv, kThreads, 0, st>>>(g->labels, nvox, root_bits);
    STEPC(cudaGetLastError());
    STEP(scan_popc(root_bits, nwords_lin, root_rank, scratch, st));
    STEPC(cudaMemcpyAsync(h_small, root_rank + nwords_lin, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    STEPC(cudaMemcpyAsync(h_small + 1, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    STEPC(cudaStreamSynchronize(st));
    if (h_small[1]) STEP(fail(VGA_ERR_CUDA, "graph build: union-find retry bound exceeded"));
    const int32_t ncomp = h_small[0];
    g->n_components = ncomp;
    STEP(dmalloc((void **)&size, sizeof(int32_t) * (size_t)std::max(ncomp, 1), "component sizes"));
    STEPC(cudaMemsetAsync(size, 0, sizeof(int32_t) * (size_t)std::max(ncomp, 1), st));
    k_label<<<gv, kThreads, 0, st>>>(nvox, g->labels, root_bits, root_rank, size);
    if (ncomp > 0) k_largest<<<grid_for(ncomp, kThreads), kThreads, 0, st>>>(size, ncomp, best);
    STEPC(cudaGetLastError());
    unsigned long long h_best = 0;
    STEPC(cudaMemcpyAsync(&h_best, best, sizeof(h_best), cudaMemcpyDeviceToHost, st));
    STEPC(cudaStreamSynchronize(st));
    g->largest = ncomp > 0 ? (int32_t)(0xffffffffu - (uint32_t)(h_best & 0xffffffffull)) : -1;
    const int32_t keep_id = (g->flags & VGA_KEEP_LARGEST_COMPONENT) ? (ncomp > 0 ? g->largest : -2) : -1;

    if (nwords_row > 0) {
        const int64_t threads = nwords_row * 32;
        k_kept_mask<<<grid_for(threads, kThreads), kThreads, 0, st>>>(g->labels, g->nx, nrows, W, keep_id, g->mask);
        STEPC(cudaGetLastError());
    }
    STEP(scan_popc(g->mask, nwords_row, g->pre, scratch, st));
    int32_t h_n = 0;
    STEPC(cudaMemcpyAsync(&h_n, g->pre + nwords_row, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    STEPC(cudaStreamSynchronize(st));
    g->n = h_n;
    cleanup();
#undef STEP
#undef STEPC
    return VGA_OK;
}

vga_status graph_export_device(const vga_graph *g, int64_t *d_von, int32_t *d_nbr, cudaStream_t st) {
    const int64_t nq = (int64_t)g->ny * g->nz * ((g->nx + 31) / 32);
    if (nq == 0 || g->n == 0) return VGA_OK;
    k_export_nodes<<<grid_for(nq, kThreads), kThreads, 0, st>>>(g->mask, g->pre, g->nx, g->ny, g->nz,
                                                               (g->nx + 31) / 32, d_von, d_nbr);
    VGA_CHECK_LAUNCH();
    return VGA_OK;
}

}  // namespace vga

vga::Topo vga_graph::topo() const {
    vga::Topo t;
    t.nx = nx;
    t.ny = ny;
    t.nz = nz;
    t.W = (nx + 31) / 32;
    t.nrows = ny * nz;
    t.n = n;
    t.mask = mask;
    t.pre = pre;
    return t;
}
