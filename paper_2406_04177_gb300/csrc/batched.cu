// Batched simulation of many independent subvolumes (uneven node counts, per-instance parameters)
// in one persistent kernel per launch.
//
// Layout: the instances' nodes are concatenated, each instance starting at a multiple of 256 nodes
// (kTile), so a 256-node tile never straddles two instances and carries one instance id.  Every
// instance keeps its own neighbour-offset table (offsets are relative, so they remain valid in the
// concatenated index space) and its own StepParams.
//
// A launch runs passes [pass0, pass1) of a step() call of N time steps (N + 1 passes: one
// transformation-only pass, N - 1 fused passes, one diffusion-only pass; see step.cu).  Passes are
// separated by a grid-wide barrier; the launch is cooperative, so every block is resident, and
// every wait in the barrier is bounded (VGA_ERR_TIMEOUT instead of a hang).  The launches of a
// step() call are captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "grid_sync.cuh"
#include "physics.cuh"
#include "stencil.cuh"
#include "vga_internal.cuh"

namespace vga {
namespace {

constexpr int kTile = 256;
constexpr int kBatchGroup = 4;  // nodes per thread in the fused passes

struct BInst {
    int64_t start;  // first node of the instance in the concatenated range (multiple of kTile)
    int64_t n;      // node count
    StepParams p;
};

struct BatchArgs {
    int64_t ntiles;
    int64_t npad;
    const int32_t *tile_inst;  // instance of every tile
    const BInst *inst;
    NbrTable tb;
    float *h[2];
    res_t *l[2];
    unsigned *bar;  // [0] arrivals, [1] generation
    int32_t *err;
    StateIO io[2];  // a pass whose input is state buffer k reads io[k] (kept as kernel parameters)
    SparseState ss;    // the sparse fused pass of the SPARSE instantiations (compact state, rank list)
    int64_t n_active;  // marked nodes (ranks of the compact state)
    int32_t skip_block;   // test of the bounded waits: this block leaves before any barrier (-1: none)
    uint32_t spin_limit;  // polls of a grid barrier before it gives up
};

// One fused pass over the whole batch, kBatchGroup consecutive nodes per thread (table_vec).
// Instances start on tile boundaries, so a group never straddles two and the 32 K nodes of a warp
// belong to one instance, whose parameters the warp reads from shared memory (per-thread copies
// would hold a dozen registers); every thread of a block runs the same number of iterations (the
// warp-wide shuffles need all lanes).
template <int TR, int PREC, int TF, bool SPARSE>
__device__ __forceinline__ void batch_fused_pass(const BatchArgs &a, const StateIO &io) {
    constexpr int KG = kBatchGroup;
    __shared__ StepParams wp[kTile / 32];
    const int w = threadIdx.x >> 5;
    const int64_t nsuper = (a.ntiles + KG - 1) / KG;  // kTile * KG nodes per block iteration
    for (int64_t sup = blockIdx.x; sup < nsuper; sup += gridDim.x) {
        const uint32_t i0 = (uint32_t)(sup * kTile * KG + (int64_t)threadIdx.x * KG);
        const int64_t tile = (int64_t)i0 / kTile;
        uint32_t end = 0;  // one past the instance's last node (0: no instance here)
        int32_t k = -1;
        if (tile < a.ntiles) {
            k = __ldg(a.tile_inst + tile);
            end = (uint32_t)(a.inst[k].start + a.inst[k].n);
        }
        __syncwarp();
        if ((threadIdx.x & 31) == 0) wp[w] = k >= 0 ? a.inst[k].p : StepParams{};
        __syncwarp();
        if (SPARSE) table_vec<4, W_UNIT, TR, PREC, TF, KG>(i0, end, a.tb, BlockTable{}, wp[w], io, PassRecord{}, a.ss);
        else table_vec<1, W_UNIT, TR, PREC, TF, KG>(i0, end, a.tb, BlockTable{}, wp[w], io);
    }
}

// Second half of a sparse fused pass, after a grid barrier: the marked nodes in rank order, each with
// its instance's parameters, MB, SOM, FOM, CO2 from the compact state (updated in place) and its DOM
// as the first half (MODE 4) stored it; stores the DOM as the dense fused pass does.  The DOM and
// the compact state were written inside this launch, so they are read with coherent loads.
template <int TR, int PREC>
__device__ __forceinline__ void batch_transform_marked(const BatchArgs &a, const StateIO &io) {
    const SparseState &ss = a.ss;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.n_active; r += stride) {
        const uint32_t i = __ldg(ss.list + r);
        const StepParams p = a.inst[__ldg(a.tile_inst + i / kTile)].p;
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
}

// FUSED_ONLY: an instantiation for launches whose passes are all fused ones (every launch but the
// first and the last pass of a call); without the code of the other two kinds it needs fewer
// registers, so more blocks are resident.
template <int TR, int PREC, int TF, bool FUSED_ONLY, bool SPARSE>
__global__ void __launch_bounds__(kTile, SPARSE ? 5 : 1) k_batch(BatchArgs a, int32_t pass0, int32_t pass1, int32_t npass, int32_t cur0) {
    if ((int32_t)blockIdx.x == a.skip_block) return;  // the other blocks' barrier waits then run out
    for (int32_t pass = pass0; pass < pass1; ++pass) {
        // transform / fused / diffuse
        const int kind = FUSED_ONLY ? 1 : ((pass == 0) ? 0 : (pass == npass - 1 ? 2 : 1));
        const int bi = (cur0 + pass) & 1, bo = bi ^ 1;
        const float *__restrict__ Y2 = a.h[bi] + a.npad;
        if (kind == 1) {
            // fused pass: kBatchGroup consecutive nodes per thread (table_vec).  Instances start on
            // tile boundaries, so a group never straddles two; every thread of a block runs the
            // same number of iterations (the warp-wide shuffles need all lanes).
            if (bi == 0) batch_fused_pass<TR, PREC, TF, SPARSE>(a, a.io[0]);
            else batch_fused_pass<TR, PREC, TF, SPARSE>(a, a.io[1]);
            if constexpr (SPARSE) {
                if (!grid_barrier(a.bar, a.err, a.spin_limit)) return;
                if (bi == 0) batch_transform_marked<TR, PREC>(a, a.io[0]);
                else batch_transform_marked<TR, PREC>(a, a.io[1]);
            }
            if (pass + 1 < pass1 && !grid_barrier(a.bar, a.err, a.spin_limit)) return;
            continue;
        }
        if constexpr (!FUSED_ONLY) {  // first (transform) and last (diffuse-only) pass of a call
            for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
                const BInst &ins = a.inst[__ldg(a.tile_inst + tile)];
                const uint32_t i = (uint32_t)(tile * kTile + threadIdx.x);
                const bool live = (int64_t)i - ins.start < ins.n;
                const StepParams p = ins.p;
                V x[5];
                if (kind == 0) {
                    if (!live) continue;
    #pragma unroll
                    for (int c = 0; c < 5; ++c) x[c] = vload<PREC>(a.h[bi] + c * a.npad, a.l[bi] + c * a.npad, i);
                    transform<TR, PREC>(x[0], x[1], x[2], x[3], x[4], p);
                } else {
                    const uint32_t ty = live ? __ldg(a.tb.ty + i) : 0u;
                    uint32_t dzm, dzp;
                    if (TF == 1) {  // compact z offsets
                        const uint32_t tz = live ? __ldg(a.tb.tz + i) : 0u;
                        dzm = tz & 0xffffu;
                        dzp = tz >> 16;
                    } else {
                        dzm = live ? __ldg(a.tb.tzm + i) : 0u;
                        dzp = live ? __ldg(a.tb.tzp + i) : 0u;
                    }
                    x[1] = live ? vload<PREC>(Y2, a.l[bi] + a.npad, i) : V{0.0f, 0.0f};
                    const float yi = x[1].h;
                    const int lane = threadIdx.x & 31;
                    float yl = __shfl_up_sync(0xffffffffu, yi, 1);
                    float yr = __shfl_down_sync(0xffffffffu, yi, 1);
                    const uint32_t dym = ty & 0x7fffu, dyp = (ty >> 16) & 0x7fffu;
                    const bool hxm = (ty >> 15) & 1u, hxp = ty >> 31;
                    if (lane == 0 && hxm) yl = __ldg(Y2 + (i - 1));
                    if (lane == 31 && hxp) yr = __ldg(Y2 + (i + 1));
                    float ym = 0.0f, yp = 0.0f, zm = 0.0f, zp = 0.0f;
                    if (dym) ym = __ldg(Y2 + (i - dym));
                    if (dyp) yp = __ldg(Y2 + (i + dyp));
                    if (dzm) zm = __ldg(Y2 + (i - dzm));
                    if (dzp) zp = __ldg(Y2 + (i + dzp));
                    if (!live) continue;
                    float acc = 0.0f;
                    if (hxm) acc = __fadd_rn(acc, __fsub_rn(yi, yl));
                    if (hxp) acc = __fadd_rn(acc, __fsub_rn(yi, yr));
                    if (dym) acc = __fadd_rn(acc, __fsub_rn(yi, ym));
                    if (dyp) acc = __fadd_rn(acc, __fsub_rn(yi, yp));
                    if (dzm) acc = __fadd_rn(acc, __fsub_rn(yi, zm));
                    if (dzp) acc = __fadd_rn(acc, __fsub_rn(yi, zp));
                    vadd<PREC>(x[1], __fmul_rn(-p.c, acc));
                    if (kind == 2) {
                        // diffusion-only pass: DOM is new, the other compartments move bit for bit
                        vstore<PREC>(a.h[bo] + a.npad, a.l[bo] + a.npad, i, x[1]);
    #pragma unroll
                        for (int c = 0; c < 5; ++c) {
                            if (c == 1) continue;
                            a.h[bo][c * a.npad + i] = a.h[bi][c * a.npad + i];
                            if (PREC == P_COMP) a.l[bo][c * a.npad + i] = a.l[bi][c * a.npad + i];
                        }
                        continue;
                    }
                    x[0] = vload<PREC>(a.h[bi], a.l[bi], i);
                    x[2] = vload<PREC>(a.h[bi] + 2 * a.npad, a.l[bi] + 2 * a.npad, i);
                    x[3] = vload<PREC>(a.h[bi] + 3 * a.npad, a.l[bi] + 3 * a.npad, i);
                    x[4] = vload<PREC>(a.h[bi] + 4 * a.npad, a.l[bi] + 4 * a.npad, i);
                    vround<PREC>(x[1]);
                    transform<TR, PREC>(x[0], x[1], x[2], x[3], x[4], p);
                }
    #pragma unroll
                for (int c = 0; c < 5; ++c) vstore<PREC>(a.h[bo] + c * a.npad, a.l[bo] + c * a.npad, i, x[c]);
            }
            if (pass + 1 < pass1 && !grid_barrier(a.bar, a.err, a.spin_limit)) return;
        }
    }
}

// FP64 (5 x n) of one instance <-> its slice of the current state buffer
__global__ void k_batch_in(int64_t n, const double *__restrict__ x, float *h, res_t *l, int64_t start,
                           int64_t npad, int comp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < 5; ++c) {
        const double v = x[c * n + i];
        const float hv = (float)v;
        h[c * npad + start + i] = hv;
        l[c * npad + start + i] = comp ? res_encode((float)(v - (double)hv), hv) : (res_t)0;
    }
}

__global__ void k_batch_out(int64_t n, double *__restrict__ x, const float *h, const res_t *l, int64_t start,
                            int64_t npad, int comp) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int c = 0; c < 5; ++c) {
        const float hv = h[c * npad + start + i];
        double v = (double)hv;
        if (comp) v += (double)res_decode(l[c * npad + start + i], hv);
        x[c * n + i] = v;
    }
}

}  // namespace
}  // namespace vga

using namespace vga;

struct vga_batch {
    int32_t count = 0;
    std::vector<int64_t> start, nodes;
    int64_t total = 0, npad = 0, ntiles = 0;
    int transform = 0, precision = 0;
    cudaStream_t stream = nullptr;
    float *h[2] = {nullptr, nullptr};
    res_t *l[2] = {nullptr, nullptr};
    uint32_t *table = nullptr;  // 3 x npad
    uint32_t *tz = nullptr;     // compact z offsets (npad) when they fit in 16 bits
    int32_t *tile_inst = nullptr;
    BInst *inst = nullptr;
    unsigned *bar = nullptr;
    int32_t *err = nullptr;
    double *stage = nullptr;
    int64_t stage_n = 0;
    int cur = 0;
    int grid = 0;          // blocks of a fused-only launch (resident on every SM)
    int grid_edge = 0;     // blocks of a launch of the first or the last pass
    int grid_sparse = 0;   // blocks of a sparse fused-only launch
    int blocks_per_sm = 0;  // tuning knob (0: the occupancy maximum)
    int steps_per_launch = 100;
    bool use_graph = true;
    bool capture_failed = false;
    std::map<std::tuple<int64_t, int, int, int>, cudaGraphExec_t> graphs;
    int64_t launches = 0, graph_replays = 0, steps_done = 0;
    Activity act;               // the sparse fused pass (as vga_sim_set_activity_skip)
    bool activity_skip = true;
    int32_t wait_test_block = -1;  // vga_batch_set_wait_test
    uint32_t wait_test_spin = 0;
};

namespace {

template <int TFV, bool FO, bool SP>
const void *batch_kernel(const vga_batch *b) {
    return b->transform == 0 ? (b->precision == P_COMP ? (const void *)k_batch<0, P_COMP, TFV, FO, SP>
                                                       : (const void *)k_batch<0, P_F32, TFV, FO, SP>)
                             : (b->precision == P_COMP ? (const void *)k_batch<1, P_COMP, TFV, FO, SP>
                                                       : (const void *)k_batch<1, P_F32, TFV, FO, SP>);
}

template <int TFV, bool FO, bool SP>
cudaError_t batch_launch_tf(const vga_batch *b, const cudaLaunchConfig_t &cfg, const BatchArgs &a, int32_t pass0,
                            int32_t pass1, int32_t npass, int32_t cur0) {
    if (b->transform == 0) {
        if (b->precision == P_COMP)
            return cudaLaunchKernelEx(&cfg, k_batch<0, P_COMP, TFV, FO, SP>, a, pass0, pass1, npass, cur0);
        return cudaLaunchKernelEx(&cfg, k_batch<0, P_F32, TFV, FO, SP>, a, pass0, pass1, npass, cur0);
    }
    if (b->precision == P_COMP) return cudaLaunchKernelEx(&cfg, k_batch<1, P_COMP, TFV, FO, SP>, a, pass0, pass1, npass, cur0);
    return cudaLaunchKernelEx(&cfg, k_batch<1, P_F32, TFV, FO, SP>, a, pass0, pass1, npass, cur0);
}

// Resident blocks of an instantiation, limited by blocks_per_sm and the tile count.
vga_status batch_grid_of(vga_batch *b, const void *fn, int *grid) {
    int dev = 0, sms = 0, per_sm = 0;
    VGA_CUDA(cudaGetDevice(&dev));
    VGA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    VGA_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTile, 0));
    if (per_sm < 1) return fail(VGA_ERR_CUDA, "batched kernel cannot be resident");
    const int want = b->blocks_per_sm > 0 ? std::min(b->blocks_per_sm, per_sm) : per_sm;
    *grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)want * sms, b->ntiles));
    return VGA_OK;
}

vga_status batch_grid(vga_batch *b) {
    VGA_TRY(batch_grid_of(b, b->tz ? batch_kernel<1, false, false>(b) : batch_kernel<0, false, false>(b), &b->grid_edge));
    VGA_TRY(batch_grid_of(b, b->tz ? batch_kernel<1, true, true>(b) : batch_kernel<0, true, true>(b), &b->grid_sparse));
    return batch_grid_of(b, b->tz ? batch_kernel<1, true, false>(b) : batch_kernel<0, true, false>(b), &b->grid);
}

vga_status launch_batch(vga_batch *b, int32_t pass0, int32_t pass1, int32_t npass, int32_t cur0, bool sparse) {
    BatchArgs a;
    a.ntiles = b->ntiles;
    a.npad = b->npad;
    a.tile_inst = b->tile_inst;
    a.inst = b->inst;
    a.tb.ty = b->table;
    a.tb.tzm = b->table + b->npad;
    a.tb.tzp = b->table + 2 * b->npad;
    a.tb.tz = b->tz;
    for (int k = 0; k < 2; ++k) {
        a.h[k] = b->h[k];
        a.l[k] = b->l[k];
    }
    a.bar = b->bar;
    a.err = b->err;
    a.ss = activity_state(b->act);
    a.n_active = b->act.n_active;
    a.skip_block = b->wait_test_block;
    a.spin_limit = b->wait_test_spin ? b->wait_test_spin : kBarrierSpin;
    for (int k = 0; k < 2; ++k) {
        for (int c = 0; c < 5; ++c) {
            a.io[k].in[c] = b->h[k] + c * b->npad;
            a.io[k].lin[c] = b->l[k] + c * b->npad;
            a.io[k].out[c] = b->h[1 - k] + c * b->npad;
            a.io[k].lout[c] = b->l[1 - k] + c * b->npad;
        }
    }
    // the first and the last pass of a call need the full kernel; the others run the fused-only one
    const bool fused_only = pass0 > 0 && pass1 < npass;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(fused_only ? (sparse ? b->grid_sparse : b->grid) : b->grid_edge));
    cfg.blockDim = dim3(kTile);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (fused_only && sparse)
        e = b->tz ? batch_launch_tf<1, true, true>(b, cfg, a, pass0, pass1, npass, cur0)
                  : batch_launch_tf<0, true, true>(b, cfg, a, pass0, pass1, npass, cur0);
    else if (fused_only)
        e = b->tz ? batch_launch_tf<1, true, false>(b, cfg, a, pass0, pass1, npass, cur0)
                  : batch_launch_tf<0, true, false>(b, cfg, a, pass0, pass1, npass, cur0);
    else
        e = b->tz ? batch_launch_tf<1, false, false>(b, cfg, a, pass0, pass1, npass, cur0)
                  : batch_launch_tf<0, false, false>(b, cfg, a, pass0, pass1, npass, cur0);
    if (e != cudaSuccess) return cuda_fail(e, "cooperative launch of k_batch", __FILE__, __LINE__);
    return VGA_OK;
}

// Launches of one call: the first pass alone, the fused passes in launches of steps_per_launch
// passes, the last pass alone.
int64_t launches_of(const vga_batch *b, int64_t n_steps) {
    const int64_t S = std::max(1, b->steps_per_launch), mid = n_steps - 1;
    return 2 + (mid > 0 ? (mid + S - 1) / S : 0);
}

// The state arrays as the input (in) of a pass reading buffer k and as its output (out).
StateIO batch_io(const vga_batch *b, int k) {
    StateIO io;
    for (int c = 0; c < 5; ++c) {
        io.in[c] = b->h[k] + c * b->npad;
        io.lin[c] = b->l[k] + c * b->npad;
        io.out[c] = b->h[1 - k] + c * b->npad;
        io.lout[c] = b->l[1 - k] + c * b->npad;
    }
    return io;
}

// sparse: the fused passes run sparse; the marked nodes' MB, SOM, FOM, CO2 go to the compact state
// after the first pass and back before the last.
vga_status enqueue_steps(vga_batch *b, int64_t n_steps, int cur0, bool sparse) {
    const int64_t npass = n_steps + 1;
    const int S = std::max(1, b->steps_per_launch);
    const bool comp = b->precision == P_COMP;
    VGA_TRY(launch_batch(b, 0, 1, (int32_t)npass, cur0, false));
    if (sparse) VGA_TRY(activity_copy(b->act, b->total, batch_io(b, (cur0 + 1) & 1), true, comp, b->stream));
    for (int64_t p0 = 1; p0 < npass - 1; p0 += S) {
        const int64_t p1 = std::min(npass - 1, p0 + S);
        VGA_TRY(launch_batch(b, (int32_t)p0, (int32_t)p1, (int32_t)npass, cur0, sparse));
    }
    // the state after pass npass - 2 is buffer (cur0 + npass - 1) & 1: the out side of the other
    if (sparse)
        VGA_TRY(activity_copy(b->act, b->total, batch_io(b, 1 - (int)((cur0 + npass - 1) & 1)), false, comp, b->stream));
    return launch_batch(b, (int32_t)(npass - 1), (int32_t)npass, (int32_t)npass, cur0, false);
}

vga_status check_err(vga_batch *b) {
    int32_t h = 0;
    VGA_CUDA(cudaMemcpyAsync(&h, b->err, sizeof(int32_t), cudaMemcpyDeviceToHost, b->stream));
    VGA_CUDA(cudaStreamSynchronize(b->stream));
    if (h) {
        cudaMemsetAsync(b->err, 0, sizeof(int32_t), b->stream);
        cudaMemsetAsync(b->bar, 0, 2 * sizeof(unsigned), b->stream);
        cudaStreamSynchronize(b->stream);
        return fail(VGA_ERR_TIMEOUT, "a grid barrier of the batched kernel timed out");
    }
    return VGA_OK;
}

void drop_graphs(vga_batch *b) {
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

}  // namespace

extern "C" {

vga_status vga_batch_free(vga_batch *b) {
    if (!b) return VGA_OK;
    VGA_TRY(release_status("error pending before vga_batch_free"));
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    for (int k = 0; k < 2; ++k) {
        dfree(b->h[k]);
        dfree(b->l[k]);
    }
    dfree(b->table);
    dfree(b->tz);
    dfree(b->tile_inst);
    dfree(b->inst);
    dfree(b->bar);
    activity_free(&b->act);
    dfree(b->err);
    dfree(b->stage);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
    return release_status("vga_batch_free");
}

vga_status vga_batch_create(const vga_graph *const *graphs, const vga_params *params, int32_t count,
                            vga_batch **out) {
    if (!out) return fail(VGA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!graphs || !params || count < 1) return fail(VGA_ERR_INVALID_ARG, "need count >= 1 graphs and params");
    for (int k = 0; k < count; ++k) {
        const vga_params &p = params[k];
        if (!graphs[k]) return fail(VGA_ERR_INVALID_ARG, "a graph is NULL");
        if (p.scheme != VGA_SCHEME_EXPLICIT) return fail(VGA_ERR_UNSUPPORTED, "the batched path runs the explicit scheme");
        if (p.transform != params[0].transform || p.state_precision != params[0].state_precision)
            return fail(VGA_ERR_INVALID_ARG, "all instances must share transform and state_precision");
        if (graphs[k]->nx > 32767) return fail(VGA_ERR_UNSUPPORTED, "batched instances need nx <= 32767");
        if (!(std::isfinite(p.dt) && p.dt > 0 && std::isfinite(p.D) && p.D >= 0 && p.K_dom > 0 && p.beta >= 0 &&
              p.beta <= 1 && p.rho >= 0 && p.mu >= 0 && p.v_som >= 0 && p.v_fom >= 0 && p.v_dom >= 0))
            return fail(VGA_ERR_INVALID_ARG, "invalid parameters of an instance");
        if (6.0 * p.D * p.dt > 1.0 + 1e-12) return fail(VGA_ERR_UNSTABLE_DT, "an instance has 6 D dt > 1");
        if (!(p.dt_transform == 0.0 || p.dt_transform == p.dt))
            return fail(VGA_ERR_UNSUPPORTED, "batched instances need dt_transform = 0 (one common step)");
    }
    vga_batch *b = new (std::nothrow) vga_batch();
    if (!b) return fail(VGA_ERR_OOM, "host allocation failed");
    b->count = count;
    b->transform = params[0].transform;
    b->precision = params[0].state_precision;
    vga_status st = VGA_OK;
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
        st = fail(VGA_ERR_CUDA, "cudaStreamCreate failed");
    int64_t off = 0;
    std::vector<int32_t> tinst;
    std::vector<BInst> hinst(count);
    for (int k = 0; k < count && st == VGA_OK; ++k) {
        b->start.push_back(off);
        b->nodes.push_back(graphs[k]->n);
        hinst[k].start = off;
        hinst[k].n = graphs[k]->n;
        vga_sim tmp;
        sim_prepare_params(&tmp, &params[k]);
        hinst[k].p = tmp.sp;
        const int64_t tiles = (graphs[k]->n + kTile - 1) / kTile;
        for (int64_t t = 0; t < tiles; ++t) tinst.push_back(k);
        off += tiles * kTile;
    }
    if (st == VGA_OK && off >= ((int64_t)1 << 31)) st = fail(VGA_ERR_UNSUPPORTED, "a batch holds fewer than 2^31 nodes");
    b->total = off;
    b->ntiles = off / kTile;
    b->npad = std::max<int64_t>(64, ((off + 63) / 64) * 64);
    const size_t hb = sizeof(float) * 5 * (size_t)b->npad, lb = sizeof(res_t) * 5 * (size_t)b->npad;
    for (int k = 0; k < 2 && st == VGA_OK; ++k) {
        st = dmalloc((void **)&b->h[k], hb, "batch state");
        if (st == VGA_OK) st = dmalloc((void **)&b->l[k], lb, "batch state residuals");
    }
    if (st == VGA_OK) st = dmalloc((void **)&b->table, sizeof(uint32_t) * 3 * (size_t)b->npad, "batch table");
    if (st == VGA_OK) st = dmalloc((void **)&b->tile_inst, sizeof(int32_t) * std::max<size_t>(tinst.size(), 1), "tile map");
    if (st == VGA_OK) st = dmalloc((void **)&b->inst, sizeof(BInst) * (size_t)count, "instances");
    if (st == VGA_OK) st = dmalloc((void **)&b->bar, sizeof(unsigned) * 2, "barrier");
    if (st == VGA_OK) st = dmalloc((void **)&b->err, sizeof(int32_t), "error flag");
    if (st == VGA_OK) {
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            e = cudaMemsetAsync(b->h[k], 0, hb, b->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(b->l[k], 0, lb, b->stream);
        }
        if (e == cudaSuccess) e = cudaMemsetAsync(b->table, 0, sizeof(uint32_t) * 3 * (size_t)b->npad, b->stream);
        if (e == cudaSuccess && !tinst.empty())
            e = cudaMemcpyAsync(b->tile_inst, tinst.data(), sizeof(int32_t) * tinst.size(), cudaMemcpyHostToDevice,
                                b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->inst, hinst.data(), sizeof(BInst) * (size_t)count, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->bar, 0, sizeof(unsigned) * 2, b->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->err, 0, sizeof(int32_t), b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "batch set-up", __FILE__, __LINE__);
    }
    for (int k = 0; k < count && st == VGA_OK; ++k) {
        const int64_t s0 = b->start[k];
        st = build_nbr_table(graphs[k]->topo(), b->table + s0, b->table + b->npad + s0, b->table + 2 * b->npad + s0,
                             b->stream);
    }
    // padding entries between instances are zero, so the compact form covers the whole range
    if (st == VGA_OK) st = build_compact_z(b->npad, b->npad, b->table + b->npad, b->table + 2 * b->npad, &b->tz, b->stream);
    if (st == VGA_OK) st = batch_grid(b);
    if (st != VGA_OK) {
        vga_batch_free(b);
        return st;
    }
    *out = b;
    return VGA_OK;
}

vga_status vga_batch_info(const vga_batch *b, int64_t *total_nodes, int64_t *node_offsets) {
    if (!b) return fail(VGA_ERR_INVALID_ARG, "batch is NULL");
    if (total_nodes) {
        int64_t t = 0;
        for (int64_t v : b->nodes) t += v;
        *total_nodes = t;
    }
    if (node_offsets)
        for (int k = 0; k < b->count; ++k) node_offsets[k] = b->start[k];
    return VGA_OK;
}

static vga_status batch_stage(vga_batch *b, int64_t n) {
    if (b->stage_n < n) {
        dfree(b->stage);
        b->stage = nullptr;
        b->stage_n = 0;
        VGA_TRY(dmalloc((void **)&b->stage, sizeof(double) * 5 * (size_t)std::max<int64_t>(n, 1), "batch stage"));
        b->stage_n = n;
    }
    return VGA_OK;
}

vga_status vga_batch_set_masses(vga_batch *b, int32_t instance, const double *x) {
    if (!b || instance < 0 || instance >= b->count) return fail(VGA_ERR_INVALID_ARG, "bad batch or instance");
    const int64_t n = b->nodes[instance];
    if (n == 0) return VGA_OK;
    if (!x) return fail(VGA_ERR_INVALID_ARG, "x is NULL");
    for (int64_t k = 0; k < 5 * n; ++k)
        if (!std::isfinite(x[k])) return fail(VGA_ERR_NONFINITE, "non-finite value in the input masses");
    VGA_TRY(batch_stage(b, n));
    VGA_CUDA(cudaMemcpyAsync(b->stage, x, sizeof(double) * 5 * (size_t)n, cudaMemcpyHostToDevice, b->stream));
    k_batch_in<<<(unsigned)((n + 255) / 256), 256, 0, b->stream>>>(n, b->stage, b->h[b->cur], b->l[b->cur],
                                                                  b->start[instance], b->npad, b->precision == P_COMP);
    VGA_CHECK_LAUNCH();
    VGA_CUDA(cudaStreamSynchronize(b->stream));
    b->act.valid = false;
    return VGA_OK;
}

vga_status vga_batch_get_masses(vga_batch *b, int32_t instance, double *x) {
    if (!b || instance < 0 || instance >= b->count) return fail(VGA_ERR_INVALID_ARG, "bad batch or instance");
    const int64_t n = b->nodes[instance];
    if (n == 0) return VGA_OK;
    if (!x) return fail(VGA_ERR_INVALID_ARG, "x is NULL");
    VGA_TRY(batch_stage(b, n));
    k_batch_out<<<(unsigned)((n + 255) / 256), 256, 0, b->stream>>>(n, b->stage, b->h[b->cur], b->l[b->cur],
                                                                   b->start[instance], b->npad, b->precision == P_COMP);
    VGA_CHECK_LAUNCH();
    VGA_CUDA(cudaMemcpyAsync(x, b->stage, sizeof(double) * 5 * (size_t)n, cudaMemcpyDeviceToHost, b->stream));
    VGA_CUDA(cudaStreamSynchronize(b->stream));
    return VGA_OK;
}

vga_status vga_batch_set_launch(vga_batch *b, int32_t steps_per_launch, int32_t blocks_per_sm, int32_t use_graph) {
    if (!b || steps_per_launch < 1 || blocks_per_sm < 0) return fail(VGA_ERR_INVALID_ARG, "bad launch settings");
    b->steps_per_launch = steps_per_launch;
    b->blocks_per_sm = blocks_per_sm;
    b->use_graph = use_graph != 0;
    drop_graphs(b);
    return batch_grid(b);
}

vga_status vga_batch_set_activity_skip(vga_batch *b, int32_t on) {
    if (!b) return fail(VGA_ERR_INVALID_ARG, "batch is NULL");
    b->activity_skip = on != 0;
    return VGA_OK;
}

vga_status vga_batch_set_wait_test(vga_batch *b, int32_t skip_block, uint32_t spin_limit) {
    if (!b) return fail(VGA_ERR_INVALID_ARG, "batch is NULL");
    if (skip_block < -1) return fail(VGA_ERR_INVALID_ARG, "skip_block must be -1 or a block index");
    b->wait_test_block = skip_block;
    b->wait_test_spin = spin_limit;
    drop_graphs(b);  // captured launches hold the old parameters
    return VGA_OK;
}

vga_status vga_batch_step(vga_batch *b, int64_t n_steps) {
    if (!b || n_steps < 0) return fail(VGA_ERR_INVALID_ARG, "bad batch or n_steps");
    if (n_steps == 0 || b->ntiles == 0) return VGA_OK;
    if (n_steps + 1 > (int64_t)INT32_MAX) return fail(VGA_ERR_INVALID_ARG, "n_steps too large for one call");
    const int cur0 = b->cur;
    // sparse fused passes need a mask for the current state (a rebuild may move the compact state:
    // the captured graphs go with it)
    const bool sparse = b->activity_skip && n_steps > 1;
    if (sparse && !b->act.valid) {
        const StateIO cur = batch_io(b, cur0);
        VGA_TRY(activity_build(&b->act, b->total, b->npad, cur, batch_io(b, 1 - cur0), b->precision == P_COMP,
                               b->stream));
        drop_graphs(b);
    }
    if (b->use_graph) {
        const auto key = std::make_tuple(n_steps, b->steps_per_launch, b->grid, cur0 + (sparse ? 2 : 0));
        auto it = b->graphs.find(key);
        if (it == b->graphs.end()) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            VGA_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            const vga_status st = enqueue_steps(b, n_steps, cur0, sparse);
            const cudaError_t ec = cudaStreamEndCapture(b->stream, &graph);
            cudaError_t ei = cudaErrorUnknown;
            if (st == VGA_OK && ec == cudaSuccess) ei = cudaGraphInstantiate(&exec, graph, 0);
            if (graph) cudaGraphDestroy(graph);
            if (st == VGA_OK && ec == cudaSuccess && ei == cudaSuccess) {
                it = b->graphs.emplace(key, exec).first;
            } else {
                // capture of the cooperative launches failed: run them directly from now on
                cudaGetLastError();
                b->use_graph = false;
                b->capture_failed = true;
            }
        }
        if (it != b->graphs.end()) {
            VGA_CUDA(cudaGraphLaunch(it->second, b->stream));
            ++b->graph_replays;
        } else {
            VGA_TRY(enqueue_steps(b, n_steps, cur0, sparse));
        }
    } else {
        VGA_TRY(enqueue_steps(b, n_steps, cur0, sparse));
    }
    b->launches += launches_of(b, n_steps);
    b->cur = (int)((cur0 + n_steps + 1) & 1);
    b->steps_done += n_steps;
    return check_err(b);
}

vga_status vga_batch_get_stats(const vga_batch *b, vga_batch_stats *out) {
    if (!b || !out) return fail(VGA_ERR_INVALID_ARG, "batch or out is NULL");
    out->instances = b->count;
    out->total_nodes = 0;
    for (int64_t v : b->nodes) out->total_nodes += v;
    out->grid_blocks = b->activity_skip ? b->grid_sparse : b->grid;
    out->steps_per_launch = b->steps_per_launch;
    out->kernel_launches = b->launches;
    out->graph_replays = b->graph_replays;
    out->steps_done = b->steps_done;
    out->capture_failed = b->capture_failed ? 1 : 0;
    return VGA_OK;
}

vga_status vga_batch_autotune(vga_batch *b, int32_t trial_steps, vga_batch_tune *out) {
    if (!b || !out || trial_steps < 2) return fail(VGA_ERR_INVALID_ARG, "bad batch, out or trial_steps");
    static const int kSteps[] = {25, 100, 400};
    static const int kBlocks[] = {0, 4, 2};
    const int keep_s = b->steps_per_launch, keep_b = b->blocks_per_sm;
    // save the state (both buffers' current side) so the trials leave it untouched
    float *h = nullptr;
    res_t *l = nullptr;
    VGA_TRY(dmalloc((void **)&h, sizeof(float) * 5 * (size_t)b->npad, "autotune snapshot"));
    vga_status st = dmalloc((void **)&l, sizeof(res_t) * 5 * (size_t)b->npad, "autotune snapshot");
    const int cur_keep = b->cur;
    const int64_t steps_keep = b->steps_done, launches_keep = b->launches, replays_keep = b->graph_replays;
    if (st == VGA_OK) {
        cudaMemcpyAsync(h, b->h[b->cur], sizeof(float) * 5 * (size_t)b->npad, cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(l, b->l[b->cur], sizeof(res_t) * 5 * (size_t)b->npad, cudaMemcpyDeviceToDevice, b->stream);
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    out->count = 0;
    out->best = -1;
    double best = 1e300;
    for (int si = 0; si < 3 && st == VGA_OK; ++si) {
        for (int bi = 0; bi < 3 && st == VGA_OK; ++bi) {
            if (out->count >= VGA_TUNE_MAX) break;
            st = vga_batch_set_launch(b, kSteps[si], kBlocks[bi], 1);
            if (st == VGA_OK) st = vga_batch_step(b, trial_steps);  // capture + warm-up
            cudaEventRecord(e0, b->stream);
            if (st == VGA_OK) st = vga_batch_step(b, trial_steps);
            cudaEventRecord(e1, b->stream);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (st != VGA_OK) break;
            vga_batch_tune_entry &en = out->entries[out->count];
            en.steps_per_launch = kSteps[si];
            en.blocks_per_sm = kBlocks[bi];
            en.grid_blocks = b->activity_skip ? b->grid_sparse : b->grid;
            en.ms_per_step = ms / trial_steps;
            if (ms < best) {
                best = ms;
                out->best = out->count;
            }
            ++out->count;
        }
    }
    if (st == VGA_OK && out->best >= 0)
        st = vga_batch_set_launch(b, out->entries[out->best].steps_per_launch, out->entries[out->best].blocks_per_sm, 1);
    else
        vga_batch_set_launch(b, keep_s, keep_b, 1);
    b->cur = cur_keep;
    if (h && l) {
        cudaMemcpyAsync(b->h[b->cur], h, sizeof(float) * 5 * (size_t)b->npad, cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(b->l[b->cur], l, sizeof(res_t) * 5 * (size_t)b->npad, cudaMemcpyDeviceToDevice, b->stream);
    }
    cudaStreamSynchronize(b->stream);
    b->steps_done = steps_keep;
    b->launches = launches_keep;
    b->graph_replays = replays_keep;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(h);
    dfree(l);
    return st;
}

}  // extern "C"
