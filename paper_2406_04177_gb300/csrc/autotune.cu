// Autotuner of the explicit time step: times every (kernel variant, chunk size) candidate on the
// simulation's own graph and state with CUDA events, keeps the fastest, and leaves the state as it
// found it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "vga_internal.cuh"

namespace vga {
bool stencil_variant_supported(int variant, int cap);

namespace {

struct Candidate {
    int variant, cap, depth, ctas;  // depth, ctas: wavefront passes per block and CTAs per SM
};

constexpr Candidate kCandidates[] = {{2, 1024, 0, 0}, {4, 1024, 0, 0}, {5, 1024, 0, 0}, {6, 1024, 0, 0}, {1, 1024, 0, 0}, {1, 512, 0, 0},  {1, 2048, 0, 0},
                                     {0, 1024, 0, 0}, {0, 512, 0, 0},  {0, 2048, 0, 0}, {3, 1024, 2, 0},
                                     {3, 512, 4, 0},  {3, 256, 4, 0}};

vga_status snapshot(vga_sim *s, float *h, res_t *l, bool restore) {
    for (int c = 0; c < 5; ++c) {
        float *dh = h + (size_t)c * s->npad;
        res_t *dl = l + (size_t)c * s->npad;
        if (restore) {
            VGA_CUDA(cudaMemcpyAsync(s->comp(c), dh, sizeof(float) * (size_t)s->n, cudaMemcpyDeviceToDevice, s->stream));
            VGA_CUDA(cudaMemcpyAsync(s->lcomp(c), dl, sizeof(res_t) * (size_t)s->n, cudaMemcpyDeviceToDevice,
                                     s->stream));
        } else {
            VGA_CUDA(cudaMemcpyAsync(dh, s->comp(c), sizeof(float) * (size_t)s->n, cudaMemcpyDeviceToDevice, s->stream));
            VGA_CUDA(cudaMemcpyAsync(dl, s->lcomp(c), sizeof(res_t) * (size_t)s->n, cudaMemcpyDeviceToDevice,
                                     s->stream));
        }
    }
    return VGA_OK;
}

vga_status select_kernel(vga_sim *s, int variant, int cap, int depth = 0, int ctas = 0) {
    if (variant == 3) {
        s->wave_chunk = cap;
        s->wave_depth = depth;
        s->wave_ctas = ctas;
    } else if (s->chunks.cap != cap) {
        VGA_TRY(build_chunks(s->g->topo(), cap, &s->chunks, s->stream));
    }
    s->kernel_variant = variant;
    return VGA_OK;
}

}  // namespace
}  // namespace vga

using namespace vga;

extern "C" vga_status vga_sim_set_kernel(vga_sim *s, int32_t variant, int32_t chunk) {
    if (!s) return fail(VGA_ERR_INVALID_ARG, "sim is NULL");
    if (variant < 0 || variant > 6 || chunk < 32 || chunk > 8192 || (chunk & 31))
        return fail(VGA_ERR_INVALID_ARG, "variant must lie in [0, 6] and chunk be a multiple of 32 in [32, 8192]");
    if (variant == 3) {
        if (!wave_params_valid(chunk, 4, 0)) return fail(VGA_ERR_INVALID_ARG, "wavefront chunks are powers of two >= 256");
        VGA_TRY(select_kernel(s, 3, chunk, 4, 0));
        return VGA_OK;
    }
    if (!stencil_variant_supported(variant, chunk))
        return fail(VGA_ERR_UNSUPPORTED, "the staged kernel exists for chunks of 512, 1024 and 2048 nodes");
    VGA_TRY(select_kernel(s, variant, chunk));
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    return VGA_OK;
}

extern "C" vga_status vga_sim_set_wavefront(vga_sim *s, int32_t chunk, int32_t depth, int32_t ctas_per_sm) {
    if (!s) return fail(VGA_ERR_INVALID_ARG, "sim is NULL");
    if (!wave_params_valid(chunk, depth, ctas_per_sm))
        return fail(VGA_ERR_INVALID_ARG,
                    "chunk must be a power of two in [256, 8192], depth in [1, 64], ctas_per_sm in [0, 32]");
    return select_kernel(s, 3, chunk, depth, ctas_per_sm);
}

extern "C" vga_status vga_sim_autotune(vga_sim *s, int32_t trial_steps, vga_tune_result *out) {
    if (!s || !out) return fail(VGA_ERR_INVALID_ARG, "sim or out is NULL");
    if (trial_steps < 1) return fail(VGA_ERR_INVALID_ARG, "trial_steps must be >= 1");
    out->count = 0;
    out->best = -1;
    if (s->n == 0 || s->params.scheme != VGA_SCHEME_EXPLICIT) return VGA_OK;
    float *h = nullptr;
    res_t *l = nullptr;
    VGA_TRY(dmalloc((void **)&h, sizeof(float) * 5 * (size_t)s->npad, "autotune snapshot"));
    vga_status st = dmalloc((void **)&l, sizeof(res_t) * 5 * (size_t)s->npad, "autotune snapshot");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == VGA_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
        st = fail(VGA_ERR_CUDA, "cudaEventCreate failed");
    const int64_t steps0 = s->steps_done;
    const int keep_variant = s->kernel_variant, keep_cap = s->chunks.cap, keep_wc = s->wave_chunk,
              keep_wd = s->wave_depth, keep_wk = s->wave_ctas;
    if (st == VGA_OK) st = snapshot(s, h, l, false);
    double best = 1e300;
    int nc = 0;
    for (const Candidate &c : kCandidates) {
        if (st != VGA_OK || nc >= VGA_TUNE_MAX) break;
        st = select_kernel(s, c.variant, c.cap, c.depth, c.ctas);
        if (st == VGA_OK) st = sim_step_explicit(s, 2);  // warm-up (instantiation, attributes)
        if (st == VGA_OK) st = snapshot(s, h, l, true);
        if (st != VGA_OK) break;
        cudaEventRecord(e0, s->stream);
        st = sim_step_explicit(s, trial_steps);
        cudaEventRecord(e1, s->stream);
        if (st == VGA_OK && cudaEventSynchronize(e1) != cudaSuccess) st = fail(VGA_ERR_CUDA, "autotune timing failed");
        float ms = 0.0f;
        if (st == VGA_OK) cudaEventElapsedTime(&ms, e0, e1);
        if (st == VGA_OK) st = snapshot(s, h, l, true);
        if (st != VGA_OK) break;
        out->entries[nc].variant = c.variant;
        out->entries[nc].chunk = c.cap;
        out->entries[nc].depth = c.depth;
        out->entries[nc].ctas_per_sm = c.ctas;
        out->entries[nc].ms_per_step = ms / trial_steps;
        if (ms < best) {
            best = ms;
            out->best = nc;
        }
        ++nc;
    }
    out->count = nc;
    if (st == VGA_OK && out->best >= 0)
        st = select_kernel(s, out->entries[out->best].variant, out->entries[out->best].chunk,
                           out->entries[out->best].depth, out->entries[out->best].ctas_per_sm);
    else if (st != VGA_OK)
        keep_variant == 3 ? select_kernel(s, 3, keep_wc, keep_wd, keep_wk) : select_kernel(s, keep_variant, keep_cap);
    s->steps_done = steps0;
    if (st == VGA_OK) {
        const cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "autotune", __FILE__, __LINE__);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dfree(h);
    dfree(l);
    return st;
}
