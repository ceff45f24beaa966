// C ABI entry points of libvga (declared in include/vga.h): argument validation, ownership of the
// device buffers, stream handling and error reporting.  The arithmetic lives in the kernels of
// graph_build.cu, step.cu and pcg.cu.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>

#include "vga_internal.cuh"

namespace vga {

namespace {
thread_local std::string g_last_error = "no error";
constexpr int32_t kDefaultCap = 1024;
}  // namespace

void set_error(const std::string &msg) { g_last_error = msg; }

vga_status fail(vga_status s, const std::string &msg) {
    set_error(msg);
    return s;
}

vga_status cuda_fail(cudaError_t e, const char *what, const char *file, int line) {
    char buf[512];
    std::snprintf(buf, sizeof(buf), "%s failed: %s (%s) at %s:%d", what, cudaGetErrorName(e), cudaGetErrorString(e),
                  file, line);
    set_error(buf);
    return e == cudaErrorMemoryAllocation ? VGA_ERR_OOM : VGA_ERR_CUDA;
}

vga_status dmalloc(void **p, size_t bytes, const char *what) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        char buf[256];
        std::snprintf(buf, sizeof(buf), "cudaMalloc of %zu bytes for %s failed: %s", bytes, what, cudaGetErrorString(e));
        set_error(buf);
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? VGA_ERR_OOM : VGA_ERR_CUDA;
    }
    return VGA_OK;
}

void dfree(void *p) {
    if (p) cudaFree(p);
}

vga_status release_status(const char *what) {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, what, __FILE__, __LINE__);
    return VGA_OK;
}

vga_status graph_build_device(vga_graph *g, const uint8_t *d_img, cudaStream_t st);
vga_status graph_export_device(const vga_graph *g, int64_t *d_von, int32_t *d_nbr, cudaStream_t st);
int totals_blocks();

static cudaEvent_t pool_event(vga_sim *s) {
    if (!s->event_pool.empty()) {
        cudaEvent_t e = s->event_pool.back();
        s->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void timing_begin(vga_sim *s, int kind) {
    if (!s->timing || s->timing_hold) return;
    s->timing_a = pool_event(s);
    s->timing_kind = kind;
    if (s->timing_a) cudaEventRecord(s->timing_a, s->stream);
}

void timing_end_weighted(vga_sim *s, int64_t passes) {
    if (!s->timing || s->timing_hold || !s->timing_a) return;
    cudaEvent_t b = pool_event(s);
    if (!b) return;
    cudaEventRecord(b, s->stream);
    s->pending.push_back({s->timing_a, b, s->timing_kind, passes});
    s->timing_a = nullptr;
}

void timing_end(vga_sim *s) { timing_end_weighted(s, 1); }

static vga_status harvest_timing(vga_sim *s) {
    if (s->pending.empty()) return VGA_OK;
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    for (auto &p : s->pending) {
        float ms = 0.0f;
        VGA_CUDA(cudaEventElapsedTime(&ms, p.a, p.b));
        if (p.kind >= 0 && p.kind < VGA_KERNEL_KINDS) {
            s->kt_ms[p.kind] += ms;
            s->kt_count[p.kind] += p.passes;
        }
        s->event_pool.push_back(p.a);
        s->event_pool.push_back(p.b);
    }
    s->pending.clear();
    return VGA_OK;
}

// Reads the device error flag written by bounded waits; a nonzero value means a kernel gave up.
static vga_status check_device_error(vga_sim *s) {
    int32_t h = 0;
    VGA_CUDA(cudaMemcpyAsync(&h, s->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    if (h != 0) {
        cudaMemsetAsync(s->d_err, 0, sizeof(int32_t), s->stream);
        return fail(VGA_ERR_TIMEOUT, h == 2 ? "a bounded device wait timed out (wavefront dependency)"
                                            : "a bounded device wait timed out (bulk copy did not complete)");
    }
    return VGA_OK;
}

static bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }

static vga_status validate_params(const vga_params *p, double max_g) {
    if (!p) return fail(VGA_ERR_INVALID_ARG, "params is NULL");
    const double vals[] = {p->D, p->rho, p->mu, p->v_som, p->v_fom, p->v_dom};
    for (double v : vals)
        if (!finite_nonneg(v)) return fail(VGA_ERR_INVALID_ARG, "rates and D must be finite and >= 0");
    if (!(std::isfinite(p->dt) && p->dt > 0.0)) return fail(VGA_ERR_INVALID_ARG, "dt must be finite and > 0");
    if (!finite_nonneg(p->dt_transform)) return fail(VGA_ERR_INVALID_ARG, "dt_transform must be finite and >= 0");
    const double dtt = p->dt_transform > 0.0 ? p->dt_transform : p->dt;
    if (!(p->dt / dtt < 1.0e6)) return fail(VGA_ERR_INVALID_ARG, "dt / dt_transform must stay below 1e6");
    if (!(std::isfinite(p->beta) && p->beta >= 0.0 && p->beta <= 1.0))
        return fail(VGA_ERR_INVALID_ARG, "beta must lie in [0, 1]");
    if (!(std::isfinite(p->K_dom) && p->K_dom > 0.0)) return fail(VGA_ERR_INVALID_ARG, "K_dom must be finite and > 0");
    if (p->scheme != VGA_SCHEME_EXPLICIT && p->scheme != VGA_SCHEME_IMPLICIT_PCG)
        return fail(VGA_ERR_INVALID_ARG, "unknown scheme");
    if (p->transform != VGA_TRANSFORM_SYNC && p->transform != VGA_TRANSFORM_ASYNC)
        return fail(VGA_ERR_INVALID_ARG, "unknown transform");
    if (p->state_precision != VGA_STATE_COMPENSATED && p->state_precision != VGA_STATE_F32)
        return fail(VGA_ERR_INVALID_ARG, "unknown state_precision");
    if (p->scheme == VGA_SCHEME_IMPLICIT_PCG) {
        if (!(std::isfinite(p->cg_rtol) && p->cg_rtol > 0.0)) return fail(VGA_ERR_INVALID_ARG, "cg_rtol must be > 0");
        if (p->cg_maxit < 1) return fail(VGA_ERR_INVALID_ARG, "cg_maxit must be >= 1");
    }
    // products that become FP32 constants must stay finite
    const double prods[] = {p->D * p->dt, p->rho * dtt, p->mu * dtt, p->v_som * dtt, p->v_fom * dtt,
                            p->v_dom * dtt};
    for (double v : prods)
        if (!(v < 3.0e38)) return fail(VGA_ERR_INVALID_ARG, "rate * dt overflows FP32");
    if (p->scheme == VGA_SCHEME_EXPLICIT && 6.0 * p->D * p->dt * max_g > 1.0 + 1e-12) {
        char buf[200];
        std::snprintf(buf, sizeof(buf),
                      "explicit scheme unstable: 6 * D * dt * max g = %.6g > 1 (Q would have negative entries)",
                      6.0 * p->D * p->dt * max_g);
        return fail(VGA_ERR_UNSTABLE_DT, buf);
    }
    return VGA_OK;
}

}  // namespace vga

using namespace vga;

extern "C" {

const char *vga_strerror(int status) {
    switch (status) {
        case VGA_OK: return "VGA_OK";
        case VGA_ERR_INVALID_ARG: return "VGA_ERR_INVALID_ARG";
        case VGA_ERR_OOM: return "VGA_ERR_OOM";
        case VGA_ERR_CUDA: return "VGA_ERR_CUDA";
        case VGA_ERR_UNSTABLE_DT: return "VGA_ERR_UNSTABLE_DT";
        case VGA_ERR_NOT_CONVERGED: return "VGA_ERR_NOT_CONVERGED";
        case VGA_ERR_TIMEOUT: return "VGA_ERR_TIMEOUT";
        case VGA_ERR_NONFINITE: return "VGA_ERR_NONFINITE";
        case VGA_ERR_UNSUPPORTED: return "VGA_ERR_UNSUPPORTED";
        default: return "VGA_ERR_UNKNOWN";
    }
}

const char *vga_last_error(void) { return g_last_error.c_str(); }

int32_t vga_version(void) { return 10000; }

// ------------------------------------------------------------------------------------------------
vga_status vga_graph_build(const uint8_t *img, int32_t nx, int32_t ny, int32_t nz, uint32_t flags, void *stream,
                           vga_graph **out) {
    if (!out) return fail(VGA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!img) return fail(VGA_ERR_INVALID_ARG, "img is NULL");
    if (nx < 1 || ny < 1 || nz < 1 || nx > 32768 || ny > 32768 || nz > 32768)
        return fail(VGA_ERR_INVALID_ARG, "each image dimension must lie in [1, 32768]");
    const int64_t nvox = (int64_t)nx * ny * nz;
    if (nvox >= (int64_t)1 << 31) return fail(VGA_ERR_INVALID_ARG, "nx*ny*nz must be < 2^31");
    if (flags & ~(VGA_KEEP_LARGEST_COMPONENT | VGA_IMAGE_ON_DEVICE)) return fail(VGA_ERR_INVALID_ARG, "unknown flags");
    cudaStream_t st = (cudaStream_t)stream;
    vga_graph *g = new (std::nothrow) vga_graph();
    if (!g) return fail(VGA_ERR_OOM, "host allocation of the graph handle failed");
    g->nx = nx;
    g->ny = ny;
    g->nz = nz;
    g->nvox = nvox;
    g->flags = flags;
    g->stream = st;
    uint8_t *d_img = nullptr;
    vga_status s = VGA_OK;
    if (flags & VGA_IMAGE_ON_DEVICE) {
        s = graph_build_device(g, img, st);
    } else {
        s = dmalloc((void **)&d_img, (size_t)nvox, "image");
        if (s == VGA_OK) {
            const cudaError_t e = cudaMemcpyAsync(d_img, img, (size_t)nvox, cudaMemcpyHostToDevice, st);
            s = e == cudaSuccess ? graph_build_device(g, d_img, st) : cuda_fail(e, "image upload", __FILE__, __LINE__);
        }
    }
    if (s == VGA_OK) {
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(e, "graph build", __FILE__, __LINE__);
    }
    dfree(d_img);
    if (s != VGA_OK) {
        vga_graph_free(g);
        return s;
    }
    *out = g;
    return VGA_OK;
}

vga_status vga_graph_info(const vga_graph *g, int64_t *n_nodes, int32_t *n_components, int32_t *largest) {
    if (!g) return fail(VGA_ERR_INVALID_ARG, "graph is NULL");
    if (n_nodes) *n_nodes = g->n;
    if (n_components) *n_components = g->n_components;
    if (largest) *largest = g->largest;
    return VGA_OK;
}

vga_status vga_graph_export(const vga_graph *g, int32_t *labels, int64_t *voxel_of_node, int32_t *nbr) {
    if (!g) return fail(VGA_ERR_INVALID_ARG, "graph is NULL");
    cudaStream_t st = g->stream;
    if (labels) VGA_CUDA(cudaMemcpyAsync(labels, g->labels, sizeof(int32_t) * (size_t)g->nvox, cudaMemcpyDeviceToHost, st));
    if ((voxel_of_node || nbr) && g->n > 0) {
        int64_t *d_von = nullptr;
        int32_t *d_nbr = nullptr;
        vga_status s = VGA_OK;
        if (voxel_of_node) s = dmalloc((void **)&d_von, sizeof(int64_t) * (size_t)g->n, "export nodes");
        if (s == VGA_OK && nbr) s = dmalloc((void **)&d_nbr, sizeof(int32_t) * 6 * (size_t)g->n, "export nbr");
        if (s == VGA_OK) s = graph_export_device(g, d_von, d_nbr, st);
        if (s == VGA_OK && voxel_of_node) {
            const cudaError_t e =
                cudaMemcpyAsync(voxel_of_node, d_von, sizeof(int64_t) * (size_t)g->n, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) s = cuda_fail(e, "export copy", __FILE__, __LINE__);
        }
        if (s == VGA_OK && nbr) {
            const cudaError_t e =
                cudaMemcpyAsync(nbr, d_nbr, sizeof(int32_t) * 6 * (size_t)g->n, cudaMemcpyDeviceToHost, st);
            if (e != cudaSuccess) s = cuda_fail(e, "export copy", __FILE__, __LINE__);
        }
        const cudaError_t e = cudaStreamSynchronize(st);
        if (s == VGA_OK && e != cudaSuccess) s = cuda_fail(e, "export", __FILE__, __LINE__);
        dfree(d_von);
        dfree(d_nbr);
        return s;
    }
    VGA_CUDA(cudaStreamSynchronize(st));
    return VGA_OK;
}

vga_status vga_graph_free(vga_graph *g) {
    if (!g) return VGA_OK;
    VGA_TRY(release_status("error pending before vga_graph_free"));
    if (g->stream) cudaStreamSynchronize(g->stream);
    dfree(g->labels);
    dfree(g->mask);
    dfree(g->pre);
    delete g;
    return release_status("vga_graph_free");
}

// ------------------------------------------------------------------------------------------------
vga_status vga_sim_create(const vga_graph *g, const vga_params *p, void *stream, vga_sim **out) {
    if (!out) return fail(VGA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!g) return fail(VGA_ERR_INVALID_ARG, "graph is NULL");
    VGA_TRY(validate_params(p, 1.0));
    vga_sim *s = new (std::nothrow) vga_sim();
    if (!s) return fail(VGA_ERR_OOM, "host allocation of the simulation handle failed");
    s->g = g;
    s->stream = (cudaStream_t)stream;
    s->n = g->n;
    s->npad = ((g->n + 63) / 64) * 64;
    sim_prepare_params(s, p);
    vga_status st = VGA_OK;
    const size_t bytes = sizeof(float) * 5 * (size_t)std::max<int64_t>(s->npad, 64);
    const size_t lbytes = sizeof(res_t) * 5 * (size_t)std::max<int64_t>(s->npad, 64);
    for (int b = 0; b < 2 && st == VGA_OK; ++b) st = dmalloc((void **)&s->buf[b], bytes, "state");
    for (int b = 0; b < 2 && st == VGA_OK; ++b) st = dmalloc((void **)&s->lbuf[b], lbytes, "state residuals");
    if (st == VGA_OK) st = dmalloc((void **)&s->partials, sizeof(double) * 5 * (size_t)totals_blocks(), "partials");
    if (st == VGA_OK) st = dmalloc((void **)&s->d_totals, sizeof(double) * 8, "totals");
    if (st == VGA_OK) st = dmalloc((void **)&s->d_err, sizeof(int32_t) * 4, "error flag");
    if (st == VGA_OK) {
        const cudaError_t e = cudaMemsetAsync(s->d_err, 0, sizeof(int32_t) * 4, s->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync", __FILE__, __LINE__);
    }
    if (st == VGA_OK) {
        const cudaError_t e = cudaMallocHost((void **)&s->h_totals, sizeof(double) * 8);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMallocHost", __FILE__, __LINE__);
    }
    if (st == VGA_OK) st = build_chunks(g->topo(), kDefaultCap, &s->chunks, s->stream);
    for (int b = 0; b < 2 && st == VGA_OK; ++b) {
        cudaError_t e = cudaMemsetAsync(s->buf[b], 0, bytes, s->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(s->lbuf[b], 0, lbytes, s->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync", __FILE__, __LINE__);
    }
    if (st == VGA_OK) {
        const cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "sim create", __FILE__, __LINE__);
    }
    if (st != VGA_OK) {
        vga_sim_free(s);
        return st;
    }
    *out = s;
    return VGA_OK;
}

vga_status vga_sim_set_params(vga_sim *s, const vga_params *p) {
    if (!s) return fail(VGA_ERR_INVALID_ARG, "sim is NULL");
    VGA_TRY(validate_params(p, s->max_g));
    ++s->param_gen;
    if (p->state_precision != s->params.state_precision) {
        // residuals are meaningless across a precision change: start them at zero
        for (int b = 0; b < 2; ++b)
            VGA_CUDA(cudaMemsetAsync(s->lbuf[b], 0, sizeof(res_t) * 5 * (size_t)std::max<int64_t>(s->npad, 64),
                                     s->stream));
    }
    return sim_prepare_params(s, p);
}

// Shared by the host and device forms of vga_sim_set_block_conductances: the block grid of the
// image and its interface count, checked against n_theta.
static vga_status block_grid_check(const vga_sim *s, int32_t block_side, int64_t n_theta, int32_t (&nb)[3],
                                   int64_t (&cnt)[3]) {
    const vga_graph *g = s->g;
    nb[0] = (g->nx + block_side - 1) / block_side;
    nb[1] = (g->ny + block_side - 1) / block_side;
    nb[2] = (g->nz + block_side - 1) / block_side;
    cnt[0] = (int64_t)nb[2] * nb[1] * (nb[0] - 1);
    cnt[1] = (int64_t)nb[2] * (nb[1] - 1) * nb[0];
    cnt[2] = (int64_t)(nb[2] - 1) * nb[1] * nb[0];
    if (n_theta != cnt[0] + cnt[1] + cnt[2]) {
        char buf[160];
        std::snprintf(buf, sizeof(buf), "n_theta = %lld but the block grid has %lld interfaces", (long long)n_theta,
                      (long long)(cnt[0] + cnt[1] + cnt[2]));
        return fail(VGA_ERR_INVALID_ARG, buf);
    }
    return VGA_OK;
}

static vga_status block_stability_check(const vga_sim *s, float mx) {
    if (s->params.scheme == VGA_SCHEME_EXPLICIT && 6.0 * s->params.D * s->params.dt * mx > 1.0 + 1e-12)
        return fail(VGA_ERR_UNSTABLE_DT, "explicit scheme unstable with these conductances (6 D dt max theta > 1)");
    return VGA_OK;
}

static vga_status block_theta_buffer(vga_sim *s, int64_t n_theta) {
    if (s->n_theta < n_theta) {
        dfree(s->theta);
        s->theta = nullptr;
        s->n_theta = 0;
        VGA_TRY(dmalloc((void **)&s->theta, sizeof(float) * (size_t)std::max<int64_t>(n_theta, 1), "theta"));
        s->n_theta = n_theta;
    }
    return VGA_OK;
}

static void block_apply(vga_sim *s, int32_t block_side, const int32_t (&nb)[3], const int64_t (&cnt)[3], float mx) {
    if (s->bw.bs != block_side || s->face_mode) s->btable_bs = 0;
    s->face_mode = false;
    s->bw.g6 = nullptr;
    s->bw.bs = block_side;
    s->bw.nbx = nb[0];
    s->bw.nby = nb[1];
    s->bw.nbz = nb[2];
    s->bw.off_y = cnt[0];
    s->bw.off_z = cnt[0] + cnt[1];
    s->bw.theta = s->theta;
    s->wmode = W_BLOCK;
    s->max_g = mx;
    ++s->param_gen;
}

vga_status vga_sim_set_block_conductances(vga_sim *s, int32_t block_side, const float *theta, int64_t n_theta) {
    if (!s) return fail(VGA_ERR_INVALID_ARG, "sim is NULL");
    if (block_side < 1 || !theta) return fail(VGA_ERR_INVALID_ARG, "block_side must be >= 1 and theta non-NULL");
    int32_t nb[3];
    int64_t cnt[3];
    VGA_TRY(block_grid_check(s, block_side, n_theta, nb, cnt));
    float mx = 1.0f;
    for (int64_t k = 0; k < n_theta; ++k) {
        if (!(std::isfinite(theta[k]) && theta[k] >= 0.0f))
            return fail(VGA_ERR_INVALID_ARG, "theta values must be finite and >= 0");
        mx = std::max(mx, theta[k]);
    }
    VGA_TRY(block_stability_check(s, mx));
    VGA_TRY(block_theta_buffer(s, n_theta));
    if (n_theta > 0)
        VGA_CUDA(cudaMemcpyAsync(s->theta, theta, sizeof(float) * (size_t)n_theta, cudaMemcpyHostToDevice, s->stream));
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    block_apply(s, block_side, nb, cnt, mx);
    return VGA_OK;
}

vga_status vga_sim_set_block_conductances_device(vga_sim *s, int32_t block_side, const float *d_theta,
                                                 int64_t n_theta) {
    if (!s) return fail(VGA_ERR_INVALID_ARG, "sim is NULL");
    if (block_side < 1 || (!d_theta && n_theta > 0))
        return fail(VGA_ERR_INVALID_ARG, "block_side must be >= 1 and d_theta non-NULL");
    int32_t nb[3];
    int64_t cnt[3];
    VGA_TRY(block_grid_check(s, block_side, n_theta, nb, cnt));
    bool valid = true;
    float vmax = 0.0f;
    VGA_TRY(sim_theta_check(s, d_theta, n_theta, &valid, &vmax));  // the caller's buffer, before any copy
    if (!valid) return fail(VGA_ERR_INVALID_ARG, "theta values must be finite and >= 0");
    const float mx = std::max(1.0f, vmax);
    VGA_TRY(block_stability_check(s, mx));
    VGA_TRY(block_theta_buffer(s, n_theta));
    if (n_theta > 0)
        VGA_CUDA(cudaMemcpyAsync(s->theta, d_theta, sizeof(float) * (size_t)n_theta, cudaMemcpyDeviceToDevice,
                                 s->stream));
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    block_apply(s, block_side, nb, cnt, mx);
    return VGA_OK;
}

vga_status vga_sim_clear_conductances(vga_sim *s) {
    if (!s) return fail(VGA_ERR_INVALID_ARG, "sim is NULL");
    s->wmode = W_UNIT;
    s->face_mode = false;
    s->bw.g6 = nullptr;
    s->max_g = 1.0f;
    ++s->param_gen;
    return VGA_OK;
}

vga_status vga_sim_set_face_conductances(vga_sim *s, const float *g_face) {
    if (!s) return fail(VGA_ERR_INVALID_ARG, "sim is NULL");
    if (!g_face && s->n > 0) return fail(VGA_ERR_INVALID_ARG, "g_face is NULL");
    if (s->g->nx > 32767 || s->n >= kMaxTableBlocks)
        return fail(VGA_ERR_UNSUPPORTED, "per-face conductances need nx <= 32767 and fewer than 2^26 nodes");
    const int64_t m = 6 * s->n;
    for (int64_t k = 0; k < m; ++k)
        if (!(std::isfinite(g_face[k]) && g_face[k] >= 0.0f))
            return fail(VGA_ERR_INVALID_ARG, "face conductances must be finite and >= 0");
    float *d = nullptr;
    VGA_TRY(dmalloc((void **)&d, sizeof(float) * (size_t)std::max<int64_t>(m, 6), "face conductances"));
    vga_status st = VGA_OK;
    if (m > 0) {
        const cudaError_t e = cudaMemcpyAsync(d, g_face, sizeof(float) * (size_t)m, cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "face conductances upload", __FILE__, __LINE__);
    }
    bool sym = true;
    float rowmax = 0.0f;
    if (st == VGA_OK) st = sim_face_check(s, d, &sym, &rowmax);
    if (st == VGA_OK && !sym)
        st = fail(VGA_ERR_INVALID_ARG, "face conductances differ between the two slots of an edge (g_ij != g_ji)");
    if (st == VGA_OK && s->params.scheme == VGA_SCHEME_EXPLICIT && s->params.D * s->params.dt * rowmax > 1.0 + 1e-12)
        st = fail(VGA_ERR_UNSTABLE_DT, "explicit scheme unstable with these conductances (D dt sum_j g_ij > 1)");
    if (st != VGA_OK) {
        dfree(d);
        return st;
    }
    dfree(s->g6);
    s->g6 = d;
    s->bw = BlockWeights{};
    s->bw.g6 = d;
    s->face_mode = true;
    s->wmode = W_BLOCK;
    s->n_theta = m;
    s->max_g = std::max(rowmax / 6.0f, 0.0f);  // the 6 D dt max_g bound of the parameter checks
    ++s->param_gen;
    return VGA_OK;
}

static vga_status ensure_stage(vga_sim *s) {
    if (!s->stage) VGA_TRY(dmalloc((void **)&s->stage, sizeof(double) * 5 * (size_t)std::max<int64_t>(s->n, 1), "stage"));
    return VGA_OK;
}

vga_status vga_sim_set_masses(vga_sim *s, const double *x, int32_t on_device) {
    if (!s || (!x && s->n > 0)) return fail(VGA_ERR_INVALID_ARG, "sim or x is NULL");
    if (s->n == 0) return VGA_OK;
    if (on_device) {
        VGA_TRY(sim_convert_in(s, x));
        return VGA_OK;
    }
    for (int64_t k = 0; k < 5 * s->n; ++k)
        if (!std::isfinite(x[k])) return fail(VGA_ERR_NONFINITE, "non-finite value in the input masses");
    VGA_TRY(ensure_stage(s));
    VGA_CUDA(cudaMemcpyAsync(s->stage, x, sizeof(double) * 5 * (size_t)s->n, cudaMemcpyHostToDevice, s->stream));
    VGA_TRY(sim_convert_in(s, s->stage));
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    return VGA_OK;
}

vga_status vga_sim_get_masses(vga_sim *s, double *x, int32_t on_device) {
    if (!s || (!x && s->n > 0)) return fail(VGA_ERR_INVALID_ARG, "sim or x is NULL");
    if (s->n == 0) return VGA_OK;
    if (on_device) return sim_convert_out(s, x);
    VGA_TRY(ensure_stage(s));
    VGA_TRY(sim_convert_out(s, s->stage));
    VGA_CUDA(cudaMemcpyAsync(x, s->stage, sizeof(double) * 5 * (size_t)s->n, cudaMemcpyDeviceToHost, s->stream));
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    return VGA_OK;
}

vga_status vga_sim_set_state_f32(vga_sim *s, const float *x, int32_t on_device) {
    if (!s || (!x && s->n > 0)) return fail(VGA_ERR_INVALID_ARG, "sim or x is NULL");
    if (s->n == 0) return VGA_OK;
    if (on_device) return sim_pack_f32(s, const_cast<float *>(x), true);
    VGA_TRY(ensure_stage(s));
    float *st = reinterpret_cast<float *>(s->stage);
    VGA_CUDA(cudaMemcpyAsync(st, x, sizeof(float) * 5 * (size_t)s->n, cudaMemcpyHostToDevice, s->stream));
    VGA_TRY(sim_pack_f32(s, st, true));
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    return VGA_OK;
}

vga_status vga_sim_get_state_f32(vga_sim *s, float *x, int32_t on_device) {
    if (!s || (!x && s->n > 0)) return fail(VGA_ERR_INVALID_ARG, "sim or x is NULL");
    if (s->n == 0) return VGA_OK;
    if (on_device) return sim_pack_f32(s, x, false);
    VGA_TRY(ensure_stage(s));
    float *st = reinterpret_cast<float *>(s->stage);
    VGA_TRY(sim_pack_f32(s, st, false));
    VGA_CUDA(cudaMemcpyAsync(x, st, sizeof(float) * 5 * (size_t)s->n, cudaMemcpyDeviceToHost, s->stream));
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    return VGA_OK;
}

namespace {
struct StateHeader {
    char magic[8];
    int64_t n;
    int64_t steps_done;
    int32_t precision;
    int32_t pad;
};
}  // namespace

vga_status vga_sim_state_bytes(const vga_sim *s, int64_t *bytes) {
    if (!s || !bytes) return fail(VGA_ERR_INVALID_ARG, "sim or bytes is NULL");
    *bytes = (int64_t)sizeof(StateHeader) + 5 * s->n * (int64_t)(sizeof(float) + sizeof(uint16_t));
    return VGA_OK;
}

vga_status vga_sim_save_state(vga_sim *s, void *buf, int64_t bytes) {
    int64_t need = 0;
    VGA_TRY(vga_sim_state_bytes(s, &need));
    if (!buf || bytes < need) return fail(VGA_ERR_INVALID_ARG, "buffer NULL or smaller than vga_sim_state_bytes");
    StateHeader hd{};
    std::memcpy(hd.magic, "VGASTATE", 8);
    hd.n = s->n;
    hd.steps_done = s->steps_done;
    hd.precision = s->params.state_precision;
    std::memcpy(buf, &hd, sizeof(hd));
    char *p = static_cast<char *>(buf) + sizeof(hd);
    for (int c = 0; c < 5; ++c)
        VGA_CUDA(cudaMemcpyAsync(p + (size_t)c * s->n * sizeof(float), s->comp(c), sizeof(float) * (size_t)s->n,
                                 cudaMemcpyDeviceToHost, s->stream));
    p += 5 * (size_t)s->n * sizeof(float);
    // residuals leave as BF16 bits (the documented format), converted on the device
    VGA_TRY(ensure_stage(s));
    uint16_t *st = reinterpret_cast<uint16_t *>(s->stage);
    VGA_TRY(sim_res_export(s, st));
    VGA_CUDA(cudaMemcpyAsync(p, st, sizeof(uint16_t) * 5 * (size_t)s->n, cudaMemcpyDeviceToHost, s->stream));
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    return VGA_OK;
}

vga_status vga_sim_load_state(vga_sim *s, const void *buf, int64_t bytes) {
    int64_t need = 0;
    VGA_TRY(vga_sim_state_bytes(s, &need));
    if (!buf || bytes < need) return fail(VGA_ERR_INVALID_ARG, "buffer NULL or smaller than vga_sim_state_bytes");
    StateHeader hd;
    std::memcpy(&hd, buf, sizeof(hd));
    if (std::memcmp(hd.magic, "VGASTATE", 8) != 0 || hd.n != s->n)
        return fail(VGA_ERR_INVALID_ARG, "not a state of this graph (magic or node count differs)");
    if (hd.precision != s->params.state_precision)
        return fail(VGA_ERR_INVALID_ARG, "state was saved with another state_precision");
    const char *p = static_cast<const char *>(buf) + sizeof(hd);
    for (int c = 0; c < 5; ++c)
        VGA_CUDA(cudaMemcpyAsync(s->comp(c), p + (size_t)c * s->n * sizeof(float), sizeof(float) * (size_t)s->n,
                                 cudaMemcpyHostToDevice, s->stream));
    p += 5 * (size_t)s->n * sizeof(float);
    VGA_TRY(ensure_stage(s));
    uint16_t *st = reinterpret_cast<uint16_t *>(s->stage);
    VGA_CUDA(cudaMemcpyAsync(st, p, sizeof(uint16_t) * 5 * (size_t)s->n, cudaMemcpyHostToDevice, s->stream));
    VGA_TRY(sim_res_import(s, st));
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    s->steps_done = hd.steps_done;
    return VGA_OK;
}

vga_status vga_sim_set_activity_skip(vga_sim *s, int32_t on) {
    if (!s) return fail(VGA_ERR_INVALID_ARG, "sim is NULL");
    s->activity_skip = on != 0;
    return VGA_OK;
}

vga_status vga_sim_set_solver(vga_sim *s, int32_t solver) {
    if (!s) return fail(VGA_ERR_INVALID_ARG, "sim is NULL");
    if (solver != VGA_SOLVER_FP64_PCG && solver != VGA_SOLVER_MIXED_REFINEMENT && solver != VGA_SOLVER_MIXED_HOST_LOOP)
        return fail(VGA_ERR_INVALID_ARG, "unknown solver");
    s->cg_mixed = solver != VGA_SOLVER_FP64_PCG;
    s->cg_host_loop = solver == VGA_SOLVER_MIXED_HOST_LOOP;
    return VGA_OK;
}

vga_status vga_sim_step(vga_sim *s, int64_t n_steps) {
    if (!s) return fail(VGA_ERR_INVALID_ARG, "sim is NULL");
    if (n_steps < 0) return fail(VGA_ERR_INVALID_ARG, "n_steps must be >= 0");
    if (s->params.scheme == VGA_SCHEME_IMPLICIT_PCG) return sim_step_implicit(s, n_steps);
    return sim_step_explicit(s, n_steps);
}

vga_status vga_sim_totals(vga_sim *s, double *totals) {
    if (!s || !totals) return fail(VGA_ERR_INVALID_ARG, "sim or totals is NULL");
    VGA_TRY(sim_totals(s, totals));
    return check_device_error(s);
}

vga_status vga_sim_sync(vga_sim *s) {
    if (!s) return fail(VGA_ERR_INVALID_ARG, "sim is NULL");
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    return check_device_error(s);
}

vga_status vga_sim_get_stats(vga_sim *s, vga_sim_stats *out) {
    if (!s || !out) return fail(VGA_ERR_INVALID_ARG, "sim or out is NULL");
    out->steps_done = s->steps_done;
    out->cg_iterations = s->cg_iterations;
    out->cg_last_relres = s->cg_last_relres;
    out->kernel_launches = s->launches;
    out->graph_launches = s->graph_launches;
    out->active_nodes = s->act.n_active;
    out->blocked_passes = s->blocked_passes;
    out->negative_reports = s->negative_reports;
    return VGA_OK;
}

vga_status vga_adjoint_forward(vga_sim *s, int64_t n_steps, int32_t ckpt_every) {
    if (!s) return fail(VGA_ERR_INVALID_ARG, "sim is NULL");
    if (n_steps < 0 || ckpt_every < 1) return fail(VGA_ERR_INVALID_ARG, "n_steps must be >= 0 and ckpt_every >= 1");
    if (s->params.scheme != VGA_SCHEME_EXPLICIT || s->params.transform != VGA_TRANSFORM_SYNC ||
        s->params.state_precision != VGA_STATE_COMPENSATED)
        return fail(VGA_ERR_UNSUPPORTED,
                    "the adjoint covers the explicit scheme, synchronous transformation, compensated state");
    if (s->subcycled()) return fail(VGA_ERR_UNSUPPORTED, "the adjoint needs dt_transform = 0 (one common step)");
    return sim_adjoint_forward(s, n_steps, ckpt_every);
}

vga_status vga_adjoint_backward(vga_sim *s, const double *dL_dXN, int32_t on_device, double *dL_dX0,
                                double *grad_params, double *grad_theta) {
    if (!s || !grad_params || (!dL_dXN && s->n > 0)) return fail(VGA_ERR_INVALID_ARG, "sim, dL_dXN or grad_params is NULL");
    const double *d_in = dL_dXN;
    double *d_out = dL_dX0;
    if (!on_device && s->n > 0) {
        VGA_TRY(ensure_stage(s));
        VGA_CUDA(cudaMemcpyAsync(s->stage, dL_dXN, sizeof(double) * 5 * (size_t)s->n, cudaMemcpyHostToDevice,
                                 s->stream));
        d_in = s->stage;
        d_out = dL_dX0 ? s->stage : nullptr;  // overwritten only after lambda^N has been read
    }
    VGA_TRY(sim_adjoint_backward(s, d_in, d_out, grad_params, grad_theta));
    if (!on_device && dL_dX0 && s->n > 0) {
        VGA_CUDA(cudaMemcpyAsync(dL_dX0, s->stage, sizeof(double) * 5 * (size_t)s->n, cudaMemcpyDeviceToHost,
                                 s->stream));
        VGA_CUDA(cudaStreamSynchronize(s->stream));
    }
    return VGA_OK;
}

vga_status vga_adjoint_grad_theta(vga_sim *s, double *grad_theta, int32_t on_device, int64_t n) {
    if (!s || (!grad_theta && n > 0)) return fail(VGA_ERR_INVALID_ARG, "sim or grad_theta is NULL");
    return sim_adjoint_grad_theta(s, grad_theta, on_device != 0, n);
}

vga_status vga_sgd_block_conductances(vga_sim *s, double lr, double theta_min, double theta_max) {
    if (!s) return fail(VGA_ERR_INVALID_ARG, "sim is NULL");
    if (!(std::isfinite(lr) && lr >= 0.0 && std::isfinite(theta_min) && std::isfinite(theta_max) && theta_min >= 0.0 &&
          theta_min <= theta_max))
        return fail(VGA_ERR_INVALID_ARG, "need lr >= 0 and 0 <= theta_min <= theta_max, all finite");
    if (s->params.scheme == VGA_SCHEME_EXPLICIT && 6.0 * s->params.D * s->params.dt * theta_max > 1.0 + 1e-12)
        return fail(VGA_ERR_UNSTABLE_DT, "theta_max would make the explicit scheme unstable");
    VGA_TRY(sim_sgd_theta(s, lr, theta_min, theta_max));
    s->max_g = (float)std::max(1.0, theta_max);
    ++s->param_gen;
    return VGA_OK;
}

vga_status vga_sim_get_block_conductances(vga_sim *s, float *theta, int64_t n_theta) {
    if (s && s->face_mode) return fail(VGA_ERR_UNSUPPORTED, "per-face conductances are set: no block conductances to read");
    if (!s || !theta) return fail(VGA_ERR_INVALID_ARG, "sim or theta is NULL");
    if (s->wmode != W_BLOCK || n_theta != s->n_theta) return fail(VGA_ERR_INVALID_ARG, "no block conductances of that size");
    VGA_CUDA(cudaMemcpyAsync(theta, s->theta, sizeof(float) * (size_t)n_theta, cudaMemcpyDeviceToHost, s->stream));
    VGA_CUDA(cudaStreamSynchronize(s->stream));
    return VGA_OK;
}

vga_status vga_loss_block_mass(vga_sim *s, int32_t block_side, uint32_t comp_mask, const double *target,
                               double *loss, double *block_mass, double *dL_dX) {
    if (!s || !target || !loss) return fail(VGA_ERR_INVALID_ARG, "sim, target or loss is NULL");
    if (block_side < 1 || comp_mask == 0 || (comp_mask & ~31u))
        return fail(VGA_ERR_INVALID_ARG, "block_side must be >= 1 and comp_mask a non-empty subset of 0..4");
    const vga_graph *g = s->g;
    const int64_t nb = (int64_t)((g->nx + block_side - 1) / block_side) * ((g->ny + block_side - 1) / block_side) *
                       ((g->nz + block_side - 1) / block_side);
    int nsel = 0;
    for (int c = 0; c < 5; ++c) nsel += (comp_mask >> c) & 1;
    const int64_t count = nsel * nb;
    const int64_t need = 3 * count + 64;
    if (s->loss_cap < need) {
        dfree(s->loss_work);
        s->loss_work = nullptr;
        s->loss_cap = 0;
        VGA_TRY(dmalloc((void **)&s->loss_work, sizeof(double) * (size_t)need, "loss work"));
        s->loss_cap = need;
    }
    double *d_target = s->loss_work + 2 * count + 64;
    VGA_CUDA(cudaMemcpyAsync(d_target, target, sizeof(double) * (size_t)count, cudaMemcpyHostToDevice, s->stream));
    return sim_block_mass_loss(s, block_side, comp_mask, d_target, s->loss_work, loss, block_mass, dL_dX);
}

vga_status vga_sim_enable_timing(vga_sim *s, int32_t on) {
    if (!s) return fail(VGA_ERR_INVALID_ARG, "sim is NULL");
    s->timing = on != 0;
    return VGA_OK;
}

vga_status vga_sim_read_timing(vga_sim *s, vga_kernel_timing *out, int32_t reset) {
    if (!s || !out) return fail(VGA_ERR_INVALID_ARG, "sim or out is NULL");
    VGA_TRY(harvest_timing(s));
    for (int k = 0; k < VGA_KERNEL_KINDS; ++k) {
        out->ms[k] = s->kt_ms[k];
        out->launches[k] = s->kt_count[k];
        if (reset) {
            s->kt_ms[k] = 0.0;
            s->kt_count[k] = 0;
        }
    }
    return VGA_OK;
}

vga_status vga_sim_free(vga_sim *s) {
    if (!s) return VGA_OK;
    VGA_TRY(release_status("error pending before vga_sim_free"));
    cudaStreamSynchronize(s->stream);
    for (auto &p : s->pending) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : s->event_pool) cudaEventDestroy(e);
    dfree(s->buf[0]);
    dfree(s->buf[1]);
    dfree(s->lbuf[0]);
    dfree(s->lbuf[1]);
    dfree(s->partials);
    dfree(s->d_totals);
    dfree(s->d_err);
    dfree(s->nbr_table);
    step_graphs_free(s);
    dfree(s->nbr_tz);
    activity_free(&s->act);
    dfree(s->bnode);
    dfree(s->bface);
    dfree(s->btheta6);
    if (s->h_totals) cudaFreeHost(s->h_totals);
    dfree(s->stage);
    dfree(s->theta);
    dfree(s->cg);
    sim_mx_graph_release(s);
    dfree(s->cg_scalars);
    dfree(s->loss_work);
    dfree(s->wave_dep);
    dfree(s->wave_order);
    dfree(s->g6);
    dfree(s->fnode);
    block_free(s);
    adjoint_free(s->adj);
    if (s->h_cg) cudaFreeHost(s->h_cg);
    free_chunks(&s->chunks);
    delete s;
    return release_status("vga_sim_free");
}

}  // extern "C"
