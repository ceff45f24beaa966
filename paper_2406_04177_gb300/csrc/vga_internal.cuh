// Internal declarations shared by the CUDA translation units of libvga (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/vga.h"

namespace vga {

// ---------------------------------------------------------------------------------------------
// Error reporting: every failing path records a detail string and returns a vga_status.
// ---------------------------------------------------------------------------------------------
void set_error(const std::string &msg);
vga_status fail(vga_status s, const std::string &msg);
vga_status cuda_fail(cudaError_t e, const char *what, const char *file, int line);
// Status of the release calls (cudaFree, cudaFreeHost, event and stream destruction) made since the
// last check: reads and clears the runtime's error state, so a failed release is reported by the
// *_free call that made it and never surfaces in a later, unrelated call.
vga_status release_status(const char *what);

#define VGA_CUDA(call)                                                         \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) return ::vga::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define VGA_CHECK_LAUNCH() VGA_CUDA(cudaGetLastError())

#define VGA_TRY(expr)                                \
    do {                                             \
        vga_status s_ = (expr);                      \
        if (s_ != VGA_OK) return s_;                 \
    } while (0)

// ---------------------------------------------------------------------------------------------
// Topology of the node set on the device.
//
// The image is seen as nrows = ny*nz rows of nx voxels; each row is padded to W = ceil(nx/32)
// 32-bit words.  Bit b of word (r, w) is set iff voxel x = 32w + b of row r is a node.  pre[q] is
// the node index of the first node at or after word q in raster order (an exclusive prefix sum of
// the word popcounts), with pre[nrows*W] = n.  A node's index is pre[q] + popc(word below its bit),
// so the neighbour in any row is found from two words without a per-node table.
// ---------------------------------------------------------------------------------------------
struct Topo {
    int32_t nx, ny, nz, W;
    int32_t nrows;
    int64_t n;
    const uint32_t *mask;  // nrows*W words
    const int32_t *pre;    // nrows*W + 1
};

// Chunking of the node range for the stencil kernels: chunk g holds nodes [g*cap, (g+1)*cap) and
// spans image rows chunk_row[g] .. chunk_row[g+1] (inclusive; chunk_row[G] is the row of node n-1).
struct Chunks {
    int32_t cap = 0;
    int32_t count = 0;
    int32_t *row = nullptr;  // count + 1 entries (device)
};

// Compact neighbour-offset table of a node set (built once from the row bitmask).  Per node i:
//   ty[i]   bits 0..14 = i - (index of the -y neighbour), 0 if none; bit 15 = has -x neighbour;
//           bits 16..30 = (index of the +y neighbour) - i, 0 if none; bit 31 = has +x neighbour
//   tzm[i]  i - (index of the -z neighbour), 0 if none
//   tzp[i]  (index of the +z neighbour) - i, 0 if none
// The -x / +x neighbours are i - 1 / i + 1.  Requires nx <= 32767 (y offsets are below nx).
struct NbrTable {
    const uint32_t *ty = nullptr, *tzm = nullptr, *tzp = nullptr;
    // Compact form of the z offsets, present when every one is below 2^16: tz[i] = tzm | tzp << 16
    // (8 bytes per node with ty instead of 12).
    const uint32_t *tz = nullptr;
};

// Block conductances in table form.  node[i] = block id (bits 0..25) | bit 26+d set when the edge
// leaving node i through slot d crosses a block face; face[6*b + d] = index into theta of face d of
// block b (or -1 at the image border); theta6[6*b + d] = theta[face[6*b + d]] (1 at the border), so
// a pass reads a crossing edge's conductance with one dependent load instead of two.
struct BlockTable {
    const uint32_t *node = nullptr;
    const int32_t *face = nullptr;
    const float *theta = nullptr;
    const float *theta6 = nullptr;
};
constexpr int64_t kMaxTableBlocks = (int64_t)1 << 26;

// Float parameters of one time step (products with dt taken in FP64 on the host, then rounded).
struct StepParams {
    float a;      // v_dom * dt
    float K;      // K_dom
    float r;      // rho * dt
    float m;      // mu * dt
    float beta;   // beta
    float omb;    // 1 - beta
    float f;      // v_fom * dt
    float s;      // v_som * dt
    float c;      // D * dt
    int transform;
    int ntrans;   // transformations applied per pass (1; 0 or more when the steps differ)
};

// Stored residual of a compensated value: the BF16 bits of its value (physics.cuh).
typedef uint16_t res_t;

// Input and output compartment arrays of one pass over the state.
struct StateIO {
    const float *in[5];   // FP32 values
    float *out[5];
    const res_t *lin[5];  // residuals (compensated precision only)
    res_t *lout[5];
};

// Compact state of the sparse fused pass (vga_sim_set_activity_skip): MB, SOM, FOM and CO2 of the
// marked nodes, in the order of the activity mask (node i has rank prefix[i / 32] + the marked nodes
// before it in its mask word), updated in place during one step call.
struct SparseState {
    const uint32_t *mask = nullptr;    // activity bits
    const uint32_t *prefix = nullptr;  // marked nodes before each mask word
    const uint32_t *list = nullptr;    // node of each rank
    float *h[4] = {nullptr, nullptr, nullptr, nullptr};  // MB, SOM, FOM, CO2 values
    res_t *l[4] = {nullptr, nullptr, nullptr, nullptr};  // and residuals
};

// Activity mask of the sparse fused pass: bit i set when node i may change under the
// transformation (MB, SOM, FOM or CO2 nonzero, or a negative-zero DOM; such a set never grows while
// stepping), the marked nodes before each mask word, and the compact state they use during a step
// call.  One per simulation or batch; built per state upload.
struct Activity {
    uint32_t *words = nullptr;  // nw mask words, nw prefix words, then a 64-bit counter
    int64_t nw = 0;
    char *state = nullptr;      // compact MB, SOM, FOM, CO2: 4 x cap values, 4 x cap residuals, cap nodes
    int64_t cap = 0;
    int64_t n_active = -1;      // marked nodes (-1: not built)
    bool valid = false;         // built for the current state
    int64_t builds = 0;         // id of the last build, unique in the process (consumers cache per build)
};

// Builds the mask, the prefix and the compact state for nodes [0, n) of the state `cur` (`spare`
// gets zeros in MB, SOM, FOM, CO2 of the unmarked nodes).  One synchronisation.
vga_status activity_build(Activity *a, int64_t n, int64_t npad, const StateIO &cur, const StateIO &spare, bool comp,
                          cudaStream_t st);
SparseState activity_state(const Activity &a);
// Marked nodes' MB, SOM, FOM, CO2: state (io.in) -> compact, or compact -> state (io.out).
vga_status activity_copy(const Activity &a, int64_t n, const StateIO &io, bool to_compact, bool comp, cudaStream_t st);
void activity_free(Activity *a);

// Edge-weight modes of the stencil.
enum WeightMode { W_UNIT = 0, W_BLOCK = 1 };

struct BlockWeights {
    int32_t bs = 0;              // block side
    int32_t nbx = 0, nby = 0, nbz = 0;
    int64_t off_y = 0, off_z = 0;  // offsets of the y- and z-normal faces in theta
    const float *theta = nullptr;  // device
    // Per-face conductances (vga_sim_set_face_conductances): g6[6 i + d] is the conductance of the edge
    // leaving node i through slot d; when set, it replaces the block lookup and the gradient of that
    // edge goes to index 6 i + d (odd slots: each edge once).
    const float *g6 = nullptr;
};

// ---------------------------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------------------------
template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t count = 0;
};

vga_status dmalloc(void **p, size_t bytes, const char *what);
void dfree(void *p);

// Exclusive prefix sum of popcount(words[q]) over q in [0, nwords): out[q], out[nwords] = total.
// `scratch` must hold scan_scratch_ints(nwords) ints.
size_t scan_scratch_ints(int64_t nwords);
vga_status scan_popc(const uint32_t *words, int64_t nwords, int32_t *out, int32_t *scratch,
                     cudaStream_t st);

// Builds the chunk table of `topo` for chunk size cap (device work, one launch).
vga_status build_chunks(const Topo &topo, int32_t cap, Chunks *ch, cudaStream_t st);
// Builds the neighbour-offset table of the simulation's graph (step.cu).
void free_chunks(Chunks *ch);

struct AdjointBuffers;
void adjoint_free(AdjointBuffers *a);

}  // namespace vga

// ---------------------------------------------------------------------------------------------
// Library-owned handle types (opaque in the C ABI).
// ---------------------------------------------------------------------------------------------
struct vga_graph {
    int32_t nx = 0, ny = 0, nz = 0;
    int64_t nvox = 0;
    int64_t n = 0;
    int32_t n_components = 0;
    int32_t largest = -1;
    uint32_t flags = 0;
    int32_t *labels = nullptr;  // device, nvox
    uint32_t *mask = nullptr;   // device, nrows*W
    int32_t *pre = nullptr;     // device, nrows*W + 1
    cudaStream_t stream = nullptr;
    vga::Topo topo() const;
};

// A captured explicit step call and its shape (sim_step_explicit on small graphs).
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    int64_t n_steps = -1, param_gen = -1, builds = -1, launches = 0;
    uint32_t cur_in = 0, cur_xor = 0;
    int variant = -1;
    bool sparse = false;
    uint64_t use = 0;
};

struct vga_sim {
    const vga_graph *g = nullptr;
    vga_params params{};
    vga::StepParams sp{};
    cudaStream_t stream = nullptr;
    int64_t n = 0;
    int64_t npad = 0;         // row stride of the state arrays (multiple of 64 floats)
    float *buf[2] = {nullptr, nullptr};     // two state buffers of 5*npad FP32 values
    vga::res_t *lbuf[2] = {nullptr, nullptr};  // their residuals (compensated precision)
    int cur[5] = {0, 0, 0, 0, 0};           // which buffer holds compartment c
    StepGraph step_graphs[4];               // graphs of whole explicit step calls (small graphs)
    uint64_t step_graph_clock = 0;
    bool step_graphs_ok = true;             // cleared when a capture fails
    cudaStream_t step_cap = nullptr;        // private capture stream
    vga::Chunks chunks;
    // conductances
    int wmode = vga::W_UNIT;
    vga::BlockWeights bw;
    float *theta = nullptr;
    int64_t n_theta = 0;
    float max_g = 1.0f;
    float *g6 = nullptr;            // per-face conductances (6 x n, device) when face_mode
    bool face_mode = false;         // W_BLOCK kernels read g6 instead of the block faces
    uint32_t *fnode = nullptr;      // BlockTable.node of the per-face table (node i, every slot crossing)
    // reductions
    double *partials = nullptr;  // per-block FP64 partial sums
    int64_t partials_cap = 0;
    double *d_totals = nullptr;  // 8 doubles (device)
    double *h_totals = nullptr;  // pinned host mirror
    // staging for FP64 input/output
    double *stage = nullptr;
    // implicit-scheme work vectors (FP64), allocated on first use
    double *cg = nullptr;
    int64_t cg_count = 0;
    double *cg_scalars = nullptr;  // device scalars of the PCG recurrence
    double *h_cg = nullptr;        // pinned mirror of the PCG scalars
    bool cg_mixed = true;          // implicit solve: float-float refinement around FP32 PCG (unit conductances)
    bool cg_host_loop = false;     // mixed solve: loop driven from the host instead of one CUDA graph
    bool mx_graph_failed = false;  // graph construction failed once: host-driven loop from then on
    void *mx_graph = nullptr;      // cached graphs of the mixed solve (pcg.cu)
    int64_t graph_launches = 0;    // CUDA graph launches of the mixed solve
    // Sparse fused pass (stencil.cuh MODE 4 and the marked-node half): activity mask and compact state
    vga::Activity act;
    bool activity_skip = true;     // use it (vga_sim_set_activity_skip)
    bool sparse_call = false;      // the fused passes of the running step call are sparse
    int64_t steps_done = 0;
    int64_t cg_iterations = 0;
    double cg_last_relres = 0.0;
    int64_t launches = 0;
    // optional per-kernel CUDA-event timing (vga_sim_enable_timing)
    bool timing = false;
    struct Pending {
        cudaEvent_t a, b;
        int kind;
        int64_t passes;  // time steps the timed launch covered (a wavefront launch runs many)
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> event_pool;
    double kt_ms[VGA_KERNEL_KINDS] = {};
    int64_t kt_count[VGA_KERNEL_KINDS] = {};
    cudaEvent_t timing_a = nullptr;
    int timing_kind = -1;
    bool timing_hold = false;      // inside a span timed as a whole (per-launch events off)
    // adjoint work buffers (adjoint.cu), allocated on first use
    vga::AdjointBuffers *adj = nullptr;
    int32_t *d_err = nullptr;     // device error flag of bounded waits (nonzero: timed out)
    int kernel_variant = 5;       // explicit stencil: 0 decode + direct loads, 1 decode + staged, 2 table,
                                  // 3 table passes as an L2 wavefront (wave.cu), 4 / 5 table, two /
                                  // four nodes per thread
    int wave_chunk = 512, wave_depth = 4, wave_ctas = 0;  // wavefront chunk, passes per block, CTAs/SM
    void *blk = nullptr;          // tile-order layout of the temporally blocked passes (block.cu)
    int64_t blocked_passes = 0;   // fused passes run by it
    int64_t negative_reports = 0;  // totals passes that found a negative mass
    int32_t *wave_dep = nullptr;      // per chunk: lowest and highest chunk its neighbours lie in; flags
    int32_t *wave_order = nullptr;    // skewed item order of one block of passes
    int wave_built_chunk = 0, wave_built_depth = 0, wave_built_lag = -1;
    int32_t wave_reach = 0;
    uint32_t *nbr_table = nullptr;  // 3 x npad words (NbrTable), built on first use
    uint32_t *nbr_tz = nullptr;     // compact z offsets (NbrTable.tz) when they fit in 16 bits
    int nbr_tz_state = 0;           // 0 not examined, 1 built, 2 offsets too large
    uint32_t *bnode = nullptr;      // BlockTable.node (npad), built for the current block side
    int32_t *bface = nullptr;       // BlockTable.face (6 x blocks)
    float *btheta6 = nullptr;       // BlockTable.theta6 (6 x blocks), rebuilt when param_gen moves
    int64_t btheta6_gen = -1;       // param_gen btheta6 was built for
    int32_t btable_bs = 0;          // block side the block table was built for (0: none)
    double *loss_work = nullptr;  // block-mass objective scratch
    int64_t loss_cap = 0;
    int64_t param_gen = 0;  // bumped by every change of parameters or conductances

    float *comp(int c) { return buf[cur[c]] + (size_t)c * npad; }
    float *spare(int c) { return buf[1 - cur[c]] + (size_t)c * npad; }
    vga::res_t *lcomp(int c) { return lbuf[cur[c]] + (size_t)c * npad; }
    vga::res_t *lspare(int c) { return lbuf[1 - cur[c]] + (size_t)c * npad; }
    int precision() const { return params.state_precision; }
    // transformation and diffusion on different steps (global clock of vga_params.dt_transform)
    bool subcycled() const { return params.dt_transform > 0.0 && params.dt_transform != params.dt; }
};

namespace vga {
// capi.cu: event timing around one kernel launch (no-op unless timing is enabled)
void timing_begin(vga_sim *s, int kind);
void timing_end(vga_sim *s);
void timing_end_weighted(vga_sim *s, int64_t passes);  // the launch covered `passes` time steps
// step.cu
vga_status sim_prepare_params(vga_sim *s, const vga_params *p);
void step_graphs_free(vga_sim *s);
vga_status sim_step_explicit(vga_sim *s, int64_t n_steps);
vga_status sim_diffuse_pass(vga_sim *s);  // last pass of a step call (DOM diffusion only)
vga_status sim_totals(vga_sim *s, double *h_out);
vga_status sim_convert_in(vga_sim *s, const double *d_x);    // device FP64 (5 x n) -> state
vga_status sim_convert_out(vga_sim *s, double *d_x);         // state -> device FP64 (5 x n)
vga_status sim_pack_f32(vga_sim *s, float *d_x, bool to_state);
// Residuals of the current state as / from BF16 bits (5 x n, device), the checkpoint format.
vga_status sim_res_export(vga_sim *s, uint16_t *d_out);
vga_status sim_res_import(vga_sim *s, const uint16_t *d_in);
vga_status sim_transform_pass(vga_sim *s);  // Y = T(X) for every node, all compartments swapped
int64_t sim_ticks_before(const vga_sim *s, int64_t k);  // transformations in the first k steps
int sim_ticks_of_step(const vga_sim *s, int64_t k);      // transformations before diffusion step k
vga_status sim_nbr_table(vga_sim *s, NbrTable *out);  // builds the table on first use
// Per-face conductances (6 x n, device): symmetric across every edge?, largest sum over a node's edges.
vga_status sim_face_check(vga_sim *s, const float *d_g6, bool *symmetric, float *rowmax);
// Copies each edge's gradient from its +x/+y/+z slot into the neighbour's opposite slot (6 x n, device).
vga_status sim_theta_check(vga_sim *s, const float *d_theta, int64_t n, bool *valid, float *maxv);
vga_status sim_face_mirror(vga_sim *s, double *d_g);
// block.cu: P fused passes of a sparse step call as temporally blocked launches (variant 6); *done
// is false (and nothing ran) when the graph, the conductances or the marked nodes do not allow it.
vga_status sim_block_fused(vga_sim *s, int64_t P, bool *done);
void block_free(vga_sim *s);
// wave.cu: P fused passes as one wavefront launch (flips the buffers when P is odd)
vga_status sim_wave_fused(vga_sim *s, int64_t P);
bool wave_params_valid(int chunk, int depth, int ctas_per_sm);
// Builds (if needed) and returns the block table of the current block conductances; false if the
// block grid is too large for it (the decode kernels are used then).
vga_status sim_block_table(vga_sim *s, BlockTable *out, bool *ok);
// Writes the neighbour-offset table of a node set (offsets are relative, so the arrays may start at
// any node offset of a larger concatenated range).  Synchronises the stream.
vga_status build_nbr_table(const Topo &t, uint32_t *ty, uint32_t *tzm, uint32_t *tzp, cudaStream_t st);
// Compact z offsets (NbrTable.tz) of a table of n entries (allocating cap entries) when every z
// offset is below 2^16; *out stays NULL otherwise.
vga_status build_compact_z(int64_t n, int64_t cap, const uint32_t *tzm, const uint32_t *tzp, uint32_t **out,
                           cudaStream_t st);
StateIO state_io(vga_sim *s);          // current buffers in, spare buffers out
StateIO state_io_inplace(vga_sim *s);  // current buffers in and out
// pcg.cu
vga_status sim_step_implicit(vga_sim *s, int64_t n_steps);
void sim_mx_graph_release(vga_sim *s);  // the cached graphs of the mixed solve
// adjoint.cu
vga_status sim_adjoint_forward(vga_sim *s, int64_t N, int64_t ckpt);
vga_status sim_adjoint_grad_theta(vga_sim *s, double *out, bool on_device, int64_t n);
vga_status sim_adjoint_backward(vga_sim *s, const double *d_lamN, double *d_lam0, double *grad8, double *h_gtheta);
vga_status sim_sgd_theta(vga_sim *s, double lr, double lo, double hi);
vga_status sim_block_mass_loss(vga_sim *s, int32_t bs, uint32_t comp_mask, const double *d_target, double *d_work,
                               double *h_loss, double *h_mass, double *d_dldx);
}  // namespace vga
