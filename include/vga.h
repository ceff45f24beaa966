/*
 * vga.h -- C ABI of the GB300 (sm_103a) implementation of the voxel-graph diffusion-transformation
 * method of arXiv 2406.04177 ("A Voxel-based Approach for Simulating Microbial Decomposition in
 * Soil").
 *
 * The calls follow the paper's problem statement: build the graph of pore voxels from a binary
 * image (Sec. II.A), set the parameters and initial masses (Sec. II.A, Sec. IV.C), advance N time
 * steps of transformation followed by diffusion (Sec. III), read the masses and their totals.
 *
 * Conventions common to every call
 *  - Every call returns a vga_status: VGA_OK (0) or a negative error code.  vga_strerror() names
 *    the code; vga_last_error() returns a human-readable detail string for the last failing call
 *    made by the calling thread.
 *  - Handles (vga_graph, vga_sim, vga_batch) are owned by the library and released by the matching
 *    *_free call.  Input arrays are owned by the caller and copied (or read) before the call
 *    returns unless stated otherwise; output arrays are allocated by the caller.
 *  - `stream` arguments are cudaStream_t values passed as void*; NULL means the legacy default
 *    stream.  Work is ordered on that stream.  Calls that hand data back to host memory
 *    synchronise the stream before returning.  vga_sim_step returns as soon as its work is
 *    enqueued; errors raised by that work are reported by the next synchronising call.
 *  - Node order: node i is the i-th kept pore voxel in raster order (x fastest, then y, then z).
 *    State arrays are structure-of-arrays with 5 rows, row c holding compartment c for all nodes:
 *    element (c, i) at offset c*n + i.  Compartments: 0 MB, 1 DOM, 2 SOM, 3 FOM, 4 CO2
 *    (x^1 .. x^5 of Sec. II.A).
 *  - Neighbour slots, always in this order: -x, +x, -y, +y, -z, +z.
 *  - Limits: 1 <= nx, ny, nz <= 32768 and nx*ny*nz < 2^31.
 */
#ifndef VGA_H
#define VGA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum vga_status {
    VGA_OK = 0,
    VGA_ERR_INVALID_ARG = -1,   /* bad size, NULL pointer, non-finite or out-of-range parameter */
    VGA_ERR_OOM = -2,           /* device or host allocation failed */
    VGA_ERR_CUDA = -3,          /* a CUDA runtime call failed (detail in vga_last_error) */
    VGA_ERR_UNSTABLE_DT = -4,   /* explicit step beyond the positivity limit D dt max_i sum_j g_ij <= 1 */
    VGA_ERR_NOT_CONVERGED = -5, /* the implicit solve reached cg_maxit before cg_rtol */
    VGA_ERR_TIMEOUT = -6,       /* a bounded device-side wait gave up (persistent kernels) */
    VGA_ERR_NONFINITE = -7,     /* non-finite value found in a state array */
    VGA_ERR_UNSUPPORTED = -8    /* combination of options not implemented */
} vga_status;

/* Name of a status code (static string, never NULL). */
const char *vga_strerror(int status);
/* Detail of the last failing call on this thread (static per-thread buffer, never NULL). */
const char *vga_last_error(void);
/* Library version as 10000*major + 100*minor + patch. */
int32_t vga_version(void);

/* ============================================================================================
 * Graph of pore voxels (Sec. II.A; Sec. III first paragraph; Fig. 2).
 * V = voxels with I(i,j,k) == 0 (any nonzero value is solid); E = pairs of face-adjacent voxels of
 * V (6-connectivity).  Connected components are numbered in raster order of their first voxel.
 * With VGA_KEEP_LARGEST_COMPONENT only the largest component (ties: the lowest number) becomes the
 * node set; otherwise every pore voxel is a node.  The image border carries no flux.
 * Integer-only and bit-exact: the result never depends on scheduling.
 * ============================================================================================ */
#define VGA_KEEP_LARGEST_COMPONENT 1u
#define VGA_IMAGE_ON_DEVICE 2u /* `img` is a device pointer instead of a host pointer */

typedef struct vga_graph vga_graph;

/* img: nx*ny*nz bytes in C order [z][y][x], host memory (or device memory with
 * VGA_IMAGE_ON_DEVICE).  On success *out receives a new graph.  Errors: VGA_ERR_INVALID_ARG
 * (sizes outside the limits, NULL pointers, unknown flags), VGA_ERR_OOM, VGA_ERR_CUDA. */
vga_status vga_graph_build(const uint8_t *img, int32_t nx, int32_t ny, int32_t nz, uint32_t flags,
                           void *stream, vga_graph **out);

/* Node count n, number of pore components, and the id of the largest component (-1 if none).
 * Any output pointer may be NULL. */
vga_status vga_graph_info(const vga_graph *g, int64_t *n_nodes, int32_t *n_components,
                          int32_t *largest_component);

/* Copies the graph to caller-allocated host arrays; each may be NULL to skip it.
 *   labels[nx*ny*nz]   component id of every pore voxel, -1 for solid voxels
 *   voxel_of_node[n]   raster index (x + nx*(y + ny*z)) of node i
 *   nbr[6*n]           node index of the face neighbour of node i in slot d at nbr[6*i + d], or -1
 *                      when that voxel is solid, outside the image, or not in the node set. */
vga_status vga_graph_export(const vga_graph *g, int32_t *labels, int64_t *voxel_of_node,
                            int32_t *nbr);

vga_status vga_graph_free(vga_graph *g);

/* ============================================================================================
 * Parameters (Sec. II.B, II.C; values of Sec. IV.C).  Units are the caller's, consistently: the
 * reference workloads use masses in ug C, time in days and lengths in voxels.
 * ============================================================================================ */
#define VGA_SCHEME_EXPLICIT 0      /* Scheme 1: m <- (I - D dt L_g) m */
#define VGA_SCHEME_IMPLICIT_PCG 1  /* Scheme 2: (I + D dt L_g) m_new = m, Jacobi-PCG (Sec. III) */
#define VGA_TRANSFORM_SYNC 0       /* every flux from the old state, then update (eq. 3 + clamps) */
#define VGA_TRANSFORM_ASYNC 1      /* sequential growth, mortality, respiration, SOM, FOM */
/* Storage of the state.  One explicit step changes a compartment by 1e-6 .. 1e-8 of its value at
 * the paper's time step, which FP32 rounding biases step after step.  The default keeps, next to
 * every FP32 value, a BF16 residual of its rounding error (about 33 significant bits, 6 bytes per
 * value); VGA_STATE_F32 stores the FP32 value alone (4 bytes, errors grow with the step count). */
#define VGA_STATE_COMPENSATED 0
#define VGA_STATE_F32 1

typedef struct vga_params {
    double D;       /* DOM diffusion coefficient D_DOM */
    double dt;      /* time step of the diffusion (and of the transformation unless dt_transform > 0) */
    double rho;     /* respiration rate */
    double mu;      /* mortality rate */
    double beta;    /* fraction of dead biomass returned to DOM, in [0, 1] */
    double v_som;   /* SOM hydrolysis rate */
    double v_fom;   /* FOM hydrolysis rate */
    double v_dom;   /* maximum growth rate (Monod) */
    double K_dom;   /* half-saturation constant of DOM, > 0, same unit as the masses */
    int32_t scheme;    /* VGA_SCHEME_* */
    int32_t transform; /* VGA_TRANSFORM_* */
    double cg_rtol;    /* implicit only: stop when ||r||_2 <= cg_rtol ||b||_2 */
    int32_t cg_maxit;  /* implicit only: iteration cap per step */
    int32_t state_precision; /* VGA_STATE_* */
    /* Transformation step (Sec. III: when the two processes use different steps, the one with
     * the smaller step is repeated; Table 1 test 3 uses 0.1 s diffusion, 0.43 s transformation).
     * 0 means dt.  Otherwise the simulation keeps a global clock: diffusion step k covers
     * [k dt, (k+1) dt) and is preceded by one transformation of step dt_transform for each tick
     * m * dt_transform (m = 0, 1, ...) in that interval, i.e. ceil((k+1) r - 1e-9) -
     * ceil(k r - 1e-9) of them with r = dt / dt_transform (zero, one or several).  k counts every
     * step taken since creation (vga_sim_get_stats steps_done, restored by vga_sim_load_state).
     * Supported by vga_sim_step with either scheme; the adjoint and the batch reject it
     * (VGA_ERR_UNSUPPORTED). */
    double dt_transform;
} vga_params;

/* ============================================================================================
 * Simulation on one graph (Sec. III).  One time step applies the transformation to every node,
 * then diffuses the transformed DOM with Scheme 1 or Scheme 2.  State and fluxes are FP32 on the
 * device; totals are reduced in FP64; the implicit solve iterates in FP64.
 * ============================================================================================ */
typedef struct vga_sim vga_sim;

/* Creates a simulation on graph g (which must outlive it) with all masses zero.  Errors:
 * VGA_ERR_INVALID_ARG (non-finite or negative parameter, beta outside [0,1], K_dom <= 0, dt <= 0,
 * unknown scheme/transform), VGA_ERR_UNSTABLE_DT (explicit scheme with 6 D dt > 1 under unit
 * conductances), VGA_ERR_OOM, VGA_ERR_CUDA. */
vga_status vga_sim_create(const vga_graph *g, const vga_params *p, void *stream, vga_sim **out);

/* Replaces the parameters (same validation as vga_sim_create). */
vga_status vga_sim_set_params(vga_sim *s, const vga_params *p);

/* Edge conductances g_ij (the voxel form, v_i = v_j = 1, of the Sec. V.A flux with alpha_ij).
 * Block form: the image is cut into cubes of `block_side` voxels; an edge that crosses the face
 * between two face-adjacent blocks gets that face's theta, edges inside a block keep 1.
 * theta (host, FP32) lists the faces normal to x ((nbz, nby, nbx-1) in C order), then normal to
 * y ((nbz, nby-1, nbx)), then normal to z ((nbz-1, nby, nbx)), with nb* = ceil(n* / block_side);
 * n_theta must equal that count.  Values must be finite and >= 0.  With the explicit scheme the
 * call fails with VGA_ERR_UNSTABLE_DT when 6 D dt max(1, max theta) > 1. */
vga_status vga_sim_set_block_conductances(vga_sim *s, int32_t block_side, const float *theta,
                                          int64_t n_theta);
/* The same with theta in device memory (d_theta, FP32, n_theta values, read on the simulation's
 * stream): the values are checked on the device before they are copied (VGA_ERR_INVALID_ARG for a
 * value that is not finite or is negative, leaving the previous conductances in place), and only a
 * flag and the largest value come back to the host.  The caller keeps d_theta. */
vga_status vga_sim_set_block_conductances_device(vga_sim *s, int32_t block_side, const float *d_theta,
                                                 int64_t n_theta);
/* Returns to unit conductances (g_ij = 1, Sec. II.B). */
vga_status vga_sim_clear_conductances(vga_sim *s);

/* Per-face conductances: the weighted flux of Sec. V.A, J_ij = -D g_ij (m_i - m_j) dt, with one
 * conductance per voxel edge (the voxel form of the alpha_ij of the coarse model).  g_face: host,
 * 6 x n FP32, g_face[6 i + d] = g of the edge leaving node i through slot d, slot order -x, +x, -y,
 * +y, -z, +z (as vga_graph_export's nbr); entries of absent edges are ignored.  Every value must be
 * finite and >= 0 and both slots of an edge must hold the same value (checked on the device:
 * VGA_ERR_INVALID_ARG otherwise); the explicit scheme needs D dt sum_j g_ij <= 1 at every node
 * (VGA_ERR_UNSTABLE_DT otherwise, Sec. II.B.3a).  Replaces block conductances.  Every scheme and
 * the adjoint use them; vga_adjoint_backward then returns dL/dg in grad_theta as 6 x n doubles in the
 * same layout (both slots of an edge hold the edge's derivative).  Requires nx <= 32767 and fewer
 * than 2^26 nodes (VGA_ERR_UNSUPPORTED).  vga_sgd_block_conductances and
 * vga_sim_get_block_conductances return VGA_ERR_UNSUPPORTED while they are set. */
vga_status vga_sim_set_face_conductances(vga_sim *s, const float *g_face);

/* Initial or replacement state X (5 x n, FP64, SoA).  Values are rounded to FP32.  on_device != 0
 * means x is a device pointer.  Errors: VGA_ERR_NONFINITE if a value is not finite (host input
 * only; device input is converted unchecked). */
vga_status vga_sim_set_masses(vga_sim *s, const double *x, int32_t on_device);
/* Current state X (5 x n, FP64) into caller memory (host, or device if on_device != 0). */
vga_status vga_sim_get_masses(vga_sim *s, double *x, int32_t on_device);
/* FP32 variants of the two calls above (same layout).  Set: residuals become zero.  Get: the value
 * rounded to FP32. */
vga_status vga_sim_set_state_f32(vga_sim *s, const float *x, int32_t on_device);
vga_status vga_sim_get_state_f32(vga_sim *s, float *x, int32_t on_device);

/* Implicit solver (Scheme 2).  VGA_SOLVER_FP64_PCG: Jacobi-PCG in FP64, stopping on the
 * recurrence residual.  VGA_SOLVER_MIXED_REFINEMENT (default): x, b and the residual b - B x are
 * kept in float-float (two FP32 numbers, about 48 significant bits, computed with error-free FP32
 * operations) and each correction is solved by the same Jacobi-PCG in FP32 (to a 1e-4 reduction);
 * stops when the true residual satisfies ||b - B x||_2 <= cg_rtol ||b||_2; iterations count the FP32
 * inner iterations against cg_maxit.  Used with unit conductances (block conductances run the FP64
 * solver).  The whole mixed solve runs as one CUDA graph whose outer and inner loops are
 * conditional (while) nodes set by the solver's own kernels, so the host synchronises once per
 * time step; where the driver cannot build such a graph the solve falls back to the host-driven
 * loop.  VGA_SOLVER_MIXED_HOST_LOOP: the same solver with its loops driven from the host (the done
 * flags polled every 8 inner iterations); the same kernels in the same order, so the same bits.
 * Errors: VGA_ERR_INVALID_ARG. */
#define VGA_SOLVER_FP64_PCG 0
#define VGA_SOLVER_MIXED_REFINEMENT 1
#define VGA_SOLVER_MIXED_HOST_LOOP 2
vga_status vga_sim_set_solver(vga_sim *s, int32_t solver);

/* Exact checkpoint of the state: the FP32 values, their residuals and the step counter, in a
 * caller-allocated host buffer of vga_sim_state_bytes() bytes (a 32-byte header, then the 5n FP32
 * values, then the 5n BF16 residuals, compartment-major; valid for a simulation on the same graph
 * with the same state_precision).  Restoring it and stepping reproduces an uninterrupted run bit
 * for bit. */
vga_status vga_sim_state_bytes(const vga_sim *s, int64_t *bytes);
vga_status vga_sim_save_state(vga_sim *s, void *buf, int64_t bytes);
vga_status vga_sim_load_state(vga_sim *s, const void *buf, int64_t bytes);

/* Advances n_steps >= 0 time steps (Sec. III: transformation, then diffusion of DOM).
 * Asynchronous on the simulation's stream.  Implicit scheme: synchronises to test convergence
 * and returns VGA_ERR_NOT_CONVERGED if any solve hit cg_maxit (the state then holds the last
 * iterate). */
vga_status vga_sim_step(vga_sim *s, int64_t n_steps);

/* FP64 totals of the 5 compartments over all nodes, into totals[5] (host).  Deterministic.  The
 * same pass scans the state: a non-finite value returns VGA_ERR_NONFINITE (totals still written);
 * a negative one counts in vga_sim_stats.negative_reports (within the stability bound the schemes
 * keep every compartment >= 0 in exact arithmetic; at the bound itself rounding can leave a value
 * a few ulps below zero, so a negative value is reported, not an error). */
vga_status vga_sim_totals(vga_sim *s, double *totals);

/* Waits for the simulation's stream; reports errors of previously enqueued work. */
vga_status vga_sim_sync(vga_sim *s);

typedef struct vga_sim_stats {
    int64_t steps_done;       /* time steps since creation */
    int64_t cg_iterations;    /* implicit scheme: PCG iterations since creation */
    double cg_last_relres;    /* implicit scheme: final relative residual of the last solve */
    int64_t kernel_launches;  /* kernels launched since creation (inside a graph: kernels it ran) */
    int64_t graph_launches;   /* implicit scheme: CUDA graph launches of the mixed solve */
    int64_t active_nodes;     /* nodes the sparse fused pass transforms (-1: no activity mask built) */
    int64_t blocked_passes;   /* fused passes run temporally blocked (kernel variant 6) since creation */
    int64_t negative_reports; /* vga_sim_totals calls whose scan of the state found a negative mass */
} vga_sim_stats;
vga_status vga_sim_get_stats(vga_sim *s, vga_sim_stats *out);

/* ============================================================================================
 * Discrete adjoint of the explicit scheme with synchronous transformation (compensated state).
 * The reverse of one step X^{k+1} = (y1, Q_g y2, y3, y4, y5), y = T(X^k), Q_g = I - D dt L_g:
 *   mu = (lam1, Q_g lam2, lam3, lam4, lam5), dL/dX^k = J_T(X^k)^T mu,
 * with FP64 gradients with respect to D, the seven rate constants, and the block conductances
 * theta (the voxel form of the Sec. V.A conductances; the one-step closed forms of Sec. V.A are the
 * special case of a single diffusion step).
 * ============================================================================================ */

/* Advances n_steps from the current state X^0, storing a checkpoint every ckpt_every steps; the
 * simulation ends at X^N exactly as vga_sim_step would leave it.  Device memory: one state per
 * checkpoint (30 bytes per node) plus ckpt_every recorded steps: 4 bytes per node each when the
 * activity skip is on (the default: X^k is recorded for the nodes with MB, SOM, FOM or CO2 at X^0,
 * 16 bytes per such node), else 24 bytes per node each.
 * Errors: VGA_ERR_UNSUPPORTED unless scheme = explicit, transform = sync and state_precision =
 * compensated; VGA_ERR_INVALID_ARG for n_steps < 0 or ckpt_every < 1. */
vga_status vga_adjoint_forward(vga_sim *s, int64_t n_steps, int32_t ckpt_every);

/* Back-propagates dL_dXN (5 x n FP64, host or device as on_device says) through the steps of the
 * last vga_adjoint_forward.  Outputs: dL_dX0 (5 x n FP64 in the same memory space, or NULL);
 * grad_params[8] (host) = dL/d(D, rho, mu, beta, v_som, v_fom, v_dom, K_dom); grad_theta (host,
 * n_theta doubles in the layout of vga_sim_set_block_conductances, or NULL; zero without block
 * conductances).  dL_dX0 and grad_params are the same bits on every run; the conductance gradients
 * are sums of FP64 atomics, whose last bits can depend on their order.  The state stays at X^N.
 * Errors: VGA_ERR_INVALID_ARG if no forward pass was run or the parameters or conductances changed
 * since. */
vga_status vga_adjoint_backward(vga_sim *s, const double *dL_dXN, int32_t on_device, double *dL_dX0,
                                double *grad_params, double *grad_theta);

/* Copies the conductance gradient of the last vga_adjoint_backward (block or per-face conductances,
 * FP64, the layout of grad_theta there) into grad_theta: n doubles, n = the number of conductances
 * set (n_theta, or 6 n for per-face conductances), in device memory if on_device != 0, else host.
 * Errors: VGA_ERR_INVALID_ARG without a completed backward sweep with conductances set, or for
 * another n. */
vga_status vga_adjoint_grad_theta(vga_sim *s, double *grad_theta, int32_t on_device, int64_t n);

/* Normalised gradient step of Sec. V.A on the block conductances, using the theta gradient of the
 * last vga_adjoint_backward: theta <- clamp(theta - lr * g/|g|, theta_min, theta_max) element-wise
 * (g/|g| = 0 where g = 0), on the device.  Errors: VGA_ERR_INVALID_ARG (no gradient, no block
 * conductances, bad bounds), VGA_ERR_UNSTABLE_DT (explicit scheme with 6 D dt theta_max > 1). */
vga_status vga_sgd_block_conductances(vga_sim *s, double lr, double theta_min, double theta_max);
/* Current block conductances (host copy, n_theta values). */
vga_status vga_sim_get_block_conductances(vga_sim *s, float *theta, int64_t n_theta);

/* Block-mass objective: the image is cut into cubes of block_side voxels; for every compartment c
 * in comp_mask (bit c) and block b, M_cb = sum of x^c over the nodes of b.
 * L = sum_cb (M_cb - target_cb)^2.  target (host): one row of nblocks values per selected
 * compartment, in increasing c, blocks in C order (nbz, nby, nbx).  Outputs: *loss (host),
 * block_mass (host, same layout as target, or NULL), dL_dX (device, 5 x n FP64, or NULL). */
vga_status vga_loss_block_mass(vga_sim *s, int32_t block_side, uint32_t comp_mask, const double *target,
                               double *loss, double *block_mass, double *dL_dX);

/* Explicit-step kernel selection (all variants give bit-identical results):
 *   0  chunks of `chunk` nodes decode their neighbours from the row bitmask, then load directly;
 *   1  as 0, with each chunk's own state staged in shared memory by bulk asynchronous copies and
 *      written back the same way (chunk = 512, 1024 or 2048);
 *   2  one node per thread with a precomputed neighbour-offset table (12 bytes per node, built on
 *      first use; nx <= 32767, otherwise variant 0 runs).  `chunk` is ignored;
 *   3  the table passes of one vga_sim_step call run inside one persistent cooperative launch as a
 *      wavefront over chunks of `chunk` nodes (a multiple of 256), so that each pass reads the
 *      previous pass's output from L2; 4 passes per block, CTAs per SM from the occupancy (see
 *      vga_sim_set_wavefront).  Not used when dt_transform differs from dt (variant 2 runs);
 *   4  as 2 with two consecutive nodes per thread, the per-node streams moved as 8-byte vectors
 *      (FP32 values, table words) and 4-byte vectors (residuals);
 *   5  as 2 with four consecutive nodes per thread, 16-byte and 8-byte vectors;
 *   6  as 5, except that the fused passes of a sparse step call (see vga_sim_set_activity_skip) run
 *      temporally blocked: the DOM is permuted into tile order (tiles of 32 x 16 x 16 voxels) for the
 *      call, and each launch advances every tile by up to 3 passes in shared memory, recomputing a
 *      3-voxel halo (Scheme 1 applied repeatedly, Sec. II.B.3a; the transformation of the marked
 *      nodes of Sec. II.C between the diffusions).  Unit conductances and equal transformation and
 *      diffusion steps only; otherwise, and when a tile's halo region holds more nodes or marked
 *      nodes than its shared-memory capacity, the call runs as 5.
 * For 4, 5 and 6 `chunk` is ignored.  The default is 5. */
vga_status vga_sim_set_kernel(vga_sim *s, int32_t variant, int32_t chunk);

/* Sparse fused pass of variant 5 (on by default).  Every flux of the transformation (Sec. II.C) is
 * proportional to MB, SOM or FOM, so at nodes where MB, SOM, FOM and CO2 are all zero the
 * transformation is the identity, and it stays so while stepping (no flux can make them nonzero).
 * The first step after a state upload (vga_sim_set_masses, vga_sim_set_state_f32,
 * vga_sim_load_state) marks the other nodes in a bit mask (one extra pass, one synchronisation); a
 * fused pass then diffuses the DOM of every node, transforms only the marked nodes (a second kernel
 * over them in rank order, their MB, SOM, FOM and CO2 held in a compact rank-ordered copy during the
 * call), and leaves the MB, SOM, FOM and CO2 of the others unread and unwritten.  Results are bit-identical with the mask off (also a node whose values are negative
 * zeros is marked).  on = 0 transforms every node every pass. */
vga_status vga_sim_set_activity_skip(vga_sim *s, int32_t on);

/* Selects variant 3 with `chunk` nodes per work item (a power of two in [256, 8192]; CTAs of
 * min(chunk, 1024) threads), `depth`
 * passes per block of the skewed order (1..64: the passes whose intermediate states stay in L2),
 * and ctas_per_sm persistent CTAs per SM (0 = as many as fit).  Every wait of the persistent
 * kernel is bounded; one that gives up makes the next synchronising call return VGA_ERR_TIMEOUT
 * (the state is then undefined). */
vga_status vga_sim_set_wavefront(vga_sim *s, int32_t chunk, int32_t depth, int32_t ctas_per_sm);

#define VGA_TUNE_MAX 16
typedef struct vga_tune_entry {
    int32_t variant;
    int32_t chunk;
    int32_t depth;        /* variant 3: passes per block; 0 otherwise */
    int32_t ctas_per_sm;  /* variant 3: CTAs per SM (0 = occupancy); 0 otherwise */
    double ms_per_step;
} vga_tune_entry;
typedef struct vga_tune_result {
    int32_t count;  /* entries filled */
    int32_t best;   /* index of the selected entry (-1 if nothing was timed) */
    vga_tune_entry entries[VGA_TUNE_MAX];
} vga_tune_result;
/* Times trial_steps explicit steps for every candidate (variant x chunk) on this simulation with
 * CUDA events, selects the fastest, and restores the state and step counter.  Allocates a
 * temporary copy of the state. */
vga_status vga_sim_autotune(vga_sim *s, int32_t trial_steps, vga_tune_result *out);

/* ============================================================================================
 * Batched simulation: many independent graphs (uneven node counts, per-instance parameters)
 * advanced together by one persistent cooperative kernel per launch, several time steps per
 * launch with a bounded grid-wide barrier between passes, the launches of one call captured in a
 * CUDA graph and replayed.  Explicit scheme only; all instances share transform and
 * state_precision.  Results are bit-identical to vga_sim on each graph.
 * ============================================================================================ */
typedef struct vga_batch vga_batch;

/* graphs[count] (must outlive the batch) and params[count].  The batch owns a private stream.
 * Errors: VGA_ERR_INVALID_ARG, VGA_ERR_UNSUPPORTED (implicit scheme, nx > 32767),
 * VGA_ERR_UNSTABLE_DT, VGA_ERR_OOM, VGA_ERR_CUDA. */
vga_status vga_batch_create(const vga_graph *const *graphs, const vga_params *params, int32_t count,
                            vga_batch **out);
/* Total node count and (if non-NULL) the first node of every instance in the concatenated range. */
vga_status vga_batch_info(const vga_batch *b, int64_t *total_nodes, int64_t *node_offsets);
/* State of one instance, (5 x n_instance) FP64 host arrays. */
vga_status vga_batch_set_masses(vga_batch *b, int32_t instance, const double *x);
vga_status vga_batch_get_masses(vga_batch *b, int32_t instance, double *x);
/* Advances every instance n_steps; returns when done.  VGA_ERR_TIMEOUT if a barrier gave up. */
vga_status vga_batch_step(vga_batch *b, int64_t n_steps);
/* Launch shape: time steps per persistent launch, resident blocks per SM (0 = occupancy maximum),
 * CUDA-graph capture on or off. */
vga_status vga_batch_set_launch(vga_batch *b, int32_t steps_per_launch, int32_t blocks_per_sm, int32_t use_graph);

/* Sparse fused passes for the batch, as vga_sim_set_activity_skip (on by default): the first step
 * call after vga_batch_set_masses marks the nodes where the transformation can change the state;
 * the fused passes then transform only those.  Bit-identical with on = 0. */
vga_status vga_batch_set_activity_skip(vga_batch *b, int32_t on);

/* Test hook of the bounded waits (no counterpart in the paper).  The batched launches are
 * cooperative and separate their passes by grid-wide barriers whose waits are bounded.  With
 * skip_block >= 0, block skip_block of every launch of the batch returns before its first barrier
 * arrival, so the other blocks' waits run out after spin_limit polls of 64 ns each (0: the default
 * limit, 2^26 polls) and vga_batch_step returns VGA_ERR_TIMEOUT; the device error flag and the
 * barrier words are reset then, and the state is undefined until the next vga_batch_set_masses.
 * skip_block = -1 switches the hook off (spin_limit still applies).  Nothing faults, traps or hangs. */
vga_status vga_batch_set_wait_test(vga_batch *b, int32_t skip_block, uint32_t spin_limit);

typedef struct vga_batch_stats {
    int32_t instances;
    int32_t grid_blocks;
    int64_t total_nodes;
    int32_t steps_per_launch;
    int32_t capture_failed; /* 1 if graph capture was refused and launches run directly */
    int64_t kernel_launches;
    int64_t graph_replays;
    int64_t steps_done;
} vga_batch_stats;
vga_status vga_batch_get_stats(const vga_batch *b, vga_batch_stats *out);

typedef struct vga_batch_tune_entry {
    int32_t steps_per_launch;
    int32_t blocks_per_sm;
    int32_t grid_blocks;
    int32_t pad;
    double ms_per_step;
} vga_batch_tune_entry;
typedef struct vga_batch_tune {
    int32_t count;
    int32_t best;
    vga_batch_tune_entry entries[VGA_TUNE_MAX];
} vga_batch_tune;
/* Times trial_steps for each (steps per launch x blocks per SM) candidate, keeps the fastest and
 * restores the state. */
vga_status vga_batch_autotune(vga_batch *b, int32_t trial_steps, vga_batch_tune *out);
vga_status vga_batch_free(vga_batch *b);

/* Kernel timing.  When enabled, the library records a CUDA event pair on the simulation's stream
 * around every kernel it launches and accumulates the elapsed times per kernel kind; reading them
 * synchronises the stream.  The fused passes of one explicit step call are timed as one span and
 * counted as that many launches (an event pair between two passes would keep the second from being
 * scheduled during the first's tail), so ms / launches is their live mean per pass.  Kinds: */
#define VGA_KERNEL_FUSED_STEP 0    /* explicit pass: diffuse stored transformed DOM, transform */
#define VGA_KERNEL_TRANSFORM 1     /* transformation-only pass (first pass of a step call) */
#define VGA_KERNEL_DIFFUSE 2       /* diffusion-only pass (last pass of a step call) */
#define VGA_KERNEL_TOTALS 3        /* FP64 compartment totals */
#define VGA_KERNEL_PCG_STENCIL 4   /* implicit: initial residual and B p products */
#define VGA_KERNEL_PCG_VECTOR 5    /* implicit: vector updates and scalar reductions */
#define VGA_KERNEL_ADJOINT 6       /* reverse step of the discrete adjoint */
#define VGA_KERNEL_OTHER 7         /* conversions, packing, losses */
#define VGA_KERNEL_KINDS 8
typedef struct vga_kernel_timing {
    double ms[VGA_KERNEL_KINDS];        /* summed event-to-event milliseconds per kind */
    int64_t launches[VGA_KERNEL_KINDS]; /* timed launches (fused passes: passes) per kind */
} vga_kernel_timing;
vga_status vga_sim_enable_timing(vga_sim *s, int32_t on);
/* Copies the accumulated timings into *out (after synchronising); reset != 0 clears them. */
vga_status vga_sim_read_timing(vga_sim *s, vga_kernel_timing *out, int32_t reset);

vga_status vga_sim_free(vga_sim *s);

/* ============================================================================================
 * Coarse primitive-graph diffusion model (PNGM) and its calibration from voxel data (Sec. V.A).
 *
 * The pore voxels are partitioned into q primitives (one label per node).  Primitive i has volume
 * v_i = its voxel count; primitives joined by at least one voxel face are adjacent, with S_ij
 * shared faces and d_ij = distance between their voxel centroids.  Masses follow
 *   Scheme 3 (explicit)  m_i^{k+1} = m_i^k - c sum_j theta_ij (m_i^k / v_i - m_j^k / v_j)
 *   Scheme 4 (implicit)  m_i^k = m_i^{k+1} + c sum_j theta_ij (m_i^{k+1} / v_i - m_j^{k+1} / v_j)
 * with c = D dt.  The conductances theta are stored per ordered pair (i, j) in CSR order (rows
 * by i, columns ascending), "slots"; their initial value is S_ij / d_ij (Sec. V.B).  Calibration
 * minimises, over l pairs (X^p, Y^p) of primitive mass vectors one coarse step apart,
 *   Objective 1  L1 = 1/(l q) sum_p sum_i (y_i - x_i + c sum_j theta_ij (x_i/v_i - x_j/v_j))^2
 *   Objective 2  L2 = 1/(l q) sum_p sum_i (x_i - y_i - c sum_j theta_ij (y_i/v_i - y_j/v_j))^2
 * by the normalised update theta_s <- theta_s - lr sign(dL/dtheta_s) (sign(0) = 0).  The gradient
 * per slot (i, j) involves row i only; with tied != 0 slots (i, j) and (j, i) share the sum of
 * their two gradients, which keeps theta symmetric.  dL2/dtheta_ij = -(2 c / (l q)) sum_p
 * r_i (y_i/v_i - y_j/v_j): the sign is that of the residual's derivative.
 * ============================================================================================ */
typedef struct vga_pngm vga_pngm;

typedef struct vga_pngm_info {
    int32_t q;                   /* primitives */
    int32_t n_slots;             /* ordered adjacent pairs (twice the undirected pairs) */
    int64_t n_nodes;             /* nodes of the graph */
    int64_t cross_faces;         /* voxel faces between different primitives */
    int32_t symmetric;           /* 1 if theta_ij == theta_ji for every pair */
    int64_t last_cg_iterations;  /* Scheme 4: PCG iterations summed over the last vga_pngm_step */
    double last_cg_relres;       /* Scheme 4: relative residual of its last solve */
} vga_pngm_info;

/* Builds the coarse graph of graph g under the partition labels[n] (int32, values in [0, q), host
 * memory, or device memory when on_device != 0; copied, so the caller keeps ownership).  Every
 * primitive must hold at least one node.  Volumes, face counts and centroids are exact integer
 * sums; theta starts at S_ij / d_ij.  Work is ordered on `stream` (NULL = default stream), which
 * the handle keeps for its own calls; the call synchronises it.  Errors: VGA_ERR_INVALID_ARG
 * (q < 1, q > n, a label outside [0, q), an empty primitive, NULL pointers), VGA_ERR_UNSUPPORTED
 * (more than 2^31 - 1 slots), VGA_ERR_OOM, VGA_ERR_CUDA. */
vga_status vga_pngm_create(const vga_graph *g, const int32_t *labels, int32_t on_device, int32_t q, void *stream,
                           vga_pngm **out);

vga_status vga_pngm_get_info(const vga_pngm *pg, vga_pngm_info *out);

/* Copies the geometry to host arrays (each may be NULL): volumes[q], centroids[3q] as (x, y, z)
 * per primitive in voxel units, row_ptr[q+1], col[n_slots], rev[n_slots] (slot of (j, i)),
 * surface[n_slots] = S_ij, distance[n_slots] = d_ij. */
vga_status vga_pngm_export(const vga_pngm *pg, double *volumes, double *centroids, int32_t *row_ptr, int32_t *col,
                           int32_t *rev, double *surface, double *distance);

/* Replaces / reads theta[n_slots] (FP64, host, or device when on_device != 0).  Values must be
 * finite.  Errors: VGA_ERR_INVALID_ARG, VGA_ERR_CUDA. */
vga_status vga_pngm_set_theta(vga_pngm *pg, const double *theta, int32_t on_device);
vga_status vga_pngm_get_theta(const vga_pngm *pg, double *theta, int32_t on_device);

/* Primitive masses of compartment comp (0..4) of simulation s (which must run on the same graph):
 * d_out[i] = sum of the node masses of primitive i (device, FP64, q entries; overwritten), ordered
 * on the simulation's stream.  The sums are exact in fixed point (every node mass rounded to a
 * multiple of 2^(e-61), where the sum of |masses| is below 2^e), so the result is deterministic.
 * Errors: VGA_ERR_INVALID_ARG, VGA_ERR_OOM, VGA_ERR_CUDA. */
vga_status vga_pngm_restrict(vga_pngm *pg, vga_sim *s, int32_t comp, double *d_out);

/* n_steps coarse steps of d_m[q] (device, FP64, in place) with c = D dt: scheme
 * VGA_SCHEME_EXPLICIT = Scheme 3 (FP64, rounding as written), VGA_SCHEME_IMPLICIT_PCG = Scheme 4,
 * solved as (V + c L) u = m^k, m^{k+1} = V u by Jacobi-PCG (start u = m^k / v, stop when
 * ||r||_2 <= cg_rtol ||m^k||_2 or after cg_maxit iterations).  Scheme 4 needs symmetric theta.
 * Synchronises the handle's stream.  Errors: VGA_ERR_INVALID_ARG, VGA_ERR_UNSUPPORTED (Scheme 4
 * with theta_ij != theta_ji), VGA_ERR_NOT_CONVERGED (a solve hit cg_maxit; m holds its last
 * iterate), VGA_ERR_CUDA. */
vga_status vga_pngm_step(vga_pngm *pg, double *d_m, int64_t n_steps, int32_t scheme, double D, double dt, double cg_rtol,
                         int32_t cg_maxit);

/* Objective 1 or 2 (objective_kind) over the l pairs X^p = record pairs[2p], Y^p = record
 * pairs[2p+1] of d_data (device, FP64, n_records x q, row-major); pairs is a host array of 2l
 * record indices.  *loss (host, may be NULL) receives the objective; d_grad (device, n_slots,
 * may be NULL) its gradient per slot (tied: summed over (i, j) and (j, i)).  Synchronises the
 * handle's stream.  Errors: VGA_ERR_INVALID_ARG (kind, l < 1, an index outside [0, n_records),
 * D < 0, dt <= 0), VGA_ERR_CUDA. */
vga_status vga_pngm_objective(vga_pngm *pg, int32_t objective_kind, const double *d_data, int64_t n_records,
                              const int32_t *pairs, int32_t l, double D, double dt, int32_t tied, double *loss,
                              double *d_grad);

/* One normalised SGD update of theta on the objective over the given pairs (as
 * vga_pngm_objective): theta_s <- max(theta_s - lr sign(g_s), theta_min).  theta_min = -INFINITY
 * gives the paper's update; 0 keeps conductances non-negative, which Scheme 4 needs to stay
 * positive definite.  *loss_before receives the objective before the update. */
vga_status vga_pngm_sgd_step(vga_pngm *pg, int32_t objective_kind, const double *d_data, int64_t n_records,
                             const int32_t *pairs, int32_t l, double D, double dt, double lr, double theta_min,
                             int32_t tied, double *loss_before);

vga_status vga_pngm_free(vga_pngm *pg);

/* ============================================================================================
 * Allocation-free totals.  The paper has no counterpart: this entry point exists for callers that
 * cannot let a library allocate device memory -- an application that owns the GPU memory pool or
 * runs under a hard memory cap and passes its plugins only the buffers to work on, or a latency-
 * critical loop where cudaMalloc/cudaFree would stall on an implicit device synchronisation.
 *
 * Computes the FP64 totals of the 5 compartments of a state held by the caller: values (device,
 * FP32, compartment c at values + c*row_stride, n entries each), optional residuals (device, BF16
 * bits in the same layout, added to the values; NULL for none), into totals (device, 5 doubles),
 * ordered on `stream`.  It calls no cudaMalloc, cudaFree or other allocating routine: its scratch
 * is a fixed 160 KiB array in the library's device memory (present on every GPU that loads the
 * library, until the process exits), which limits n to 33,554,432 nodes; larger n returns
 * VGA_ERR_INVALID_ARG.  The first call on a device looks up that array's address (with the device
 * current), so make that first call before any stream capture.  The address is kept per device
 * ordinal for the rest of the process: it belongs to the device's primary context (the one the CUDA
 * runtime uses), so it does not survive cudaDeviceReset and is wrong under another context made
 * current through the driver API.  All calls share the array: calls that overlap on the GPU race,
 * so serialise them.  The library cannot check the caller's buffers: values (and residuals) must
 * hold 4*row_stride + n elements and totals 5.  Errors: VGA_ERR_INVALID_ARG (NULL pointers, n < 0,
 * row_stride < n, n over the limit), VGA_ERR_CUDA. */
vga_status vga_state_totals_noalloc(const float *values, const uint16_t *residuals, int64_t n,
                                    int64_t row_stride, double *totals, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* VGA_H */
