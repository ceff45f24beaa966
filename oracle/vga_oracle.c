/*
 * vga_oracle.c -- plain FP64 CPU restatement of the voxel-graph method of arXiv 2406.04177
 * ("A Voxel-based Approach for Simulating Microbial Decomposition in Soil").
 *
 * TEST INFRASTRUCTURE.  This file is the correctness oracle: only the test suite, the package's
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no code, header, table
 * or helper with the CUDA library, and the CUDA library never calls it.
 *
 * It is deliberately slow and literal: adjacency lists, one voxel at a time, FP64 throughout,
 * no blocking or fusion.  Per-voxel loops carry an OpenMP pragma, as the paper marks them
 * "Parallel loop" (Appendix A); results do not depend on the thread count except through the
 * summation order of the FP64 dot products inside the conjugate-gradient solver.
 *
 * Readings of the paper applied here (the paper is garbled or silent at these points):
 *  R1  Scheme 1 sign: the update subtracts D*dt*sum_j (m_i - m_j) (Sec. II.B.3a, the matrix form
 *      Q = I - D dt Laplacian); the intermediate line printed with "+D" is a typo.
 *  R2  Edges are the 6 face neighbours, i != j (Sec. II.A text and Fig. 2), not every pair of
 *      touching voxels.
 *  R3  The appendix titles are swapped: the algorithm that computes every flux from the old state
 *      and then updates (Appendix A, first listing) is the "synchronous" transformation of
 *      Sec. III; the sequential one (second listing) is the "asynchronous" transformation.
 *  R4  Synchronous transformation clamps exactly as printed: uptake <= DOM, resp+morta <= MB
 *      (mortality first), turnover of FOM <= FOM and of SOM <= SOM, strict ">" comparisons.
 *      The names morDOM/morSOM in the update lines mean mortaDOM/mortaSOM.
 *  R5  Asynchronous transformation: the SOM branch compares turnSOM (printed "resp") with SOM,
 *      the FOM branch compares turnFOM (printed "resp < x3") with FOM; in the exhaustion
 *      branches the compartment is added to DOM before being set to zero; when mortality
 *      exceeds the biomass, all biomass is split between DOM and SOM and MB becomes 0 (the
 *      listing omits the reset, which would create carbon).
 *  R6  Each time step applies the transformation to every voxel first, then diffuses the
 *      transformed DOM (Sec. II.A last paragraph, Sec. III); one common dt for both processes.
 *  R7  Implicit scheme: (I + D dt L_g) m^{k+1} = y solved by Jacobi-preconditioned CG with
 *      T = diag(1/b_ii) (Sec. III), initial guess y, stop when ||r||_2 <= rtol ||y||_2.
 *  R8  Weighted edges: the flux over edge (i,j) is multiplied by a symmetric conductance g_ij,
 *      the voxel form (v_i = v_j = 1) of the PNGM flux F_ij with alpha_ij (Sec. V.A).
 *  R9  Mortality split: mortaDOM = beta*morta and mortaSOM = (1-beta)*morta as printed.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    double D, dt, rho, mu, beta, v_som, v_fom, v_dom, K_dom;
} vo_params;

/* Neighbour slots, in this order for every node: -x, +x, -y, +y, -z, +z. */
enum { NB = 6 };

int vo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Thread count of the parallel loops from here on (the benchmark times one thread and all cores). */
void vo_set_num_threads(int k) {
    if (k > 0) omp_set_num_threads(k);
}

/* ------------------------------------------------------------------------------------------
 * Graph construction (Sec. II.A; Sec. III first paragraph; Fig. 2).
 * V = voxels with I == 0; edges join face-adjacent voxels of V.  Components are labelled by a
 * breadth-first search started from each still-unlabelled pore voxel in raster order, so the
 * component id is the rank of the component's smallest raster index.  With keep_largest the
 * node set is restricted to the largest component (ties: smallest id).  Node index = rank of
 * the voxel in raster order among the kept voxels.  The image border carries no flux: voxels
 * outside the image are not nodes.
 * Returns the number of nodes n, or -1 on bad arguments / allocation failure.
 * labels[nvox]: component id of each pore voxel, -1 for solid.
 * voxel_of_node[n], nbr[6n] (-1 where the face neighbour is not a node) need capacity nvox, 6nvox.
 * ---------------------------------------------------------------------------------------- */
int64_t vo_graph_build(const uint8_t *img, int nx, int ny, int nz, int keep_largest,
                       int32_t *labels, int32_t *n_components, int32_t *largest,
                       int64_t *voxel_of_node, int32_t *nbr) {
    if (nx <= 0 || ny <= 0 || nz <= 0) return -1;
    const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
    const int64_t nvox = sz * nz;
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)nvox);
    int64_t *comp_size = NULL;
    int64_t ncomp = 0, cap = 0;
    if (!queue) return -1;
    for (int64_t v = 0; v < nvox; ++v) labels[v] = -1;

    for (int64_t s = 0; s < nvox; ++s) {
        if (img[s] != 0 || labels[s] != -1) continue;
        if (ncomp == cap) {
            cap = cap ? 2 * cap : 1024;
            int64_t *tmp = (int64_t *)realloc(comp_size, sizeof(int64_t) * (size_t)cap);
            if (!tmp) { free(queue); free(comp_size); return -1; }
            comp_size = tmp;
        }
        const int32_t id = (int32_t)ncomp;
        int64_t head = 0, tail = 0;
        labels[s] = id;
        queue[tail++] = s;
        while (head < tail) {
            const int64_t v = queue[head++];
            const int64_t x = v % nx, y = (v / nx) % ny, z = v / sz;
            int64_t cand[NB];
            int has[NB];
            has[0] = x > 0;      cand[0] = v - sx;
            has[1] = x < nx - 1; cand[1] = v + sx;
            has[2] = y > 0;      cand[2] = v - sy;
            has[3] = y < ny - 1; cand[3] = v + sy;
            has[4] = z > 0;      cand[4] = v - sz;
            has[5] = z < nz - 1; cand[5] = v + sz;
            for (int d = 0; d < NB; ++d) {
                if (!has[d]) continue;
                const int64_t u = cand[d];
                if (img[u] == 0 && labels[u] == -1) {
                    labels[u] = id;
                    queue[tail++] = u;
                }
            }
        }
        comp_size[ncomp++] = tail;
    }

    int32_t best = -1;
    for (int64_t c = 0; c < ncomp; ++c)
        if (best < 0 || comp_size[c] > comp_size[best]) best = (int32_t)c;
    *n_components = (int32_t)ncomp;
    *largest = best;

    /* node index of every kept voxel; queue is reused as the voxel -> node map */
    int64_t n = 0;
    for (int64_t v = 0; v < nvox; ++v) {
        const int kept = labels[v] >= 0 && (!keep_largest || labels[v] == best);
        if (kept) {
            queue[v] = n;
            voxel_of_node[n] = v;
            ++n;
        } else {
            queue[v] = -1;
        }
    }
    for (int64_t i = 0; i < n; ++i) {
        const int64_t v = voxel_of_node[i];
        const int64_t x = v % nx, y = (v / nx) % ny, z = v / sz;
        int64_t cand[NB];
        int has[NB];
        has[0] = x > 0;      cand[0] = v - sx;
        has[1] = x < nx - 1; cand[1] = v + sx;
        has[2] = y > 0;      cand[2] = v - sy;
        has[3] = y < ny - 1; cand[3] = v + sy;
        has[4] = z > 0;      cand[4] = v - sz;
        has[5] = z < nz - 1; cand[5] = v + sz;
        for (int d = 0; d < NB; ++d)
            nbr[i * NB + d] = has[d] ? (int32_t)queue[cand[d]] : -1;
    }
    free(queue);
    free(comp_size);
    return n;
}

/* ------------------------------------------------------------------------------------------
 * Synchronous transformation of one voxel (Sec. II.C eq. 3 with the clamps of the Appendix A
 * listing that computes all fluxes from the old state; readings R3, R4, R9).
 * x[0..4] = (MB, DOM, SOM, FOM, CO2), updated in place.
 * ---------------------------------------------------------------------------------------- */
void vo_transform_sync(const vo_params *p, double *x) {
    const double x1 = x[0], x2 = x[1], x3 = x[2], x4 = x[3];
    double uptake = p->v_dom * x2 / (p->K_dom + x2) * x1 * p->dt;  /* Monod uptake */
    if (uptake > x2) uptake = x2;
    double resp = p->rho * x1 * p->dt;
    double morta = p->mu * x1 * p->dt;
    if (resp + morta > x1) {
        if (morta > x1) {
            morta = x1;
            resp = 0.0;
        } else {
            resp = x1 - morta;
        }
    }
    const double mortaSOM = (1.0 - p->beta) * morta;
    const double mortaDOM = p->beta * morta;
    double turnFOM = p->v_fom * x4 * p->dt;
    if (turnFOM > x4) turnFOM = x4;
    double turnSOM = p->v_som * x3 * p->dt;
    if (turnSOM > x3) turnSOM = x3;
    x[0] = x1 + (uptake - morta - resp);
    x[1] = x2 + (mortaDOM - uptake + turnFOM + turnSOM);
    x[2] = x3 + (mortaSOM - turnSOM);
    x[3] = x4 - turnFOM;
    x[4] = x[4] + resp;
}

/* ------------------------------------------------------------------------------------------
 * Asynchronous transformation of one voxel (Sec. III: grow on DOM, then mortality, then
 * respiration, then SOM and FOM hydrolysis, each using the values already updated; Appendix A
 * sequential listing with readings R3, R5).
 * ---------------------------------------------------------------------------------------- */
void vo_transform_async(const vo_params *p, double *x) {
    double x1 = x[0], x2 = x[1], x3 = x[2], x4 = x[3], x5 = x[4];
    if (x1 > 0.0) {
        if (x2 > 0.0) {
            const double uptake = p->v_dom * x2 / (p->K_dom + x2) * x1 * p->dt;
            if (uptake < x2) {
                x1 += uptake;
                x2 -= uptake;
            } else {
                x1 += x2;
                x2 = 0.0;
            }
        }
        const double morta = p->mu * x1 * p->dt;
        if (morta < x1) {
            x1 -= morta;
            x2 += p->beta * morta;
            x3 += (1.0 - p->beta) * morta;
        } else {
            x2 += p->beta * x1;
            x3 += (1.0 - p->beta) * x1;
            x1 = 0.0;
        }
        const double resp = p->rho * x1 * p->dt;
        if (resp < x1) {
            x1 -= resp;
            x5 += resp;
        } else {
            x5 += x1;
            x1 = 0.0;
        }
    }
    if (x3 > 0.0) {
        const double turnSOM = p->v_som * x3 * p->dt;
        if (turnSOM < x3) {
            x3 -= turnSOM;
            x2 += turnSOM;
        } else {
            x2 += x3;
            x3 = 0.0;
        }
    }
    if (x4 > 0.0) {
        const double turnFOM = p->v_fom * x4 * p->dt;
        if (turnFOM < x4) {
            x4 -= turnFOM;
            x2 += turnFOM;
        } else {
            x2 += x4;
            x4 = 0.0;
        }
    }
    x[0] = x1; x[1] = x2; x[2] = x3; x[3] = x4; x[4] = x5;
}

static void transform_all(int64_t n, const vo_params *p, int transform, double *X) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double x[5];
        for (int c = 0; c < 5; ++c) x[c] = X[c * n + i];
        if (transform == 1) vo_transform_async(p, x);
        else vo_transform_sync(p, x);
        for (int c = 0; c < 5; ++c) X[c * n + i] = x[c];
    }
}

static inline double edge_weight(const double *g6, int64_t i, int d) {
    return g6 ? g6[i * NB + d] : 1.0;
}

/* ------------------------------------------------------------------------------------------
 * Scheme 1 (Sec. II.B.3a, reading R1, weights R8): m_i <- m_i - D dt sum_j g_ij (m_i - m_j).
 * `in` and `out` must not alias.
 * ---------------------------------------------------------------------------------------- */
void vo_diffuse_explicit(int64_t n, const int32_t *nbr, const double *g6, double c,
                         const double *in, double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double flux = 0.0;
        for (int d = 0; d < NB; ++d) {
            const int32_t j = nbr[i * NB + d];
            if (j >= 0) flux += edge_weight(g6, i, d) * (in[i] - in[j]);
        }
        out[i] = in[i] - c * flux;
    }
}

/* B v = v + c * L_g v, the matrix of Scheme 2 (Sec. II.B.3b) with edge weights (R8). */
static void apply_B(int64_t n, const int32_t *nbr, const double *g6, double c, const double *v,
                    double *out) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double lv = 0.0;
        for (int d = 0; d < NB; ++d) {
            const int32_t j = nbr[i * NB + d];
            if (j >= 0) lv += edge_weight(g6, i, d) * (v[i] - v[j]);
        }
        out[i] = v[i] + c * lv;
    }
}

static double dot(int64_t n, const double *a, const double *b) {
    double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* ------------------------------------------------------------------------------------------
 * Jacobi-preconditioned conjugate gradient for B x = b (Sec. II.B.3b and Sec. III, reading R7).
 * Preconditioner t_ii = 1 / b_ii = 1 / (1 + c sum_j g_ij).  On entry x holds the initial guess.
 * Returns 0 when ||r|| <= rtol ||b|| (the recurrence residual), 1 when maxit is reached.
 * ---------------------------------------------------------------------------------------- */
int vo_pcg_solve(int64_t n, const int32_t *nbr, const double *g6, double c, const double *b,
                 double *x, double rtol, int maxit, int *iters, double *relres) {
    double *r = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *z = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *pp = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *q = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *tdiag = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    int status = 0, it = 0;
    if (!r || !z || !pp || !q || !tdiag) { status = -1; goto done; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int d = 0; d < NB; ++d)
            if (nbr[i * NB + d] >= 0) s += edge_weight(g6, i, d);
        tdiag[i] = 1.0 / (1.0 + c * s);
    }
    const double bnorm = sqrt(dot(n, b, b));
    apply_B(n, nbr, g6, c, x, q);
    for (int64_t i = 0; i < n; ++i) r[i] = b[i] - q[i];
    double rnorm = sqrt(dot(n, r, r));
    if (bnorm == 0.0) {
        for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
        rnorm = 0.0;
        goto done;
    }
    for (int64_t i = 0; i < n; ++i) { z[i] = tdiag[i] * r[i]; pp[i] = z[i]; }
    double rz = dot(n, r, z);
    while (rnorm > rtol * bnorm) {
        if (it >= maxit) { status = 1; break; }
        apply_B(n, nbr, g6, c, pp, q);
        const double alpha = rz / dot(n, pp, q);
        for (int64_t i = 0; i < n; ++i) { x[i] += alpha * pp[i]; r[i] -= alpha * q[i]; }
        ++it;
        rnorm = sqrt(dot(n, r, r));
        if (rnorm <= rtol * bnorm) break;
        for (int64_t i = 0; i < n; ++i) z[i] = tdiag[i] * r[i];
        const double rz_new = dot(n, r, z);
        const double beta = rz_new / rz;
        rz = rz_new;
        for (int64_t i = 0; i < n; ++i) pp[i] = z[i] + beta * pp[i];
    }
done:
    if (iters) *iters = it;
    if (relres) *relres = bnorm > 0.0 ? rnorm / bnorm : 0.0;
    free(r); free(z); free(pp); free(q); free(tdiag);
    return status;
}

/* ------------------------------------------------------------------------------------------
 * Time loop with Scheme 1 (Sec. III, reading R6): per step, transform every voxel, then apply
 * Scheme 1 to the transformed DOM.  X is (5, n) in SoA order: X[c*n + i].
 * transform: 0 synchronous, 1 asynchronous.
 * ---------------------------------------------------------------------------------------- */
int vo_explicit_run(int64_t n, const int32_t *nbr, const double *g6, const vo_params *p,
                    int transform, double *X, int64_t nsteps) {
    double *y2 = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    if (!y2) return -1;
    const double c = p->D * p->dt;
    for (int64_t k = 0; k < nsteps; ++k) {
        transform_all(n, p, transform, X);
        memcpy(y2, X + n, sizeof(double) * (size_t)n);
        vo_diffuse_explicit(n, nbr, g6, c, y2, X + n);
    }
    free(y2);
    return 0;
}

/* Time loop with Scheme 2 (Sec. III, readings R6, R7).  Returns 0, or 1 if a solve stopped at
 * maxit.  *total_iters accumulates CG iterations; *worst_relres is the largest final residual. */
int vo_implicit_run(int64_t n, const int32_t *nbr, const double *g6, const vo_params *p,
                    int transform, double *X, int64_t nsteps, double rtol, int maxit,
                    int64_t *total_iters, double *worst_relres) {
    double *y2 = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    if (!y2) return -1;
    const double c = p->D * p->dt;
    int status = 0;
    int64_t tot = 0;
    double worst = 0.0;
    for (int64_t k = 0; k < nsteps; ++k) {
        transform_all(n, p, transform, X);
        memcpy(y2, X + n, sizeof(double) * (size_t)n);
        int it = 0;
        double rr = 0.0;
        const int s = vo_pcg_solve(n, nbr, g6, c, y2, X + n, rtol, maxit, &it, &rr);
        if (s < 0) { free(y2); return -1; }
        if (s) status = 1;
        tot += it;
        if (rr > worst) worst = rr;
    }
    if (total_iters) *total_iters = tot;
    if (worst_relres) *worst_relres = worst;
    free(y2);
    return status;
}

/* Per-compartment totals with Neumaier compensated summation (the tracked masses of Sec. IV). */
void vo_totals(int64_t n, const double *X, double *tot) {
    for (int c = 0; c < 5; ++c) {
        double s = 0.0, comp = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            const double v = X[c * n + i];
            const double t = s + v;
            if (fabs(s) >= fabs(v)) comp += (s - t) + v;
            else comp += (v - t) + s;
            s = t;
        }
        tot[c] = s + comp;
    }
}

/* ------------------------------------------------------------------------------------------
 * Discrete adjoint of the explicit synchronous step.
 *
 * Forward step k:  Y = T(X^k) voxel by voxel (synchronous transformation), then
 *                  X^{k+1} = (y1, Q_g y2, y3, y4, y5), Q_g = I - D dt L_g (Scheme 1, R8).
 * The transformation is written as y = x + S f(x) with the five fluxes
 *   f = (uptake, morta, resp, turnFOM, turnSOM) and
 *   y1 = x1 + uptake - morta - resp
 *   y2 = x2 - uptake + beta*morta + turnFOM + turnSOM
 *   y3 = x3 + (1-beta)*morta - turnSOM
 *   y4 = x4 - turnFOM
 *   y5 = x5 + resp
 * so with w = S^T mu the reverse of one voxel is lambda_x = mu + (df/dx)^T w, and the rate
 * gradients are w . df/dtheta (plus mu2*morta - mu3*morta for beta).  The derivatives of f follow
 * the branch that the clamps (R4) took in the forward pass.  Q_g is symmetric, so the reverse of
 * the diffusion is mu2 = Q_g lambda2, with dL/dD = -dt sum_i lambda2_i (L_g y2)_i and
 * dL/dg_ij = -D dt (y2_i - y2_j)(lambda2_i - lambda2_j).
 * ---------------------------------------------------------------------------------------- */

/* Parameter order of the gradient vector. */
enum { G_D = 0, G_RHO, G_MU, G_BETA, G_VSOM, G_VFOM, G_VDOM, G_K, G_COUNT };

static void sync_transform_reverse(const vo_params *p, const double *x, const double *mu,
                                   double *lam, double *gpar) {
    const double x1 = x[0], x2 = x[1], x3 = x[2], x4 = x[3];
    const double dt = p->dt, K = p->K_dom;
    /* forward fluxes and branch flags */
    const double sat = x2 / (K + x2);
    const double u0 = p->v_dom * sat * x1 * dt;
    const int upt_clamped = u0 > x2;
    const double r0 = p->rho * x1 * dt, m0 = p->mu * x1 * dt;
    int mr_case = 0; /* 0: free, 1: morta = x1 and resp = 0, 2: resp = x1 - morta */
    if (r0 + m0 > x1) mr_case = (m0 > x1) ? 1 : 2;
    const double morta = mr_case == 1 ? x1 : m0;
    const double tF0 = p->v_fom * x4 * dt;
    const int tF_clamped = tF0 > x4;
    const double tS0 = p->v_som * x3 * dt;
    const int tS_clamped = tS0 > x3;

    const double w_upt = mu[0] - mu[1];
    const double w_mor = -mu[0] + p->beta * mu[1] + (1.0 - p->beta) * mu[2];
    const double w_resp = -mu[0] + mu[4];
    const double w_tF = mu[1] - mu[3];
    const double w_tS = mu[1] - mu[2];

    for (int c = 0; c < 5; ++c) lam[c] = mu[c];
    /* uptake */
    if (upt_clamped) {
        lam[1] += w_upt;
    } else {
        lam[0] += w_upt * p->v_dom * sat * dt;
        lam[1] += w_upt * p->v_dom * x1 * dt * K / ((K + x2) * (K + x2));
        gpar[G_VDOM] += w_upt * sat * x1 * dt;
        gpar[G_K] += w_upt * (-p->v_dom * x2 * x1 * dt / ((K + x2) * (K + x2)));
    }
    /* mortality and respiration */
    if (mr_case == 0) {
        lam[0] += w_mor * p->mu * dt + w_resp * p->rho * dt;
        gpar[G_MU] += w_mor * x1 * dt;
        gpar[G_RHO] += w_resp * x1 * dt;
    } else if (mr_case == 1) {
        lam[0] += w_mor;
    } else {
        lam[0] += w_mor * p->mu * dt + w_resp * (1.0 - p->mu * dt);
        gpar[G_MU] += w_mor * x1 * dt - w_resp * x1 * dt;
    }
    gpar[G_BETA] += (mu[1] - mu[2]) * morta;
    /* FOM and SOM hydrolysis */
    if (tF_clamped) {
        lam[3] += w_tF;
    } else {
        lam[3] += w_tF * p->v_fom * dt;
        gpar[G_VFOM] += w_tF * x4 * dt;
    }
    if (tS_clamped) {
        lam[2] += w_tS;
    } else {
        lam[2] += w_tS * p->v_som * dt;
        gpar[G_VSOM] += w_tS * x3 * dt;
    }
}

/*
 * Runs nsteps explicit synchronous steps from X0 and back-propagates lamN = dL/dX^N.
 * Forward states are stored every `ckpt` steps and each segment is recomputed before its reverse
 * sweep.  Outputs: XN (5n, optional), lam0 = dL/dX^0 (5n), grad[8] in the order
 * (D, rho, mu, beta, v_som, v_fom, v_dom, K_dom), and, if gface != NULL, gface[6n]: for the edge
 * in slot d of node i, the derivative of L with respect to that edge's conductance (the same value
 * appears in the slots of both end nodes).  Returns 0, or -1 on allocation failure.
 */
int vo_adjoint_run(int64_t n, const int32_t *nbr, const double *g6, const vo_params *p,
                   const double *X0, int64_t nsteps, int64_t ckpt, const double *lamN,
                   double *XN, double *lam0, double *grad, double *gface) {
    if (ckpt <= 0) ckpt = 1;
    const int64_t nseg = nsteps > 0 ? (nsteps + ckpt - 1) / ckpt : 0;
    const size_t st = sizeof(double) * 5 * (size_t)(n ? n : 1);
    double *ck = (double *)malloc(st * (size_t)(nseg ? nseg : 1));
    double *seg = (double *)malloc(st * (size_t)(ckpt + 1));
    double *lam = (double *)malloc(st);
    double *y2 = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    double *gthr = NULL;
    if (!ck || !seg || !lam || !y2) {
        free(ck); free(seg); free(lam); free(y2);
        return -1;
    }
    const double c = p->D * p->dt;
    for (int g = 0; g < G_COUNT; ++g) grad[g] = 0.0;
    if (gface) memset(gface, 0, sizeof(double) * NB * (size_t)n);

    /* forward pass storing checkpoints */
    memcpy(seg, X0, st);
    for (int64_t s = 0; s < nseg; ++s) {
        memcpy(ck + (size_t)s * 5 * n, seg, st);
        const int64_t len = (s == nseg - 1) ? nsteps - s * ckpt : ckpt;
        vo_explicit_run(n, nbr, g6, p, 0, seg, len);
    }
    if (XN) memcpy(XN, nseg ? seg : X0, st);

    memcpy(lam, lamN, st);
    for (int64_t s = nseg - 1; s >= 0; --s) {
        const int64_t len = (s == nseg - 1) ? nsteps - s * ckpt : ckpt;
        /* recompute X^k for the segment: seg[k] holds X^{s*ckpt + k} */
        memcpy(seg, ck + (size_t)s * 5 * n, st);
        for (int64_t k = 0; k < len; ++k) {
            memcpy(seg + (size_t)(k + 1) * 5 * n, seg + (size_t)k * 5 * n, st);
            vo_explicit_run(n, nbr, g6, p, 0, seg + (size_t)(k + 1) * 5 * n, 1);
        }
        for (int64_t k = len - 1; k >= 0; --k) {
            const double *Xk = seg + (size_t)k * 5 * n;
            /* transformed DOM of step k */
            for (int64_t i = 0; i < n; ++i) {
                double x[5];
                for (int cc = 0; cc < 5; ++cc) x[cc] = Xk[cc * n + i];
                vo_transform_sync(p, x);
                y2[i] = x[1];
            }
            /* diffusion: parameter gradients, then mu2 = Q_g lambda2 (kept in seg slot k+1,
               which is no longer needed) */
            double *mu2 = seg + (size_t)(k + 1) * 5 * n;
            for (int64_t i = 0; i < n; ++i) {
                double lflux = 0.0, yflux = 0.0;
                for (int d = 0; d < NB; ++d) {
                    const int32_t j = nbr[i * NB + d];
                    if (j < 0) continue;
                    const double g = edge_weight(g6, i, d);
                    lflux += g * (lam[n + i] - lam[n + j]);
                    yflux += g * (y2[i] - y2[j]);
                    if (gface) gface[i * NB + d] += -c * (y2[i] - y2[j]) * (lam[n + i] - lam[n + j]);
                }
                grad[G_D] += -p->dt * lam[n + i] * yflux;
                mu2[i] = lam[n + i] - c * lflux;
            }
            /* transformation reverse, voxel by voxel */
            for (int64_t i = 0; i < n; ++i) {
                double x[5], mu[5], out[5];
                for (int cc = 0; cc < 5; ++cc) {
                    x[cc] = Xk[cc * n + i];
                    mu[cc] = lam[cc * n + i];
                }
                mu[1] = mu2[i];
                sync_transform_reverse(p, x, mu, out, grad);
                for (int cc = 0; cc < 5; ++cc) lam[cc * n + i] = out[cc];
            }
        }
    }
    memcpy(lam0, lam, st);
    free(ck); free(seg); free(lam); free(y2); free(gthr);
    return 0;
}

/* ------------------------------------------------------------------------------------------
 * Different time steps for transformation and diffusion (Sec. III: the process with the smaller
 * step is iterated; Table 1 tests 2-4).  Reading: a global clock.  Diffusion advances by dt per
 * step; the transformation, with its own step dt_transform, fires once for every tick
 * m * dt_transform (m = 0, 1, ...) in [k dt, (k+1) dt), before diffusion step k.  The number of
 * ticks in [0, k dt) is ceil(k r) with r = dt / dt_transform (a 1e-9 guard absorbs rounding of r).
 * step0 is the number of diffusion steps already taken (the clock's origin).
 * ---------------------------------------------------------------------------------------- */
int64_t vo_ticks_before(int64_t k, double dt, double dt_transform) {
    if (k <= 0) return 0;
    const double r = dt / dt_transform;
    return (int64_t)ceil((double)k * r - 1e-9);
}

int vo_run_subcycled(int64_t n, const int32_t *nbr, const double *g6, const vo_params *p, int transform,
                     int scheme, double *X, int64_t nsteps, double dt_transform, int64_t step0,
                     double rtol, int maxit, int64_t *total_iters) {
    double *y2 = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    if (!y2) return -1;
    vo_params pt = *p;
    pt.dt = dt_transform;  /* the transformation uses its own step */
    const double c = p->D * p->dt;
    int status = 0;
    int64_t tot = 0;
    for (int64_t k = 0; k < nsteps; ++k) {
        const int64_t kk = step0 + k;
        const int64_t ticks = vo_ticks_before(kk + 1, p->dt, dt_transform) - vo_ticks_before(kk, p->dt, dt_transform);
        for (int64_t m = 0; m < ticks; ++m) transform_all(n, &pt, transform, X);
        memcpy(y2, X + n, sizeof(double) * (size_t)n);
        if (scheme == 0) {
            vo_diffuse_explicit(n, nbr, g6, c, y2, X + n);
        } else {
            int it = 0;
            double rr = 0.0;
            const int st = vo_pcg_solve(n, nbr, g6, c, y2, X + n, rtol, maxit, &it, &rr);
            if (st < 0) { free(y2); return -1; }
            if (st) status = 1;
            tot += it;
        }
    }
    if (total_iters) *total_iters = tot;
    free(y2);
    return status;
}
