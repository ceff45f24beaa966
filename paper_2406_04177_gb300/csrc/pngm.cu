// Coarse primitive-graph diffusion model and its calibration from voxel data (Sec. V.A).
//
// A partition of the pore voxels into q primitives (one label per node) defines a coarse graph:
// primitive i has volume v_i (its voxel count); primitives i and j are adjacent when a voxel face
// joins them, with S_ij shared faces and centroid distance d_ij; the initial conductance is
// S_ij / d_ij (Sec. V.B).  The conductances theta are stored per ordered pair (CSR slot), as the
// paper's gradient treats theta_ij and theta_ji as separate parameters; `tied` updates keep them
// equal.
//
// Kernels:
//   build     two decode passes over the node chunks: volumes, integer centroid sums and the count
//             of cross faces, then a hash table of the (lo, hi) primitive pairs with face counts
//             (warp-aggregated atomics); the pairs are compacted, sorted on the host and laid out
//             as CSR.  Every quantity is an integer sum, so the graph is bit-exact.
//   restrict  primitive masses = sums of node masses (warp-aggregated FP64 atomics).
//   scheme 3  one explicit step per launch, one row per thread, FP64, rounding as in the formula.
//   scheme 4  (V + c L) u = m^k, m^{k+1} = V u, by Jacobi-PCG inside one CTA per solve (the coarse
//             graph is small; the whole iteration runs without a host round trip).
//   objective Objective 1 or 2 over l data pairs and its gradient per slot; one row per thread
//             owns its slots, so the gradient needs no atomics; the loss is reduced in FP64.
//   sgd       theta <- theta - lr sign(g) per slot (sign(0) = 0).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "stencil.cuh"
#include "vga_internal.cuh"

using namespace vga;

struct vga_pngm {
    const vga_graph *g = nullptr;
    cudaStream_t stream = nullptr;
    int32_t q = 0;
    int64_t n = 0;
    int32_t nslots = 0;
    int64_t cross_faces = 0;
    int32_t *labels = nullptr;   // device, n
    double *vol = nullptr;       // device, q
    int32_t *row_ptr = nullptr;  // device, q + 1
    int32_t *col = nullptr;      // device, nslots
    int32_t *rev = nullptr;      // device, nslots
    double *theta = nullptr;     // device, nslots
    double *grad = nullptr;      // device, 2 * nslots (raw, tied)
    double *work = nullptr;      // device: PCG vectors (6 q) + loss partials + scalars
    int64_t work_count = 0;
    int32_t *d_pairs = nullptr;  // device pair indices
    int32_t *h_pairs = nullptr;  // pinned staging
    int32_t pairs_cap = 0;
    double *h_scal = nullptr;    // pinned: loss, PCG iterations, relres, converged
    unsigned long long *fx = nullptr;  // restriction: fixed-point sums (q), scale (2), partials
    bool symmetric = true;       // theta_ij == theta_ji for every pair
    // host copies of the geometry (export)
    std::vector<double> h_vol, h_cen, h_S, h_dist;
    std::vector<int32_t> h_row_ptr, h_col, h_rev;
    int64_t last_iters = 0;
    double last_relres = 0.0;
};

namespace {

constexpr int kThreads = 256;
constexpr int kCap = 1024;        // nodes per decoded chunk
constexpr int kObjBlocks = 1024;  // grid of the objective kernel (grid-stride over rows)
constexpr int kPcgThreads = 1024;
constexpr unsigned long long kEmpty = ~0ull;

inline unsigned grid_for(int64_t count, int threads) { return (unsigned)((count + threads - 1) / threads); }

// Sum of v over the lanes of `peers` (all lanes of `act` take part in the shuffles; must be called
// by all 32 lanes).
template <typename T>
__device__ __forceinline__ T peer_sum(unsigned act, unsigned peers, T v) {
    const int lane = threadIdx.x & 31;
    T sum = v;
    unsigned rest = act;
    while (rest) {
        const int src = __ffs(rest) - 1;
        rest &= rest - 1;
        const T t = __shfl_sync(0xffffffffu, v, src);
        if (src != lane && ((peers >> src) & 1u)) sum += t;
    }
    return sum;
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    // SplitMix64 finaliser (Steele, Lea, Flood 2014)
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Pass 1: volumes, integer coordinate sums and the number of cross faces (+x, +y, +z).
__global__ void __launch_bounds__(kThreads) k_scan_nodes(Topo t, const int32_t *__restrict__ chunk_row,
                                                         const int32_t *__restrict__ lab, int32_t q,
                                                         unsigned long long *__restrict__ acc,  // 4 q
                                                         unsigned long long *__restrict__ nfaces, int32_t *err) {
    extern __shared__ uint32_t smem[];
    int32_t *s_nb = reinterpret_cast<int32_t *>(smem + kCap);
    int64_t v0;
    const int32_t nv = decode_chunk<true>(t, chunk_row, kCap, smem, s_nb, smem + 5 * kCap, v0);
    unsigned long long faces = 0;
    for (int32_t base = 0; base < nv; base += blockDim.x) {
        const int32_t k = base + (int32_t)threadIdx.x;
        int32_t a = -1;
        uint32_t x = 0, y = 0, z = 0, bits = 0;
        if (k < nv) {
            a = __ldg(lab + v0 + k);
            if (a < 0 || a >= q) {
                atomicExch(err, 1);
                a = -1;
            }
            x = smem[k] & 0xffffu;
            bits = smem[k] >> 16;
            y = smem[5 * kCap + k] & 0xffffu;
            z = smem[5 * kCap + k] >> 16;
        }
        const unsigned act = __ballot_sync(0xffffffffu, a >= 0);
        const unsigned peers = __match_any_sync(0xffffffffu, a);
        const unsigned long long cnt = peer_sum<unsigned long long>(act, peers, a >= 0 ? 1ull : 0ull);
        const unsigned long long sx = peer_sum<unsigned long long>(act, peers, x);
        const unsigned long long sy = peer_sum<unsigned long long>(act, peers, y);
        const unsigned long long sz = peer_sum<unsigned long long>(act, peers, z);
        if (a >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) {
            atomicAdd(acc + a, cnt);
            atomicAdd(acc + q + a, sx);
            atomicAdd(acc + 2 * (int64_t)q + a, sy);
            atomicAdd(acc + 3 * (int64_t)q + a, sz);
        }
        if (a >= 0) {
            const int64_t j[3] = {(bits & 2u) ? v0 + k + 1 : -1, (bits & 8u) ? (int64_t)s_nb[kCap + k] : -1,
                                  (bits & 32u) ? (int64_t)s_nb[3 * kCap + k] : -1};
#pragma unroll
            for (int d = 0; d < 3; ++d)
                if (j[d] >= 0) {
                    const int32_t b = __ldg(lab + j[d]);
                    if (b != a && b >= 0 && b < q) ++faces;
                }
        }
    }
    double f[1] = {(double)faces};
    __shared__ double tot[1];
    block_sum_store<1>(f, tot);
    if (threadIdx.x == 0 && tot[0] > 0.0) atomicAdd(nfaces, (unsigned long long)tot[0]);
}

// Pass 2: insert every cross face's (lo, hi) pair into the hash table and count faces per pair.
__global__ void __launch_bounds__(kThreads) k_insert_pairs(Topo t, const int32_t *__restrict__ chunk_row,
                                                           const int32_t *__restrict__ lab, int32_t q,
                                                           unsigned long long *__restrict__ keys,
                                                           unsigned int *__restrict__ counts,
                                                           unsigned long long hmask, int32_t *err) {
    extern __shared__ uint32_t smem[];
    int32_t *s_nb = reinterpret_cast<int32_t *>(smem + kCap);
    int64_t v0;
    const int32_t nv = decode_chunk<false>(t, chunk_row, kCap, smem, s_nb, nullptr, v0);
    for (int32_t base = 0; base < nv; base += blockDim.x) {
        const int32_t k = base + (int32_t)threadIdx.x;
        const bool live = k < nv;
        const int32_t a = live ? __ldg(lab + v0 + k) : -1;
        const uint32_t bits = live ? (smem[k] >> 16) : 0u;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            unsigned long long key = kEmpty;
            if (live && a >= 0 && a < q) {
                const uint32_t bit = 2u << (2 * d);
                if (bits & bit) {
                    const int64_t j = d == 0 ? v0 + k + 1 : (int64_t)s_nb[(2 * d - 1) * kCap + k];
                    const int32_t b = __ldg(lab + j);
                    if (b != a && b >= 0 && b < q) {
                        const unsigned long long lo = (unsigned long long)min(a, b), hi = (unsigned long long)max(a, b);
                        key = lo * (unsigned long long)q + hi;
                    }
                }
            }
            const unsigned act = __ballot_sync(0xffffffffu, key != kEmpty);
            if (!act) continue;
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            if (key == kEmpty || (int)(threadIdx.x & 31) != __ffs(peers) - 1) continue;
            const unsigned cnt = (unsigned)__popc(peers);
            unsigned long long h = mix64(key) & hmask;
            bool done = false;
            for (unsigned long long probe = 0; probe <= hmask; ++probe) {  // bounded: table size
                const unsigned long long prev = atomicCAS(keys + h, kEmpty, key);
                if (prev == kEmpty || prev == key) {
                    atomicAdd(counts + h, cnt);
                    done = true;
                    break;
                }
                h = (h + 1) & hmask;
            }
            if (!done) atomicExch(err, 2);
        }
    }
}

__global__ void k_compact_pairs(unsigned long long hsize, const unsigned long long *__restrict__ keys,
                                const unsigned int *__restrict__ counts, unsigned long long *__restrict__ out_key,
                                unsigned int *__restrict__ out_cnt, unsigned long long *__restrict__ nout) {
    for (unsigned long long h = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; h < hsize;
         h += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[h];
        if (k == kEmpty) continue;
        const unsigned long long o = atomicAdd(nout, 1ull);
        out_key[o] = k;
        out_cnt[o] = counts[h];
    }
}

// Primitive masses: out[label[i]] = sum of m_i over the primitive's nodes, summed exactly in fixed
// point: every node's value becomes the integer round(h_i 2^k) + round(l_i 2^k) of its stored pair,
// k = 61 - e with sum_i (|h_i| + |l_i|) < 2^e (up to the FP32 rounding of that bound; int64 holds
// 2 more bits), so no partial sum can overflow int64 and the result does not depend on the order
// of the atomic additions (the restriction is deterministic).  No FP64 arithmetic per node: the
// FP64 rate of this part is a small fraction of its FP32 and integer rates.  A CTA sums a segment
// of kSeg consecutive nodes into a shared-memory hash of labels (runs of equal labels over
// consecutive lanes summed in the warp first) with 64-bit integer atomics, then flushes one global
// atomic per distinct label; a label that finds no free slot within kProbe probes goes straight to
// global memory.
constexpr int kSeg = 4096;
constexpr int kHash = 1024;
constexpr int kProbe = 16;
constexpr int kSumBlocks = 1024;
static_assert(kSeg % (4 * kThreads) == 0, "a segment is a whole number of four-row batches");

// round(x 2^k) of a finite FP32 x, ties to even, from the bits of x; the caller bounds |x| 2^k
// below 2^62 (so a left shift stays below 64 bits; a shift of 64 or more, outside that bound, gives 0).
__device__ __forceinline__ long long fixed_of_f32(float x, int k) {
    const uint32_t b = __float_as_uint(x);
    const int ex = (int)((b >> 23) & 0xffu);
    const uint64_t m = ex ? (uint64_t)((b & 0x7fffffu) | 0x800000u) : (uint64_t)(b & 0x7fffffu);
    const int sh = (ex ? ex - 150 : -149) + k;  // x 2^k = m 2^sh
    uint64_t r;
    if (sh >= 0) {
        r = sh < 64 ? m << sh : 0ull;
    } else if (sh < -40) {
        r = 0ull;  // m 2^sh < 2^-16
    } else {
        const int t = -sh;
        const uint64_t rem = m & ((1ull << t) - 1ull), half = 1ull << (t - 1);
        r = m >> t;
        if (rem > half || (rem == half && (r & 1ull))) ++r;
    }
    return (b >> 31) ? -(long long)r : (long long)r;
}

template <int PREC>
__global__ void __launch_bounds__(kThreads) k_abs_sum(int64_t n, const float *__restrict__ H,
                                                      const res_t *__restrict__ L, double *__restrict__ part) {
    float acc32 = 0.0f;  // about n / (blocks x threads) terms per thread
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {  // four independent loads in flight
        V x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = vload<PREC>(H, L, i + u * stride);
#pragma unroll
        for (int u = 0; u < 4; ++u) acc32 += fabsf(x[u].h) + fabsf(x[u].l);
    }
    for (; i < n; i += stride) {
        const V x = vload<PREC>(H, L, i);
        acc32 += fabsf(x.h) + fabsf(x.l);
    }
    double acc[1] = {(double)acc32};
    __shared__ double out[1];
    block_sum_store<1>(acc, out);
    if (threadIdx.x == 0) part[blockIdx.x] = out[0];
}

// scale[0] = 2^(61 - e), sum |m| < 2^e; scale[1] = 1 / scale[0]; scale[2] = 61 - e
__global__ void k_fx_scale(const double *__restrict__ part, int32_t count, double *__restrict__ scale) {
    double acc[1] = {0.0};
    for (int32_t k = threadIdx.x; k < count; k += blockDim.x) acc[0] += part[k];
    __shared__ double out[1];
    block_sum_store<1>(acc, out);
    if (threadIdx.x == 0) {
        const double S = out[0];
        const int e = S > 0.0 ? ilogb(S) + 1 : 0;
        scale[0] = ldexp(1.0, 61 - e);
        scale[1] = ldexp(1.0, e - 61);
        scale[2] = (double)(61 - e);
    }
}

constexpr int kRestrictBlocksPerSm = 6;  // resident blocks of k_restrict (at most 40 registers)

template <int PREC>
__global__ void __launch_bounds__(kThreads, kRestrictBlocksPerSm) k_restrict(int64_t n, const int32_t *__restrict__ lab,
                                                       const float *__restrict__ H, const res_t *__restrict__ L,
                                                       const double *__restrict__ scale,
                                                       unsigned long long *__restrict__ out) {
    __shared__ int32_t hkey[kHash];
    __shared__ unsigned long long hval[kHash];
    for (int k = threadIdx.x; k < kHash; k += blockDim.x) {
        hkey[k] = -1;
        hval[k] = 0ull;
    }
    __syncthreads();
    const int k2 = (int)scale[2];
    const int lane = (int)(threadIdx.x & 31);
    const int64_t nseg = (n + kSeg - 1) / kSeg;
    for (int64_t seg = blockIdx.x; seg < nseg; seg += gridDim.x) {
        const int64_t i0 = seg * kSeg;
        for (int k4 = 0; k4 < kSeg; k4 += 4 * kThreads) {
          // the loads of four rows of the segment first (independent), then their sums
          int32_t a4[4];
          float h4[4];
          res_t l4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
              const int64_t i = i0 + k4 + u * kThreads + threadIdx.x;
              a4[u] = i < n ? __ldg(lab + i) : -1;
              h4[u] = i < n ? __ldg(H + i) : 0.0f;
              l4[u] = (PREC == P_COMP && i < n) ? __ldg(L + i) : (res_t)0;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int64_t i = i0 + k4 + u * kThreads + threadIdx.x;
            const bool live = i < n;
            const int32_t a = a4[u];
            long long f = 0;
            if (live) {
                f = fixed_of_f32(h4[u], k2);
                if (PREC == P_COMP) f += fixed_of_f32(res_decode(l4[u], h4[u]), k2);
            }
            // inclusive sum over the run of equal labels that ends at this lane
            const int32_t a_prev = __shfl_up_sync(0xffffffffu, a, 1);
            const int32_t a_next = __shfl_down_sync(0xffffffffu, a, 1);
            const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || a_prev != a);
            const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
            unsigned long long sum = (unsigned long long)f;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long t = __shfl_up_sync(0xffffffffu, sum, d);
                if (lane - d >= start) sum += t;
            }
            if (live && (lane == 31 || a_next != a)) {
                const uint32_t h = (uint32_t)a * 2654435761u;
                bool done = false;
                for (int q = 0; q < kProbe; ++q) {
                    const int slot = (int)((h >> 22) + q) & (kHash - 1);
                    const int32_t cur = atomicCAS(hkey + slot, -1, a);
                    if (cur == -1 || cur == a) {
                        atomicAdd(hval + slot, sum);
                        done = true;
                        break;
                    }
                }
                if (!done) atomicAdd(out + a, sum);
            }
          }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kHash; k += blockDim.x) {
            const int32_t key = hkey[k];
            if (key >= 0) {
                atomicAdd(out + key, hval[k]);
                hkey[k] = -1;
                hval[k] = 0ull;
            }
        }
        __syncthreads();
    }
}

__global__ void k_fx_out(int32_t q, const unsigned long long *__restrict__ fx, const double *__restrict__ scale,
                         double *__restrict__ out) {
    const int32_t a = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (a < q) out[a] = (double)(long long)fx[a] * scale[1];
}

// Scheme 3: m_i - c sum_s theta_s (m_i / v_i - m_j / v_j), FP64 with every rounding explicit.
__global__ void __launch_bounds__(kThreads) k_scheme3(int32_t q, const int32_t *__restrict__ rp,
                                                      const int32_t *__restrict__ col, const double *__restrict__ th,
                                                      const double *__restrict__ vol, double c,
                                                      const double *__restrict__ m, double *__restrict__ out) {
    const int32_t i = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= q) return;
    const double ci = m[i] / vol[i];
    double s = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) {
        const int32_t j = col[k];
        s = __dadd_rn(s, __dmul_rn(th[k], __dsub_rn(ci, m[j] / vol[j])));
    }
    out[i] = __dsub_rn(m[i], __dmul_rn(c, s));
}

__device__ __forceinline__ double cta_sum(double v, double *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sum_d(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        t = warp_sum_d(t);
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

// (A x)_i = v_i x_i + c sum_s theta_s (x_i - x_j)
__device__ __forceinline__ double apply_row(int32_t i, const int32_t *rp, const int32_t *col, const double *th,
                                            const double *vol, double c, const double *x) {
    const double xi = x[i];
    double s = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) s += th[k] * (xi - x[col[k]]);
    return vol[i] * xi + c * s;
}

// Scheme 4 for one step: solve (V + c L) u = b by Jacobi-PCG in one CTA, then m = V u.
// w holds 5 q doubles (u, r, z, p, ap) + q (inverse diagonal).  stats: iterations, relres, converged.
__global__ void __launch_bounds__(kPcgThreads, 1) k_scheme4_pcg(int32_t q, const int32_t *__restrict__ rp,
                                                              const int32_t *__restrict__ col,
                                                              const double *__restrict__ th,
                                                              const double *__restrict__ vol, double c, double *m,
                                                              double *w, double rtol, int32_t maxit, double *stats) {
    __shared__ double sh[33];
    double *u = w, *r = w + q, *z = w + 2 * (int64_t)q, *p = w + 3 * (int64_t)q, *ap = w + 4 * (int64_t)q,
           *dinv = w + 5 * (int64_t)q;
    double bb = 0.0;
    for (int32_t i = threadIdx.x; i < q; i += blockDim.x) {
        double s = 0.0;
        for (int32_t k = rp[i]; k < rp[i + 1]; ++k) s += th[k];
        dinv[i] = 1.0 / (vol[i] + c * s);
        u[i] = m[i] / vol[i];
        bb += m[i] * m[i];
    }
    bb = cta_sum(bb, sh);
    double rz = 0.0, rr = 0.0;
    for (int32_t i = threadIdx.x; i < q; i += blockDim.x) {
        const double ri = m[i] - apply_row(i, rp, col, th, vol, c, u);
        r[i] = ri;
        const double zi = ri * dinv[i];
        z[i] = zi;
        p[i] = zi;
        rz += ri * zi;
        rr += ri * ri;
    }
    rz = cta_sum(rz, sh);
    rr = cta_sum(rr, sh);
    const double tol2 = rtol * rtol * bb;
    int32_t it = 0;
    while (rr > tol2 && it < maxit) {
        double pap = 0.0;
        for (int32_t i = threadIdx.x; i < q; i += blockDim.x) {
            const double a = apply_row(i, rp, col, th, vol, c, p);
            ap[i] = a;
            pap += p[i] * a;
        }
        pap = cta_sum(pap, sh);
        if (!(pap > 0.0)) break;  // not positive definite (or breakdown): stop, reported as not converged
        const double alpha = rz / pap;
        double rzn = 0.0, rrn = 0.0;
        for (int32_t i = threadIdx.x; i < q; i += blockDim.x) {
            u[i] += alpha * p[i];
            const double ri = r[i] - alpha * ap[i];
            r[i] = ri;
            const double zi = ri * dinv[i];
            z[i] = zi;
            rzn += ri * zi;
            rrn += ri * ri;
        }
        rzn = cta_sum(rzn, sh);
        rr = cta_sum(rrn, sh);
        const double beta = rzn / rz;
        rz = rzn;
        for (int32_t i = threadIdx.x; i < q; i += blockDim.x) p[i] = z[i] + beta * p[i];
        __syncthreads();
        ++it;
    }
    for (int32_t i = threadIdx.x; i < q; i += blockDim.x) m[i] = vol[i] * u[i];
    if (threadIdx.x == 0) {
        stats[0] += (double)it;
        const double rel = bb > 0.0 ? sqrt(rr / bb) : 0.0;
        stats[1] = rel;
        if (!(rr <= tol2)) stats[2] = 0.0;
    }
}

// Objective 1 (KIND 1) or 2 (KIND 2) over the l pairs (data[pairs[2p]], data[pairs[2p+1]]):
// residual r_i and gradient 2 r_i dr_i/dtheta_s / (l q) for the slots of row i.
template <int KIND>
__global__ void __launch_bounds__(kThreads) k_objective(int32_t q, const int32_t *__restrict__ rp,
                                                        const int32_t *__restrict__ col, const double *__restrict__ th,
                                                        const double *__restrict__ vol, double c,
                                                        const double *__restrict__ data, const int32_t *__restrict__ pairs,
                                                        int32_t l, double *__restrict__ grad, double *__restrict__ part) {
    double loss = 0.0;
    const double inv_lq = 1.0 / ((double)l * (double)q);
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < q; i += gridDim.x * blockDim.x) {
        const int32_t k0 = rp[i], k1 = rp[i + 1];
        for (int32_t k = k0; k < k1; ++k) grad[k] = 0.0;
        for (int32_t pp = 0; pp < l; ++pp) {
            const double *x = data + (int64_t)pairs[2 * pp] * q;
            const double *y = data + (int64_t)pairs[2 * pp + 1] * q;
            // the vector whose fluxes enter the residual: x for Objective 1, y for Objective 2
            const double *a = KIND == 1 ? x : y;
            const double ai = a[i] / vol[i];
            double fs = 0.0;
            for (int32_t k = k0; k < k1; ++k) fs += th[k] * (ai - a[col[k]] / vol[col[k]]);
            const double r = KIND == 1 ? (y[i] - x[i]) + c * fs : (x[i] - y[i]) - c * fs;
            loss += r * r;
            const double coef = (KIND == 1 ? 2.0 : -2.0) * c * r * inv_lq;
            for (int32_t k = k0; k < k1; ++k) grad[k] += coef * (ai - a[col[k]] / vol[col[k]]);
        }
    }
    double v[1] = {loss * inv_lq};
    block_sum_store<1>(v, part + blockIdx.x);
}

__global__ void k_sum_partials(const double *__restrict__ part, int32_t count, double *__restrict__ out) {
    double s = 0.0;
    for (int32_t i = threadIdx.x; i < count; i += blockDim.x) s += part[i];
    double v[1] = {s};
    block_sum_store<1>(v, out);
}

__global__ void k_tie(int32_t ns, const int32_t *__restrict__ rev, const double *__restrict__ g,
                      double *__restrict__ out) {
    const int32_t s = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (s < ns) out[s] = g[s] + g[rev[s]];
}

__global__ void k_sign_sgd(int32_t ns, const double *__restrict__ g, double *__restrict__ th, double lr, double tmin) {
    const int32_t s = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (s >= ns) return;
    const double gs = g[s];
    const double step = gs > 0.0 ? 1.0 : (gs < 0.0 ? -1.0 : 0.0);
    th[s] = fmax(th[s] - lr * step, tmin);
}

vga_status ensure_work(vga_pngm *pg, int64_t count) {
    if (pg->work_count >= count) return VGA_OK;
    dfree(pg->work);
    pg->work = nullptr;
    pg->work_count = 0;
    VGA_TRY(dmalloc((void **)&pg->work, sizeof(double) * (size_t)count, "coarse-graph work"));
    pg->work_count = count;
    return VGA_OK;
}

vga_status ensure_pairs(vga_pngm *pg, int32_t l) {
    if (pg->pairs_cap >= l) return VGA_OK;
    dfree(pg->d_pairs);
    if (pg->h_pairs) cudaFreeHost(pg->h_pairs);
    pg->d_pairs = nullptr;
    pg->h_pairs = nullptr;
    pg->pairs_cap = 0;
    const int32_t cap = std::max<int32_t>(64, l);
    VGA_TRY(dmalloc((void **)&pg->d_pairs, sizeof(int32_t) * 2 * (size_t)cap, "pair indices"));
    VGA_CUDA(cudaMallocHost((void **)&pg->h_pairs, sizeof(int32_t) * 2 * (size_t)cap));
    pg->pairs_cap = cap;
    return VGA_OK;
}

// Frees every buffer of the handle; returns the name of the first release call that failed (the
// runtime's error state is left set for release_status to report).
const char *pngm_release(vga_pngm *pg) {
    const char *bad = nullptr;
    auto chk = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && !bad) bad = what;
    };
    void *dev[] = {pg->labels, pg->vol, pg->row_ptr, pg->col, pg->rev, pg->theta, pg->grad, pg->work, pg->d_pairs, pg->fx};
    const char *names[] = {"labels", "vol", "row_ptr", "col", "rev", "theta", "grad", "work", "d_pairs", "fx"};
    for (int k = 0; k < 10; ++k)
        if (dev[k]) chk(cudaFree(dev[k]), names[k]);
    if (pg->h_pairs) chk(cudaFreeHost(pg->h_pairs), "h_pairs");
    if (pg->h_scal) chk(cudaFreeHost(pg->h_scal), "h_scal");
    delete pg;
    return bad;
}

vga_status check_theta_symmetry(vga_pngm *pg, const std::vector<double> &th) {
    pg->symmetric = true;
    for (int32_t s = 0; s < pg->nslots; ++s)
        if (th[s] != th[pg->h_rev[s]]) {
            pg->symmetric = false;
            break;
        }
    return VGA_OK;
}

vga_status build(vga_pngm *pg, const int32_t *labels, bool on_device) {
    const vga_graph *g = pg->g;
    cudaStream_t st = pg->stream;
    const int64_t n = g->n;
    const int32_t q = pg->q;
    VGA_TRY(dmalloc((void **)&pg->labels, sizeof(int32_t) * (size_t)std::max<int64_t>(n, 1), "primitive labels"));
    if (n > 0)
        VGA_CUDA(cudaMemcpyAsync(pg->labels, labels, sizeof(int32_t) * (size_t)n,
                                 on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    // pass 1
    unsigned long long *acc = nullptr;
    int32_t *err = nullptr;
    VGA_TRY(dmalloc((void **)&acc, sizeof(unsigned long long) * (4 * (size_t)q + 2), "coarse-graph sums"));
    vga_status status = dmalloc((void **)&err, sizeof(int32_t), "error flag");
    Chunks ch;
    if (status == VGA_OK && n > 0) status = build_chunks(g->topo(), kCap, &ch, st);
    std::vector<unsigned long long> h_acc(4 * (size_t)q + 2, 0);
    int32_t h_err = 0;
    if (status == VGA_OK) {
        cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * (4 * (size_t)q + 2), st);
        cudaMemsetAsync(err, 0, sizeof(int32_t), st);
        if (n > 0) {
            const size_t smem = sizeof(uint32_t) * kCap * decode_words(true);
            k_scan_nodes<<<ch.count, kThreads, smem, st>>>(g->topo(), ch.row, pg->labels, q, acc, acc + 4 * (size_t)q, err);
        }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h_acc.data(), acc, sizeof(unsigned long long) * h_acc.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) status = cuda_fail(e, "coarse-graph pass 1", __FILE__, __LINE__);
    }
    dfree(acc);
    if (status == VGA_OK && h_err) status = fail(VGA_ERR_INVALID_ARG, "a primitive label lies outside [0, q)");
    pg->h_vol.assign(q, 0.0);
    pg->h_cen.assign(3 * (size_t)q, 0.0);
    for (int32_t a = 0; a < q && status == VGA_OK; ++a) {
        if (h_acc[a] == 0) status = fail(VGA_ERR_INVALID_ARG, "every primitive needs at least one node");
        const double v = (double)h_acc[a];
        pg->h_vol[a] = v;
        for (int d = 0; d < 3; ++d) pg->h_cen[3 * (size_t)a + d] = (double)h_acc[(size_t)(d + 1) * q + a] / v;
    }
    const unsigned long long nf = h_acc[4 * (size_t)q];
    pg->cross_faces = (int64_t)nf;
    // pass 2: hash table of at least twice the face count (so it never fills)
    unsigned long long hsize = 1024;
    while (hsize < 2 * nf) hsize <<= 1;
    unsigned long long *keys = nullptr, *okey = nullptr, *nout = nullptr;
    unsigned int *cnts = nullptr, *ocnt = nullptr;
    if (status == VGA_OK) status = dmalloc((void **)&keys, sizeof(unsigned long long) * hsize, "pair table");
    if (status == VGA_OK) status = dmalloc((void **)&cnts, sizeof(unsigned int) * hsize, "pair table");
    const size_t maxpairs = (size_t)std::max<unsigned long long>(nf, 1);
    if (status == VGA_OK) status = dmalloc((void **)&okey, sizeof(unsigned long long) * maxpairs, "pair list");
    if (status == VGA_OK) status = dmalloc((void **)&ocnt, sizeof(unsigned int) * maxpairs, "pair list");
    if (status == VGA_OK) status = dmalloc((void **)&nout, sizeof(unsigned long long), "pair count");
    unsigned long long np = 0;
    std::vector<unsigned long long> hk;
    std::vector<unsigned int> hc;
    if (status == VGA_OK) {
        cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * hsize, st);
        cudaMemsetAsync(cnts, 0, sizeof(unsigned int) * hsize, st);
        cudaMemsetAsync(nout, 0, sizeof(unsigned long long), st);
        if (n > 0 && nf > 0) {
            const size_t smem = sizeof(uint32_t) * kCap * decode_words(false);
            k_insert_pairs<<<ch.count, kThreads, smem, st>>>(g->topo(), ch.row, pg->labels, q, keys, cnts, hsize - 1, err);
            k_compact_pairs<<<(unsigned)std::min<unsigned long long>(4096, (hsize + kThreads - 1) / kThreads), kThreads, 0,
                              st>>>(hsize, keys, cnts, okey, ocnt, nout);
        }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&np, nout, sizeof(np), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && h_err) status = fail(VGA_ERR_CUDA, "coarse-graph pair table overflow (device-side)");
        if (e == cudaSuccess && status == VGA_OK) {
            hk.resize(np);
            hc.resize(np);
            if (np > 0) e = cudaMemcpy(hk.data(), okey, sizeof(unsigned long long) * np, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && np > 0) e = cudaMemcpy(hc.data(), ocnt, sizeof(unsigned int) * np, cudaMemcpyDeviceToHost);
        }
        if (e != cudaSuccess && status == VGA_OK) status = cuda_fail(e, "coarse-graph pass 2", __FILE__, __LINE__);
    }
    dfree(keys);
    dfree(cnts);
    dfree(okey);
    dfree(ocnt);
    dfree(nout);
    dfree(err);
    if (n > 0) free_chunks(&ch);
    VGA_TRY(status);
    if (2 * np > (unsigned long long)INT32_MAX) return fail(VGA_ERR_UNSUPPORTED, "more than 2^31 - 1 coarse-graph slots");
    // CSR of the ordered pairs: sorting the (lo, hi) keys and appending (lo -> hi) and (hi -> lo)
    // in that order leaves every row sorted by column.
    std::vector<size_t> order(np);
    for (size_t k = 0; k < np; ++k) order[k] = k;
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) { return hk[a] < hk[b]; });
    const int32_t ns = (int32_t)(2 * np);
    pg->nslots = ns;
    pg->h_row_ptr.assign((size_t)q + 1, 0);
    for (size_t k = 0; k < np; ++k) {
        const int64_t lo = (int64_t)(hk[k] / (unsigned long long)q), hi = (int64_t)(hk[k] % (unsigned long long)q);
        ++pg->h_row_ptr[lo + 1];
        ++pg->h_row_ptr[hi + 1];
    }
    for (int32_t a = 0; a < q; ++a) pg->h_row_ptr[a + 1] += pg->h_row_ptr[a];
    std::vector<int32_t> fill(pg->h_row_ptr.begin(), pg->h_row_ptr.end() - 1);
    pg->h_col.assign(ns, 0);
    pg->h_rev.assign(ns, 0);
    pg->h_S.assign(ns, 0.0);
    pg->h_dist.assign(ns, 0.0);
    for (size_t o = 0; o < np; ++o) {
        const size_t k = order[o];
        const int32_t lo = (int32_t)(hk[k] / (unsigned long long)q), hi = (int32_t)(hk[k] % (unsigned long long)q);
        const int32_t s1 = fill[lo]++, s2 = fill[hi]++;
        pg->h_col[s1] = hi;
        pg->h_col[s2] = lo;
        pg->h_rev[s1] = s2;
        pg->h_rev[s2] = s1;
        pg->h_S[s1] = pg->h_S[s2] = (double)hc[k];
    }
    std::vector<double> th(ns);
    for (int32_t a = 0; a < q; ++a)
        for (int32_t s = pg->h_row_ptr[a]; s < pg->h_row_ptr[a + 1]; ++s) {
            const int32_t b = pg->h_col[s];
            const double dx = pg->h_cen[3 * (size_t)a] - pg->h_cen[3 * (size_t)b];
            const double dy = pg->h_cen[3 * (size_t)a + 1] - pg->h_cen[3 * (size_t)b + 1];
            const double dz = pg->h_cen[3 * (size_t)a + 2] - pg->h_cen[3 * (size_t)b + 2];
            const double dxx = dx * dx, dyy = dy * dy, dzz = dz * dz;
            const double sum = dxx + dyy;
            pg->h_dist[s] = std::sqrt(sum + dzz);
            th[s] = pg->h_S[s] / pg->h_dist[s];
        }
    const size_t ns1 = (size_t)std::max(ns, 1);
    VGA_TRY(dmalloc((void **)&pg->vol, sizeof(double) * (size_t)q, "volumes"));
    VGA_TRY(dmalloc((void **)&pg->row_ptr, sizeof(int32_t) * ((size_t)q + 1), "row pointers"));
    VGA_TRY(dmalloc((void **)&pg->col, sizeof(int32_t) * ns1, "columns"));
    VGA_TRY(dmalloc((void **)&pg->rev, sizeof(int32_t) * ns1, "reverse slots"));
    VGA_TRY(dmalloc((void **)&pg->theta, sizeof(double) * ns1, "conductances"));
    VGA_TRY(dmalloc((void **)&pg->grad, sizeof(double) * 2 * ns1, "gradients"));
    VGA_CUDA(cudaMallocHost((void **)&pg->h_scal, sizeof(double) * 8));
    VGA_CUDA(cudaMemcpy(pg->vol, pg->h_vol.data(), sizeof(double) * (size_t)q, cudaMemcpyHostToDevice));
    VGA_CUDA(cudaMemcpy(pg->row_ptr, pg->h_row_ptr.data(), sizeof(int32_t) * ((size_t)q + 1), cudaMemcpyHostToDevice));
    if (ns > 0) {
        VGA_CUDA(cudaMemcpy(pg->col, pg->h_col.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice));
        VGA_CUDA(cudaMemcpy(pg->rev, pg->h_rev.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice));
        VGA_CUDA(cudaMemcpy(pg->theta, th.data(), sizeof(double) * ns, cudaMemcpyHostToDevice));
    }
    return check_theta_symmetry(pg, th);
}

vga_status check_pairs(const vga_pngm *pg, const int32_t *pairs, int32_t l, int64_t n_records) {
    if (l < 1 || !pairs) return fail(VGA_ERR_INVALID_ARG, "need l >= 1 pairs");
    for (int32_t k = 0; k < 2 * l; ++k)
        if (pairs[k] < 0 || pairs[k] >= n_records) return fail(VGA_ERR_INVALID_ARG, "a pair index lies outside [0, n_records)");
    (void)pg;
    return VGA_OK;
}

// Loss and gradient (raw per slot in grad[0..ns), tied in grad[ns..2ns) when requested).  The loss
// stays on the device at h_scal[0] after the copy; the stream is synchronised.
vga_status objective(vga_pngm *pg, int32_t kind, const double *d_data, int64_t n_records, const int32_t *pairs, int32_t l,
                     double D, double dt, bool tied, double *loss) {
    if (kind != 1 && kind != 2) return fail(VGA_ERR_INVALID_ARG, "objective must be 1 or 2");
    if (!d_data) return fail(VGA_ERR_INVALID_ARG, "data is NULL");
    if (!(std::isfinite(D) && D >= 0.0 && std::isfinite(dt) && dt > 0.0)) return fail(VGA_ERR_INVALID_ARG, "need D >= 0, dt > 0");
    VGA_TRY(check_pairs(pg, pairs, l, n_records));
    VGA_TRY(ensure_pairs(pg, l));
    VGA_TRY(ensure_work(pg, 6 * (int64_t)pg->q + kObjBlocks + 8));
    cudaStream_t st = pg->stream;
    std::memcpy(pg->h_pairs, pairs, sizeof(int32_t) * 2 * (size_t)l);
    VGA_CUDA(cudaMemcpyAsync(pg->d_pairs, pg->h_pairs, sizeof(int32_t) * 2 * (size_t)l, cudaMemcpyHostToDevice, st));
    const double c = D * dt;
    double *part = pg->work + 6 * (int64_t)pg->q;
    double *d_loss = part + kObjBlocks;
    const unsigned G = (unsigned)std::min<int64_t>(kObjBlocks, std::max<int64_t>(1, grid_for(pg->q, kThreads)));
    if (kind == 1)
        k_objective<1><<<G, kThreads, 0, st>>>(pg->q, pg->row_ptr, pg->col, pg->theta, pg->vol, c, d_data, pg->d_pairs, l,
                                               pg->grad, part);
    else
        k_objective<2><<<G, kThreads, 0, st>>>(pg->q, pg->row_ptr, pg->col, pg->theta, pg->vol, c, d_data, pg->d_pairs, l,
                                               pg->grad, part);
    k_sum_partials<<<1, kThreads, 0, st>>>(part, (int32_t)G, d_loss);
    if (tied && pg->nslots > 0)
        k_tie<<<grid_for(pg->nslots, kThreads), kThreads, 0, st>>>(pg->nslots, pg->rev, pg->grad, pg->grad + pg->nslots);
    VGA_CHECK_LAUNCH();
    VGA_CUDA(cudaMemcpyAsync(pg->h_scal, d_loss, sizeof(double), cudaMemcpyDeviceToHost, st));
    VGA_CUDA(cudaStreamSynchronize(st));
    if (loss) *loss = pg->h_scal[0];
    return VGA_OK;
}

}  // namespace

extern "C" {

vga_status vga_pngm_create(const vga_graph *g, const int32_t *labels, int32_t on_device, int32_t q, void *stream,
                           vga_pngm **out) {
    if (!out) return fail(VGA_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!g) return fail(VGA_ERR_INVALID_ARG, "graph is NULL");
    if (q < 1) return fail(VGA_ERR_INVALID_ARG, "q must be >= 1");
    if (!labels && g->n > 0) return fail(VGA_ERR_INVALID_ARG, "labels is NULL");
    if ((int64_t)q > g->n) return fail(VGA_ERR_INVALID_ARG, "q exceeds the node count (every primitive needs a node)");
    if ((unsigned long long)q * (unsigned long long)q >= kEmpty) return fail(VGA_ERR_INVALID_ARG, "q too large");
    vga_pngm *pg = new (std::nothrow) vga_pngm();
    if (!pg) return fail(VGA_ERR_OOM, "host allocation failed");
    pg->g = g;
    pg->stream = (cudaStream_t)stream;
    pg->q = q;
    pg->n = g->n;
    const vga_status st = build(pg, labels, on_device != 0);
    if (st != VGA_OK) {
        pngm_release(pg);
        return st;
    }
    *out = pg;
    return VGA_OK;
}

vga_status vga_pngm_get_info(const vga_pngm *pg, vga_pngm_info *out) {
    if (!pg || !out) return fail(VGA_ERR_INVALID_ARG, "pngm or out is NULL");
    out->q = pg->q;
    out->n_slots = pg->nslots;
    out->n_nodes = pg->n;
    out->cross_faces = pg->cross_faces;
    out->symmetric = pg->symmetric ? 1 : 0;
    out->last_cg_iterations = pg->last_iters;
    out->last_cg_relres = pg->last_relres;
    return VGA_OK;
}

vga_status vga_pngm_export(const vga_pngm *pg, double *volumes, double *centroids, int32_t *row_ptr, int32_t *col,
                           int32_t *rev, double *surface, double *distance) {
    if (!pg) return fail(VGA_ERR_INVALID_ARG, "pngm is NULL");
    const size_t q = (size_t)pg->q, ns = (size_t)pg->nslots;
    if (volumes) std::memcpy(volumes, pg->h_vol.data(), sizeof(double) * q);
    if (centroids) std::memcpy(centroids, pg->h_cen.data(), sizeof(double) * 3 * q);
    if (row_ptr) std::memcpy(row_ptr, pg->h_row_ptr.data(), sizeof(int32_t) * (q + 1));
    if (col && ns) std::memcpy(col, pg->h_col.data(), sizeof(int32_t) * ns);
    if (rev && ns) std::memcpy(rev, pg->h_rev.data(), sizeof(int32_t) * ns);
    if (surface && ns) std::memcpy(surface, pg->h_S.data(), sizeof(double) * ns);
    if (distance && ns) std::memcpy(distance, pg->h_dist.data(), sizeof(double) * ns);
    return VGA_OK;
}

vga_status vga_pngm_set_theta(vga_pngm *pg, const double *theta, int32_t on_device) {
    if (!pg || (!theta && pg->nslots > 0)) return fail(VGA_ERR_INVALID_ARG, "pngm or theta is NULL");
    if (pg->nslots == 0) return VGA_OK;
    std::vector<double> th(pg->nslots);
    if (on_device)
        VGA_CUDA(cudaMemcpy(th.data(), theta, sizeof(double) * pg->nslots, cudaMemcpyDeviceToHost));
    else
        std::memcpy(th.data(), theta, sizeof(double) * pg->nslots);
    for (double v : th)
        if (!std::isfinite(v)) return fail(VGA_ERR_INVALID_ARG, "conductances must be finite");
    VGA_CUDA(cudaMemcpy(pg->theta, th.data(), sizeof(double) * pg->nslots, cudaMemcpyHostToDevice));
    return check_theta_symmetry(pg, th);
}

vga_status vga_pngm_get_theta(const vga_pngm *pg, double *theta, int32_t on_device) {
    if (!pg || (!theta && pg->nslots > 0)) return fail(VGA_ERR_INVALID_ARG, "pngm or theta is NULL");
    if (pg->nslots == 0) return VGA_OK;
    VGA_CUDA(cudaStreamSynchronize(pg->stream));
    VGA_CUDA(cudaMemcpy(theta, pg->theta, sizeof(double) * pg->nslots,
                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
    return VGA_OK;
}

vga_status vga_pngm_restrict(vga_pngm *pg, vga_sim *s, int32_t comp, double *d_out) {
    if (!pg || !s || !d_out) return fail(VGA_ERR_INVALID_ARG, "pngm, sim or out is NULL");
    if (s->g != pg->g) return fail(VGA_ERR_INVALID_ARG, "the simulation runs on another graph");
    if (comp < 0 || comp > 4) return fail(VGA_ERR_INVALID_ARG, "comp must lie in [0, 4]");
    cudaStream_t st = s->stream;
    if (pg->n == 0) {
        VGA_CUDA(cudaMemsetAsync(d_out, 0, sizeof(double) * (size_t)pg->q, st));
        return VGA_OK;
    }
    if (!pg->fx) VGA_TRY(dmalloc((void **)&pg->fx, sizeof(unsigned long long) * (size_t)pg->q + 4 * sizeof(double) +
                                                       sizeof(double) * kSumBlocks, "restriction scratch"));
    double *scale = reinterpret_cast<double *>(pg->fx + pg->q);
    double *part = scale + 4;
    VGA_CUDA(cudaMemsetAsync(pg->fx, 0, sizeof(unsigned long long) * (size_t)pg->q, st));
    const unsigned Gs = (unsigned)std::min<int64_t>(kSumBlocks, grid_for(pg->n, kThreads));
    int dev = 0, sms = 0;
    VGA_CUDA(cudaGetDevice(&dev));
    VGA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    // one resident wave of segment-striding blocks
    const unsigned G = (unsigned)std::min<int64_t>((pg->n + kSeg - 1) / kSeg, (int64_t)sms * kRestrictBlocksPerSm);
    if (s->precision() == P_COMP) {
        k_abs_sum<P_COMP><<<Gs, kThreads, 0, st>>>(pg->n, s->comp(comp), s->lcomp(comp), part);
        k_fx_scale<<<1, kThreads, 0, st>>>(part, (int32_t)Gs, scale);
        k_restrict<P_COMP><<<G, kThreads, 0, st>>>(pg->n, pg->labels, s->comp(comp), s->lcomp(comp), scale, pg->fx);
    } else {
        k_abs_sum<P_F32><<<Gs, kThreads, 0, st>>>(pg->n, s->comp(comp), s->lcomp(comp), part);
        k_fx_scale<<<1, kThreads, 0, st>>>(part, (int32_t)Gs, scale);
        k_restrict<P_F32><<<G, kThreads, 0, st>>>(pg->n, pg->labels, s->comp(comp), s->lcomp(comp), scale, pg->fx);
    }
    k_fx_out<<<grid_for(pg->q, kThreads), kThreads, 0, st>>>(pg->q, pg->fx, scale, d_out);
    VGA_CHECK_LAUNCH();
    s->launches += 4;
    return VGA_OK;
}

vga_status vga_pngm_step(vga_pngm *pg, double *d_m, int64_t n_steps, int32_t scheme, double D, double dt, double cg_rtol,
                         int32_t cg_maxit) {
    if (!pg || !d_m) return fail(VGA_ERR_INVALID_ARG, "pngm or masses is NULL");
    if (n_steps < 0) return fail(VGA_ERR_INVALID_ARG, "n_steps must be >= 0");
    if (!(std::isfinite(D) && D >= 0.0 && std::isfinite(dt) && dt > 0.0)) return fail(VGA_ERR_INVALID_ARG, "need D >= 0, dt > 0");
    if (scheme != VGA_SCHEME_EXPLICIT && scheme != VGA_SCHEME_IMPLICIT_PCG) return fail(VGA_ERR_INVALID_ARG, "unknown scheme");
    const double c = D * dt;
    cudaStream_t st = pg->stream;
    const int32_t q = pg->q;
    if (scheme == VGA_SCHEME_EXPLICIT) {
        VGA_TRY(ensure_work(pg, 6 * (int64_t)q + kObjBlocks + 8));
        double *a = d_m, *b = pg->work;
        for (int64_t k = 0; k < n_steps; ++k) {
            k_scheme3<<<grid_for(q, kThreads), kThreads, 0, st>>>(q, pg->row_ptr, pg->col, pg->theta, pg->vol, c, a, b);
            std::swap(a, b);
        }
        VGA_CHECK_LAUNCH();
        if (a != d_m) VGA_CUDA(cudaMemcpyAsync(d_m, a, sizeof(double) * (size_t)q, cudaMemcpyDeviceToDevice, st));
        VGA_CUDA(cudaStreamSynchronize(st));
        return VGA_OK;
    }
    if (!pg->symmetric) return fail(VGA_ERR_UNSUPPORTED, "Scheme 4 by PCG needs tied conductances (theta_ij = theta_ji)");
    if (!(std::isfinite(cg_rtol) && cg_rtol > 0.0) || cg_maxit < 1) return fail(VGA_ERR_INVALID_ARG, "need cg_rtol > 0, cg_maxit >= 1");
    VGA_TRY(ensure_work(pg, 6 * (int64_t)q + kObjBlocks + 8));
    double *stats = pg->work + 6 * (int64_t)q + kObjBlocks;
    const double init[3] = {0.0, 0.0, 1.0};
    VGA_CUDA(cudaMemcpyAsync(stats, init, sizeof(init), cudaMemcpyHostToDevice, st));
    for (int64_t k = 0; k < n_steps; ++k)
        k_scheme4_pcg<<<1, kPcgThreads, 0, st>>>(q, pg->row_ptr, pg->col, pg->theta, pg->vol, c, d_m, pg->work, cg_rtol,
                                                 cg_maxit, stats);
    VGA_CHECK_LAUNCH();
    VGA_CUDA(cudaMemcpyAsync(pg->h_scal, stats, sizeof(double) * 3, cudaMemcpyDeviceToHost, st));
    VGA_CUDA(cudaStreamSynchronize(st));
    pg->last_iters = (int64_t)pg->h_scal[0];
    pg->last_relres = pg->h_scal[1];
    if (n_steps > 0 && pg->h_scal[2] == 0.0) return fail(VGA_ERR_NOT_CONVERGED, "Scheme 4 solve reached cg_maxit before cg_rtol");
    return VGA_OK;
}

vga_status vga_pngm_objective(vga_pngm *pg, int32_t objective_kind, const double *d_data, int64_t n_records,
                              const int32_t *pairs, int32_t l, double D, double dt, int32_t tied, double *loss,
                              double *d_grad) {
    if (!pg) return fail(VGA_ERR_INVALID_ARG, "pngm is NULL");
    VGA_TRY(objective(pg, objective_kind, d_data, n_records, pairs, l, D, dt, tied != 0, loss));
    if (d_grad && pg->nslots > 0)
        VGA_CUDA(cudaMemcpy(d_grad, pg->grad + (tied ? pg->nslots : 0), sizeof(double) * pg->nslots,
                            cudaMemcpyDeviceToDevice));
    return VGA_OK;
}

vga_status vga_pngm_sgd_step(vga_pngm *pg, int32_t objective_kind, const double *d_data, int64_t n_records,
                             const int32_t *pairs, int32_t l, double D, double dt, double lr, double theta_min,
                             int32_t tied, double *loss_before) {
    if (!pg) return fail(VGA_ERR_INVALID_ARG, "pngm is NULL");
    if (!(std::isfinite(lr) && lr >= 0.0)) return fail(VGA_ERR_INVALID_ARG, "lr must be finite and >= 0");
    if (std::isnan(theta_min) || theta_min == INFINITY) return fail(VGA_ERR_INVALID_ARG, "theta_min must be < +inf");
    VGA_TRY(objective(pg, objective_kind, d_data, n_records, pairs, l, D, dt, tied != 0, loss_before));
    if (pg->nslots > 0) {
        k_sign_sgd<<<grid_for(pg->nslots, kThreads), kThreads, 0, pg->stream>>>(
            pg->nslots, pg->grad + (tied ? pg->nslots : 0), pg->theta, lr, theta_min);
        VGA_CHECK_LAUNCH();
    }
    if (!tied) pg->symmetric = false;  // a raw update may break the symmetry; re-checked by set_theta
    return VGA_OK;
}

vga_status vga_pngm_free(vga_pngm *pg) {
    if (!pg) return VGA_OK;
    VGA_TRY(release_status("error pending before vga_pngm_free"));
    if (pg->stream) cudaStreamSynchronize(pg->stream);
    const char *bad = pngm_release(pg);
    if (bad) {
        const std::string what = std::string("vga_pngm_free (") + bad + ")";
        return release_status(what.c_str());
    }
    return release_status("vga_pngm_free");
}

}  // extern "C"
