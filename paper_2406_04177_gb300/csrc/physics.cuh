// Per-voxel arithmetic of one time step in FP32, shared by every kernel that advances the state.
//
// All operations use explicit round-to-nearest intrinsics, so the compiler cannot contract or
// reorder them differently in different kernels: a voxel transformed in the single-step kernel,
// in the batched kernel or in a halo of a multi-step tile yields the same bits.
#pragma once

#include "vga_internal.cuh"

namespace vga {

// Synchronous transformation (Sec. II.C eq. 3 with the clamps of the Appendix A listing that
// computes every flux from the old state): uptake <= DOM; respiration + mortality <= MB with
// mortality served first; FOM and SOM turnover <= FOM and SOM.
__device__ __forceinline__ void transform_sync(float &x1, float &x2, float &x3, float &x4, float &x5,
                                               const StepParams &p) {
    const float sat = __fdividef(x2, __fadd_rn(p.K, x2));        // Monod term x2 / (K + x2)
    float uptake = __fmul_rn(__fmul_rn(p.a, sat), x1);          // v_dom dt x2/(K+x2) x1
    if (uptake > x2) uptake = x2;
    float resp = __fmul_rn(p.r, x1);
    float morta = __fmul_rn(p.m, x1);
    if (__fadd_rn(resp, morta) > x1) {
        if (morta > x1) {
            morta = x1;
            resp = 0.0f;
        } else {
            resp = __fsub_rn(x1, morta);
        }
    }
    const float mDOM = __fmul_rn(p.beta, morta);
    const float mSOM = __fmul_rn(p.omb, morta);
    float tF = __fmul_rn(p.f, x4);
    if (tF > x4) tF = x4;
    float tS = __fmul_rn(p.s, x3);
    if (tS > x3) tS = x3;
    x1 = __fadd_rn(x1, __fsub_rn(__fsub_rn(uptake, morta), resp));
    x2 = __fadd_rn(x2, __fadd_rn(__fadd_rn(__fsub_rn(mDOM, uptake), tF), tS));
    x3 = __fadd_rn(x3, __fsub_rn(mSOM, tS));
    x4 = __fsub_rn(x4, tF);
    x5 = __fadd_rn(x5, resp);
}

// Asynchronous transformation (Appendix A sequential listing, Sec. III): growth on DOM, then
// mortality, then respiration, then SOM and FOM hydrolysis, each on the values already updated.
// Readings: the SOM/FOM branches compare their own turnover with their own stock, exhausted
// compartments are added to DOM before being zeroed, and MB is zeroed when mortality exceeds it.
__device__ __forceinline__ void transform_async(float &x1, float &x2, float &x3, float &x4, float &x5,
                                                const StepParams &p) {
    if (x1 > 0.0f) {
        if (x2 > 0.0f) {
            const float sat = __fdividef(x2, __fadd_rn(p.K, x2));
            const float up = __fmul_rn(__fmul_rn(p.a, sat), x1);
            if (up < x2) {
                x1 = __fadd_rn(x1, up);
                x2 = __fsub_rn(x2, up);
            } else {
                x1 = __fadd_rn(x1, x2);
                x2 = 0.0f;
            }
        }
        const float mo = __fmul_rn(p.m, x1);
        if (mo < x1) {
            x1 = __fsub_rn(x1, mo);
            x2 = __fadd_rn(x2, __fmul_rn(p.beta, mo));
            x3 = __fadd_rn(x3, __fmul_rn(p.omb, mo));
        } else {
            x2 = __fadd_rn(x2, __fmul_rn(p.beta, x1));
            x3 = __fadd_rn(x3, __fmul_rn(p.omb, x1));
            x1 = 0.0f;
        }
        const float re = __fmul_rn(p.r, x1);
        if (re < x1) {
            x1 = __fsub_rn(x1, re);
            x5 = __fadd_rn(x5, re);
        } else {
            x5 = __fadd_rn(x5, x1);
            x1 = 0.0f;
        }
    }
    if (x3 > 0.0f) {
        const float ts = __fmul_rn(p.s, x3);
        if (ts < x3) {
            x3 = __fsub_rn(x3, ts);
            x2 = __fadd_rn(x2, ts);
        } else {
            x2 = __fadd_rn(x2, x3);
            x3 = 0.0f;
        }
    }
    if (x4 > 0.0f) {
        const float tf = __fmul_rn(p.f, x4);
        if (tf < x4) {
            x4 = __fsub_rn(x4, tf);
            x2 = __fadd_rn(x2, tf);
        } else {
            x2 = __fadd_rn(x2, x4);
            x4 = 0.0f;
        }
    }
}

template <int TR>
__device__ __forceinline__ void transform(float &x1, float &x2, float &x3, float &x4, float &x5,
                                          const StepParams &p) {
    if (TR == 0) transform_sync(x1, x2, x3, x4, x5, p);
    else transform_async(x1, x2, x3, x4, x5, p);
}

// Node index of voxel x in image row `row`, or -1 when it is not a node (see Topo).
__device__ __forceinline__ int64_t node_in_row(const Topo &t, int32_t row, int32_t x) {
    const int32_t q = row * t.W + (x >> 5);
    const uint32_t m = __ldg(t.mask + q);
    const uint32_t bit = 1u << (x & 31);
    if (!(m & bit)) return -1;
    return (int64_t)__ldg(t.pre + q) + __popc(m & (bit - 1u));
}

__device__ __forceinline__ bool is_node(const Topo &t, int32_t row, int32_t x) {
    const uint32_t m = __ldg(t.mask + row * t.W + (x >> 5));
    return (m >> (x & 31)) & 1u;
}

}  // namespace vga
