// Per-voxel arithmetic of one time step in FP32, shared by every kernel that advances the state.
//
// All operations use explicit round-to-nearest intrinsics, so the compiler cannot contract or
// reorder them differently in different kernels: a voxel transformed in the single-step kernel,
// in the batched kernel or in a multi-step tile yields the same bits.
//
// Compensated state.  With the paper's time step (D dt = 0.15, dt ~ 1.5e-6 day) one step changes a
// compartment by 1e-6 .. 1e-8 of its value (SOM hydrolysis: v_SOM dt = 1.5e-8, below half an FP32
// ulp).  Rounding x + d to FP32 then errs the same way step after step and the error grows
// linearly with the number of steps.  Each compartment is therefore carried as a pair (h, l): an
// FP32 value h and a residual l (FP32 in registers, BF16 in memory), value = h + l.  Increments are
// added with an error-free TwoSum whose rounding error goes into l, so the stored significand has
// about 24 + 9 bits.  Fluxes are computed from h alone: their relative error (~1e-7 of a flux that
// is itself ~1e-6 of the value) does not accumulate.
#pragma once

#include <cuda_bf16.h>

#include "vga_internal.cuh"

namespace vga {

struct V {
    float h, l;
};

// State precision modes (vga_params.state_precision).
enum Precision { P_COMP = 0, P_F32 = 1 };

// v += d.  P_COMP: TwoSum, the rounding error of h + d is added to the residual.
template <int PREC>
__device__ __forceinline__ void vadd(V &v, float d) {
    const float s = __fadd_rn(v.h, d);
    if (PREC == P_COMP) {
        const float bp = __fsub_rn(s, v.h);
        const float e = __fadd_rn(__fsub_rn(v.h, __fsub_rn(s, bp)), __fsub_rn(d, bp));
        v.l = __fadd_rn(v.l, e);
    }
    v.h = s;
}

// v += w (a full pair).
template <int PREC>
__device__ __forceinline__ void vaddv(V &v, const V &w) {
    vadd<PREC>(v, w.h);
    if (PREC == P_COMP) v.l = __fadd_rn(v.l, w.l);
}

__device__ __forceinline__ float bf16_bits_to_float(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

__device__ __forceinline__ uint16_t float_to_bf16_bits(float f) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}

// Load / store of one compartment value.
template <int PREC>
__device__ __forceinline__ V vload(const float *__restrict__ H, const uint16_t *__restrict__ L, int64_t i) {
    V v;
    v.h = __ldg(H + i);
    v.l = (PREC == P_COMP) ? bf16_bits_to_float(__ldg(L + i)) : 0.0f;
    return v;
}

template <int PREC>
__device__ __forceinline__ void vstore(float *__restrict__ H, uint16_t *__restrict__ L, int64_t i, V v) {
    if (PREC == P_COMP) {
        const float s = __fadd_rn(v.h, v.l);  // renormalise: h = RN(h + l), l = exact remainder
        const float r = __fadd_rn(__fsub_rn(v.h, s), v.l);
        H[i] = s;
        L[i] = float_to_bf16_bits(r);
    } else {
        H[i] = v.h;
    }
}

// Synchronous transformation (Sec. II.C eq. 3 with the clamps of the Appendix A listing that
// computes every flux from the old state): uptake <= DOM; respiration + mortality <= MB with
// mortality served first; FOM and SOM turnover <= FOM and SOM.  Fluxes use the FP32 part h.
template <int PREC>
__device__ __forceinline__ void transform_sync(V &x1, V &x2, V &x3, V &x4, V &x5, const StepParams &p) {
    const float sat = __fdividef(x2.h, __fadd_rn(p.K, x2.h));  // Monod term x2 / (K + x2)
    float uptake = __fmul_rn(__fmul_rn(p.a, sat), x1.h);       // v_dom dt x2/(K+x2) x1
    if (uptake > x2.h) uptake = x2.h;
    float resp = __fmul_rn(p.r, x1.h);
    float morta = __fmul_rn(p.m, x1.h);
    if (__fadd_rn(resp, morta) > x1.h) {
        if (morta > x1.h) {
            morta = x1.h;
            resp = 0.0f;
        } else {
            resp = __fsub_rn(x1.h, morta);
        }
    }
    const float mDOM = __fmul_rn(p.beta, morta);
    const float mSOM = __fmul_rn(p.omb, morta);
    float tF = __fmul_rn(p.f, x4.h);
    if (tF > x4.h) tF = x4.h;
    float tS = __fmul_rn(p.s, x3.h);
    if (tS > x3.h) tS = x3.h;
    vadd<PREC>(x1, __fsub_rn(__fsub_rn(uptake, morta), resp));
    vadd<PREC>(x2, __fadd_rn(__fadd_rn(__fsub_rn(mDOM, uptake), tF), tS));
    vadd<PREC>(x3, __fsub_rn(mSOM, tS));
    vadd<PREC>(x4, -tF);
    vadd<PREC>(x5, resp);
}

// Asynchronous transformation (Appendix A sequential listing, Sec. III): growth on DOM, then
// mortality, then respiration, then SOM and FOM hydrolysis, each on the values already updated.
// Readings: the SOM/FOM branches compare their own turnover with their own stock, exhausted
// compartments are added to DOM before being zeroed, and MB is zeroed when mortality exceeds it.
template <int PREC>
__device__ __forceinline__ void transform_async(V &x1, V &x2, V &x3, V &x4, V &x5, const StepParams &p) {
    const V zero = {0.0f, 0.0f};
    if (x1.h > 0.0f) {
        if (x2.h > 0.0f) {
            const float sat = __fdividef(x2.h, __fadd_rn(p.K, x2.h));
            const float up = __fmul_rn(__fmul_rn(p.a, sat), x1.h);
            if (up < x2.h) {
                vadd<PREC>(x1, up);
                vadd<PREC>(x2, -up);
            } else {
                vaddv<PREC>(x1, x2);
                x2 = zero;
            }
        }
        const float mo = __fmul_rn(p.m, x1.h);
        if (mo < x1.h) {
            vadd<PREC>(x1, -mo);
            vadd<PREC>(x2, __fmul_rn(p.beta, mo));
            vadd<PREC>(x3, __fmul_rn(p.omb, mo));
        } else {
            vadd<PREC>(x2, __fmul_rn(p.beta, x1.h));
            vadd<PREC>(x3, __fmul_rn(p.omb, x1.h));
            x1 = zero;
        }
        const float re = __fmul_rn(p.r, x1.h);
        if (re < x1.h) {
            vadd<PREC>(x1, -re);
            vadd<PREC>(x5, re);
        } else {
            vaddv<PREC>(x5, x1);
            x1 = zero;
        }
    }
    if (x3.h > 0.0f) {
        const float ts = __fmul_rn(p.s, x3.h);
        if (ts < x3.h) {
            vadd<PREC>(x3, -ts);
            vadd<PREC>(x2, ts);
        } else {
            vaddv<PREC>(x2, x3);
            x3 = zero;
        }
    }
    if (x4.h > 0.0f) {
        const float tf = __fmul_rn(p.f, x4.h);
        if (tf < x4.h) {
            vadd<PREC>(x4, -tf);
            vadd<PREC>(x2, tf);
        } else {
            vaddv<PREC>(x2, x4);
            x4 = zero;
        }
    }
}

template <int TR, int PREC>
__device__ __forceinline__ void transform(V &x1, V &x2, V &x3, V &x4, V &x5, const StepParams &p) {
    if (TR == 0) transform_sync<PREC>(x1, x2, x3, x4, x5, p);
    else transform_async<PREC>(x1, x2, x3, x4, x5, p);
}

}  // namespace vga
