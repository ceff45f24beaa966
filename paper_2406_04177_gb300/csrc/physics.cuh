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
// is itself ~1e-6 of the value) does not accumulate.  (A fixed-point 8-bit residual in units of
// ulp(h)/256 was measured as well: it rounds a constant per-step decrement the same way every step,
// which biases slow decays about 4x more, and its encoding costs more instructions than the
// bytes it saves.)
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

// Packed pairs (PTX .f32x2, sm_100 and later): each lane is one round-to-nearest IEEE addition or
// subtraction, as __fadd_rn / __fsub_rn, so a pair gives the bits of the two scalar operations in
// one instruction (subnormals kept: no .ftz).  There is no packed multiply here: a packed multiply
// whose result feeds a packed add is contracted into a fused multiply-add by the code generator in
// spite of the .rn modifiers (measured: 14% of the results of x + c*y differed), while scalar
// __fmul_rn is never contracted, so products are formed in scalar.
__device__ __forceinline__ float2 add2_rn(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}
__device__ __forceinline__ float2 sub2_rn(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// BF16 bits of a (low half) and b (high half), each rounded to nearest as float_to_bf16_bits.
__device__ __forceinline__ uint32_t bf16x2_bits(float a, float b) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    uint32_t u;
    memcpy(&u, &v, sizeof(u));
    return u;
}

// Stored residual r of a value whose FP32 part is h (the BF16 encoding does not need h).
__device__ __forceinline__ res_t res_encode(float r, float /*h*/) { return float_to_bf16_bits(r); }
__device__ __forceinline__ float res_decode(res_t q, float /*h*/) { return bf16_bits_to_float(q); }

// Value h + l of a stored pair in FP64.
template <int PREC>
__device__ __forceinline__ double ld_value_d(const float *__restrict__ H, const res_t *__restrict__ L, int64_t i) {
    const float h = __ldg(H + i);
    return (double)h + (PREC == P_COMP ? (double)res_decode(__ldg(L + i), h) : 0.0);
}

// Load / store of one compartment value.
template <int PREC>
__device__ __forceinline__ V vload(const float *__restrict__ H, const res_t *__restrict__ L, int64_t i) {
    V v;
    v.h = __ldg(H + i);
    v.l = (PREC == P_COMP) ? res_decode(__ldg(L + i), v.h) : 0.0f;
    return v;
}

template <int PREC>
__device__ __forceinline__ void vstore(float *__restrict__ H, res_t *__restrict__ L, int64_t i, V v) {
    if (PREC == P_COMP) {
        const float s = __fadd_rn(v.h, v.l);  // renormalise: h = RN(h + l), l = exact remainder
        const float r = __fadd_rn(__fsub_rn(v.h, s), v.l);
        H[i] = s;
        L[i] = res_encode(r, s);
    } else {
        H[i] = v.h;
    }
}

// Rounds a pair to exactly what vstore followed by vload yields, so a value kept in registers across
// two stages of one pass behaves as if it had been stored in between (a run split into several
// calls then reproduces an uninterrupted run bit for bit).
template <int PREC>
__device__ __forceinline__ void vround(V &v) {
    if (PREC == P_COMP) {
        const float s = __fadd_rn(v.h, v.l);
        const float r = __fadd_rn(__fsub_rn(v.h, s), v.l);
        v.h = s;
        v.l = res_decode(res_encode(r, s), s);
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

// p.ntrans transformations of step dt_transform (the rates in p are already scaled by it).
template <int TR, int PREC>
__device__ __forceinline__ void transform_n(V &x1, V &x2, V &x3, V &x4, V &x5, const StepParams &p) {
#pragma unroll 1
    for (int t = 0; t < p.ntrans; ++t) transform<TR, PREC>(x1, x2, x3, x4, x5, p);
}

}  // namespace vga

namespace vga {

// Rate-gradient slots accumulated by the reverse transformation.  The first five are derivatives
// with respect to the dt-products (v_dom dt, rho dt, mu dt, v_fom dt, v_som dt); the caller scales
// them by dt to obtain derivatives with respect to the rates.
enum { GR_A = 0, GR_R, GR_M, GR_F, GR_S, GR_BETA, GR_K, GR_COUNT };

// Reverse of transform_sync at the pre-transformation state x (FP32 values).  The transformation
// is y = x + S f(x) with fluxes f = (uptake, morta, resp, turnFOM, turnSOM); with w = S^T mu the
// adjoint of x is mu + (df/dx)^T w, and w . df/dtheta are the rate gradients.  Every derivative
// follows the branch the forward clamps took at x.
template <int PREC>
__device__ __forceinline__ void transform_sync_reverse(const float (&x)[5], const V (&mu)[5], V (&lam)[5],
                                                       float (&gr)[GR_COUNT], const StepParams &p) {
    const float x1 = x[0], x2 = x[1], x3 = x[2], x4 = x[3];
    const float kx = __fadd_rn(p.K, x2);
    const float sat = __fdividef(x2, kx);
    const float u0 = __fmul_rn(__fmul_rn(p.a, sat), x1);
    const bool upt_clamped = u0 > x2;
    const float r0 = __fmul_rn(p.r, x1), m0 = __fmul_rn(p.m, x1);
    int mr_case = 0;  // 0: free, 1: morta = x1 and resp = 0, 2: resp = x1 - morta
    if (__fadd_rn(r0, m0) > x1) mr_case = (m0 > x1) ? 1 : 2;
    const float morta = (mr_case == 1) ? x1 : m0;
    const bool tF_clamped = __fmul_rn(p.f, x4) > x4;
    const bool tS_clamped = __fmul_rn(p.s, x3) > x3;

    const float w_upt = __fsub_rn(mu[0].h, mu[1].h);
    const float w_mor = __fadd_rn(__fadd_rn(-mu[0].h, __fmul_rn(p.beta, mu[1].h)), __fmul_rn(p.omb, mu[2].h));
    const float w_resp = __fsub_rn(mu[4].h, mu[0].h);
    const float w_tF = __fsub_rn(mu[1].h, mu[3].h);
    const float w_tS = __fsub_rn(mu[1].h, mu[2].h);

    float d[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    if (upt_clamped) {
        d[1] = __fadd_rn(d[1], w_upt);
    } else {
        const float inv2 = __fdividef(1.0f, __fmul_rn(kx, kx));
        d[0] = __fadd_rn(d[0], __fmul_rn(w_upt, __fmul_rn(p.a, sat)));
        d[1] = __fadd_rn(d[1], __fmul_rn(w_upt, __fmul_rn(__fmul_rn(__fmul_rn(p.a, x1), p.K), inv2)));
        gr[GR_A] = __fadd_rn(gr[GR_A], __fmul_rn(w_upt, __fmul_rn(sat, x1)));
        gr[GR_K] = __fsub_rn(gr[GR_K], __fmul_rn(w_upt, __fmul_rn(__fmul_rn(__fmul_rn(p.a, x2), x1), inv2)));
    }
    if (mr_case == 0) {
        d[0] = __fadd_rn(d[0], __fadd_rn(__fmul_rn(w_mor, p.m), __fmul_rn(w_resp, p.r)));
        gr[GR_M] = __fadd_rn(gr[GR_M], __fmul_rn(w_mor, x1));
        gr[GR_R] = __fadd_rn(gr[GR_R], __fmul_rn(w_resp, x1));
    } else if (mr_case == 1) {
        d[0] = __fadd_rn(d[0], w_mor);
    } else {
        d[0] = __fadd_rn(d[0], __fadd_rn(__fmul_rn(w_mor, p.m), __fmul_rn(w_resp, __fsub_rn(1.0f, p.m))));
        gr[GR_M] = __fadd_rn(gr[GR_M], __fmul_rn(__fsub_rn(w_mor, w_resp), x1));
    }
    gr[GR_BETA] = __fadd_rn(gr[GR_BETA], __fmul_rn(__fsub_rn(mu[1].h, mu[2].h), morta));
    if (tF_clamped) {
        d[3] = __fadd_rn(d[3], w_tF);
    } else {
        d[3] = __fadd_rn(d[3], __fmul_rn(w_tF, p.f));
        gr[GR_F] = __fadd_rn(gr[GR_F], __fmul_rn(w_tF, x4));
    }
    if (tS_clamped) {
        d[2] = __fadd_rn(d[2], w_tS);
    } else {
        d[2] = __fadd_rn(d[2], __fmul_rn(w_tS, p.s));
        gr[GR_S] = __fadd_rn(gr[GR_S], __fmul_rn(w_tS, x3));
    }
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        lam[c] = mu[c];
        vadd<PREC>(lam[c], d[c]);
    }
}

}  // namespace vga
