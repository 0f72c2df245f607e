// Bloch propagation on the GPU (Appendix, Eq. A2 with the hard-pulse RF form,
// or the off-resonant form for pulses of finite duration, and the recovery
// term of Eq. A1), FP32, one fingerprint per thread.
//
// State (mx, my, w) with w = 1 - Mz. Per timepoint j:
//   RF:  M <- R_z(phi_j) R_x(-alpha_j) R_z(-phi_j) M     (coefficients from SeqDev;
//        finite pulses: the effective-field rotation, per candidate df)
//   evolve TE_j:         (mx + i my) <- E2 e^{i theta} (mx + i my),  w <- E1 w
//   sample s_j = mx + i my
//   evolve TR_j - TE_j
// with E1 = exp(-tau/T1), E2 = exp(-tau/T2), theta = 2 pi df tau / 1000.
#pragma once

#include <cuda_runtime.h>

#include "mrf_internal.h"

struct Bloch {
    float mx, my, w;
};

__device__ __forceinline__ void bloch_init(Bloch &s) { s.mx = 0.f; s.my = 0.f; s.w = 0.f; }

// Ideal 180 degree inversion about x from equilibrium: Mz = -1, i.e. w = 2.
__device__ __forceinline__ void bloch_invert(Bloch &s) { s.mx = 0.f; s.my = 0.f; s.w = 2.f; }

// x-rotation by beta in deficit form: my' = c my + s w - s, w' = (1 - c) + c w - s my.
__device__ __forceinline__ void bloch_rf_x(Bloch &st, float4 r)
{
    const float c = r.x, s = r.y, omc = r.z;
    const float my = fmaf(c, st.my, fmaf(s, st.w, -s));
    const float w = fmaf(c, st.w, fmaf(-s, st.my, omc));
    st.my = my;
    st.w = w;
}

// General rotation R (row-major 3x3) in deficit form, q[9] = 1 - R22.
__device__ __forceinline__ void bloch_rf_general(Bloch &st, const float *q)
{
    const float mx = st.mx, my = st.my, w = st.w;
    st.mx = fmaf(q[0], mx, fmaf(q[1], my, fmaf(-q[2], w, q[2])));
    st.my = fmaf(q[3], mx, fmaf(q[4], my, fmaf(-q[5], w, q[5])));
    st.w = fmaf(q[8], w, fmaf(-q[6], mx, fmaf(-q[7], my, q[9])));
}

// RF pulse of finite duration tau off resonance by df (Appendix): R_RF =
// R_z(phi) R_y(beta) R_x(alpha') R_y(-beta) R_z(-phi) is the counterclockwise
// rotation by theta = |a| about a = (-alpha cos phi, -alpha sin phi, tau dw),
// dw = 2 pi df / 1000 rad/ms (the RF and off-resonance fields acting
// together), written in Rodrigues' form with half-angle factors,
//   R = cos(theta) I + k1 [a]x + k2 a a^T,  h = theta / 2,
//   k1 = sin(theta) / theta = sinc(h) cos(h),  k2 = (1 - cos theta) / theta^2 = sinc(h)^2 / 2,
// and 1 - R22 = k2 alpha^2 in deficit form. p = (-alpha cos phi, -alpha sin
// phi, alpha^2, 2 pi tau), f = df / 1000 (cycles per ms). Accurate sqrtf and
// sincosf.
__device__ __forceinline__ void bloch_rf_finite(Bloch &st, float4 p, float f)
{
    const float ax = p.x, ay = p.y, az = p.w * f;
    const float h = 0.5f * sqrtf(fmaf(az, az, p.z));
    float sh, ch;
    sincosf(h, &sh, &ch);
    const float sc = h > 0.f ? sh / h : 1.f;
    const float k1 = sc * ch, k2 = 0.5f * sc * sc;
    const float cth = fmaf(-2.f * sh, sh, 1.f);
    float q[10];
    q[0] = fmaf(k2 * ax, ax, cth);
    q[1] = fmaf(k2 * ax, ay, -k1 * az);
    q[2] = fmaf(k2 * ax, az, k1 * ay);
    q[3] = fmaf(k2 * ay, ax, k1 * az);
    q[4] = fmaf(k2 * ay, ay, cth);
    q[5] = fmaf(k2 * ay, az, -k1 * ax);
    q[6] = fmaf(k2 * az, ax, -k1 * ay);
    q[7] = fmaf(k2 * az, ay, k1 * ax);
    q[8] = fmaf(k2 * az, az, cth);
    q[9] = k2 * p.z;
    bloch_rf_general(st, q);
}

// Free evolution with precomputed z = E2 e^{i theta} and E1.
__device__ __forceinline__ void bloch_evolve(Bloch &st, float e1, float zr, float zi)
{
    const float mx = fmaf(zr, st.mx, -zi * st.my);
    const float my = fmaf(zi, st.mx, zr * st.my);
    st.mx = mx;
    st.my = my;
    st.w *= e1;
}

// 2^x on the SFU (PTX ex2.approx.ftz; relative error about 2^-22).
__device__ __forceinline__ float ex2_fast(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Per-fingerprint constants for on-the-fly evolution factors.
struct Relax {
    float k1;   // -log2(e) / T1
    float k2;   // -log2(e) / T2
    float f;    // df / 1000  (cycles per ms)
};

__device__ __forceinline__ Relax relax_make(float T1, float T2, float df)
{
    Relax r;
    r.k1 = -1.4426950408889634f / T1;
    r.k2 = -1.4426950408889634f / T2;
    r.f = df * 1.0e-3f;
    return r;
}

// Evolution factors for an interval of tau ms, computed with CUDA's exp2f and
// sincospif (argument reduced to [-1/2, 1/2] cycles first).
__device__ __forceinline__ void relax_factors(const Relax &r, float tau, float &e1, float &zr, float &zi)
{
    e1 = exp2f(r.k1 * tau);
    const float e2 = exp2f(r.k2 * tau);
    float t = r.f * tau;
    t -= rintf(t);
    float sn, cs;
    sincospif(2.0f * t, &sn, &cs);
    zr = e2 * cs;
    zi = e2 * sn;
}

// e^{i 2 pi f tau} on the SFU, the argument first reduced to [-1/2, 1/2] cycles.
__device__ __forceinline__ void cis_sfu(float f, float tau, float &cs, float &sn)
{
    float t = f * tau;
    t -= rintf(t);
    __sincosf(6.283185307179586f * t, &sn, &cs);
}

// RF pulse of timepoint j for a candidate off resonance by f = df / 1000
// cycles per ms (dispatch on the sequence kind; `xonly` and `finite` are
// uniform).
template <bool XONLY>
__device__ __forceinline__ void bloch_rf(Bloch &st, const SeqDev &s, int j, float f)
{
    if (XONLY) {
        bloch_rf_x(st, __ldg(&s.rfx[j]));
    } else if (s.finite) {
        bloch_rf_finite(st, __ldg(&s.rff[j]), f);
    } else {
        float q[10];
        const float4 *p = reinterpret_cast<const float4 *>(s.rfg + 12 * j);
        float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
        q[0] = a.x; q[1] = a.y; q[2] = a.z; q[3] = a.w;
        q[4] = b.x; q[5] = b.y; q[6] = b.z; q[7] = b.w;
        q[8] = c.x; q[9] = c.y;
        bloch_rf_general(st, q);
    }
}

// Start of a fingerprint: equilibrium, then optional inversion + delay.
__device__ __forceinline__ void bloch_start(Bloch &st, const SeqDev &s, const Relax &r)
{
    bloch_init(st);
    if (s.inversion) {
        bloch_invert(st);
        float e1, zr, zi;
        relax_factors(r, s.inv_delay, e1, zr, zi);
        bloch_evolve(st, e1, zr, zi);
    }
}

// One full timepoint with on-the-fly factors; returns the sample in (sr, si).
template <bool XONLY>
__device__ __forceinline__ void bloch_step_otf(Bloch &st, const SeqDev &s, const Relax &r, int j, float &sr,
                                               float &si)
{
    bloch_rf<XONLY>(st, s, j, r.f);
    const float2 tau = __ldg(&s.tau[j]);
    float e1, zr, zi;
    relax_factors(r, tau.x, e1, zr, zi);
    bloch_evolve(st, e1, zr, zi);
    sr = st.mx;
    si = st.my;
    if (s.symmetric) {
        bloch_evolve(st, e1, zr, zi);
    } else {
        relax_factors(r, tau.y, e1, zr, zi);
        bloch_evolve(st, e1, zr, zi);
    }
}
