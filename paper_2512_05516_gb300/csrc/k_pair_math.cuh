// Per-pair arithmetic of the SPH kernels, in FP32: the M4 spline (support
// 2h, sigma = 1/pi in 3D), compensated accumulation and one symmetric force
// pair with Monaghan viscosity (Eq. 7, Eq. 5).  Shared by the cell-list pair
// kernels (k_pairs.cu) and the buffer kernels (k_buffers.cu).
#pragma once

#include "sph_internal.cuh"

namespace sph {

// M4 spline w(q) and w'(q), branch-free, for any q >= 0: with the clamped
// linear terms p = sat(1 - q/2) = max(2 - q, 0) / 2 and u = sat(1 - q)
// (sat clamps to [0, 1], so both run on the FMA pipe),
//   w = 2 p^3 - u^3,   w' = 3 (u^2 - p^2),
// which is 1 - 3q^2/2 + 3q^3/4 on [0, 1), (2 - q)^3 / 4 on [1, 2) and 0 beyond.
struct SplineTerms {
    float p, u, p2, u2;
};

__device__ __forceinline__ SplineTerms spline_terms(float q)
{
    SplineTerms s;
    s.p = __saturatef(fmaf(q, -0.5f, 1.0f));
    s.u = __saturatef(1.0f - q);
    s.p2 = s.p * s.p;
    s.u2 = s.u * s.u;
    return s;
}

__device__ __forceinline__ void spline(float q, float &w, float &dw)
{
    const SplineTerms s = spline_terms(q);
    w = fmaf(s.p2 + s.p2, s.p, -(s.u2 * s.u));
    dw = 3.0f * (s.u2 - s.p2);
}

// 1 / sqrt(x) for x >= 1e-30 (a normal number), the approximate hardware
// reciprocal square root (the same result as rsqrtf for such x, without the
// handling of subnormal inputs)
__device__ __forceinline__ float rsqrt_normal(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Kahan compensated accumulation: s - c carries the running sum; c holds the
// low-order part lost by the last addition (the terms are non-negative)
__device__ __forceinline__ void kahan_add(float &s, float &c, float x)
{
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
}

// One interacting force pair: separation d = x_i - x_j, hs = h_i + h_j,
// qb = (v_j, m_j), qc = (P_j / rho_j^2, rho_j, c_j, -).  A pair at r = 0 (the
// particle itself, or a coincident one) adds exactly zero: w'(0) = 0 and
// v_ij . d = 0.
__device__ __forceinline__ void force_pair(float &ax, float &ay, float &az, float &du, float vxi, float vyi,
                                           float vzi, float rhoi, float Pr2i, float ci, float dx, float dy,
                                           float dz, float r2, float hs, const float4 qb, const float4 qc,
                                           float alpha, float beta, float eps)
{
    const float rinv = rsqrt_normal(fmaxf(r2, 1.0e-30f));
    const float r = r2 * rinv;
    const float hb = 0.5f * hs;
    const float hbinv = __fdividef(2.0f, hs);
    const float qq = r * hbinv;
    float w, dw;
    spline(qq, w, dw);
    const float hb2 = hbinv * hbinv;
    const float gw = kSigma * hb2 * hb2 * dw * rinv;   // grad_i W = d * gw
    const float vx = vxi - qb.x, vy = vyi - qb.y, vz = vzi - qb.z;
    const float vdotr = fmaf(vx, dx, fmaf(vy, dy, vz * dz));
    // Monaghan viscosity, branch-free: a receding pair (v_ij . d >= 0) gets
    // mu = 0 and so visc = 0 exactly (a branch costs more here: the lanes of
    // a warp disagree on it)
    const float mu = __fdividef(hb * fminf(vdotr, 0.0f), fmaf(eps * hb, hb, r2));
    const float cbar = 0.5f * (ci + qc.z);
    const float rbar = 0.5f * (rhoi + qc.y);
    const float visc = __fdividef(fmaf(-alpha * cbar, mu, beta * mu * mu), rbar);
    const float fac = qb.w * (Pr2i + qc.x + visc) * gw;
    ax = fmaf(-fac, dx, ax);
    ay = fmaf(-fac, dy, ay);
    az = fmaf(-fac, dz, az);
    du = fmaf(qb.w * fmaf(0.5f, visc, Pr2i), vdotr * gw, du);
}

}  // namespace sph
