// Euler fluxes of the record-path kernels (kernels_fast.cu, kernels_tc.cu).
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace sdrt {
namespace {

// Euler / Rusanov on the record path with fewer instructions than the
// generic helpers of device_math.cuh: one reciprocal of the density per state
// (FP32: the hardware approximation refined by one Newton-Raphson step
// r <- r + r (1 - x r)), the sound speed from the reciprocal square root, and
// the factor s / 2 of the transformed flux folded into the combination.
__device__ __forceinline__ float recip(float x) {
    const float r = __fdividef(1.0f, x);
    return fmaf(r, fmaf(-x, r, 1.0f), r);
}
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float pos_sqrt(float x) { return x * rsqrtf(x); }   // x > 0
__device__ __forceinline__ double pos_sqrt(double x) { return sqrt(x); }

// Velocity, |v|^2-weighted pressure and 1/rho of one conserved state.
template <typename T, int ND>
__device__ __forceinline__ void prim_rec(const T* u, T gamma, T& inv, T* v, T& p) {
    inv = recip(u[0]);
    T ke = T(0);
    #pragma unroll
    for (int d = 0; d < ND; ++d) {
        v[d] = u[1 + d] * inv;
        ke = fma(u[1 + d], v[d], ke);
    }
    p = (gamma - T(1)) * fma(T(-0.5), ke, u[ND + 1]);
}

// FP32: the primitive variables, normal velocities and sound speeds of the
// left and right states as the two lanes of float2 pairs on the paired FP32
// instructions of sm_100 and later (__fmul2_rn / __ffma2_rn: IEEE
// round-to-nearest per lane), in the same operations and order as the scalar
// code below, so the results are bit-identical.
template <int ND>
__device__ __forceinline__ void rusanov_rec_pair(const float* uL, const float* uR, const float* n, float gamma, float s,
                                                 float* F) {
    constexpr int V = ND + 2;
    float2 u[V];
    #pragma unroll
    for (int v = 0; v < V; ++v) u[v] = make_float2(uL[v], uR[v]);
    float2 inv = make_float2(__fdividef(1.0f, u[0].x), __fdividef(1.0f, u[0].y));
    inv = __ffma2_rn(inv, __ffma2_rn(make_float2(-u[0].x, -u[0].y), inv, make_float2(1.f, 1.f)), inv);
    float2 vv[ND];
    float2 ke = make_float2(0.f, 0.f);
    #pragma unroll
    for (int d = 0; d < ND; ++d) {
        vv[d] = __fmul2_rn(u[1 + d], inv);
        ke = __ffma2_rn(u[1 + d], vv[d], ke);
    }
    const float g1 = gamma - 1.0f;
    const float2 p = __fmul2_rn(make_float2(g1, g1), __ffma2_rn(make_float2(-0.5f, -0.5f), ke, u[V - 1]));
    float2 vn = __fmul2_rn(vv[0], make_float2(n[0], n[0]));
    #pragma unroll
    for (int d = 1; d < ND; ++d) vn = __ffma2_rn(vv[d], make_float2(n[d], n[d]), vn);
    const float2 c2 = __fmul2_rn(__fmul2_rn(make_float2(gamma, gamma), p), inv);
    const float cL = c2.x * rsqrtf(c2.x), cR = c2.y * rsqrtf(c2.y);
    // + 0 (cL + cR): a non-physical state (negative pressure or density, NaN
    // sound speed) stays NaN instead of being dropped by fmaxf.
    const float phi = fmaxf(fabsf(vn.x) + cL, fabsf(vn.y) + cR) + 0.0f * (cL + cR);
    const float hs = 0.5f * s;
    F[0] = hs * fmaf(phi, u[0].x - u[0].y, fmaf(u[0].x, vn.x, u[0].y * vn.y));
    const float pp = p.x + p.y;
    #pragma unroll
    for (int i = 0; i < ND; ++i)
        F[1 + i] = hs * fmaf(phi, u[1 + i].x - u[1 + i].y, fmaf(pp, n[i], fmaf(u[1 + i].x, vn.x, u[1 + i].y * vn.y)));
    F[V - 1] = hs * fmaf(phi, u[V - 1].x - u[V - 1].y, fmaf(u[V - 1].x + p.x, vn.x, (u[V - 1].y + p.y) * vn.y));
}

// s F_Rusanov(u_L, u_R, n): F = (n.f_L + n.f_R)/2 + phi/2 (u_L - u_R).
template <typename T, int ND>
__device__ __forceinline__ void rusanov_rec(const T* uL, const T* uR, const T* n, T gamma, T s, T* F) {
    if constexpr (std::is_same<T, float>::value) {
        rusanov_rec_pair<ND>(uL, uR, n, gamma, s, F);
        return;
    }
    constexpr int V = ND + 2;
    T iL, iR, vL[ND], vR[ND], pL, pR;
    prim_rec<T, ND>(uL, gamma, iL, vL, pL);
    prim_rec<T, ND>(uR, gamma, iR, vR, pR);
    T vnL = vL[0] * n[0], vnR = vR[0] * n[0];
    #pragma unroll
    for (int d = 1; d < ND; ++d) {
        vnL = fma(vL[d], n[d], vnL);
        vnR = fma(vR[d], n[d], vnR);
    }
    const T cL = pos_sqrt(gamma * pL * iL);
    const T cR = pos_sqrt(gamma * pR * iR);
    const T phi = fmax(fabs(vnL) + cL, fabs(vnR) + cR) + T(0) * (cL + cR);
    const T hs = T(0.5) * s;
    F[0] = hs * fma(phi, uL[0] - uR[0], fma(uL[0], vnL, uR[0] * vnR));
    const T pp = pL + pR;
    #pragma unroll
    for (int i = 0; i < ND; ++i)
        F[1 + i] = hs * fma(phi, uL[1 + i] - uR[1 + i], fma(pp, n[i], fma(uL[1 + i], vnL, uR[1 + i] * vnR)));
    F[V - 1] = hs * fma(phi, uL[V - 1] - uR[V - 1], fma(uL[V - 1] + pL, vnL, (uR[V - 1] + pR) * vnR));
}

}  // namespace
}  // namespace sdrt
