// Euler fluxes of the record-path kernels (kernels_fast.cu, kernels_tc.cu).
#pragma once

#include <cuda_runtime.h>

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

// s F_Rusanov(u_L, u_R, n): F = (n.f_L + n.f_R)/2 + phi/2 (u_L - u_R).
template <typename T, int ND>
__device__ __forceinline__ void rusanov_rec(const T* uL, const T* uR, const T* n, T gamma, T s, T* F) {
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
    const T phi = fmax(fabs(vnL) + cL, fabs(vnR) + cR);
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
