// Scalar helpers for the SDRT kernels: a forward-mode dual number for the JVP,
// branch-by-primal |.| and max (ties take the non-negative / first branch), and
// the physical / common fluxes of paper Sec. 2.1, 3, 5.
#pragma once

#include <cuda_runtime.h>

namespace sdrt {

template <typename T>
struct Dual {
    T v, d;
};

template <typename T> __device__ __forceinline__ T pval(T x) { return x; }
template <typename T> __device__ __forceinline__ T pval(Dual<T> x) { return x.v; }

template <typename T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, Dual<T> b) { return {a.v + b.v, a.d + b.d}; }
template <typename T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, Dual<T> b) { return {a.v - b.v, a.d - b.d}; }
template <typename T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a) { return {-a.v, -a.d}; }
template <typename T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, Dual<T> b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }
template <typename T> __device__ __forceinline__ Dual<T> operator/(Dual<T> a, Dual<T> b) {
    T q = a.v / b.v;
    return {q, (a.d - q * b.d) / b.v};
}
template <typename T> __device__ __forceinline__ Dual<T> operator+(Dual<T> a, T b) { return {a.v + b, a.d}; }
template <typename T> __device__ __forceinline__ Dual<T> operator+(T a, Dual<T> b) { return {a + b.v, b.d}; }
template <typename T> __device__ __forceinline__ Dual<T> operator-(Dual<T> a, T b) { return {a.v - b, a.d}; }
template <typename T> __device__ __forceinline__ Dual<T> operator-(T a, Dual<T> b) { return {a - b.v, -b.d}; }
template <typename T> __device__ __forceinline__ Dual<T> operator*(Dual<T> a, T b) { return {a.v * b, a.d * b}; }
template <typename T> __device__ __forceinline__ Dual<T> operator*(T a, Dual<T> b) { return {a * b.v, a * b.d}; }
template <typename T> __device__ __forceinline__ Dual<T> operator/(Dual<T> a, T b) { return {a.v / b, a.d / b}; }
template <typename T> __device__ __forceinline__ Dual<T> operator/(T a, Dual<T> b) {
    T q = a / b.v;
    return {q, -q * b.d / b.v};
}
template <typename T> __device__ __forceinline__ Dual<T>& operator+=(Dual<T>& a, Dual<T> b) { a = a + b; return a; }

__device__ __forceinline__ float ssqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double ssqrt(double x) { return sqrt(x); }
template <typename T> __device__ __forceinline__ Dual<T> ssqrt(Dual<T> x) {
    T r = ssqrt(x.v);
    return {r, x.d / (T(2) * r)};
}

template <typename S> __device__ __forceinline__ S sabs(S x) { return pval(x) >= 0 ? x : -x; }
template <typename S> __device__ __forceinline__ S smax(S a, S b) { return pval(a) >= pval(b) ? a : b; }
template <typename T> __device__ __forceinline__ bool sfinite(T x) { return isfinite(x); }

// acc += a * b with a real operator entry a.
template <typename T> __device__ __forceinline__ void mac(T& acc, T a, T b) { acc = fma(a, b, acc); }
template <typename T> __device__ __forceinline__ void mac(Dual<T>& acc, T a, Dual<T> b) {
    acc.v = fma(a, b.v, acc.v);
    acc.d = fma(a, b.d, acc.d);
}
template <typename S> __device__ __forceinline__ S szero() { return S(0); }
template <> __device__ __forceinline__ Dual<float> szero<Dual<float>>() { return {0.f, 0.f}; }
template <> __device__ __forceinline__ Dual<double> szero<Dual<double>>() { return {0.0, 0.0}; }

// (u_L, u_R) of a face point from its own and its partner's state (own is L
// when `left`), selected value by value so that a warp whose points have both
// orientations evaluates the common flux once instead of on two divergent
// paths.  Both sides of a face still pass the same operands in the same order.
template <int V, typename S>
__device__ __forceinline__ void orient(bool left, const S* own, const S* nbr, S* uL, S* uR) {
    #pragma unroll
    for (int v = 0; v < V; ++v) {
        uL[v] = left ? own[v] : nbr[v];
        uR[v] = left ? nbr[v] : own[v];
    }
}

// ---------------------------------------------------------------------------
// Euler: primitive velocity and pressure of u = (rho, rho v, rho E).
template <typename S, typename T, int ND>
__device__ __forceinline__ void euler_prim(const S* u, S* v, S& p, T gamma) {
    S inv = T(1) / u[0];
    S ke = szero<S>();
    #pragma unroll
    for (int d = 0; d < ND; ++d) {
        v[d] = u[1 + d] * inv;
        ke = ke + u[1 + d] * v[d];
    }
    p = (gamma - T(1)) * (u[ND + 1] - T(0.5) * ke);
}

// n . f(u) for an arbitrary (not necessarily unit) vector n.
template <typename S, typename NV, int ND>
__device__ __forceinline__ void euler_nflux(const S* u, const S* v, S p, const NV* n, S* fn) {
    S vn = v[0] * n[0];
    #pragma unroll
    for (int d = 1; d < ND; ++d) vn = vn + v[d] * n[d];
    fn[0] = u[0] * vn;
    #pragma unroll
    for (int i = 0; i < ND; ++i) fn[1 + i] = u[1 + i] * vn + p * n[i];
    fn[ND + 1] = (u[ND + 1] + p) * vn;
}

// Rusanov common flux along the unit normal n: n.(fL+fR)/2 + phi/2 (uL - uR),
// phi = max(|vL.n| + cL, |vR.n| + cR).
template <typename S, typename T, int ND>
__device__ __forceinline__ void rusanov(const S* uL, const S* uR, const T* n, T gamma, S* F) {
    constexpr int V = ND + 2;
    S vL[ND], vR[ND], pL, pR, fL[V], fR[V];
    euler_prim<S, T, ND>(uL, vL, pL, gamma);
    euler_prim<S, T, ND>(uR, vR, pR, gamma);
    euler_nflux<S, T, ND>(uL, vL, pL, n, fL);
    euler_nflux<S, T, ND>(uR, vR, pR, n, fR);
    S vnL = vL[0] * n[0], vnR = vR[0] * n[0];
    #pragma unroll
    for (int d = 1; d < ND; ++d) {
        vnL = vnL + vL[d] * n[d];
        vnR = vnR + vR[d] * n[d];
    }
    S cL = ssqrt(gamma * pL / uL[0]);
    S cR = ssqrt(gamma * pR / uR[0]);
    S phi = smax(sabs(vnL) + cL, sabs(vnR) + cR);
    #pragma unroll
    for (int k = 0; k < V; ++k) F[k] = T(0.5) * (fL[k] + fR[k]) + T(0.5) * phi * (uL[k] - uR[k]);
}

// Roe common flux with a Harten entropy fix (delta = 0.1 c~) on the acoustic waves.
template <typename S, typename T, int ND>
__device__ __forceinline__ void roe(const S* uL, const S* uR, const T* n, T gamma, S* F) {
    constexpr int V = ND + 2;
    S vL[ND], vR[ND], pL, pR, fL[V], fR[V];
    euler_prim<S, T, ND>(uL, vL, pL, gamma);
    euler_prim<S, T, ND>(uR, vR, pR, gamma);
    euler_nflux<S, T, ND>(uL, vL, pL, n, fL);
    euler_nflux<S, T, ND>(uR, vR, pR, n, fR);
    S HL = (uL[ND + 1] + pL) / uL[0];
    S HR = (uR[ND + 1] + pR) / uR[0];
    S sL = ssqrt(uL[0]), sR = ssqrt(uR[0]);
    S w = sL + sR;
    S vt[ND];
    S q2 = szero<S>(), vnt = szero<S>(), dvn = szero<S>();
    S dv[ND];
    #pragma unroll
    for (int d = 0; d < ND; ++d) {
        vt[d] = (sL * vL[d] + sR * vR[d]) / w;
        q2 = q2 + vt[d] * vt[d];
        vnt = vnt + vt[d] * n[d];
        dv[d] = vR[d] - vL[d];
        dvn = dvn + dv[d] * n[d];
    }
    S Ht = (sL * HL + sR * HR) / w;
    S rt = sL * sR;
    S ct = ssqrt((gamma - T(1)) * (Ht - T(0.5) * q2));
    S dr = uR[0] - uL[0];
    S dp = pR - pL;
    S delta = T(0.1) * ct;
    auto fix = [&](S lam) {
        S a = sabs(lam);
        return pval(a) < pval(delta) ? (a * a + delta * delta) / (T(2) * delta) : a;
    };
    S l1 = fix(vnt - ct), l2 = sabs(vnt), l5 = fix(vnt + ct);
    S c2 = ct * ct;
    S a1 = (dp - rt * ct * dvn) / (T(2) * c2);
    S a5 = (dp + rt * ct * dvn) / (T(2) * c2);
    S a2 = dr - dp / c2;
    S w1 = l1 * a1, w5 = l5 * a5, w2 = l2 * a2, ws = l2 * rt;
    S vtdvt = szero<S>();
    S dvt[ND];
    #pragma unroll
    for (int d = 0; d < ND; ++d) {
        dvt[d] = dv[d] - dvn * n[d];
        vtdvt = vtdvt + vt[d] * dvt[d];
    }
    S diss[V];
    diss[0] = w1 + w5 + w2;
    #pragma unroll
    for (int d = 0; d < ND; ++d)
        diss[1 + d] = w1 * (vt[d] - ct * n[d]) + w5 * (vt[d] + ct * n[d]) + w2 * vt[d] + ws * dvt[d];
    diss[ND + 1] = w1 * (Ht - ct * vnt) + w5 * (Ht + ct * vnt) + w2 * (T(0.5) * q2) + ws * vtdvt;
    #pragma unroll
    for (int k = 0; k < V; ++k) F[k] = T(0.5) * (fL[k] + fR[k]) - T(0.5) * diss[k];
}

// ---------------------------------------------------------------------------
// Viscous fluxes (paper Eq. "fluxOperatorNavierStokes"; mu dynamic,
// mu c_p / Pr grad T = mu gamma / Pr grad e with e = E/rho - |v|^2/2).
// q[d][v]: physical gradient of conserved variable v along x_d.
// fv[d][v]: viscous part of the flux along x_d (zero for the density).
template <typename S, typename T, int ND>
__device__ __forceinline__ void ns_viscous(const S* u, const S (*q)[ND + 2], T mu, T gamma, T prandtl,
                                           S (*fv)[ND + 2]) {
    const S inv = T(1) / u[0];
    S v[ND];
    #pragma unroll
    for (int i = 0; i < ND; ++i) v[i] = u[1 + i] * inv;
    S gv[ND][ND];                 // gv[d][i] = d v_i / d x_d
    #pragma unroll
    for (int d = 0; d < ND; ++d)
        #pragma unroll
        for (int i = 0; i < ND; ++i) gv[d][i] = (q[d][1 + i] - q[d][0] * v[i]) * inv;
    S div = gv[0][0];
    #pragma unroll
    for (int i = 1; i < ND; ++i) div = div + gv[i][i];
    S tau[ND][ND];
    #pragma unroll
    for (int i = 0; i < ND; ++i)
        #pragma unroll
        for (int j = 0; j < ND; ++j) tau[i][j] = mu * (gv[j][i] + gv[i][j]);
    #pragma unroll
    for (int i = 0; i < ND; ++i) tau[i][i] = tau[i][i] - T(2.0 / 3.0) * mu * div;
    const S Eo = u[ND + 1] * inv;
    const T kap = mu * gamma / prandtl;
    #pragma unroll
    for (int d = 0; d < ND; ++d) {
        S ge = (q[d][ND + 1] - Eo * q[d][0]) * inv;
        #pragma unroll
        for (int i = 0; i < ND; ++i) ge = ge - v[i] * gv[d][i];
        fv[d][0] = szero<S>();
        S w = szero<S>();
        #pragma unroll
        for (int i = 0; i < ND; ++i) {
            fv[d][1 + i] = -tau[i][d];
            w = w + tau[d][i] * v[i];
        }
        fv[d][ND + 1] = -w - kap * ge;
    }
}

}  // namespace sdrt
