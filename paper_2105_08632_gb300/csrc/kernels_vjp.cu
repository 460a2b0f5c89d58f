// Vector-Jacobian product W^T (dR/dU) of the inviscid residual (generic path).
//
// With R = -(1/det J) ([M14 | M13] [F~_fe; F~_fi]) per element (paper App. B,
// Eq. "residual_sdrt_matrices"), the adjoint of the divergence is
//   G_j   = -(1/det J) (M14^T W)_j      at the external points,
//   Fb_nu = -(1/det J) (M13^T W)_nu     at the internal DOFs.
// Both sides of a face pair (j, p) evaluate the same common flux
// F(u_L, u_R, n_L), scaled by s_j and s_p, so the adjoint reaching the state
// of either side through that pair is H = s_j G_j + s_p G_p, and
//   ub_fe,j  = (dF / du_own)^T H,
//   ub_fiu,k = sum over the DOFs nu of point k of (d(S_axis . f) / du)^T Fb_nu,
//   W^T J    = M0^T ub_fe + M12^T ub_fiu.
// Two launches (each over every block) after the forward interpolation k_interp_ext:
//   k_vjp_face : GS_j = s_j G_j for every external point (UFE layout);
//   k_vjp_elem : the flux Jacobians (V forward-mode dual evaluations per point,
//                one per input variable, so the branch taken at ties of |.| and
//                max is the JVP's) and the transposed interpolation.
#include <cstdint>

#include "generic.cuh"
#include "launch.hpp"

namespace sdrt {

// GS = s * (-(1/det J) M14^T W) at the external points of a tile.
template <typename T, int V, int ND>
__global__ void __launch_bounds__(256) k_vjp_face(KTable<T> tab, const T* __restrict__ W, T* __restrict__ GS,
                                                  int64_t Ftot) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* RW = reinterpret_cast<T*>(smem_raw);
    constexpr int ND2 = ND * ND;
    for (int gt = blockIdx.x;; gt += gridDim.x) {
        int bi, tile;
        if (!locate(tab, TK_VJP, gt, bi, tile)) break;
        const KBlock<T>& B = tab.blocks[bi];
        const int TE = B.te_vjp;
        const int NCOL = V * TE;
        const int e0 = tile * TE;
        __syncthreads();
        load_tile<T, T, V>(B, W, nullptr, e0, TE, RW);
        __syncthreads();
        tile_gemm<T, T>(B.Adt, B.Mdt_pad, B.nfe, B.nsol, RW, B.nsol, RW, NCOL,
                        [&](int m0, int col, const T* acc) {
                            const int v = col / TE, te = col - v * TE, e = e0 + te;
                            if (e >= B.nelem) return;
                            const T inv = __ldg(B.metric + e);
                            #pragma unroll
                            for (int i = 0; i < kMR; ++i) {
                                const int m = m0 + i;
                                if (m >= B.nfe) break;
                                const int f = __ldg(B.fe_face + m);
                                const T s = __ldg(B.metric + (size_t)(1 + ND2 + f * (ND + 1) + ND) * B.ld + e);
                                GS[(size_t)v * Ftot + B.fe_base + (size_t)m * B.ld + e] = -(inv * s) * acc[i];
                            }
                        });
    }
}

// Shared memory (columns (v, te)): RA = U, then W (nsol rows); RB = u_fiu,
// then ub_fiu (nfiu rows); RC = Fb (nfi rows); RD = ub_fe (nfe rows).
template <typename T, int V, int ND, int SYS, int RIE>
__global__ void __launch_bounds__(256) k_vjp_elem(KTable<T> tab, const T* __restrict__ U, const T* __restrict__ W,
                                                  const T* __restrict__ UFE, const T* __restrict__ GS, int64_t Ftot,
                                                  KPhys<T> P, T* __restrict__ out, int* flag) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using D = Dual<T>;
    constexpr int ND2 = ND * ND;
    for (int gt = blockIdx.x;; gt += gridDim.x) {
        int bi, tile;
        if (!locate(tab, TK_VJP, gt, bi, tile)) break;
        const KBlock<T>& B = tab.blocks[bi];
        const int TE = B.te_vjp;
        const int NCOL = V * TE;
        T* RA = reinterpret_cast<T*>(smem_raw);
        T* RB = RA + (size_t)B.nsol * NCOL;
        T* RC = RB + (size_t)B.nfiu * NCOL;
        T* RD = RC + (size_t)B.nfi * NCOL;
        const int nfe_pad = (B.nfe + kMR - 1) / kMR * kMR;
        const int e0 = tile * TE;
        __syncthreads();
        load_tile<T, T, V>(B, U, nullptr, e0, TE, RA);
        __syncthreads();
        // u_fiu = M12 U (rows nfe .. Mi - 1 of the transposed interpolation operator).
        tile_gemm<T, T>(B.Ai + B.nfe, B.Mi_pad, B.nfiu, B.nsol, RA, B.nsol, RA, NCOL,
                        [&](int m0, int col, const T* acc) {
                            #pragma unroll
                            for (int i = 0; i < kMR; ++i)
                                if (m0 + i < B.nfiu) RB[(size_t)(m0 + i) * NCOL + col] = acc[i];
                        });
        __syncthreads();
        load_tile<T, T, V>(B, W, nullptr, e0, TE, RA);
        __syncthreads();
        // Fb = -(1/det J) M13^T W
        tile_gemm<T, T>(B.Adt + nfe_pad, B.Mdt_pad, B.nfi, B.nsol, RA, B.nsol, RA, NCOL,
                        [&](int m0, int col, const T* acc) {
                            const int te = col % TE;
                            const int e = min(e0 + te, B.nelem - 1);
                            const T inv = __ldg(B.metric + e);
                            #pragma unroll
                            for (int i = 0; i < kMR; ++i)
                                if (m0 + i < B.nfi) RC[(size_t)(m0 + i) * NCOL + col] = -inv * acc[i];
                        });
        // External points: ub_fe = (dF / du_own)^T (GS_own + GS_partner).
        for (int it = threadIdx.x; it < B.nfe * TE; it += blockDim.x) {
            const int sg = it / TE;
            const int te = it - sg * TE;
            const int e = min(e0 + te, B.nelem - 1);
            const int f = __ldg(B.fe_face + sg);
            const int mrow = 1 + ND2 + f * (ND + 1);
            T n[ND];
            #pragma unroll
            for (int c = 0; c < ND; ++c) n[c] = __ldg(B.metric + (size_t)(mrow + c) * B.ld + e);
            const bool left = __ldg(B.metric + (size_t)(mrow + ND) * B.ld + e) > T(0);
            const size_t oi = (size_t)B.fe_base + (size_t)sg * B.ld + e;
            const size_t pi = (size_t)__ldg(B.map + (size_t)sg * B.ld + e);
            T own[V], nbr[V], H[V];
            #pragma unroll
            for (int v = 0; v < V; ++v) {
                own[v] = UFE[(size_t)v * Ftot + oi];
                nbr[v] = UFE[(size_t)v * Ftot + pi];
                H[v] = GS[(size_t)v * Ftot + oi] + GS[(size_t)v * Ftot + pi];
            }
            #pragma unroll 1
            for (int c = 0; c < V; ++c) {
                D uo[V], un[V], F[V];
                #pragma unroll
                for (int v = 0; v < V; ++v) {
                    uo[v] = {own[v], v == c ? T(1) : T(0)};
                    un[v] = {nbr[v], T(0)};
                }
                D uL[V], uR[V];
                orient<V>(left, uo, un, uL, uR);
                common_flux<SYS, RIE, ND>(uL, uR, n, P, F);
                T a = T(0);
                #pragma unroll
                for (int v = 0; v < V; ++v) a = fma(F[v].d, H[v], a);
                RD[(size_t)sg * NCOL + c * TE + te] = a;
            }
        }
        __syncthreads();
        // Internal points: ub_fiu = sum over the point's DOFs of (d(S_axis . f)/du)^T Fb.
        for (int it = threadIdx.x; it < B.nfiu * TE; it += blockDim.x) {
            const int k = it / TE;
            const int te = it - k * TE;
            const int e = min(e0 + te, B.nelem - 1);
            T u[V];
            #pragma unroll
            for (int v = 0; v < V; ++v) u[v] = RB[(size_t)k * NCOL + v * TE + te];
            const int4 tab = __ldg(reinterpret_cast<const int4*>(B.fi_tab) + k);
            const int dofs[3] = {tab.y, tab.z, tab.w};
            T ub[V];
            #pragma unroll
            for (int c = 0; c < V; ++c) ub[c] = T(0);
            for (int q = 0; q < tab.x; ++q) {
                const int nu = dofs[q] & 0xffff;
                const int ax = dofs[q] >> 16;
                T Srow[ND], Fb[V];
                #pragma unroll
                for (int i = 0; i < ND; ++i) Srow[i] = __ldg(B.metric + (size_t)(1 + ax * ND + i) * B.ld + e);
                #pragma unroll
                for (int v = 0; v < V; ++v) Fb[v] = RC[(size_t)nu * NCOL + v * TE + te];
                #pragma unroll
                for (int c = 0; c < V; ++c) {
                    D ud[V], Ft[V];
                    #pragma unroll
                    for (int v = 0; v < V; ++v) ud[v] = {u[v], v == c ? T(1) : T(0)};
                    internal_flux<SYS, ND>(ud, Srow, P, Ft);
                    T a = ub[c];
                    #pragma unroll
                    for (int v = 0; v < V; ++v) a = fma(Ft[v].d, Fb[v], a);
                    ub[c] = a;
                }
            }
            #pragma unroll
            for (int v = 0; v < V; ++v) RB[(size_t)k * NCOL + v * TE + te] = ub[v];
        }
        __syncthreads();
        // W^T J = [M0; M12]^T [ub_fe; ub_fiu]  (row-major [M0; M12] is the transposed operator).
        tile_gemm<T, T>(B.Air, B.Md_pad, B.nsol, B.Mi, RD, B.nfe, RB, NCOL,
                        [&](int m0, int col, const T* acc) {
                            const int v = col / TE, te = col - v * TE, e = e0 + te;
                            if (e >= B.nelem) return;
                            bool bad = false;
                            #pragma unroll
                            for (int i = 0; i < kMR; ++i) {
                                const int m = m0 + i;
                                if (m >= B.nsol) break;
                                bad |= !isfinite(acc[i]);
                                out[(size_t)B.u_off + ((size_t)m * V + v) * B.ld + e] = acc[i];
                            }
                            if (bad) *flag = 1;
                        });
    }
}

// ---------------------------------------------------------------------------
// Host launchers.

template <typename T>
int vjp_smem(const KBlock<T>& B, int V, int TE) {
    return (B.nsol + B.nfiu + B.nfi + B.nfe) * V * TE * (int)sizeof(T);
}

template <typename T, int V, int ND, int SYS, int RIE>
static void launch_vjp_pass(const KSet<T>& ks, int pass, const T* U, const T* W, const T* UFE, T* GS, int64_t Ftot,
                            const KPhys<T>& P, T* out, int* flag, int nsm, cudaStream_t st) {
    const int tiles = ks.tiles(TK_VJP);
    const int grid = tiles < 2 * nsm ? tiles : 2 * nsm;
    const KTable<T> tab = ks.table();
    int smem = 0;
    for (int i = 0; i < ks.n; ++i) {
        const int b = pass == 0 ? ks.host[i].nsol * V * ks.host[i].te_vjp * (int)sizeof(T)
                                : vjp_smem(ks.host[i], V, ks.host[i].te_vjp);
        smem = b > smem ? b : smem;
    }
    if (pass == 0) {
        auto kf = k_vjp_face<T, V, ND>;
        cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        kf<<<grid, 256, smem, st>>>(tab, W, GS, Ftot);
    } else {
        auto ke = k_vjp_elem<T, V, ND, SYS, RIE>;
        cudaFuncSetAttribute(ke, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        ke<<<grid, 256, smem, st>>>(tab, U, W, UFE, GS, Ftot, P, out, flag);
    }
}

template <typename T>
int launch_vjp(const KSet<T>& ks, int pass, int system, int riemann, int nd, const T* U, const T* W, const T* UFE,
               T* GS, int64_t Ftot, const KPhys<T>& P, T* out, int* flag, int nsm, cudaStream_t st) {
    if (!ks.all_tiled(TK_VJP)) return -2;
#define SDRT_VJP(VV, NDD, SYSS, RIEE) \
    launch_vjp_pass<T, VV, NDD, SYSS, RIEE>(ks, pass, U, W, UFE, GS, Ftot, P, out, flag, nsm, st)
    if (system == SYS_ADVECTION) {
        if (nd == 2) SDRT_VJP(1, 2, SYS_ADVECTION, RIE_UPWIND);
        else SDRT_VJP(1, 3, SYS_ADVECTION, RIE_UPWIND);
        return 0;
    }
    if (system == SYS_EULER) {
        if (nd == 2) {
            if (riemann == RIE_ROE) SDRT_VJP(4, 2, SYS_EULER, RIE_ROE);
            else SDRT_VJP(4, 2, SYS_EULER, RIE_RUSANOV);
        } else {
            if (riemann == RIE_ROE) SDRT_VJP(5, 3, SYS_EULER, RIE_ROE);
            else SDRT_VJP(5, 3, SYS_EULER, RIE_RUSANOV);
        }
        return 0;
    }
#undef SDRT_VJP
    return -1;
}

template int vjp_smem<float>(const KBlock<float>&, int, int);
template int vjp_smem<double>(const KBlock<double>&, int, int);
template int launch_vjp<float>(const KSet<float>&, int, int, int, int, const float*, const float*, const float*,
                               float*, int64_t, const KPhys<float>&, float*, int*, int, cudaStream_t);
template int launch_vjp<double>(const KSet<double>&, int, int, int, int, const double*, const double*,
                                const double*, double*, int64_t, const KPhys<double>&, double*, int*, int,
                                cudaStream_t);

}  // namespace sdrt
