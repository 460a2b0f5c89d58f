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
//
// Viscous systems (LDG, Sec. 2.1) add the gradient chain: the fluxes also
// depend on the physical gradients q at the flux points, q = [M0; M12] J^{-T}
// q~, q~ = [M16 | M15 P M12] [C; U], with the common value C = (1/2 - beta)
// u_L + (1/2 + beta) u_R shared by the two sides of a face.  After the
// forward interpolation and gradient kernels (UFE, QFE, QFIU) and k_vjp_face:
//   k_vjp_elem_visc : ub_fe, qb_fe = (dF / d(u, q)_own)^T H at the external
//                     points and ub_fiu, qb_fiu at the internal points (dual
//                     evaluations of the total flux, convective + viscous,
//                     per own input), qb = [M0; M12]^T qb_fe|fiu at the
//                     solution points, qb~_d = sum_i (J^{-1})_{di} qb_i,
//                     [Cb; Ub_g] = [M16 | M15 P M12]^T qb~; writes Cb (face
//                     buffer CB) and W^T J without the C term:
//                     [M0; M12]^T [ub_fe; ub_fiu] + Ub_g;
//   k_vjp_cbar      : adds the C term, M0^T (w_own (Cb_own + Cb_partner)),
//                     w_own = dC / du_own.
#include <cstdint>

#include "generic.cuh"
#include "launch.hpp"

namespace sdrt {

// R[s][col] *= 1/det J at solution point s of the column's element: the W
// tile scaled by the semi-discrete form's factor (one per element on affine
// blocks, one per point on curved ones).
template <typename T>
__device__ __forceinline__ void scale_inv_det(const KBlock<T>& B, T* R, int e0, int TE, int NCOL) {
    for (int it = threadIdx.x; it < B.nsol * NCOL; it += blockDim.x) {
        const int sp = it / NCOL;
        const int e = min(e0 + (it - sp * NCOL) % TE, B.nelem - 1);
        R[it] *= __ldg(B.metric + (size_t)sp * B.mr_inv * B.ld + e);
    }
}

// GS = s * (-M14^T (W / det J)) at the external points of a tile.
template <typename T, int V, int ND>
__global__ void __launch_bounds__(256) k_vjp_face(KTable<T> tab, const T* __restrict__ W, T* __restrict__ GS,
                                                  int64_t Ftot) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* RW = reinterpret_cast<T*>(smem_raw);
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
        scale_inv_det(B, RW, e0, TE, NCOL);
        __syncthreads();
        tile_gemm<T, T>(B.Adt, B.Mdt_pad, B.nfe, B.nsol, RW, B.nsol, RW, NCOL,
                        [&](int m0, int col, const T* acc) {
                            const int v = col / TE, te = col - v * TE, e = e0 + te;
                            if (e >= B.nelem) return;
                            #pragma unroll
                            for (int i = 0; i < kMR; ++i) {
                                const int m = m0 + i;
                                if (m >= B.nfe) break;
                                const int f = __ldg(B.fe_face + m);
                                const T s = __ldg(B.metric + (size_t)(B.mr_f + f * B.mr_ff + m * B.mr_fp + ND) * B.ld + e);
                                GS[(size_t)v * Ftot + B.fe_base + (size_t)m * B.ld + e] = -s * acc[i];
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
        scale_inv_det(B, RA, e0, TE, NCOL);
        __syncthreads();
        // Fb = -M13^T (W / det J)
        tile_gemm<T, T>(B.Adt + nfe_pad, B.Mdt_pad, B.nfi, B.nsol, RA, B.nsol, RA, NCOL,
                        [&](int m0, int col, const T* acc) {
                            #pragma unroll
                            for (int i = 0; i < kMR; ++i)
                                if (m0 + i < B.nfi) RC[(size_t)(m0 + i) * NCOL + col] = -acc[i];
                        });
        // External points: ub_fe = (dF / du_own)^T (GS_own + GS_partner).
        for (int it = threadIdx.x; it < B.nfe * TE; it += blockDim.x) {
            const int sg = it / TE;
            const int te = it - sg * TE;
            const int e = min(e0 + te, B.nelem - 1);
            const int f = __ldg(B.fe_face + sg);
            const int mrow = B.mr_f + f * B.mr_ff + sg * B.mr_fp;
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
                for (int i = 0; i < ND; ++i)
                    Srow[i] = __ldg(B.metric + (size_t)(B.mr_si + k * B.mr_sik + ax * ND + i) * B.ld + e);
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
                            if (bad) atomicOr(flag, 1);
                        });
    }
}

// Total common flux along n_L of a face point (convective + LDG viscous),
// the same operations in the same order as the residual kernel's.
template <int SYS, int RIE, int ND, int V, typename S, typename T>
__device__ __forceinline__ void face_flux_total(const S* own, const S (*qo)[V], const S* nbr, const S (*qn)[V],
                                                const T* n, bool left, const KPhys<T>& P, S* F) {
    S uL[V], uR[V];
    orient<V>(left, own, nbr, uL, uR);
    common_flux<SYS, RIE, ND>(uL, uR, n, P, F);
    S fv[ND][V], g[V];
    viscous_flux<SYS, ND, V, S, T>(own, qo, P, fv);
    viscous_normal<ND, V, S, T>(fv, n, g);
    const T wo = left ? T(0.5) + P.beta : T(0.5) - P.beta;
    #pragma unroll
    for (int v = 0; v < V; ++v) F[v] = F[v] + wo * g[v];
    viscous_flux<SYS, ND, V, S, T>(nbr, qn, P, fv);
    viscous_normal<ND, V, S, T>(fv, n, g);
    const T wn = T(1) - wo;
    const T eo = left ? P.eta : -P.eta;
    #pragma unroll
    for (int v = 0; v < V; ++v) F[v] = F[v] + wn * g[v] + eo * (own[v] - nbr[v]);
}

// Shared memory (columns (v, te) or (d, v, te)): RA = U, then W, then Ub_g
// (nsol rows); RB = u_fiu, then ub_fiu (nfiu rows); RC = Fb (nfi rows);
// RD = ub_fe (nfe rows); QE = qb_fe (nfe rows), QI = qb_fiu (nfiu rows),
// QS = qb, then qb~ (nsol rows), each of ND V TE columns.
template <typename T, int V, int ND, int SYS, int RIE>
__global__ void __launch_bounds__(256) k_vjp_elem_visc(KTable<T> tab, const T* __restrict__ U,
                                                       const T* __restrict__ W, const T* __restrict__ UFE,
                                                       const T* __restrict__ QFE, const T* __restrict__ QFIU,
                                                       const T* __restrict__ GS, int64_t Ftot, KPhys<T> P,
                                                       T* __restrict__ CB, T* __restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using D = Dual<T>;
    for (int gt = blockIdx.x;; gt += gridDim.x) {
        int bi, tile;
        if (!locate(tab, TK_VJP, gt, bi, tile)) break;
        const KBlock<T>& B = tab.blocks[bi];
        const int TE = B.te_vjp;
        const int NCOL = V * TE;
        const int QCOL = ND * NCOL;
        T* RA = reinterpret_cast<T*>(smem_raw);
        T* RB = RA + (size_t)B.nsol * NCOL;
        T* RC = RB + (size_t)B.nfiu * NCOL;
        T* RD = RC + (size_t)B.nfi * NCOL;
        T* QE = RD + (size_t)B.nfe * NCOL;
        T* QI = QE + (size_t)B.nfe * QCOL;
        T* QS = QI + (size_t)B.nfiu * QCOL;
        const int nfe_pad = (B.nfe + kMR - 1) / kMR * kMR;
        const int e0 = tile * TE;
        __syncthreads();
        load_tile<T, T, V>(B, U, nullptr, e0, TE, RA);
        __syncthreads();
        // u_fiu = M12 U
        tile_gemm<T, T>(B.Ai + B.nfe, B.Mi_pad, B.nfiu, B.nsol, RA, B.nsol, RA, NCOL,
                        [&](int m0, int col, const T* acc) {
                            #pragma unroll
                            for (int i = 0; i < kMR; ++i)
                                if (m0 + i < B.nfiu) RB[(size_t)(m0 + i) * NCOL + col] = acc[i];
                        });
        __syncthreads();
        load_tile<T, T, V>(B, W, nullptr, e0, TE, RA);
        __syncthreads();
        scale_inv_det(B, RA, e0, TE, NCOL);
        __syncthreads();
        // Fb = -M13^T (W / det J)
        tile_gemm<T, T>(B.Adt + nfe_pad, B.Mdt_pad, B.nfi, B.nsol, RA, B.nsol, RA, NCOL,
                        [&](int m0, int col, const T* acc) {
                            #pragma unroll
                            for (int i = 0; i < kMR; ++i)
                                if (m0 + i < B.nfi) RC[(size_t)(m0 + i) * NCOL + col] = -acc[i];
                        });
        // External points: (ub_fe, qb_fe) = (dF / d(u, q)_own)^T (GS_own + GS_partner).
        for (int it = threadIdx.x; it < B.nfe * TE; it += blockDim.x) {
            const int sg = it / TE;
            const int te = it - sg * TE;
            const int e = min(e0 + te, B.nelem - 1);
            const int f = __ldg(B.fe_face + sg);
            const int mrow = B.mr_f + f * B.mr_ff + sg * B.mr_fp;
            T n[ND];
            #pragma unroll
            for (int c = 0; c < ND; ++c) n[c] = __ldg(B.metric + (size_t)(mrow + c) * B.ld + e);
            const bool left = __ldg(B.metric + (size_t)(mrow + ND) * B.ld + e) > T(0);
            const size_t oi = (size_t)B.fe_base + (size_t)sg * B.ld + e;
            const size_t pi = (size_t)__ldg(B.map + (size_t)sg * B.ld + e);
            T own[V], nbr[V], H[V], qo[ND][V], qn[ND][V];
            #pragma unroll
            for (int v = 0; v < V; ++v) {
                own[v] = UFE[(size_t)v * Ftot + oi];
                nbr[v] = UFE[(size_t)v * Ftot + pi];
                H[v] = GS[(size_t)v * Ftot + oi] + GS[(size_t)v * Ftot + pi];
                #pragma unroll
                for (int d = 0; d < ND; ++d) {
                    qo[d][v] = QFE[(size_t)(d * V + v) * Ftot + oi];
                    qn[d][v] = QFE[(size_t)(d * V + v) * Ftot + pi];
                }
            }
            // seed c < V: own state variable c; seed V + d V + w: own gradient (d, w)
            #pragma unroll 1
            for (int c = 0; c < V + ND * V; ++c) {
                D uo[V], un[V], go[ND][V], gn[ND][V], F[V];
                #pragma unroll
                for (int v = 0; v < V; ++v) {
                    uo[v] = {own[v], v == c ? T(1) : T(0)};
                    un[v] = {nbr[v], T(0)};
                    #pragma unroll
                    for (int d = 0; d < ND; ++d) {
                        go[d][v] = {qo[d][v], V + d * V + v == c ? T(1) : T(0)};
                        gn[d][v] = {qn[d][v], T(0)};
                    }
                }
                face_flux_total<SYS, RIE, ND, V>(uo, go, un, gn, n, left, P, F);
                T a = T(0);
                #pragma unroll
                for (int v = 0; v < V; ++v) a = fma(F[v].d, H[v], a);
                if (c < V) RD[(size_t)sg * NCOL + c * TE + te] = a;
                else QE[(size_t)sg * QCOL + (c - V) * TE + te] = a;     // column (d, w, te), d V + w = c - V
            }
        }
        __syncthreads();
        // Internal points: (ub_fiu, qb_fiu) = sum over the point's DOFs of
        // (d(S_axis . (f + f_v)) / d(u, q))^T Fb.
        for (int it = threadIdx.x; it < B.nfiu * TE; it += blockDim.x) {
            const int k = it / TE;
            const int te = it - k * TE;
            const int e = min(e0 + te, B.nelem - 1);
            T u[V], q[ND][V];
            #pragma unroll
            for (int v = 0; v < V; ++v) {
                u[v] = RB[(size_t)k * NCOL + v * TE + te];
                #pragma unroll
                for (int d = 0; d < ND; ++d)
                    q[d][v] = QFIU[(size_t)B.qfiu_off + ((size_t)k * (ND * V) + d * V + v) * B.ld + e];
            }
            const int4 ftab = __ldg(reinterpret_cast<const int4*>(B.fi_tab) + k);
            const int dofs[3] = {ftab.y, ftab.z, ftab.w};
            T ub[V + ND * V];
            #pragma unroll
            for (int c = 0; c < V + ND * V; ++c) ub[c] = T(0);
            for (int j = 0; j < ftab.x; ++j) {
                const int nu = dofs[j] & 0xffff;
                const int ax = dofs[j] >> 16;
                T Srow[ND], Fb[V];
                #pragma unroll
                for (int i = 0; i < ND; ++i)
                    Srow[i] = __ldg(B.metric + (size_t)(B.mr_si + k * B.mr_sik + ax * ND + i) * B.ld + e);
                #pragma unroll
                for (int v = 0; v < V; ++v) Fb[v] = RC[(size_t)nu * NCOL + v * TE + te];
                #pragma unroll 1
                for (int c = 0; c < V + ND * V; ++c) {
                    D ud[V], qd[ND][V], Ft[V], fv[ND][V], g[V];
                    #pragma unroll
                    for (int v = 0; v < V; ++v) {
                        ud[v] = {u[v], v == c ? T(1) : T(0)};
                        #pragma unroll
                        for (int d = 0; d < ND; ++d) qd[d][v] = {q[d][v], V + d * V + v == c ? T(1) : T(0)};
                    }
                    internal_flux<SYS, ND>(ud, Srow, P, Ft);
                    viscous_flux<SYS, ND, V, D, T>(ud, qd, P, fv);
                    viscous_normal<ND, V, D, T>(fv, Srow, g);
                    T a = ub[c];
                    #pragma unroll
                    for (int v = 0; v < V; ++v) a = fma((Ft[v] + g[v]).d, Fb[v], a);
                    ub[c] = a;
                }
            }
            #pragma unroll
            for (int v = 0; v < V; ++v) RB[(size_t)k * NCOL + v * TE + te] = ub[v];
            #pragma unroll
            for (int c = 0; c < ND * V; ++c) QI[(size_t)k * QCOL + c * TE + te] = ub[V + c];
        }
        __syncthreads();
        // qb = [M0; M12]^T [qb_fe; qb_fiu] at the solution points, columns (d, v, te).
        tile_gemm<T, T>(B.Air, B.Md_pad, B.nsol, B.Mi, QE, B.nfe, QI, QCOL,
                        [&](int m0, int col, const T* acc) {
                            #pragma unroll
                            for (int i = 0; i < kMR; ++i)
                                if (m0 + i < B.nsol) QS[(size_t)(m0 + i) * QCOL + col] = acc[i];
                        });
        __syncthreads();
        // qb~_d = sum_i (J^{-1})_{di} qb_i = (1/det J) sum_i S_di qb_i, in place.
        for (int it = threadIdx.x; it < B.nsol * NCOL; it += blockDim.x) {
            const int sp = it / NCOL;
            const int col = it - sp * NCOL;
            const int te = col % TE;
            const int e = min(e0 + te, B.nelem - 1);
            const T inv = __ldg(B.metric + (size_t)sp * B.mr_inv * B.ld + e);
            const T* Sp = B.metric + (size_t)(B.mr_ss + sp * B.mr_ssk) * B.ld + e;
            T qb[ND];
            #pragma unroll
            for (int i = 0; i < ND; ++i) qb[i] = QS[(size_t)sp * QCOL + i * NCOL + col];
            #pragma unroll
            for (int d = 0; d < ND; ++d) {
                T a = qb[0] * (__ldg(Sp + (size_t)(d * ND) * B.ld) * inv);
                #pragma unroll
                for (int i = 1; i < ND; ++i) a = a + qb[i] * (__ldg(Sp + (size_t)(d * ND + i) * B.ld) * inv);
                QS[(size_t)sp * QCOL + d * NCOL + col] = a;
            }
        }
        __syncthreads();
        // [Cb; Ub_g] = [M16 | M15 P M12]^T qb~  (rows (rho, d) of QS are its K index).
        tile_gemm<T, T>(B.Agr, B.Agr_pad, B.nfe + B.nsol, ND * B.nsol, QS, ND * B.nsol, QS, NCOL,
                        [&](int m0, int col, const T* acc) {
                            const int v = col / TE, te = col - v * TE, e = e0 + te;
                            #pragma unroll
                            for (int i = 0; i < kMR; ++i) {
                                const int m = m0 + i;
                                if (m >= B.nfe + B.nsol) break;
                                if (m < B.nfe) {
                                    if (e < B.nelem) CB[(size_t)v * Ftot + B.fe_base + (size_t)m * B.ld + e] = acc[i];
                                } else {
                                    RA[(size_t)(m - B.nfe) * NCOL + col] = acc[i];
                                }
                            }
                        });
        __syncthreads();
        // W^T J (without the C term) = [M0; M12]^T [ub_fe; ub_fiu] + Ub_g.
        tile_gemm<T, T>(B.Air, B.Md_pad, B.nsol, B.Mi, RD, B.nfe, RB, NCOL,
                        [&](int m0, int col, const T* acc) {
                            const int v = col / TE, te = col - v * TE, e = e0 + te;
                            if (e >= B.nelem) return;
                            #pragma unroll
                            for (int i = 0; i < kMR; ++i) {
                                const int m = m0 + i;
                                if (m >= B.nsol) break;
                                out[(size_t)B.u_off + ((size_t)m * V + v) * B.ld + e] =
                                    acc[i] + RA[(size_t)m * NCOL + col];
                            }
                        });
    }
}

// The common value's term: out += M0^T (w_own (Cb_own + Cb_partner)), w_own =
// dC / du_own = 1/2 - beta on the face's L side, 1/2 + beta on its R side.
template <typename T, int V, int ND>
__global__ void __launch_bounds__(256) k_vjp_cbar(KTable<T> tab, const T* __restrict__ CB, int64_t Ftot, KPhys<T> P,
                                                  T* __restrict__ out, int* flag) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* RD = reinterpret_cast<T*>(smem_raw);
    for (int gt = blockIdx.x;; gt += gridDim.x) {
        int bi, tile;
        if (!locate(tab, TK_VJP, gt, bi, tile)) break;
        const KBlock<T>& B = tab.blocks[bi];
        const int TE = B.te_vjp;
        const int NCOL = V * TE;
        const int e0 = tile * TE;
        __syncthreads();
        for (int it = threadIdx.x; it < B.nfe * TE; it += blockDim.x) {
            const int sg = it / TE;
            const int te = it - sg * TE;
            const int e = min(e0 + te, B.nelem - 1);
            const int f = __ldg(B.fe_face + sg);
            const bool left = __ldg(B.metric + (size_t)(B.mr_f + f * B.mr_ff + sg * B.mr_fp + ND) * B.ld + e) > T(0);
            const T wo = left ? T(0.5) - P.beta : T(0.5) + P.beta;
            const size_t oi = (size_t)B.fe_base + (size_t)sg * B.ld + e;
            const size_t pi = (size_t)__ldg(B.map + (size_t)sg * B.ld + e);
            #pragma unroll
            for (int v = 0; v < V; ++v)
                RD[(size_t)sg * NCOL + v * TE + te] = wo * (CB[(size_t)v * Ftot + oi] + CB[(size_t)v * Ftot + pi]);
        }
        __syncthreads();
        tile_gemm<T, T>(B.Air, B.Md_pad, B.nsol, B.nfe, RD, B.nfe, RD, NCOL,
                        [&](int m0, int col, const T* acc) {
                            const int v = col / TE, te = col - v * TE, e = e0 + te;
                            if (e >= B.nelem) return;
                            bool bad = false;
                            #pragma unroll
                            for (int i = 0; i < kMR; ++i) {
                                const int m = m0 + i;
                                if (m >= B.nsol) break;
                                T& o = out[(size_t)B.u_off + ((size_t)m * V + v) * B.ld + e];
                                o = o + acc[i];
                                bad |= !isfinite(o);
                            }
                            if (bad) atomicOr(flag, 1);
                        });
    }
}

// ---------------------------------------------------------------------------
// Host launchers.

template <typename T>
int vjp_smem(const KBlock<T>& B, int V, int TE) {
    return (B.nsol + B.nfiu + B.nfi + B.nfe) * V * TE * (int)sizeof(T);
}

template <typename T>
int vjp_visc_smem(const KBlock<T>& B, int V, int nd, int TE) {
    return (B.nsol + B.nfiu + B.nfi + B.nfe + nd * (B.nfe + B.nfiu + B.nsol)) * V * TE * (int)sizeof(T);
}

template <typename T, int V, int ND, int SYS, int RIE>
static void launch_vjp_visc_pass(const KSet<T>& ks, int pass, const T* U, const T* W, const T* UFE, const T* QFE,
                                 const T* QFIU, T* GS, T* CB, int64_t Ftot, const KPhys<T>& P, T* out, int* flag,
                                 int nsm, cudaStream_t st) {
    const int tiles = ks.tiles(TK_VJP);
    const int grid = tiles < 2 * nsm ? tiles : 2 * nsm;
    const KTable<T> tab = ks.table();
    int smem = 0;
    for (int i = 0; i < ks.n; ++i) {
        const KBlock<T>& B = ks.host[i];
        const int b = pass == 0 ? B.nsol * V * B.te_vjp * (int)sizeof(T)
                    : pass == 1 ? vjp_visc_smem(B, V, ND, B.te_vjp)
                                : B.nfe * V * B.te_vjp * (int)sizeof(T);
        smem = b > smem ? b : smem;
    }
    if (pass == 0) {
        auto kf = k_vjp_face<T, V, ND>;
        cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        kf<<<grid, 256, smem, st>>>(tab, W, GS, Ftot);
    } else if (pass == 1) {
        auto ke = k_vjp_elem_visc<T, V, ND, SYS, RIE>;
        cudaFuncSetAttribute(ke, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        ke<<<grid, 256, smem, st>>>(tab, U, W, UFE, QFE, QFIU, GS, Ftot, P, CB, out);
    } else {
        auto kc = k_vjp_cbar<T, V, ND>;
        cudaFuncSetAttribute(kc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        kc<<<grid, 256, smem, st>>>(tab, CB, Ftot, P, out, flag);
    }
}

template <typename T>
int launch_vjp_visc(const KSet<T>& ks, int pass, int system, int riemann, int nd, const T* U, const T* W,
                    const T* UFE, const T* QFE, const T* QFIU, T* GS, T* CB, int64_t Ftot, const KPhys<T>& P, T* out,
                    int* flag, int nsm, cudaStream_t st) {
    if (!ks.all_tiled(TK_VJP)) return -2;
#define SDRT_VJPV(VV, NDD, SYSS, RIEE) \
    launch_vjp_visc_pass<T, VV, NDD, SYSS, RIEE>(ks, pass, U, W, UFE, QFE, QFIU, GS, CB, Ftot, P, out, flag, nsm, st)
    if (system == SYS_ADVDIFF) {
        if (nd == 2) SDRT_VJPV(1, 2, SYS_ADVDIFF, RIE_UPWIND);
        else SDRT_VJPV(1, 3, SYS_ADVDIFF, RIE_UPWIND);
        return 0;
    }
    if (system == SYS_NS) {
        if (nd == 2) {
            if (riemann == RIE_ROE) SDRT_VJPV(4, 2, SYS_NS, RIE_ROE);
            else SDRT_VJPV(4, 2, SYS_NS, RIE_RUSANOV);
        } else {
            if (riemann == RIE_ROE) SDRT_VJPV(5, 3, SYS_NS, RIE_ROE);
            else SDRT_VJPV(5, 3, SYS_NS, RIE_RUSANOV);
        }
        return 0;
    }
#undef SDRT_VJPV
    return -1;
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
template int vjp_visc_smem<float>(const KBlock<float>&, int, int, int);
template int vjp_visc_smem<double>(const KBlock<double>&, int, int, int);
template int launch_vjp_visc<float>(const KSet<float>&, int, int, int, int, const float*, const float*, const float*,
                                    const float*, const float*, float*, float*, int64_t, const KPhys<float>&, float*,
                                    int*, int, cudaStream_t);
template int launch_vjp_visc<double>(const KSet<double>&, int, int, int, int, const double*, const double*,
                                     const double*, const double*, const double*, double*, double*, int64_t,
                                     const KPhys<double>&, double*, int*, int, cudaStream_t);
template int launch_vjp<float>(const KSet<float>&, int, int, int, int, const float*, const float*, const float*,
                               float*, int64_t, const KPhys<float>&, float*, int*, int, cudaStream_t);
template int launch_vjp<double>(const KSet<double>&, int, int, int, int, const double*, const double*,
                                const double*, double*, int64_t, const KPhys<double>&, double*, int*, int,
                                cudaStream_t);

}  // namespace sdrt
