// Viscous systems (advection-diffusion, Navier-Stokes) on the generic FMA path.
//
// The viscous flux needs the gradient of the solution at the flux points
// (paper Sec. 3 and App. B).  Per block and tile of TE elements, k_grad forms
//   C  = (1/2 - beta) u_L + (1/2 + beta) u_R     common value at the external
//                                                points (u_L, u_R: the face's sides)
//   q~ = M16 C + (M15 P M12) U                   transformed gradient at the
//                                                solution points, rows (axis d, point)
//   q  = J^{-T} q~, i.e. q_i = sum_d (J^{-1})_{di} q~_d
//   [q_fe; q_fiu] = [M0; M12] q                  written to QFE / QFIU
// after which k_residual (generic.cuh) adds the LDG viscous common flux at the
// external points and the viscous part of the transformed flux at the
// internal DOFs.  One evaluation is three launches, each walking the tiles of
// every block: k_interp_ext, k_grad (after the interpolation) and k_residual
// (after the gradients).
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "generic.cuh"
#include "launch.hpp"

namespace sdrt {

namespace {

template <typename T>
__device__ __forceinline__ void store_state(T* X, T*, size_t i, T v) { X[i] = v; }
template <typename T>
__device__ __forceinline__ void store_state(T* X, T* dX, size_t i, Dual<T> v) {
    X[i] = v.v;
    dX[i] = v.d;
}

}  // namespace

// Shared memory: RU = U tile (nsol rows), RC = C (nfe rows), both of V * TE
// columns (v, te); RQ = q (nsol rows of ND * V * TE columns (d, v, te)).
template <typename S, typename T, int V, int ND>
__global__ void __launch_bounds__(256) k_grad(KTable<T> tab, const T* __restrict__ U, const T* __restrict__ dU,
                                              const T* __restrict__ UFE, const T* __restrict__ dUFE, int64_t Ftot,
                                              KPhys<T> P, T* __restrict__ QFE, T* __restrict__ dQFE,
                                              T* __restrict__ QFIU, T* __restrict__ dQFIU, T* __restrict__ QSOL) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int kind = std::is_same<S, T>::value ? TK_GRAD : TK_GRAD_DUAL;
    for (int gt = blockIdx.x;; gt += gridDim.x) {
        int bi, tile;
        if (!locate(tab, kind, gt, bi, tile)) break;
        const KBlock<T>& B = tab.blocks[bi];
        const int TE = tile_width(B, kind);
        const int NCOL = V * TE;
        const int QCOL = ND * NCOL;
        S* RU = reinterpret_cast<S*>(smem_raw);
        S* RC = RU + (size_t)B.nsol * NCOL;
        S* RQ = RC + (size_t)B.nfe * NCOL;
        const int e0 = tile * TE;
        __syncthreads();
        load_tile<S, T, V>(B, U, dU, e0, TE, RU);
        // Common value at the external points.
        for (int it = threadIdx.x; it < B.nfe * TE; it += blockDim.x) {
            const int sg = it / TE;
            const int te = it - sg * TE;
            const int e = min(e0 + te, B.nelem - 1);
            const int f = __ldg(B.fe_face + sg);
            const T s = __ldg(B.metric + (size_t)(B.mr_f + f * B.mr_ff + sg * B.mr_fp + ND) * B.ld + e);
            const T wo = s > T(0) ? T(0.5) - P.beta : T(0.5) + P.beta;   // own side is L when s > 0
            const T wn = T(1) - wo;
            S own[V], nbr[V];
            gather_partner<S, T, V>(UFE, dUFE, Ftot, (int)(B.fe_base + (int64_t)sg * B.ld + e), own);
            gather_partner<S, T, V>(UFE, dUFE, Ftot, __ldg(B.map + (size_t)sg * B.ld + e), nbr);
            #pragma unroll
            for (int v = 0; v < V; ++v) RC[(size_t)sg * NCOL + v * TE + te] = wo * own[v] + wn * nbr[v];
        }
        __syncthreads();
        // q~ = [M16 | M15 P M12] [C; U]; row m = d * nsol + s goes to RQ row s, column block d.
        tile_gemm<S, T>(B.Ag, B.Mg_pad, ND * B.nsol, B.nfe + B.nsol, RC, B.nfe, RU, NCOL,
                        [&](int m0, int col, const S* acc) {
                            #pragma unroll
                            for (int i = 0; i < kMR; ++i) {
                                const int m = m0 + i;
                                if (m >= ND * B.nsol) break;
                                const int d = m / B.nsol, sp = m - d * B.nsol;
                                RQ[(size_t)sp * QCOL + d * NCOL + col] = acc[i];
                            }
                        });
        __syncthreads();
        // q = J^{-T} q~ at every solution point (metric rows S_di = det J (J^{-1})_di).
        for (int it = threadIdx.x; it < B.nsol * NCOL; it += blockDim.x) {
            const int sp = it / NCOL;
            const int col = it - sp * NCOL;
            const int te = col % TE;
            const int e = min(e0 + te, B.nelem - 1);
            const T inv = __ldg(B.metric + (size_t)sp * B.mr_inv * B.ld + e);
            const T* Sp = B.metric + (size_t)(B.mr_ss + sp * B.mr_ssk) * B.ld + e;
            S qt[ND];
            #pragma unroll
            for (int d = 0; d < ND; ++d) qt[d] = RQ[(size_t)sp * QCOL + d * NCOL + col];
            #pragma unroll
            for (int i = 0; i < ND; ++i) {
                S q = qt[0] * (__ldg(Sp + (size_t)i * B.ld) * inv);
                #pragma unroll
                for (int d = 1; d < ND; ++d) q = q + qt[d] * (__ldg(Sp + (size_t)(d * ND + i) * B.ld) * inv);
                RQ[(size_t)sp * QCOL + i * NCOL + col] = q;
                if constexpr (std::is_same<S, T>::value) {
                    // optional copy of the solution-point gradients, [N_s][ND][V][ld] per block
                    if (QSOL && e0 + te < B.nelem)
                        QSOL[(size_t)ND * B.u_off + ((size_t)(sp * ND + i) * V + col / TE) * B.ld + e] = q;
                }
            }
        }
        __syncthreads();
        // [q_fe; q_fiu] = [M0; M12] q; column (d, v, te) -> d * V + v = col / TE.
        tile_gemm<S, T>(B.Ai, B.Mi_pad, B.Mi, B.nsol, RQ, B.nsol, RQ, QCOL,
                        [&](int m0, int col, const S* acc) {
                            const int dv = col / TE, te = col - dv * TE, e = e0 + te;
                            if (e >= B.nelem) return;
                            #pragma unroll
                            for (int i = 0; i < kMR; ++i) {
                                const int m = m0 + i;
                                if (m >= B.Mi) break;
                                if (m < B.nfe)
                                    store_state(QFE, dQFE, (size_t)dv * Ftot + B.fe_base + (size_t)m * B.ld + e, acc[i]);
                                else
                                    store_state(QFIU, dQFIU,
                                                (size_t)B.qfiu_off + ((size_t)(m - B.nfe) * (ND * V) + dv) * B.ld + e,
                                                acc[i]);
                            }
                        });
    }
}

// ---------------------------------------------------------------------------
// Taylor-Green vortex diagnostics (paper Sec. 5.3): per element, the state
// U, the LDG gradients q at the solution points and the residual R are
// interpolated to the points of the element quadrature (degree 10) and
//   sums[0] += w det J                                   (volume)
//   sums[1] += w det J (1/2) rho |v|^2                    (kinetic energy)
//   sums[2] += w det J (v . R_m - (1/2) |v|^2 R_rho)      (its time derivative)
//   sums[3] += w det J S^d : S^d,  S^d = (grad v + grad v^T)/2 - (div v / 3) I
//   sums[4] += w det J p div v
// with grad v from q: d v_i / d x_d = (q_d,1+i - v_i q_d,0) / rho.
template <typename T>
__global__ void __launch_bounds__(256) k_tgv_diag(KBlock<T> B, const T* __restrict__ U, const T* __restrict__ Q,
                                                  const T* __restrict__ R, const T* __restrict__ Mq,
                                                  const T* __restrict__ wq, int nq, T gamma, double* sums) {
    constexpr int ND = 3, V = 5, NF = 2 * V + ND * V;    // fields per point: U, R, q
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* F = reinterpret_cast<T*>(smem_raw);              // [N_s][NF]
    double acc[5] = {0, 0, 0, 0, 0};
    for (int e = blockIdx.x; e < B.nelem; e += gridDim.x) {
        __syncthreads();
        for (int i = threadIdx.x; i < B.nsol * NF; i += blockDim.x) {
            const int r = i / NF, f = i - r * NF;
            T x;
            if (f < V) x = U[(size_t)B.u_off + ((size_t)r * V + f) * B.ld + e];
            else if (f < 2 * V) x = R[(size_t)B.u_off + ((size_t)r * V + (f - V)) * B.ld + e];
            else x = Q[(size_t)ND * B.u_off + ((size_t)r * ND * V + (f - 2 * V)) * B.ld + e];
            F[i] = x;
        }
        __syncthreads();
        const double detJ = 1.0 / (double)__ldg(B.metric + e);
        for (int k = threadIdx.x; k < nq; k += blockDim.x) {
            double val[NF];
            #pragma unroll
            for (int f = 0; f < NF; ++f) val[f] = 0.0;
            for (int r = 0; r < B.nsol; ++r) {
                const double m = (double)__ldg(Mq + (size_t)k * B.nsol + r);
                #pragma unroll
                for (int f = 0; f < NF; ++f) val[f] += m * (double)F[r * NF + f];
            }
            const double w = (double)__ldg(wq + k) * detJ;
            const double rho = val[0];
            double v[ND], ke = 0;
            #pragma unroll
            for (int i = 0; i < ND; ++i) {
                v[i] = val[1 + i] / rho;
                ke += v[i] * val[1 + i];
            }
            const double p = ((double)gamma - 1.0) * (val[V - 1] - 0.5 * ke);
            double dke = -0.5 * (ke / rho) * val[V];
            #pragma unroll
            for (int i = 0; i < ND; ++i) dke += v[i] * val[V + 1 + i];
            double gv[ND][ND];                           // gv[d][i] = d v_i / d x_d
            #pragma unroll
            for (int d = 0; d < ND; ++d)
                #pragma unroll
                for (int i = 0; i < ND; ++i)
                    gv[d][i] = (val[2 * V + d * V + 1 + i] - v[i] * val[2 * V + d * V]) / rho;
            const double div = gv[0][0] + gv[1][1] + gv[2][2];
            double ss = 0;
            #pragma unroll
            for (int i = 0; i < ND; ++i)
                #pragma unroll
                for (int j = 0; j < ND; ++j) {
                    const double sd = 0.5 * (gv[j][i] + gv[i][j]) - (i == j ? div / 3.0 : 0.0);
                    ss += sd * sd;
                }
            acc[0] += w;
            acc[1] += w * 0.5 * ke;
            acc[2] += w * dke;
            acc[3] += w * ss;
            acc[4] += w * p * div;
        }
    }
    __syncthreads();
    double* red = reinterpret_cast<double*>(smem_raw);
    for (int c = 0; c < 5; ++c) {
        red[threadIdx.x] = acc[c];
        __syncthreads();
        for (int s2 = blockDim.x / 2; s2 > 0; s2 >>= 1) {
            if (threadIdx.x < s2) red[threadIdx.x] += red[threadIdx.x + s2];
            __syncthreads();
        }
        if (threadIdx.x == 0) atomicAdd(sums + c, red[0]);
        __syncthreads();
    }
}

template <typename T>
void launch_tgv_diag(const KBlock<T>& B, const T* U, const T* Q, const T* R, const T* Mq, const T* wq, int nq, T gamma,
                     double* sums, int nsm, cudaStream_t st) {
    const int smem = (int)std::max(sizeof(T) * B.nsol * 25, sizeof(double) * 256);
    const int grid = B.nelem < 4 * nsm ? B.nelem : 4 * nsm;
    k_tgv_diag<T><<<grid, 256, smem, st>>>(B, U, Q, R, Mq, wq, nq, gamma, sums);
}

template void launch_tgv_diag<float>(const KBlock<float>&, const float*, const float*, const float*, const float*,
                                     const float*, int, float, double*, int, cudaStream_t);
template void launch_tgv_diag<double>(const KBlock<double>&, const double*, const double*, const double*,
                                      const double*, const double*, int, double, double*, int, cudaStream_t);

// ---------------------------------------------------------------------------
// Host launchers.

template <typename T>
int grad_smem(const KBlock<T>& B, int V, int nd, int TE, bool dual) {
    return (B.nsol + B.nfe + nd * B.nsol) * V * TE * (int)sizeof(T) * (dual ? 2 : 1);
}

template <typename S, typename T, int V, int ND>
static void launch_grad_impl(const KTable<T>& tab, const T* U, const T* dU, const T* UFE, const T* dUFE, int64_t Ftot,
                             const KPhys<T>& P, T* QFE, T* dQFE, T* QFIU, T* dQFIU, T* QSOL, int smem, int tiles,
                             int nsm, cudaStream_t st) {
    auto k = k_grad<S, T, V, ND>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k<<<persistent_grid(k, smem, tiles, nsm), 256, smem, st>>>(tab, U, dU, UFE, dUFE, Ftot, P, QFE, dQFE, QFIU, dQFIU,
                                                               QSOL);
}

template <typename T>
int launch_grad(const KSet<T>& ks, int system, int nd, const T* U, const T* dU, const T* UFE, const T* dUFE,
                int64_t Ftot, const KPhys<T>& P, T* QFE, T* dQFE, T* QFIU, T* dQFIU, int nsm, cudaStream_t st,
                T* QSOL) {
    const bool dual = dU != nullptr;
    const int kind = dual ? TK_GRAD_DUAL : TK_GRAD;
    if (!ks.all_tiled(kind)) return -2;
    const int V = system == SYS_ADVDIFF ? 1 : nd + 2;
    int smem = 0;
    for (int i = 0; i < ks.n; ++i) {
        const int b = grad_smem(ks.host[i], V, nd, tile_width(ks.host[i], kind), dual);
        smem = b > smem ? b : smem;
    }
    const int tiles = ks.tiles(kind);
    const KTable<T> tab = ks.table();
#define SDRT_GRAD(VV, NDD)                                                                                          \
    do {                                                                                                            \
        if (dual)                                                                                                   \
            launch_grad_impl<Dual<T>, T, VV, NDD>(tab, U, dU, UFE, dUFE, Ftot, P, QFE, dQFE, QFIU, dQFIU, nullptr, \
                                                  smem, tiles, nsm, st);                                                  \
        else                                                                                                        \
            launch_grad_impl<T, T, VV, NDD>(tab, U, dU, UFE, dUFE, Ftot, P, QFE, dQFE, QFIU, dQFIU, QSOL, smem, tiles, \
                                            nsm, st);                                                             \
    } while (0)
    if (system == SYS_ADVDIFF) {
        if (nd == 2) SDRT_GRAD(1, 2);
        else SDRT_GRAD(1, 3);
        return 0;
    }
    if (system == SYS_NS) {
        if (nd == 2) SDRT_GRAD(4, 2);
        else SDRT_GRAD(5, 3);
        return 0;
    }
#undef SDRT_GRAD
    return -1;
}

template <typename T>
int launch_residual_visc(const KSet<T>& ks, int system, int riemann, int nd, const T* U, const T* dU,
                         const T* UFE, const T* dUFE, int64_t Ftot, const KPhys<T>& P, const KEpi<T>& E,
                         const KVisc<T>& Q, int nsm, cudaStream_t st) {
    const bool dual = dU != nullptr;
    const int kind = dual ? TK_RES_DUAL : TK_RES;
    if (!ks.all_tiled(kind)) return -2;
    const int V = system == SYS_ADVDIFF ? 1 : nd + 2;
    int smem = 0;
    for (int i = 0; i < ks.n; ++i) {
        const int b = residual_smem(ks.host[i], V, tile_width(ks.host[i], kind), dual, nullptr);
        smem = b > smem ? b : smem;
    }
    const int tiles = ks.tiles(kind);
    const KTable<T> tab = ks.table();
#define SDRT_RES(VV, NDD, SYSS, RIEE)                                                                             \
    do {                                                                                                          \
        if (dual)                                                                                                 \
            launch_res_impl<Dual<T>, T, VV, NDD, SYSS, RIEE>(tab, U, dU, UFE, dUFE, Ftot, P, E, Q, smem, tiles, nsm,    \
                                                             st);                                                 \
        else                                                                                                      \
            launch_res_impl<T, T, VV, NDD, SYSS, RIEE>(tab, U, dU, UFE, dUFE, Ftot, P, E, Q, smem, tiles, nsm, st);     \
    } while (0)
    if (system == SYS_ADVDIFF) {
        if (nd == 2) SDRT_RES(1, 2, SYS_ADVDIFF, RIE_UPWIND);
        else SDRT_RES(1, 3, SYS_ADVDIFF, RIE_UPWIND);
        return 0;
    }
    if (system == SYS_NS) {
        if (nd == 2) {
            if (riemann == RIE_ROE) SDRT_RES(4, 2, SYS_NS, RIE_ROE);
            else SDRT_RES(4, 2, SYS_NS, RIE_RUSANOV);
        } else {
            if (riemann == RIE_ROE) SDRT_RES(5, 3, SYS_NS, RIE_ROE);
            else SDRT_RES(5, 3, SYS_NS, RIE_RUSANOV);
        }
        return 0;
    }
#undef SDRT_RES
    return -1;
}

template int grad_smem<float>(const KBlock<float>&, int, int, int, bool);
template int grad_smem<double>(const KBlock<double>&, int, int, int, bool);
template int launch_grad<float>(const KSet<float>&, int, int, const float*, const float*, const float*,
                                const float*, int64_t, const KPhys<float>&, float*, float*, float*, float*, int,
                                cudaStream_t, float*);
template int launch_grad<double>(const KSet<double>&, int, int, const double*, const double*, const double*,
                                 const double*, int64_t, const KPhys<double>&, double*, double*, double*, double*,
                                 int, cudaStream_t, double*);
template int launch_residual_visc<float>(const KSet<float>&, int, int, int, const float*, const float*,
                                         const float*, const float*, int64_t, const KPhys<float>&,
                                         const KEpi<float>&, const KVisc<float>&, int, cudaStream_t);
template int launch_residual_visc<double>(const KSet<double>&, int, int, int, const double*, const double*,
                                          const double*, const double*, int64_t, const KPhys<double>&,
                                          const KEpi<double>&, const KVisc<double>&, int, cudaStream_t);

}  // namespace sdrt
