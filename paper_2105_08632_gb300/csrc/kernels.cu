// SDRT residual kernels for sm_103a (FMA path).
//
// One residual evaluation (paper Sec. 2.1 and App. B) is two launches per block:
//   k_interp_ext : U -> u_fe = M0 U at the external flux points (written to UFE,
//                  the only data exchanged between elements);
//   k_residual   : per tile of TE elements, entirely in shared memory:
//                  [u_fe; u_fiu] = [M0; M12] U                       (Eqs. "interpolation_procedure")
//                  common flux at external points with the partner's u_fe
//                  gathered through the face map, F~ = s F(u_L, u_R, n_L)
//                  normal transformed flux at internal DOFs F~ = (S f(u)) . e_axis
//                                                                  (Eq. "normal_transformed_flux")
//                  R~ = [M14 | M13] [F~_fe; F~_fi], dU/dt = -R~ / det J
//                                                                  (Eq. "residual_sdrt_matrices")
//                  and an optional fused RK4 stage update.
// The same kernels instantiated with a dual-number scalar give the JVP.
#include <cstdint>

#include "device_math.cuh"
#include "kargs.hpp"
#include "launch.hpp"

namespace sdrt {

namespace {

constexpr int kMR = 8;   // rows of a GEMM micro tile

// C[m][col] = sum_k At[k * ldA + m] * B(k)[col]  for m < M, col < NCOL.
// B rows k < ksplit live at B0 + k * NCOL, the others at B1 + (k - ksplit) * NCOL.
// Work items are (row block of kMR rows, chunk of 32 columns); each warp takes
// items round-robin, each lane one column of the chunk.
template <typename S, typename T, typename Store>
__device__ __forceinline__ void tile_gemm(const T* __restrict__ At, int ldA, int M, int K,
                                          const S* B0, int ksplit, const S* B1, int NCOL, Store store) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int nrb = (M + kMR - 1) / kMR;
    const int ncc = (NCOL + 31) >> 5;
    for (int item = warp; item < nrb * ncc; item += nwarps) {
        const int rb = item / ncc;
        const int col = (item - rb * ncc) * 32 + lane;
        const bool colok = col < NCOL;
        const int c = colok ? col : 0;
        S acc[kMR];
        #pragma unroll
        for (int i = 0; i < kMR; ++i) acc[i] = szero<S>();
        const T* a = At + rb * kMR;
        #pragma unroll 2
        for (int k = 0; k < K; ++k) {
            const S b = (k < ksplit) ? B0[k * NCOL + c] : B1[(k - ksplit) * NCOL + c];
            T av[kMR];
            #pragma unroll
            for (int i = 0; i < kMR; ++i) av[i] = __ldg(a + (size_t)k * ldA + i);
            #pragma unroll
            for (int i = 0; i < kMR; ++i) mac(acc[i], av[i], b);
        }
        if (colok) {
            #pragma unroll
            for (int i = 0; i < kMR; ++i)
                if (rb * kMR + i < M) store(rb * kMR + i, col, acc[i]);
        }
    }
}

template <typename S, typename T>
__device__ __forceinline__ S load_state(const T* U, const T* dU, size_t idx);
template <>
__device__ __forceinline__ float load_state<float, float>(const float* U, const float*, size_t i) { return U[i]; }
template <>
__device__ __forceinline__ double load_state<double, double>(const double* U, const double*, size_t i) { return U[i]; }
template <>
__device__ __forceinline__ Dual<float> load_state<Dual<float>, float>(const float* U, const float* dU, size_t i) {
    return {U[i], dU[i]};
}
template <>
__device__ __forceinline__ Dual<double> load_state<Dual<double>, double>(const double* U, const double* dU, size_t i) {
    return {U[i], dU[i]};
}

// Stage the tile's solution values U[rho][v][e0 .. e0+TE) in shared memory
// (columns v * TE + te).  Lanes past the end of the block repeat the last
// element so that every lane works on a physical state.
template <typename S, typename T, int V>
__device__ __forceinline__ void load_tile(const KBlock<T>& B, const T* U, const T* dU, int e0, int TE, S* Us) {
    const int n = B.nsol * V * TE;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int row = i / TE;             // rho * V + v
        const int te = i - row * TE;
        const int e = min(e0 + te, B.nelem - 1);
        Us[i] = load_state<S, T>(U, dU, (size_t)B.u_off + (size_t)row * B.ld + e);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// u_fe = M0 U for every element of the block, written to UFE.
template <typename T, int V>
__global__ void __launch_bounds__(256) k_interp_ext(KBlock<T> B, const T* __restrict__ U, T* __restrict__ UFE,
                                                    int64_t Ftot, int TE) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Us = reinterpret_cast<T*>(smem_raw);
    const int ntiles = (B.nelem + TE - 1) / TE;
    const int NCOL = V * TE;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int e0 = tile * TE;
        __syncthreads();
        load_tile<T, T, V>(B, U, nullptr, e0, TE, Us);
        __syncthreads();
        tile_gemm<T, T>(B.Ai, B.Mi_pad, B.nfe, B.nsol, Us, B.nsol, Us, NCOL,
                        [&](int m, int col, T acc) {
                            const int v = col / TE, te = col - v * TE, e = e0 + te;
                            if (e < B.nelem) UFE[(size_t)v * Ftot + B.fe_base + (size_t)m * B.ld + e] = acc;
                        });
    }
}

// ---------------------------------------------------------------------------
// Fluxes of one system at one point.
template <int SYS, int RIE, int ND, typename S, typename T>
__device__ __forceinline__ void common_flux(const S* uL, const S* uR, const T* n, const KPhys<T>& P, S* F) {
    if constexpr (SYS == SYS_EULER) {
        if constexpr (RIE == RIE_ROE) roe<S, T, ND>(uL, uR, n, P.gamma, F);
        else rusanov<S, T, ND>(uL, uR, n, P.gamma, F);
    } else {
        T an = P.a[0] * n[0];
        #pragma unroll
        for (int d = 1; d < ND; ++d) an = fma(P.a[d], n[d], an);
        const T aa = an >= T(0) ? an : -an;
        F[0] = T(0.5) * an * (uL[0] + uR[0]) + T(0.5) * aa * (uL[0] - uR[0]);
    }
}

// (S_axis . f(u)) for the transformed flux component along one reference axis.
template <int SYS, int ND, typename S, typename T>
__device__ __forceinline__ void internal_flux(const S* u, const T* Srow, const KPhys<T>& P, S* Ft) {
    if constexpr (SYS == SYS_EULER) {
        S v[ND], p;
        euler_prim<S, T, ND>(u, v, p, P.gamma);
        euler_nflux<S, T, ND>(u, v, p, Srow, Ft);
    } else {
        T an = P.a[0] * Srow[0];
        #pragma unroll
        for (int d = 1; d < ND; ++d) an = fma(P.a[d], Srow[d], an);
        Ft[0] = an * u[0];
    }
}

template <typename T>
__device__ __forceinline__ void epilogue(const KEpi<T>& E, size_t idx, T r) {
    if (!isfinite(r)) *E.flag = 1;
    switch (E.mode) {
        case EPI_STORE: E.out[idx] = r; break;
        case EPI_RK_FIRST: {
            const T u0 = E.u0[idx];
            E.uacc[idx] = fma(E.cacc, r, u0);
            E.unext[idx] = fma(E.cnext, r, u0);
            break;
        }
        case EPI_RK_MID: {
            E.uacc[idx] = fma(E.cacc, r, E.uacc[idx]);
            E.unext[idx] = fma(E.cnext, r, E.u0[idx]);
            break;
        }
        default: E.out[idx] = fma(E.cacc, r, E.uacc[idx]); break;
    }
}
template <typename T>
__device__ __forceinline__ void epilogue(const KEpi<T>& E, size_t idx, Dual<T> r) {
    if (!isfinite(r.d)) *E.flag = 1;
    E.out[idx] = r.d;
}

template <typename S, typename T, int V>
__device__ __forceinline__ void gather_partner(const T* UFE, const T* dUFE, int64_t Ftot, int fp, S* out) {
    #pragma unroll
    for (int v = 0; v < V; ++v) out[v] = load_state<S, T>(UFE, dUFE, (size_t)v * Ftot + fp);
}

// Full inviscid residual of one block (S = T: value; S = Dual<T>: JVP).
template <typename S, typename T, int V, int ND, int SYS, int RIE>
__global__ void __launch_bounds__(256) k_residual(KBlock<T> B, const T* __restrict__ U, const T* __restrict__ dU,
                                                  const T* __restrict__ UFE, const T* __restrict__ dUFE, int64_t Ftot,
                                                  KPhys<T> P, KEpi<T> E, int TE, int rowsA) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NCOL = V * TE;
    S* RA = reinterpret_cast<S*>(smem_raw);            // U tile, then internal F~ (rowsA rows)
    S* RB = RA + (size_t)rowsA * NCOL;                  // [u_fe; u_fiu], F~_fe in place of u_fe
    const int ntiles = (B.nelem + TE - 1) / TE;
    constexpr int ND2 = ND * ND;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int e0 = tile * TE;
        __syncthreads();
        load_tile<S, T, V>(B, U, dU, e0, TE, RA);
        __syncthreads();
        // [u_fe; u_fiu] = [M0; M12] U
        tile_gemm<S, T>(B.Ai, B.Mi_pad, B.Mi, B.nsol, RA, B.nsol, RA, NCOL,
                        [&](int m, int col, S acc) { RB[(size_t)m * NCOL + col] = acc; });
        __syncthreads();
        // External points: common flux with the partner state.
        for (int it = threadIdx.x; it < B.nfe * TE; it += blockDim.x) {
            const int sg = it / TE;
            const int te = it - sg * TE;
            const int e = min(e0 + te, B.nelem - 1);
            const int f = __ldg(B.fe_face + sg);
            const int mrow = 1 + ND2 + f * (ND + 1);
            T n[ND];
            #pragma unroll
            for (int c = 0; c < ND; ++c) n[c] = __ldg(B.metric + (size_t)(mrow + c) * B.ld + e);
            const T s = __ldg(B.metric + (size_t)(mrow + ND) * B.ld + e);
            S own[V], nbr[V], F[V];
            #pragma unroll
            for (int v = 0; v < V; ++v) own[v] = RB[(size_t)sg * NCOL + v * TE + te];
            gather_partner<S, T, V>(UFE, dUFE, Ftot, __ldg(B.map + (size_t)sg * B.ld + e), nbr);
            if (s > T(0)) common_flux<SYS, RIE, ND>(own, nbr, n, P, F);
            else common_flux<SYS, RIE, ND>(nbr, own, n, P, F);
            #pragma unroll
            for (int v = 0; v < V; ++v) RB[(size_t)sg * NCOL + v * TE + te] = s * F[v];
        }
        // Internal DOFs: transformed flux component along the DOF's axis.
        for (int it = threadIdx.x; it < B.nfiu * TE; it += blockDim.x) {
            const int k = it / TE;
            const int te = it - k * TE;
            const int e = min(e0 + te, B.nelem - 1);
            S u[V];
            #pragma unroll
            for (int v = 0; v < V; ++v) u[v] = RB[(size_t)(B.nfe + k) * NCOL + v * TE + te];
            const int4 tab = __ldg(reinterpret_cast<const int4*>(B.fi_tab) + k);
            const int dofs[3] = {tab.y, tab.z, tab.w};
            for (int q = 0; q < tab.x; ++q) {
                const int nu = dofs[q] & 0xffff;
                const int ax = dofs[q] >> 16;
                T Srow[ND];
                #pragma unroll
                for (int i = 0; i < ND; ++i) Srow[i] = __ldg(B.metric + (size_t)(1 + ax * ND + i) * B.ld + e);
                S Ft[V];
                internal_flux<SYS, ND>(u, Srow, P, Ft);
                #pragma unroll
                for (int v = 0; v < V; ++v) RA[(size_t)nu * NCOL + v * TE + te] = Ft[v];
            }
        }
        __syncthreads();
        // R~ = [M14 | M13] [F~_fe; F~_fi];  dU/dt = -R~ / det J
        tile_gemm<S, T>(B.Ad, B.Md_pad, B.nsol, B.nfe + B.nfi, RB, B.nfe, RA, NCOL,
                        [&](int m, int col, S acc) {
                            const int v = col / TE, te = col - v * TE, e = e0 + te;
                            if (e < B.nelem) {
                                const T inv = __ldg(B.metric + e);
                                const size_t idx = (size_t)B.u_off + (size_t)(m * V + v) * B.ld + e;
                                epilogue(E, idx, acc * (-inv));
                            }
                        });
    }
}

// ---------------------------------------------------------------------------
// Host launchers.

template <typename T>
static int smem_interp(const KBlock<T>& B, int V, int TE) {
    return B.nsol * V * TE * (int)sizeof(T);
}

template <typename T>
void launch_interp_ext(const KBlock<T>& B, int V, const T* U, T* UFE, int64_t Ftot, int TE, int grid,
                       cudaStream_t st) {
    const int smem = smem_interp(B, V, TE);
    switch (V) {
#define SDRT_CASE(VV)                                                                                   \
    case VV:                                                                                            \
        cudaFuncSetAttribute(k_interp_ext<T, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);   \
        k_interp_ext<T, VV><<<grid, 256, smem, st>>>(B, U, UFE, Ftot, TE);                               \
        break;
        SDRT_CASE(1)
        SDRT_CASE(4)
        SDRT_CASE(5)
#undef SDRT_CASE
        default: break;
    }
}

template <typename S, typename T, int V, int ND, int SYS, int RIE>
static void launch_res_impl(const KBlock<T>& B, const T* U, const T* dU, const T* UFE, const T* dUFE, int64_t Ftot,
                            const KPhys<T>& P, const KEpi<T>& E, int TE, int rowsA, int smem, int grid,
                            cudaStream_t st) {
    auto k = k_residual<S, T, V, ND, SYS, RIE>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k<<<grid, 256, smem, st>>>(B, U, dU, UFE, dUFE, Ftot, P, E, TE, rowsA);
}

template <typename T>
int residual_smem(const KBlock<T>& B, int V, int TE, bool dual, int* rowsA) {
    const int ra = B.nsol > B.nfi ? B.nsol : B.nfi;
    if (rowsA) *rowsA = ra;
    return (ra + B.Mi) * V * TE * (int)sizeof(T) * (dual ? 2 : 1);
}

template <typename T>
int launch_residual(const KBlock<T>& B, int system, int riemann, int nd, const T* U, const T* dU, const T* UFE,
                    const T* dUFE, int64_t Ftot, const KPhys<T>& P, const KEpi<T>& E, int TE, int grid,
                    cudaStream_t st) {
    const bool dual = dU != nullptr;
    int rowsA = 0;
    const int V = (system == SYS_ADVECTION) ? 1 : nd + 2;
    const int smem = residual_smem(B, V, TE, dual, &rowsA);
#define SDRT_DISPATCH(SS, VV, NDD, SYSS, RIEE) \
    launch_res_impl<SS, T, VV, NDD, SYSS, RIEE>(B, U, dU, UFE, dUFE, Ftot, P, E, TE, rowsA, smem, grid, st)
    if (system == SYS_ADVECTION) {
        if (nd == 2) {
            if (dual) SDRT_DISPATCH(Dual<T>, 1, 2, SYS_ADVECTION, RIE_UPWIND);
            else SDRT_DISPATCH(T, 1, 2, SYS_ADVECTION, RIE_UPWIND);
        } else {
            if (dual) SDRT_DISPATCH(Dual<T>, 1, 3, SYS_ADVECTION, RIE_UPWIND);
            else SDRT_DISPATCH(T, 1, 3, SYS_ADVECTION, RIE_UPWIND);
        }
        return 0;
    }
    if (system == SYS_EULER) {
        if (nd == 2) {
            if (riemann == RIE_ROE) {
                if (dual) SDRT_DISPATCH(Dual<T>, 4, 2, SYS_EULER, RIE_ROE);
                else SDRT_DISPATCH(T, 4, 2, SYS_EULER, RIE_ROE);
            } else {
                if (dual) SDRT_DISPATCH(Dual<T>, 4, 2, SYS_EULER, RIE_RUSANOV);
                else SDRT_DISPATCH(T, 4, 2, SYS_EULER, RIE_RUSANOV);
            }
        } else {
            if (riemann == RIE_ROE) {
                if (dual) SDRT_DISPATCH(Dual<T>, 5, 3, SYS_EULER, RIE_ROE);
                else SDRT_DISPATCH(T, 5, 3, SYS_EULER, RIE_ROE);
            } else {
                if (dual) SDRT_DISPATCH(Dual<T>, 5, 3, SYS_EULER, RIE_RUSANOV);
                else SDRT_DISPATCH(T, 5, 3, SYS_EULER, RIE_RUSANOV);
            }
        }
        return 0;
    }
#undef SDRT_DISPATCH
    return -1;
}

template void launch_interp_ext<float>(const KBlock<float>&, int, const float*, float*, int64_t, int, int,
                                       cudaStream_t);
template void launch_interp_ext<double>(const KBlock<double>&, int, const double*, double*, int64_t, int, int,
                                        cudaStream_t);
template int launch_residual<float>(const KBlock<float>&, int, int, int, const float*, const float*, const float*,
                                    const float*, int64_t, const KPhys<float>&, const KEpi<float>&, int, int,
                                    cudaStream_t);
template int launch_residual<double>(const KBlock<double>&, int, int, int, const double*, const double*,
                                     const double*, const double*, int64_t, const KPhys<double>&,
                                     const KEpi<double>&, int, int, cudaStream_t);
template int residual_smem<float>(const KBlock<float>&, int, int, bool, int*);
template int residual_smem<double>(const KBlock<double>&, int, int, bool, int*);

}  // namespace sdrt
