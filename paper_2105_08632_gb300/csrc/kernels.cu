// Host launchers of the generic inviscid kernels (advection, Euler).
#include <cstdint>

#include "generic.cuh"
#include "launch.hpp"

namespace sdrt {

// ---------------------------------------------------------------------------
// Host launchers.

template <typename T>
void launch_interp_ext(const KSet<T>& ks, int V, const T* U, T* UFE, int64_t Ftot, int nsm, cudaStream_t st) {
    int smem = 0;
    for (int i = 0; i < ks.n; ++i) {
        const int b = ks.host[i].nsol * V * ks.host[i].te_interp * (int)sizeof(T);
        smem = b > smem ? b : smem;
    }
    const int tiles = ks.tiles(TK_INTERP);
    const KTable<T> tab = ks.table();
    switch (V) {
#define SDRT_CASE(VV)                                                                                   \
    case VV:                                                                                            \
        cudaFuncSetAttribute(k_interp_ext<T, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);   \
        k_interp_ext<T, VV><<<persistent_grid(k_interp_ext<T, VV>, smem, tiles, nsm), 256, smem, st>>>(   \
            tab, U, UFE, Ftot);                                                                         \
        break;
        SDRT_CASE(1)
        SDRT_CASE(4)
        SDRT_CASE(5)
#undef SDRT_CASE
        default: break;
    }
}

template <typename T>
__global__ void k_gather_values(const T* __restrict__ src, T* __restrict__ dst, const int* __restrict__ idx, int64_t n,
                                int scatter) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int j = idx[i];
        if (scatter) {
            if (j >= 0) dst[j] = src[i];
        } else {
            dst[i] = j >= 0 ? src[j] : T(0);
        }
    }
}

template <typename T>
void launch_gather_values(const T* src, T* dst, const int* idx, int64_t n, bool scatter, int nsm, cudaStream_t st) {
    if (n <= 0) return;
    int64_t grid = (n + 255) / 256;
    if (grid > 8 * (int64_t)nsm) grid = 8 * (int64_t)nsm;
    k_gather_values<T><<<(int)grid, 256, 0, st>>>(src, dst, idx, n, scatter ? 1 : 0);
}
template void launch_gather_values<float>(const float*, float*, const int*, int64_t, bool, int, cudaStream_t);
template void launch_gather_values<double>(const double*, double*, const int*, int64_t, bool, int, cudaStream_t);

template <typename T>
int residual_smem(const KBlock<T>& B, int V, int TE, bool dual, int* rowsA) {
    const int ra = B.nsol > B.nfi ? B.nsol : B.nfi;
    if (rowsA) *rowsA = ra;
    return (ra + B.Mi) * V * TE * (int)sizeof(T) * (dual ? 2 : 1);
}

template <typename T>
int launch_residual(const KSet<T>& ks, int system, int riemann, int nd, const T* U, const T* dU, const T* UFE,
                    const T* dUFE, int64_t Ftot, const KPhys<T>& P, const KEpi<T>& E, const KVisc<T>& Q, int nsm,
                    cudaStream_t st) {
    if (system == SYS_ADVDIFF || system == SYS_NS)
        return launch_residual_visc<T>(ks, system, riemann, nd, U, dU, UFE, dUFE, Ftot, P, E, Q, nsm, st);
    const bool dual = dU != nullptr;
    const int kind = dual ? TK_RES_DUAL : TK_RES;
    if (!ks.all_tiled(kind)) return -2;
    const int V = (system == SYS_ADVECTION) ? 1 : nd + 2;
    int smem = 0;
    for (int i = 0; i < ks.n; ++i) {
        const int b = residual_smem(ks.host[i], V, tile_width(ks.host[i], kind), dual, nullptr);
        smem = b > smem ? b : smem;
    }
    const int tiles = ks.tiles(kind);
    const KTable<T> tab = ks.table();
#define SDRT_DISPATCH(SS, VV, NDD, SYSS, RIEE) \
    launch_res_impl<SS, T, VV, NDD, SYSS, RIEE>(tab, U, dU, UFE, dUFE, Ftot, P, E, Q, smem, tiles, nsm, st)
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

template void launch_interp_ext<float>(const KSet<float>&, int, const float*, float*, int64_t, int, cudaStream_t);
template void launch_interp_ext<double>(const KSet<double>&, int, const double*, double*, int64_t, int,
                                        cudaStream_t);
template int launch_residual<float>(const KSet<float>&, int, int, int, const float*, const float*, const float*,
                                    const float*, int64_t, const KPhys<float>&, const KEpi<float>&,
                                    const KVisc<float>&, int, cudaStream_t);
template int launch_residual<double>(const KSet<double>&, int, int, int, const double*, const double*,
                                     const double*, const double*, int64_t, const KPhys<double>&,
                                     const KEpi<double>&, const KVisc<double>&, int, cudaStream_t);
template int residual_smem<float>(const KBlock<float>&, int, int, bool, int*);
template int residual_smem<double>(const KBlock<double>&, int, int, bool, int*);

}  // namespace sdrt
