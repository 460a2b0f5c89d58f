// Host launchers of the generic inviscid kernels (advection, Euler).
#include <cstdint>

#include "generic.cuh"
#include "launch.hpp"

namespace sdrt {

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

template <typename T>
int residual_smem(const KBlock<T>& B, int V, int TE, bool dual, int* rowsA) {
    const int ra = B.nsol > B.nfi ? B.nsol : B.nfi;
    if (rowsA) *rowsA = ra;
    return (ra + B.Mi) * V * TE * (int)sizeof(T) * (dual ? 2 : 1);
}

template <typename T>
int launch_residual(const KBlock<T>& B, int system, int riemann, int nd, const T* U, const T* dU, const T* UFE,
                    const T* dUFE, int64_t Ftot, const KPhys<T>& P, const KEpi<T>& E, const KVisc<T>& Q, int TE,
                    int grid, cudaStream_t st) {
    if (system == SYS_ADVDIFF || system == SYS_NS)
        return launch_residual_visc<T>(B, system, riemann, nd, U, dU, UFE, dUFE, Ftot, P, E, Q, TE, grid, st);
    const bool dual = dU != nullptr;
    int rowsA = 0;
    const int V = (system == SYS_ADVECTION) ? 1 : nd + 2;
    const int smem = residual_smem(B, V, TE, dual, &rowsA);
#define SDRT_DISPATCH(SS, VV, NDD, SYSS, RIEE) \
    launch_res_impl<SS, T, VV, NDD, SYSS, RIEE>(B, U, dU, UFE, dUFE, Ftot, P, E, Q, TE, rowsA, smem, grid, st)
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
                                    const float*, int64_t, const KPhys<float>&, const KEpi<float>&,
                                    const KVisc<float>&, int, int, cudaStream_t);
template int launch_residual<double>(const KBlock<double>&, int, int, int, const double*, const double*,
                                     const double*, const double*, int64_t, const KPhys<double>&,
                                     const KEpi<double>&, const KVisc<double>&, int, int, cudaStream_t);
template int residual_smem<float>(const KBlock<float>&, int, int, bool, int*);
template int residual_smem<double>(const KBlock<double>&, int, int, bool, int*);

}  // namespace sdrt
