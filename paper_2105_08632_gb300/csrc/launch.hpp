// Host-side launchers of the CUDA kernels (implemented in kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kargs.hpp"

namespace sdrt {

// u_fe = M0 U for one block (V variables), written to UFE.
template <typename T>
void launch_interp_ext(const KBlock<T>& B, int V, const T* U, T* UFE, int64_t Ftot, int TE, int grid,
                       cudaStream_t st);

// Residual of one block with a fused epilogue.  dU / dUFE non-null: JVP mode
// (tangent of the residual written to E.out, E.mode must be EPI_STORE).
// Returns -1 for an unsupported (system, riemann, nd) combination.
template <typename T>
int launch_residual(const KBlock<T>& B, int system, int riemann, int nd, const T* U, const T* dU, const T* UFE,
                    const T* dUFE, int64_t Ftot, const KPhys<T>& P, const KEpi<T>& E, int TE, int grid,
                    cudaStream_t st);

// Dynamic shared memory of the residual kernel for tile width TE.
template <typename T>
int residual_smem(const KBlock<T>& B, int V, int TE, bool dual, int* rowsA);

}  // namespace sdrt
