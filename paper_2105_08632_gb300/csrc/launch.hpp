// Host-side launchers of the CUDA kernels (implemented in kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kargs.hpp"

namespace sdrt {

// The blocks of a mesh for the generic kernels, which walk all blocks' tiles
// in one launch per kernel kind: host copies (tile counts, shared-memory
// sizes) and the same array in device memory.
template <typename T>
struct KSet {
    const KBlock<T>* host;
    const KBlock<T>* dev;
    int n;
    KTable<T> table() const { return {dev, n}; }
    int tiles(int kind) const {
        int t = 0;
        for (int i = 0; i < n; ++i) {
            const int te = tile_width(host[i], kind);
            if (te > 0) t += (host[i].nelem + te - 1) / te;
        }
        return t;
    }
    bool all_tiled(int kind) const {
        for (int i = 0; i < n; ++i)
            if (tile_width(host[i], kind) <= 0) return false;
        return true;
    }
};

// u_fe = M0 U for every block (V variables), written to UFE.  One launch.
template <typename T>
void launch_interp_ext(const KSet<T>& ks, int V, const T* U, T* UFE, int64_t Ftot, int nsm, cudaStream_t st);

// Residual of every block with a fused epilogue, one launch.  dU / dUFE
// non-null: JVP mode (tangent of the residual written to E.out, E.mode must be
// EPI_STORE).  Returns -1 for an unsupported (system, riemann, nd)
// combination, -2 if a block has no tile width for the mode.
// Viscous systems read the flux-point gradients from Q (written by launch_grad).
template <typename T>
int launch_residual(const KSet<T>& ks, int system, int riemann, int nd, const T* U, const T* dU, const T* UFE,
                    const T* dUFE, int64_t Ftot, const KPhys<T>& P, const KEpi<T>& E, const KVisc<T>& Q, int nsm,
                    cudaStream_t st);

// The viscous instantiations of launch_residual (kernels_visc.cu).
template <typename T>
int launch_residual_visc(const KSet<T>& ks, int system, int riemann, int nd, const T* U, const T* dU,
                         const T* UFE, const T* dUFE, int64_t Ftot, const KPhys<T>& P, const KEpi<T>& E,
                         const KVisc<T>& Q, int nsm, cudaStream_t st);

// Physical gradients of a viscous system at the flux points of every block
// (UFE must hold u_fe of every block): QFE / QFIU (kargs.hpp layout), and with
// dU / dUFE non-null also their tangents dQFE / dQFIU.  One launch.  Returns
// -1 for an unsupported (system, nd) combination, -2 without tile widths.
// QSOL non-null (value mode): also the solution-point gradients, per block
// [N_s][ND][V][ld] at ND * u_off.
template <typename T>
int launch_grad(const KSet<T>& ks, int system, int nd, const T* U, const T* dU, const T* UFE, const T* dUFE,
                int64_t Ftot, const KPhys<T>& P, T* QFE, T* dQFE, T* QFIU, T* dQFIU, int nsm, cudaStream_t st,
                T* QSOL = nullptr);

// Gradient chain of one block on the tensor cores (kernels_tc_grad.cu): the
// value-mode output of launch_grad (QFE / QFIU) for FP32 3D Navier-Stokes on
// affine blocks of the instantiated element types (tetrahedra p3 / p4,
// hexahedra p2, prisms p2).  Returns -1 if the block is not of that kind.
bool grad_tc_available(const KBlock<float>& B, int V, int nd);
int launch_grad_tc(const KBlock<float>& B, int V, int nd, const float* U, const float* UFE, int64_t Ftot,
                   const KPhys<float>& P, float* QFE, float* QFIU, int* err, int nsm, cudaStream_t st);

// Taylor-Green diagnostics integrals of one block (kernels_visc.cu), added to
// sums[5] = {volume, kinetic energy, its time derivative from R, S^d : S^d,
// p div v}; 3D Navier-Stokes.
template <typename T>
void launch_tgv_diag(const KBlock<T>& B, const T* U, const T* Q, const T* R, const T* Mq, const T* wq, int nq, T gamma,
                     double* sums, int nsm, cudaStream_t st);

// Vector-Jacobian product of the inviscid residual, every block in one launch
// per pass (kernels_vjp.cu).  pass 0: GS (UFE layout) = s G at the external
// points from W; pass 1: out = W^T dR/dU, with UFE = u_fe of every block.
// Returns -1 for an unsupported combination, -2 without tile widths.
template <typename T>
int launch_vjp(const KSet<T>& ks, int pass, int system, int riemann, int nd, const T* U, const T* W, const T* UFE,
               T* GS, int64_t Ftot, const KPhys<T>& P, T* out, int* flag, int nsm, cudaStream_t st);
template <typename T>
int vjp_smem(const KBlock<T>& B, int V, int TE);

// Vector-Jacobian product of the viscous residual (advection-diffusion,
// Navier-Stokes; kernels_vjp.cu), every block in one launch per pass, after
// the forward interpolation (UFE) and gradients (QFE, QFIU): pass 0 GS = s G;
// pass 1 out = W^T J without the common value's term and CB = its adjoint at
// the external points (UFE layout); pass 2 out += that term.  Returns -1 for
// an unsupported combination, -2 without tile widths.
template <typename T>
int launch_vjp_visc(const KSet<T>& ks, int pass, int system, int riemann, int nd, const T* U, const T* W,
                    const T* UFE, const T* QFE, const T* QFIU, T* GS, T* CB, int64_t Ftot, const KPhys<T>& P, T* out,
                    int* flag, int nsm, cudaStream_t st);
template <typename T>
int vjp_visc_smem(const KBlock<T>& B, int V, int nd, int TE);

// Dynamic shared memory of the gradient kernel for tile width TE.
template <typename T>
int grad_smem(const KBlock<T>& B, int V, int nd, int TE, bool dual);

// Dynamic shared memory of the residual kernel for tile width TE.
template <typename T>
int residual_smem(const KBlock<T>& B, int V, int TE, bool dual, int* rowsA);

// Register-blocked record path (kernels_fast.cu) for the element types
// instantiated there (tetrahedra of degree 3 and 4).
bool fast_path_available(int shape, int nsol, int nd, int system, int riemann);

// Whether the JVP variant of the record path fits in shared memory for this
// block (FP64 degree-4 tetrahedra do not: their JVP takes the generic path).
template <typename T>
bool fast_jvp_available(const KBlock<T>& B, int V);

// [u_fe; u_fiu] = [M0; M12] U written as element records (REC, FIUR).
// Returns -1 if not instantiated.
template <typename T>
int launch_interp_rec(const KBlock<T>& B, int V, const T* U, T* REC, T* FIUR, int* err, int nsm, cudaStream_t st);

// Tensor-core (tcgen05, 3xTF32) variant of launch_interp_rec for FP32
// tetrahedra of degree 3 with 5 variables (kernels_tc.cu).  Returns -1 if
// the block is not of that kind.
bool tc_interp_available(int shape, int nsol, int nvar);
int launch_interp_tc(const KBlock<float>& B, int V, const float* U, float* REC, float* FIUR, int* err, int nsm,
                     cudaStream_t st);

// Fluxes on the CUDA cores and divergence on the tensor cores (tcgen05,
// 3xTF32) from the records, for FP32 Euler / Rusanov on tetrahedra of degree 3
// (kernels_tc.cu).  Returns -1 if the block is not of that kind.
bool tc_flux_available(int shape, int nsol, int nvar, int system, int riemann);
int launch_flux_tc(const KBlock<float>& B, const float* REC, const float* FIUR, const KPhys<float>& P,
                   const KEpi<float>& E, int nsm, cudaStream_t st);

// Whether launch_flux_rec can interpolate the next RK stage's state in its
// epilogue (E.rec_next / E.fiur_next non-null; FP32 Euler, tetrahedra of degree 3).
bool flux_rec_fusable(const KBlock<float>& B, int V, int system);

// n face records of len values between the record array and a packed buffer:
// gather (buf[i len + k] = rec[off[i] + k]) or scatter (rec[off[i] + k] = buf[i len + k]).
template <typename T>
void launch_face_records(const T* src, T* dst, const int* off, int64_t n, int len, bool scatter, int nsm,
                         cudaStream_t st);

// n values between an array and a packed buffer through an index list (-1:
// padding, gathered as zero, not scattered): gather dst[i] = src[idx[i]],
// scatter dst[idx[i]] = src[i].
template <typename T>
void launch_gather_values(const T* src, T* dst, const int* idx, int64_t n, bool scatter, int nsm, cudaStream_t st);

// RK54 stage update (kernels_rk.cu): dU = a dU + dt R (dU = dt R when
// first), U += b dU, and with E non-null E = (first ? 0 : E) + ne dt R.
template <typename T>
void launch_rk2n(int64_t n, T* U, T* dU, const T* R, T* E, double a, double b, double ne, double dt, bool first,
                 int nsm, cudaStream_t st);
// Per-CTA maxima of |E| / (atol + rtol max(|U0|, |U|)) over n values, part[nparts].
template <typename T>
void launch_err_linf(int64_t n, const T* E, const T* U0, const T* U, double atol, double rtol, double* part, int nparts,
                     cudaStream_t st);

// Fluxes and divergence from the records (dREC / dFIUR non-null: JVP mode) with epilogue E.
template <typename T>
int launch_flux_rec(const KBlock<T>& B, int system, const T* REC, const T* dREC, const T* FIUR, const T* dFIUR,
                    const KPhys<T>& P, const KEpi<T>& E, int nsm, cudaStream_t st);

}  // namespace sdrt
