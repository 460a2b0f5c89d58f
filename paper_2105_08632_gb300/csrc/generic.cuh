// Generic (any element type) SDRT kernel templates for sm_103a, FMA path.
//
// One residual evaluation (paper Sec. 2.1 and App. B) is two launches, each a
// persistent grid walking the tiles of every block of the mesh (block table
// KTable, tile widths per block from the autotuner; viscous systems add k_grad
// in between):
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
#pragma once

#include <cstdint>
#include <type_traits>

#include "device_math.cuh"
#include "kargs.hpp"

namespace sdrt {

namespace {

constexpr int kMR = 8;   // rows of a GEMM micro tile

__device__ __forceinline__ bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// Grid of a persistent kernel (256 threads, blocks walking tiles): every CTA
// that fits on an SM at this shared-memory size, at most one per tile.
template <typename K>
inline int persistent_grid(K kernel, int smem, int tiles, int nsm) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 256, smem) != cudaSuccess || per < 1) per = 1;
    const int cap = per * nsm;
    return tiles < 1 ? 1 : (tiles < cap ? tiles : cap);
}

// 8 consecutive operator entries (16-byte loads when aligned).
__device__ __forceinline__ void ld_a8(const float* p, float (&a)[8], bool vec) {
    if (vec) {
        const float4 x = __ldg(reinterpret_cast<const float4*>(p));
        const float4 y = __ldg(reinterpret_cast<const float4*>(p) + 1);
        a[0] = x.x; a[1] = x.y; a[2] = x.z; a[3] = x.w;
        a[4] = y.x; a[5] = y.y; a[6] = y.z; a[7] = y.w;
    } else {
        #pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = __ldg(p + i);
    }
}
__device__ __forceinline__ void ld_a8(const double* p, double (&a)[8], bool vec) {
    if (vec) {
        #pragma unroll
        for (int i = 0; i < 4; ++i) {
            const double2 x = __ldg(reinterpret_cast<const double2*>(p) + i);
            a[2 * i] = x.x;
            a[2 * i + 1] = x.y;
        }
    } else {
        #pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = __ldg(p + i);
    }
}
// CW consecutive values of a shared-memory row (16-byte loads for float / double).
template <int CW>
__device__ __forceinline__ void ld_b(const float* p, float (&b)[CW]) {
    if constexpr (CW == 4) {
        const float4 x = *reinterpret_cast<const float4*>(p);
        b[0] = x.x; b[1] = x.y; b[2] = x.z; b[3] = x.w;
    } else {
        #pragma unroll
        for (int j = 0; j < CW; ++j) b[j] = p[j];
    }
}
template <int CW>
__device__ __forceinline__ void ld_b(const double* p, double (&b)[CW]) {
    if constexpr (CW == 4) {
        const double2 x = *reinterpret_cast<const double2*>(p);
        const double2 y = *(reinterpret_cast<const double2*>(p) + 1);
        b[0] = x.x; b[1] = x.y; b[2] = y.x; b[3] = y.y;
    } else {
        #pragma unroll
        for (int j = 0; j < CW; ++j) b[j] = p[j];
    }
}
template <int CW, typename T>
__device__ __forceinline__ void ld_b(const Dual<T>* p, Dual<T> (&b)[CW]) {
    #pragma unroll
    for (int j = 0; j < CW; ++j) b[j] = p[j];
}

template <int CW, bool PAIRED, typename S, typename T, typename Store>
__device__ __forceinline__ void tile_gemm_cw(const T* __restrict__ At, int ldA, int M, int K, const S* B0, int ksplit,
                                             const S* B1, int NCOL, Store store) {
    const int nrb = (M + kMR - 1) / kMR;
    const int ncw = NCOL / CW;
    const bool avec = aligned16(At) && ((size_t)ldA * sizeof(T)) % 16 == 0;
    for (int u = threadIdx.x; u < nrb * ncw; u += blockDim.x) {
        const int rb = u / ncw;
        const int col0 = (u - rb * ncw) * CW;
        S acc[kMR][CW];
        #pragma unroll
        for (int i = 0; i < kMR; ++i)
            #pragma unroll
            for (int j = 0; j < CW; ++j) acc[i][j] = szero<S>();
        const T* a = At + rb * kMR;
        if constexpr (PAIRED && std::is_same<S, float>::value && std::is_same<T, float>::value && CW == 4) {
            // Paired FP32 FMA (two IEEE fmas per instruction, sm_100+), rows and
            // columns paired crosswise: D = (r c, r+1 c+1) += (a_r, a_r+1)(b_c, b_c+1),
            // X = (r c+1, r+1 c) += (a_r, a_r+1)(b_c+1, b_c) -- the same sums, in
            // the same order, as the scalar loop below.
            float2 d[kMR / 2][2], x[kMR / 2][2];
            #pragma unroll
            for (int q = 0; q < kMR / 2; ++q)
                #pragma unroll
                for (int w = 0; w < 2; ++w) d[q][w] = x[q][w] = make_float2(0.f, 0.f);
            #pragma unroll 2
            for (int k = 0; k < K; ++k) {
                float b[4];
                ld_b<4>((k < ksplit ? B0 + (size_t)k * NCOL : B1 + (size_t)(k - ksplit) * NCOL) + col0, b);
                float av[kMR];
                ld_a8(a + (size_t)k * ldA, av, avec);
                const float2 P[2] = {make_float2(b[0], b[1]), make_float2(b[2], b[3])};
                const float2 Q[2] = {make_float2(b[1], b[0]), make_float2(b[3], b[2])};
                #pragma unroll
                for (int q = 0; q < kMR / 2; ++q) {
                    const float2 A2 = make_float2(av[2 * q], av[2 * q + 1]);
                    #pragma unroll
                    for (int w = 0; w < 2; ++w) {
                        d[q][w] = __ffma2_rn(A2, P[w], d[q][w]);
                        x[q][w] = __ffma2_rn(A2, Q[w], x[q][w]);
                    }
                }
            }
            #pragma unroll
            for (int q = 0; q < kMR / 2; ++q)
                #pragma unroll
                for (int w = 0; w < 2; ++w) {
                    acc[2 * q][2 * w] = d[q][w].x;
                    acc[2 * q + 1][2 * w + 1] = d[q][w].y;
                    acc[2 * q][2 * w + 1] = x[q][w].x;
                    acc[2 * q + 1][2 * w] = x[q][w].y;
                }
        } else {
            #pragma unroll 2
            for (int k = 0; k < K; ++k) {
                S b[CW];
                ld_b<CW>((k < ksplit ? B0 + (size_t)k * NCOL : B1 + (size_t)(k - ksplit) * NCOL) + col0, b);
                T av[kMR];
                ld_a8(a + (size_t)k * ldA, av, avec);
                #pragma unroll
                for (int i = 0; i < kMR; ++i)
                    #pragma unroll
                    for (int j = 0; j < CW; ++j) mac(acc[i][j], av[i], b[j]);
            }
        }
        #pragma unroll
        for (int j = 0; j < CW; ++j) {
            S c[kMR];
            #pragma unroll
            for (int i = 0; i < kMR; ++i) c[i] = acc[i][j];
            store(rb * kMR, col0 + j, c);          // rows rb * kMR .. + kMR - 1 (those < M)
        }
    }
}

// C[m][col] = sum_k At[k * ldA + m] * B(k)[col]  for m < M, col < NCOL.
// B rows k < ksplit live at B0 + k * NCOL, the others at B1 + (k - ksplit) * NCOL.
// Work units are (row block of kMR rows, CW consecutive columns), spread over
// all threads of the block: each unit takes 8 operator entries per k (16-byte
// loads, cached) and CW values of the B row (one 16-byte shared-memory load),
// i.e. kMR x CW FMAs per three loads.  CW = 4 when NCOL is a multiple of 4
// (B rows then start 16-byte aligned), else 1.  Every thread must call it
// (no barrier inside); rows >= M of the last block read zero-padded operator
// entries and are dropped by the store functor.  PAIRED (FP32, CW = 4): the
// paired FP32 FMA, bit-identical sums; it pays where the GEMM is issue-bound
// (the interpolation kernel) and not where the tile is latency-bound.
template <typename S, typename T, bool PAIRED = false, typename Store>
__device__ __forceinline__ void tile_gemm(const T* __restrict__ At, int ldA, int M, int K, const S* B0, int ksplit,
                                          const S* B1, int NCOL, Store store) {
    if (NCOL % 4 == 0 && aligned16(B0) && aligned16(B1))
        tile_gemm_cw<4, PAIRED>(At, ldA, M, K, B0, ksplit, B1, NCOL, store);
    else
        tile_gemm_cw<1, false>(At, ldA, M, K, B0, ksplit, B1, NCOL, store);
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

// Block and tile of the global tile g of a work table (false past the last
// tile).  Every thread of a CTA gets the same answer for the same g.
template <typename T>
__device__ __forceinline__ bool locate(const KTable<T>& tab, int kind, int g, int& b, int& tile) {
    for (int i = 0; i < tab.nblocks; ++i) {
        const KBlock<T>& B = tab.blocks[i];
        const int te = tile_width(B, kind);
        const int n = (B.nelem + te - 1) / te;
        if (g < n) {
            b = i;
            tile = g;
            return true;
        }
        g -= n;
    }
    return false;
}

}  // namespace

// ---------------------------------------------------------------------------
// u_fe = M0 U for every element of every block of the table, written to UFE.
template <typename T, int V>
__global__ void __launch_bounds__(256) k_interp_ext(KTable<T> tab, const T* __restrict__ U, T* __restrict__ UFE,
                                                    int64_t Ftot) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* Us = reinterpret_cast<T*>(smem_raw);
    for (int gt = blockIdx.x;; gt += gridDim.x) {
        int bi, tile;
        if (!locate(tab, TK_INTERP, gt, bi, tile)) break;
        const KBlock<T>& B = tab.blocks[bi];
        const int TE = B.te_interp;
        const int NCOL = V * TE;
        const int e0 = tile * TE;
        __syncthreads();
        load_tile<T, T, V>(B, U, nullptr, e0, TE, Us);
        __syncthreads();
        tile_gemm<T, T, true>(B.Ai, B.Mi_pad, B.nfe, B.nsol, Us, B.nsol, Us, NCOL,
                        [&](int m0, int col, const T* acc) {
                            const int v = col / TE, te = col - v * TE, e = e0 + te;
                            if (e >= B.nelem) return;
                            #pragma unroll
                            for (int i = 0; i < kMR; ++i)
                                if (m0 + i < B.nfe)
                                    UFE[(size_t)v * Ftot + B.fe_base + (size_t)(m0 + i) * B.ld + e] = acc[i];
                        });
    }
}

// ---------------------------------------------------------------------------
// Fluxes of one system at one point.
template <int SYS>
constexpr bool is_gas() { return SYS == SYS_EULER || SYS == SYS_NS; }
template <int SYS>
constexpr bool is_viscous() { return SYS == SYS_ADVDIFF || SYS == SYS_NS; }

template <int SYS, int RIE, int ND, typename S, typename T>
__device__ __forceinline__ void common_flux(const S* uL, const S* uR, const T* n, const KPhys<T>& P, S* F) {
    if constexpr (is_gas<SYS>()) {
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
    if constexpr (is_gas<SYS>()) {
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

// Stage update of the kMR rows m0 + i (< nrows) of one column: value at
// base + (m0 + i) * rstride.  Loads are issued before stores (the state arrays
// are distinct but the compiler cannot prove it).
template <typename T>
__device__ __forceinline__ void epilogue_rows(const KEpi<T>& E, const T* acc, const T* minv, size_t istride,
                                              size_t base, size_t rstride, int m0, int nrows) {
    // minv: 1/det J of solution point 0; point m at minv[m * istride] (0: one value)
    const T inv0 = -__ldg(minv);
    T a[kMR], b[kMR];
    const bool need_u0 = E.mode == EPI_RK_FIRST || E.mode == EPI_RK_MID;
    const bool need_acc = E.mode == EPI_RK_MID || E.mode == EPI_RK_LAST;
    #pragma unroll
    for (int i = 0; i < kMR; ++i) {
        const bool ok = m0 + i < nrows;
        const size_t idx = base + (size_t)(m0 + i) * rstride;
        a[i] = (ok && need_u0) ? __ldg(E.u0 + idx) : T(0);
        b[i] = (ok && need_acc) ? E.uacc[idx] : T(0);
    }
    bool bad = false;
    #pragma unroll
    for (int i = 0; i < kMR; ++i) {
        if (m0 + i >= nrows) continue;
        const size_t idx = base + (size_t)(m0 + i) * rstride;
        const T inv = istride ? -__ldg(minv + (size_t)(m0 + i) * istride) : inv0;
        const T r = acc[i] * inv;
        bad |= !isfinite(r);
        switch (E.mode) {
            case EPI_STORE: E.out[idx] = r; break;
            case EPI_RK_FIRST:
                E.uacc[idx] = fma(E.cacc, r, a[i]);
                E.unext[idx] = fma(E.cnext, r, a[i]);
                break;
            case EPI_RK_MID:
                E.uacc[idx] = fma(E.cacc, r, b[i]);
                E.unext[idx] = fma(E.cnext, r, a[i]);
                break;
            default: E.out[idx] = fma(E.cacc, r, b[i]); break;
        }
    }
    if (bad) atomicOr(E.flag, 1);
}
template <typename T>
__device__ __forceinline__ void epilogue_rows(const KEpi<T>& E, const Dual<T>* acc, const T* minv, size_t istride,
                                              size_t base, size_t rstride, int m0, int nrows) {
    const T inv0 = -__ldg(minv);
    bool bad = false;
    #pragma unroll
    for (int i = 0; i < kMR; ++i) {
        if (m0 + i >= nrows) continue;
        const T inv = istride ? -__ldg(minv + (size_t)(m0 + i) * istride) : inv0;
        const T d = acc[i].d * inv;
        bad |= !isfinite(d);
        E.out[base + (size_t)(m0 + i) * rstride] = d;
    }
    if (bad) atomicOr(E.flag, 1);
}

template <typename S, typename T, int V>
__device__ __forceinline__ void gather_partner(const T* UFE, const T* dUFE, int64_t Ftot, int fp, S* out) {
    #pragma unroll
    for (int v = 0; v < V; ++v) out[v] = load_state<S, T>(UFE, dUFE, (size_t)v * Ftot + fp);
}

// Viscous flux f_v[d][v] (ND x V) of a viscous system from u (V) and the
// physical gradient q[d][v].
template <int SYS, int ND, int V, typename S, typename T>
__device__ __forceinline__ void viscous_flux(const S* u, const S (*q)[V], const KPhys<T>& P, S (*fv)[V]) {
    if constexpr (SYS == SYS_NS) {
        ns_viscous<S, T, ND>(u, q, P.mu, P.gamma, P.prandtl, fv);
    } else {
        #pragma unroll
        for (int d = 0; d < ND; ++d) fv[d][0] = (-P.mu) * q[d][0];
    }
}

// n . f_v for an arbitrary vector n.
template <int ND, int V, typename S, typename NV>
__device__ __forceinline__ void viscous_normal(const S (*fv)[V], const NV* n, S* out) {
    #pragma unroll
    for (int v = 0; v < V; ++v) {
        S a = fv[0][v] * n[0];
        #pragma unroll
        for (int d = 1; d < ND; ++d) a = a + fv[d][v] * n[d];
        out[v] = a;
    }
}

// Gradient states (ND x V) of one point: q[d][v] at base + (d * V + v) * stride.
template <int ND, int V, typename S, typename T>
__device__ __forceinline__ void load_grad(const T* Q, const T* dQ, size_t base, size_t stride, S (*q)[V]) {
    #pragma unroll
    for (int d = 0; d < ND; ++d)
        #pragma unroll
        for (int v = 0; v < V; ++v) q[d][v] = load_state<S, T>(Q, dQ, base + (size_t)(d * V + v) * stride);
}

// Full residual of one block (S = T: value; S = Dual<T>: JVP).  Viscous systems
// read the physical gradients at the flux points from Q (written by k_grad).
template <typename S, typename T, int V, int ND, int SYS, int RIE>
__global__ void __launch_bounds__(256, (std::is_same<S, float>::value && (SYS == SYS_EULER || SYS == SYS_ADVECTION))
                                               ? 3    // inviscid FP32: three CTAs per SM (a few spills; measured faster)
                                               : 1) k_residual(KTable<T> tab, const T* __restrict__ U, const T* __restrict__ dU,
                                                  const T* __restrict__ UFE, const T* __restrict__ dUFE, int64_t Ftot,
                                                  KPhys<T> P, KEpi<T> E, KVisc<T> Q) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool dual = !std::is_same<S, T>::value;
    constexpr int kind = dual ? TK_RES_DUAL : TK_RES;
    for (int gt = blockIdx.x;; gt += gridDim.x) {
        int bi, tile;
        if (!locate(tab, kind, gt, bi, tile)) break;
        const KBlock<T>& B = tab.blocks[bi];
        const int TE = tile_width(B, kind);
        const int NCOL = V * TE;
        const int rowsA = B.nsol > B.nfi ? B.nsol : B.nfi;
        S* RA = reinterpret_cast<S*>(smem_raw);         // U tile, then internal F~ (rowsA rows)
        S* RB = RA + (size_t)rowsA * NCOL;               // [u_fe; u_fiu], F~_fe in place of u_fe
        const int e0 = tile * TE;
        __syncthreads();
        load_tile<S, T, V>(B, U, dU, e0, TE, RA);
        __syncthreads();
        // [u_fe; u_fiu] = [M0; M12] U
        tile_gemm<S, T>(B.Ai, B.Mi_pad, B.Mi, B.nsol, RA, B.nsol, RA, NCOL,
                        [&](int m0, int col, const S* acc) {
                            #pragma unroll
                            for (int i = 0; i < kMR; ++i)
                                if (m0 + i < B.Mi) RB[(size_t)(m0 + i) * NCOL + col] = acc[i];
                        });
        __syncthreads();
        // External points: common flux with the partner state.
        for (int it = threadIdx.x; it < B.nfe * TE; it += blockDim.x) {
            const int sg = it / TE;
            const int te = it - sg * TE;
            const int e = min(e0 + te, B.nelem - 1);
            const int f = __ldg(B.fe_face + sg);
            const int mrow = B.mr_f + f * B.mr_ff + sg * B.mr_fp;
            T n[ND];
            #pragma unroll
            for (int c = 0; c < ND; ++c) n[c] = __ldg(B.metric + (size_t)(mrow + c) * B.ld + e);
            const T s = __ldg(B.metric + (size_t)(mrow + ND) * B.ld + e);
            S own[V], nbr[V], F[V];
            #pragma unroll
            for (int v = 0; v < V; ++v) own[v] = RB[(size_t)sg * NCOL + v * TE + te];
            const int fp = __ldg(B.map + (size_t)sg * B.ld + e);
            gather_partner<S, T, V>(UFE, dUFE, Ftot, fp, nbr);
            const bool left = s > T(0);       // this point is on its face's L side
            {
                S uL[V], uR[V];
                orient<V>(left, own, nbr, uL, uR);
                common_flux<SYS, RIE, ND>(uL, uR, n, P, F);
            }
            if constexpr (is_viscous<SYS>()) {
                // LDG flux n.[(1/2 + beta) f_v(u_L, q_L) + (1/2 - beta) f_v(u_R, q_R)] + eta (u_L - u_R).
                const size_t own_q = (size_t)B.fe_base + (size_t)sg * B.ld + e;
                S q[ND][V], fv[ND][V], g[V];
                load_grad<ND, V, S, T>(Q.qfe, Q.dqfe, own_q, (size_t)Ftot, q);
                viscous_flux<SYS, ND, V, S, T>(own, q, P, fv);
                viscous_normal<ND, V, S, T>(fv, n, g);
                const T wo = left ? T(0.5) + P.beta : T(0.5) - P.beta;
                #pragma unroll
                for (int v = 0; v < V; ++v) F[v] = F[v] + wo * g[v];
                load_grad<ND, V, S, T>(Q.qfe, Q.dqfe, (size_t)fp, (size_t)Ftot, q);
                viscous_flux<SYS, ND, V, S, T>(nbr, q, P, fv);
                viscous_normal<ND, V, S, T>(fv, n, g);
                const T wn = T(1) - wo;
                const T eo = left ? P.eta : -P.eta;
                #pragma unroll
                for (int v = 0; v < V; ++v) F[v] = F[v] + wn * g[v] + eo * (own[v] - nbr[v]);
            }
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
            S fv[ND][V];
            if constexpr (is_viscous<SYS>()) {
                S q[ND][V];
                load_grad<ND, V, S, T>(Q.qfiu, Q.dqfiu,
                                       (size_t)B.qfiu_off + (size_t)k * (ND * V) * B.ld + e, (size_t)B.ld, q);
                viscous_flux<SYS, ND, V, S, T>(u, q, P, fv);
            }
            const int4 tab = __ldg(reinterpret_cast<const int4*>(B.fi_tab) + k);
            const int dofs[3] = {tab.y, tab.z, tab.w};
            for (int q = 0; q < tab.x; ++q) {
                const int nu = dofs[q] & 0xffff;
                const int ax = dofs[q] >> 16;
                T Srow[ND];
                #pragma unroll
                for (int i = 0; i < ND; ++i)
                    Srow[i] = __ldg(B.metric + (size_t)(B.mr_si + k * B.mr_sik + ax * ND + i) * B.ld + e);
                S Ft[V];
                internal_flux<SYS, ND>(u, Srow, P, Ft);
                if constexpr (is_viscous<SYS>()) {
                    S g[V];
                    viscous_normal<ND, V, S, T>(fv, Srow, g);
                    #pragma unroll
                    for (int v = 0; v < V; ++v) Ft[v] = Ft[v] + g[v];
                }
                #pragma unroll
                for (int v = 0; v < V; ++v) RA[(size_t)nu * NCOL + v * TE + te] = Ft[v];
            }
        }
        __syncthreads();
        // R~ = [M14 | M13] [F~_fe; F~_fi];  dU/dt = -R~ / det J
        tile_gemm<S, T>(B.Ad, B.Md_pad, B.nsol, B.nfe + B.nfi, RB, B.nfe, RA, NCOL,
                        [&](int m0, int col, const S* acc) {
                            const int v = col / TE, te = col - v * TE, e = e0 + te;
                            if (e >= B.nelem) return;
                            epilogue_rows(E, acc, B.metric + e,
                                          (size_t)B.mr_inv * B.ld, (size_t)B.u_off + (size_t)v * B.ld + e,
                                          (size_t)V * B.ld, m0, B.nsol);
                        });
    }
}

// Launch of one k_residual instantiation (host side).
template <typename S, typename T, int V, int ND, int SYS, int RIE>
inline void launch_res_impl(const KTable<T>& tab, const T* U, const T* dU, const T* UFE, const T* dUFE, int64_t Ftot,
                            const KPhys<T>& P, const KEpi<T>& E, const KVisc<T>& Q, int smem, int tiles, int nsm,
                            cudaStream_t st) {
    auto k = k_residual<S, T, V, ND, SYS, RIE>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k<<<persistent_grid(k, smem, tiles, nsm), 256, smem, st>>>(tab, U, dU, UFE, dUFE, Ftot, P, E, Q);
}

}  // namespace sdrt
