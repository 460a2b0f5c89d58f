// Fused SDRT stage kernel with the element type's operators compiled in
// (sm_103a, FP32).  Included by the per-element-type translation units that
// csrc/gen/opgen.cpp writes at build time; K supplies the operator code:
//   K::NS, NFE, NG, GR          sizes, number of flux-point groups, the largest
//                                group's point + DOF rows
//   K::Grp<g>::interp(u, ldu, x, ldx)   point states of group g, x = A_g u
//                                        (rows of [M0; M12], structural
//                                        non-zeros only, FP32 immediates)
//   K::Grp<g>::div(f, ldf, r)   r += D_g f (columns of [M14 | M13] of the
//                                group's DOFs)
//   K::desc(i)                  point descriptors: external point sigma and
//                                its face, or internal point with its DOF axes,
//                                and the first DOF row of the point
//   K::ext(w, o, ldo)           o = M0 w (external points)
//
// A CTA works on a tile of 32 consecutive elements of one block with V warps:
// thread (lane, v) owns variable v of element e0 + lane for the operator
// applications (one column of the paper's state matrix, App. B), and the
// threads share the tile's points for the flux evaluation:
//   1. the tile's state, metric rows and partner map go to shared memory
//      with asynchronous copies (coalesced rows);
//   2. per group: the partners' states of its external points are copied
//      asynchronously (face records FRin) while the group is interpolated
//      (each thread its column); then the common fluxes at external points
//      (Sec. 2.1) and the normal transformed fluxes at internal DOFs (Eq.
//      "normal_transformed_flux"), then the divergence accumulated in
//      registers, column by column;
//   3. dU/dt = -R~ / det J, the RK stage epilogue, and (FRout) the new state's
//      external-point values, staged in shared memory and written as the
//      tile's contiguous face records.
#pragma once

#include "flux_rec.cuh"
#include "gen_api.hpp"
#include "generic.cuh"

namespace sdrt {
namespace gen {

constexpr int TE = 32;   // elements per tile (one per lane)

template <class K, int V>
struct Smem {
    static constexpr int LDX = V * TE;                       // row stride (values) of US / group rows
    static constexpr int NM = 1 + 9 + K::NF * 4;             // metric rows (3D, kargs.hpp layout)
    static constexpr int NREC = K::NFE * V;                  // values of one element's face records
    static constexpr int PADREC = NREC % 2 == 0 ? NREC + 1 : NREC;   // odd: conflict-free staging
    static constexpr int STAGE = TE * PADREC;
    // [US: NS rows][group rows: GR][metric: NM x TE][partner map: NFE x TE (int)]
    static constexpr int US = 0;
    static constexpr int XS = K::NS * LDX;
    static constexpr int MS = XS + K::GR * LDX;
    static constexpr int PM = MS + NM * TE;
    static constexpr int MAIN = PM + K::NFE * TE;
    static constexpr int FLOATS = MAIN > STAGE ? MAIN : STAGE;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// 4-byte asynchronous global -> shared copy (no register staging).
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// External-point values of the tile (thread (lane, v) holds w[NS] of its
// column) into the face-record array: staged per element with an odd stride,
// then written as one contiguous run (the tile's elements are consecutive).
template <class K, int V>
__device__ __forceinline__ void write_records(const float (&w)[K::NS], float* S, float* dst, int nvalid, int v,
                                              int lane) {
    using SM = Smem<K, V>;
    K::ext(w, S + lane * SM::PADREC + v, V);
    __syncthreads();
    const int n = nvalid * SM::NREC;
    for (int i = threadIdx.x; i < n; i += V * TE) {
        const int el = i / SM::NREC;
        dst[i] = S[el * SM::PADREC + (i - el * SM::NREC)];
    }
}

// One group of flux points: the partners' states of its external points are
// copied asynchronously into the DOF-flux rows those points will overwrite
// (each item's copy and use by the same thread), overlapping the
// interpolation; then the fluxes, then the divergence.
template <class K, int V, int SYS, int RIE, int G>
__device__ __forceinline__ void run_groups(const GenArgs& a, float* sm, float (&acc)[K::NS], int v, int lane) {
    using Grp = typename K::template Grp<G>;
    using SM = Smem<K, V>;
    constexpr int LDX = V * TE, ND = 3, ND2 = ND * ND;
    const float* US = sm + SM::US;
    float* XS = sm + SM::XS;
    float* FS = XS + Grp::NP * LDX;
    const float* MS = sm + SM::MS;
    const int* PM = reinterpret_cast<const int*>(sm + SM::PM);
    __syncthreads();                                    // previous group's rows consumed
    for (int it = threadIdx.x; it < Grp::NP * TE; it += V * TE) {
        const int4 d = K::desc(Grp::OFF + (it >> 5));
        if (d.x >= 0) {
            const int te = it & 31;
            const float* src = a.FRin + PM[d.x * TE + te];
            #pragma unroll
            for (int q = 0; q < V; ++q) cp_async4(FS + (d.z * V + q) * TE + te, src + q);
        }
    }
    Grp::interp(US + v * TE + lane, LDX, XS + v * TE + lane, LDX);
    cp_async_wait_all();
    __syncthreads();
    for (int it = threadIdx.x; it < Grp::NP * TE; it += V * TE) {
        const int r = it >> 5;                          // point row (warp-uniform)
        const int te = it & 31;
        const int4 d = K::desc(Grp::OFF + r);
        float u[V];
        #pragma unroll
        for (int q = 0; q < V; ++q) u[q] = XS[(r * V + q) * TE + te];
        if (d.x >= 0) {
            // external point sigma = d.x of face d.y: common flux with the partner
            const int mrow = 1 + ND2 + d.y * (ND + 1);
            float n[ND];
            #pragma unroll
            for (int c = 0; c < ND; ++c) n[c] = MS[(mrow + c) * TE + te];
            const float s = MS[(mrow + ND) * TE + te];
            float nb[V], uL[V], uR[V], F[V];
            #pragma unroll
            for (int q = 0; q < V; ++q) nb[q] = FS[(d.z * V + q) * TE + te];
            orient<V>(s > 0.f, u, nb, uL, uR);          // this point on its face's L side when s > 0
            if constexpr (SYS == SYS_EULER && RIE == RIE_RUSANOV) {
                rusanov_rec<float, ND>(uL, uR, n, a.P.gamma, s, F);   // s F, one reciprocal per state
                #pragma unroll
                for (int q = 0; q < V; ++q) FS[(d.z * V + q) * TE + te] = F[q];
            } else {
                common_flux<SYS, RIE, ND>(uL, uR, n, a.P, F);
                #pragma unroll
                for (int q = 0; q < V; ++q) FS[(d.z * V + q) * TE + te] = s * F[q];
            }
        } else {
            // internal point: one transformed flux component per DOF axis
            const int ndof = d.w & 3;
            if constexpr (SYS == SYS_EULER) {
                // primitive state once per point (one reciprocal), then n . f per axis
                float inv, vel[ND], p;
                prim_rec<float, ND>(u, a.P.gamma, inv, vel, p);
                for (int k = 0; k < ndof; ++k) {
                    const int ax = (d.w >> (2 + 2 * k)) & 3;
                    float Srow[ND];
                    #pragma unroll
                    for (int i = 0; i < ND; ++i) Srow[i] = MS[(1 + ax * ND + i) * TE + te];
                    float vn = vel[0] * Srow[0];
                    #pragma unroll
                    for (int i = 1; i < ND; ++i) vn = fmaf(vel[i], Srow[i], vn);
                    float* o = FS + (d.z + k) * V * TE + te;
                    o[0] = u[0] * vn;
                    #pragma unroll
                    for (int i = 0; i < ND; ++i) o[(1 + i) * TE] = fmaf(u[1 + i], vn, p * Srow[i]);
                    o[(V - 1) * TE] = (u[V - 1] + p) * vn;
                }
            } else {
                for (int k = 0; k < ndof; ++k) {
                    const int ax = (d.w >> (2 + 2 * k)) & 3;
                    float Srow[ND], Ft[V];
                    #pragma unroll
                    for (int i = 0; i < ND; ++i) Srow[i] = MS[(1 + ax * ND + i) * TE + te];
                    internal_flux<SYS, ND>(u, Srow, a.P, Ft);
                    #pragma unroll
                    for (int q = 0; q < V; ++q) FS[((d.z + k) * V + q) * TE + te] = Ft[q];
                }
            }
        }
    }
    __syncthreads();
    Grp::div(FS + v * TE + lane, LDX, acc);
    if constexpr (G + 1 < K::NG) run_groups<K, V, SYS, RIE, G + 1>(a, sm, acc, v, lane);
}

template <class K, int V, int SYS, int RIE>
__global__ void __launch_bounds__(V * TE, 2) k_gen_stage(const GenArgs a) {
    extern __shared__ __align__(16) float smem[];
    using SM = Smem<K, V>;
    constexpr int NS = K::NS;
    const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const KEpi<float>& E = a.E;
    for (int tile = blockIdx.x; tile * TE < a.nelem; tile += gridDim.x) {
        const int e0 = tile * TE;
        const bool valid = e0 + lane < a.nelem;
        const int e = valid ? e0 + lane : a.nelem - 1;  // lanes past the end repeat the last element
        __syncthreads();                                // previous tile's shared memory free
        // The tile's state, metric rows and partner map, copied asynchronously.
        #pragma unroll 4
        for (int r = 0; r < NS; ++r)
            cp_async4(smem + SM::US + (r * V + v) * TE + lane, a.U + a.u_off + (size_t)(r * V + v) * a.ld + e);
        for (int i = threadIdx.x; i < SM::NM * TE; i += V * TE) {
            const int k = i >> 5, te = i & 31;
            cp_async4(smem + SM::MS + i, a.metric + (size_t)k * a.ld + min(e0 + te, a.nelem - 1));
        }
        for (int i = threadIdx.x; i < K::NFE * TE; i += V * TE) {
            const int k = i >> 5, te = i & 31;
            cp_async4(smem + SM::PM + i, a.pmap + (size_t)k * a.ld + min(e0 + te, a.nelem - 1));
        }
        cp_async_wait_all();
        float acc[NS];
        #pragma unroll
        for (int r = 0; r < NS; ++r) acc[r] = 0.f;
        run_groups<K, V, SYS, RIE, 0>(a, smem, acc, v, lane);   // its first barrier publishes the copies
        // dU/dt = -R~ / det J and the stage update; acc becomes the new state.
        const float inv = -smem[SM::MS + lane];
        bool bad = false;
        const size_t base = a.u_off + (size_t)v * a.ld + e;
        const size_t rs = (size_t)V * a.ld;           // row stride of one solution point
        if (E.mode == EPI_STORE) {
            #pragma unroll
            for (int r = 0; r < NS; ++r) {
                acc[r] *= inv;
                bad |= !isfinite(acc[r]);
                if (valid) E.out[base + r * rs] = acc[r];
            }
        } else if (E.mode == EPI_RK_FIRST) {
            #pragma unroll
            for (int r = 0; r < NS; ++r) {
                const float R = acc[r] * inv;
                const float u0 = __ldg(E.u0 + base + r * rs);
                bad |= !isfinite(R);
                acc[r] = fmaf(E.cnext, R, u0);
                if (valid) {
                    E.uacc[base + r * rs] = fmaf(E.cacc, R, u0);
                    E.unext[base + r * rs] = acc[r];
                }
            }
        } else if (E.mode == EPI_RK_MID) {
            #pragma unroll
            for (int r = 0; r < NS; ++r) {
                const float R = acc[r] * inv;
                const float u0 = __ldg(E.u0 + base + r * rs);
                const float ua = E.uacc[base + r * rs];
                bad |= !isfinite(R);
                acc[r] = fmaf(E.cnext, R, u0);
                if (valid) {
                    E.uacc[base + r * rs] = fmaf(E.cacc, R, ua);
                    E.unext[base + r * rs] = acc[r];
                }
            }
        } else {
            #pragma unroll
            for (int r = 0; r < NS; ++r) {
                const float R = acc[r] * inv;
                bad |= !isfinite(R);
                acc[r] = fmaf(E.cacc, R, E.uacc[base + r * rs]);
                if (valid) E.out[base + r * rs] = acc[r];
            }
        }
        if (bad && valid) *E.flag = 1;
        if (a.FRout) {
            __syncthreads();                            // every group's shared rows consumed
            write_records<K, V>(acc, smem, a.FRout + a.fr_base + (size_t)e0 * SM::NREC, min(TE, a.nelem - e0), v,
                                lane);
        }
    }
}

template <class K, int V>
__global__ void __launch_bounds__(V * TE) k_gen_interp(const GenArgs a) {
    extern __shared__ __align__(16) float smem[];
    using SM = Smem<K, V>;
    const int v = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int tile = blockIdx.x; tile * TE < a.nelem; tile += gridDim.x) {
        const int e0 = tile * TE;
        const int e = min(e0 + lane, a.nelem - 1);
        float w[K::NS];
        #pragma unroll
        for (int r = 0; r < K::NS; ++r) w[r] = __ldg(a.U + a.u_off + (size_t)(r * V + v) * a.ld + e);
        __syncthreads();                                // previous tile's staging read
        write_records<K, V>(w, smem, a.FRout + a.fr_base + (size_t)e0 * SM::NREC, min(TE, a.nelem - e0), v, lane);
    }
}

template <class K, int V, int SYS, int RIE>
int launch_gen_v(int kind, const GenArgs& a, cudaStream_t st) {
    using SM = Smem<K, V>;
    const int tiles = (a.nelem + TE - 1) / TE;
    if (kind == 0) {
        auto k = k_gen_interp<K, V>;
        const int smem = SM::STAGE * (int)sizeof(float);
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k<<<tiles, V * TE, smem, st>>>(a);
    } else {
        auto k = k_gen_stage<K, V, SYS, RIE>;
        const int smem = SM::FLOATS * (int)sizeof(float);
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k<<<tiles, V * TE, smem, st>>>(a);
    }
    return 0;
}

// Instantiated combinations: 3D Euler with the Rusanov flux (five variables).
template <class K>
int launch_gen(int kind, const GenArgs& a, int V, int sys, int rie, int /*nsm*/, cudaStream_t st) {
    if (V == 5 && sys == SYS_EULER && rie == RIE_RUSANOV) return launch_gen_v<K, 5, SYS_EULER, RIE_RUSANOV>(kind, a, st);
    return -1;
}

}  // namespace gen
}  // namespace sdrt
