// Fused SDRT stage kernel with the element type's operators compiled in
// (sm_103a, FP32).  Included by the per-element-type translation units that
// csrc/gen/opgen.cpp writes at build time; K supplies the operator code:
//   K::NS, NFE, NG, GR          sizes, number of flux-point groups, the largest
//                                group's point + DOF rows
//   K::SPLIT, NSH               threads per (element, variable) column and the
//                                divergence rows each of them owns
//   K::Grp<g>::interp(h, u, x, ldx)  point states of group g, x = A_g u,
//                                        part h of the rows (rows of
//                                        [M0; M12], structural non-zeros
//                                        only, FP32 immediates)
//   K::Grp<g>::div(h, f, ldf, r)  r += D_g f for the rows of part h (columns
//                                of [M14 | M13] of the group's DOFs)
//   K::desc(i)                  point descriptors: external point sigma and
//                                its face, or internal point with its DOF axes,
//                                and the first DOF row of the point
//   K::ext(c, h, u, x, ldx)     x = M0 u for chunk c of the external points,
//                                part h
//
// A CTA works on a tile of 32 consecutive elements of one block with
// SPLIT x V warps: thread (lane, v, h) owns part h of the rows of variable v
// of element e0 + lane for the operator applications (one column of the
// paper's state matrix, App. B), and the threads share the tile's points for
// the flux evaluation.  Persistent CTAs walk the tiles and prefetch the next
// tile's rows into L2:
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
    static constexpr int NT = K::SPLIT * V * TE;             // threads of a CTA
    static constexpr int LDX = V * TE;                       // row stride (values) of US / group rows
    static constexpr int NM = 1 + 9 + K::NF * 4;             // metric rows (3D, kargs.hpp layout)
    // The tile's state US is stored column by column, [V][TE][CS]: each
    // thread's solution column contiguous (float4 reads), CS = 4 k with k odd
    // so that the 16-byte reads of 8 consecutive lanes hit distinct banks.
    static constexpr int CS = (K::NS + 3) / 4 % 2 ? (K::NS + 3) / 4 * 4 : (K::NS + 3) / 4 * 4 + 4;
    // [US: V TE CS][group rows: GR][metric: NM x TE][partner map: NFE x TE (int)]
    static constexpr int US = 0;
    static constexpr int XS = V * TE * CS;
    static constexpr int MS = XS + K::GR * LDX;
    static constexpr int PM = MS + NM * TE;
    static constexpr int MAIN = PM + K::NFE * TE;
    // face-record staging of one chunk of ECH external points per element
    // (odd element stride: conflict-free), after US
    static constexpr int CREC = K::ECH * V;
    static constexpr int PADREC = CREC % 2 == 0 ? CREC + 1 : CREC;
    static constexpr int STAGE_END = XS + TE * PADREC;
    static constexpr int FLOATS = MAIN > STAGE_END ? MAIN : STAGE_END;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// 4-byte asynchronous global -> shared copy (no register staging).
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// 16-byte asynchronous copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// The tile's rows of a [rows][ld] array (element fastest) into shared memory,
// [rows][TE], with asynchronous copies.  A full tile of an array whose start
// is 16-byte aligned moves each row as eight 16-byte copies (ld and the block
// offsets are multiples of 32 elements); otherwise, and on the last, partial
// tile, value by value, the lanes past the end repeating the last element.
template <int NT, typename E>
__device__ __forceinline__ void stage_rows(E* dst, const E* src, int rows, int ld, int e0, int nelem) {
    if (e0 + TE <= nelem && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
        for (int i = threadIdx.x; i < rows * (TE / 4); i += NT)
            cp_async16(dst + 4 * i, src + (size_t)(i >> 3) * ld + e0 + 4 * (i & 7));
    } else {
        for (int i = threadIdx.x; i < rows * TE; i += NT)
            cp_async4(dst + i, src + (size_t)(i >> 5) * ld + min(e0 + (i & 31), nelem - 1));
    }
}
// The tile's state (rows (rho, v) of a block's [N_s][V][ld] array) into the
// column layout [V][TE][CS] with asynchronous copies; lanes past the end
// repeat the last element.  A warp's copies take 8 consecutive elements of 4
// consecutive rows rho of one variable: with CS an odd multiple of 4 the 32
// destinations fall on 32 distinct banks (eight 32-byte row segments read).
template <int NT, int NS, int V, int CS>
__device__ __forceinline__ void stage_state(float* dst, const float* src, int ld, int e0, int nelem) {
    constexpr int RG = (NS + 3) / 4;                    // groups of 4 rows rho
    for (int i = threadIdx.x; i < RG * V * TE * 4; i += NT) {
        const int lane = i & 31, w = i >> 5;
        const int te = (w & 3) * 8 + (lane & 7);
        const int q = w >> 2;                           // (rho group, v), v fastest
        const int rg = q / V, v = q - rg * V;
        const int rho = rg * 4 + (lane >> 3);
        if (rho < NS)
            cp_async4(dst + (v * TE + te) * CS + rho,
                      src + (size_t)(rho * V + v) * ld + min(e0 + te, nelem - 1));
    }
}

// L2 prefetch of the same rows for a later tile (one 128-byte line per row).
template <int NT, typename E>
__device__ __forceinline__ void prefetch_rows(const E* src, int rows, int ld, int e0) {
    for (int i = threadIdx.x; i < rows; i += NT) prefetch_l2(src + (size_t)i * ld + e0);
}

// The external-point values of the tile's state (in US) into the face-record
// array, chunk by chunk: each chunk staged per element with an odd stride and
// written point by point, the tile's records being one contiguous block
// (dst: the tile's records, [point][element of the tile][variable]).
template <class K, int V>
__device__ __forceinline__ void write_records(float* sm, float* dst, int nvalid, int v, int h, int lane) {
    using SM = Smem<K, V>;
    float* S = sm + SM::XS;
    #pragma unroll 1
    for (int c = 0; c < K::NECH; ++c) {
        const int c0 = c * K::ECH;
        const int rows = min(K::ECH, K::NFE - c0);
        __syncthreads();                                // staging free, US complete
        K::ext(c, h, sm + SM::US + (v * TE + lane) * SM::CS, S + lane * SM::PADREC + v, V);
        __syncthreads();
        constexpr int RUN = TE * V;                     // one point's values of the tile
        for (int i = threadIdx.x; i < rows * RUN; i += SM::NT) {
            const int pt = i / RUN;
            const int j = i - pt * RUN;
            const int el = j / V;
            if (el < nvalid) dst[(size_t)(c0 + pt) * RUN + j] = S[el * SM::PADREC + pt * V + (j - el * V)];
        }
    }
}

// One group of flux points: the partners' states of its external points are
// copied asynchronously into the DOF-flux rows those points will overwrite
// (each item's copy and use by the same thread), overlapping the
// interpolation; then the fluxes, then the divergence.
template <class K, int V, int SYS, int RIE, int G>
__device__ __forceinline__ void run_groups(const GenArgs& a, float* sm, float (&acc)[K::NSH], int v, int h, int lane) {
    using Grp = typename K::template Grp<G>;
    using SM = Smem<K, V>;
    constexpr int LDX = V * TE, ND = 3, ND2 = ND * ND, NT = SM::NT;
    const float* US = sm + SM::US;
    float* XS = sm + SM::XS;
    float* FS = XS + Grp::NP * LDX;
    const float* MS = sm + SM::MS;
    const int* PM = reinterpret_cast<const int*>(sm + SM::PM);
    __syncthreads();                                    // previous group's rows consumed
    for (int it = threadIdx.x; it < Grp::NP * TE; it += NT) {
        const int4 d = K::desc(Grp::OFF + (it >> 5));
        if (d.x >= 0) {
            const int te = it & 31;
            const float* src = a.FRin + PM[d.x * TE + te];
            #pragma unroll
            for (int q = 0; q < V; ++q) cp_async4(FS + (d.z * V + q) * TE + te, src + q);
        }
    }
    Grp::interp(h, US + (v * TE + lane) * SM::CS, XS + v * TE + lane, LDX);
    cp_async_wait_all();
    __syncthreads();
    for (int it = threadIdx.x; it < Grp::NP * TE; it += NT) {
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
    Grp::div(h, FS + v * TE + lane, LDX, acc);
    if constexpr (G + 1 < K::NG) run_groups<K, V, SYS, RIE, G + 1>(a, sm, acc, v, h, lane);
}

// CTAs per SM the stage kernel is compiled for (the register cap follows):
// as many as its shared memory allows, at most 5 for the element types with
// one thread per column (5 x 160 threads at <= 72 registers, no spills) and 3
// for those with two (3 x 320 threads at <= 64 registers).
template <class K, int V>
constexpr int stage_min_blocks() {
    constexpr int fit = (228 * 1024) / (Smem<K, V>::FLOATS * (int)sizeof(float) + 1024);
    constexpr int want = K::SPLIT > 1 ? 3 : 5;
    return fit < 1 ? 1 : fit < want ? fit : want;
}

template <class K, int V, int SYS, int RIE>
__global__ void __launch_bounds__(K::SPLIT * V * TE, (stage_min_blocks<K, V>())) k_gen_stage(const GenArgs a) {
    extern __shared__ __align__(16) float smem[];
    using SM = Smem<K, V>;
    constexpr int NS = K::NS, NSH = K::NSH, NT = SM::NT;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int v = w % V, h = w / V;                      // thread (lane, v, h): rows of part h of column (e, v)
    const KEpi<float>& E = a.E;
    const float* Ub = a.U + a.u_off;
    for (int tile = blockIdx.x; tile * TE < a.nelem; tile += gridDim.x) {
        const int e0 = tile * TE;
        const bool valid = e0 + lane < a.nelem;
        const int e = valid ? e0 + lane : a.nelem - 1;  // lanes past the end repeat the last element
        __syncthreads();                                // previous tile's shared memory free
        // The tile's state, metric rows and partner map, copied asynchronously;
        // the next tile's rows prefetched into L2 meanwhile.
        stage_state<NT, NS, V, SM::CS>(smem + SM::US, Ub, a.ld, e0, a.nelem);
        stage_rows<NT>(smem + SM::MS, a.metric, SM::NM, a.ld, e0, a.nelem);
        stage_rows<NT>(reinterpret_cast<int*>(smem + SM::PM), a.pmap, K::NFE, a.ld, e0, a.nelem);
        const int en = (tile + gridDim.x) * TE;
        if (en < a.nelem) {
            prefetch_rows<NT>(Ub, NS * V, a.ld, en);
            prefetch_rows<NT>(a.metric, SM::NM, a.ld, en);
            prefetch_rows<NT>(a.pmap, K::NFE, a.ld, en);
        }
        // The RK inputs of this tile's epilogue into L2 while the groups run.
        if (E.mode == EPI_RK_FIRST || E.mode == EPI_RK_MID)
            prefetch_rows<NT>(E.u0 + a.u_off, NS * V, a.ld, e0);
        if (E.mode == EPI_RK_MID || E.mode == EPI_RK_LAST)
            prefetch_rows<NT>(E.uacc + a.u_off, NS * V, a.ld, e0);
        cp_async_wait_all();
        __syncthreads();
        // The partners' face records of the whole tile into L2 (the map has
        // arrived), ahead of the groups' copies into shared memory.
        {
            const int* PMt = reinterpret_cast<const int*>(smem + SM::PM);
            for (int i = threadIdx.x; i < K::NFE * TE; i += NT) prefetch_l2(a.FRin + PMt[i]);
        }
        float acc[NSH];
        #pragma unroll
        for (int r = 0; r < NSH; ++r) acc[r] = 0.f;
        run_groups<K, V, SYS, RIE, 0>(a, smem, acc, v, h, lane);   // its first barrier publishes the copies
        // dU/dt = -R~ / det J and the stage update of this thread's rows
        // rho = h NSH + r; acc becomes the new state.
        const float inv = -smem[SM::MS + lane];
        bool bad = false;
        const size_t rs = (size_t)V * a.ld;           // row stride of one solution point
        const size_t base = a.u_off + (size_t)v * a.ld + e + (size_t)(h * NSH) * rs;
        const int nrow = min(NSH, NS - h * NSH);
        if (E.mode == EPI_STORE) {
            #pragma unroll
            for (int r = 0; r < NSH; ++r) {
                if (r >= nrow) break;
                acc[r] *= inv;
                bad |= !isfinite(acc[r]);
                if (valid) E.out[base + r * rs] = acc[r];
            }
        } else if (E.mode == EPI_RK_FIRST) {
            #pragma unroll
            for (int r = 0; r < NSH; ++r) {
                if (r >= nrow) break;
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
            for (int r = 0; r < NSH; ++r) {
                if (r >= nrow) break;
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
            for (int r = 0; r < NSH; ++r) {
                if (r >= nrow) break;
                const float R = acc[r] * inv;
                bad |= !isfinite(R);
                acc[r] = fmaf(E.cacc, R, E.uacc[base + r * rs]);
                if (valid) E.out[base + r * rs] = acc[r];
            }
        }
        if (bad && valid) atomicOr(E.flag, 1);
        if (a.FRout) {
            // the new state into US (every group has read it), then its face records
            __syncthreads();
            #pragma unroll
            for (int r = 0; r < NSH; ++r)
                if (r < nrow) smem[SM::US + (v * TE + lane) * SM::CS + h * NSH + r] = acc[r];
            write_records<K, V>(smem, a.FRout + a.fr_base + (size_t)e0 * K::NFE * V, min(TE, a.nelem - e0), v, h,
                                lane);
        }
    }
}

template <class K, int V>
__global__ void __launch_bounds__(K::SPLIT * V * TE) k_gen_interp(const GenArgs a) {
    extern __shared__ __align__(16) float smem[];
    using SM = Smem<K, V>;
    constexpr int NT = SM::NT;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int v = w % V, h = w / V;
    for (int tile = blockIdx.x; tile * TE < a.nelem; tile += gridDim.x) {
        const int e0 = tile * TE;
        __syncthreads();                                // previous tile's staging read
        stage_state<NT, K::NS, V, SM::CS>(smem + SM::US, a.U + a.u_off, a.ld, e0, a.nelem);
        cp_async_wait_all();
        write_records<K, V>(smem, a.FRout + a.fr_base + (size_t)e0 * K::NFE * V, min(TE, a.nelem - e0), v, h, lane);
    }
}

// Persistent grid: every CTA that fits on the SMs at once, at most one per tile.
template <typename Kern>
int persistent_ctas(Kern k, int threads, int smem, int tiles, int nsm) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, threads, smem) != cudaSuccess || per < 1) per = 1;
    return tiles < per * nsm ? tiles : per * nsm;
}

template <class K, int V, int SYS, int RIE>
int launch_gen_v(int kind, const GenArgs& a, int nsm, cudaStream_t st) {
    using SM = Smem<K, V>;
    const int tiles = (a.nelem + TE - 1) / TE;
    if (kind == 0) {
        auto k = k_gen_interp<K, V>;
        const int smem = SM::STAGE_END * (int)sizeof(float);
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k<<<persistent_ctas(k, SM::NT, smem, tiles, nsm), SM::NT, smem, st>>>(a);
    } else {
        auto k = k_gen_stage<K, V, SYS, RIE>;
        const int smem = SM::FLOATS * (int)sizeof(float);
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        k<<<persistent_ctas(k, SM::NT, smem, tiles, nsm), SM::NT, smem, st>>>(a);
    }
    return 0;
}

// Instantiated combinations: 3D Euler with the Rusanov flux (five variables).
template <class K>
int launch_gen(int kind, const GenArgs& a, int V, int sys, int rie, int nsm, cudaStream_t st) {
    if (V == 5 && sys == SYS_EULER && rie == RIE_RUSANOV)
        return launch_gen_v<K, 5, SYS_EULER, RIE_RUSANOV>(kind, a, nsm, st);
    return -1;
}

}  // namespace gen
}  // namespace sdrt
