// Register-blocked SDRT residual kernels for tetrahedra of degree 3 and 4
// (sm_103a), exchanging face states through per-element records staged with
// bulk asynchronous copies.
//
// One residual evaluation (paper Sec. 2.1, App. B) is two launches per block:
//   k_interp_pipe : [u_fe; u_fiu] = [M0; M12] U (Eq. "interpolation_procedure"),
//                   FP32: one producer lane streams each tile of U with a 2D
//                   tensor copy into a two-stage ring, consumer warps compute
//                   all variables of their elements' rows and assemble the
//                   records (REC: external points, FIUR: internal points) in
//                   shared memory, written with bulk stores;
//   k_interp_rec  : the same for FP64 (two threads per element, no TMA);
//   k_flux_rec    : per tile, cp.async.bulk loads (completing on an mbarrier)
//                   bring the tile's own records, the four partner face records
//                   of every element, the metric rows and the partner
//                   permutations into shared memory; G threads per element
//                   compute the common fluxes (Sec. 2.1) and the normal
//                   transformed internal fluxes (Eq. "normal_transformed_flux")
//                   of their share of the points, exchange them with warp
//                   shuffles and accumulate their share of the rows of
//                   R~ = [M14 | M13] [F~_fe; F~_fi] (Eq. "residual_sdrt_matrices")
//                   in registers (paired FP32 FMA); dU/dt = -R~ / det J goes
//                   through the fused RK4 stage epilogue.  With FUSE (RK4 stages
//                   1-3) the epilogue keeps the next stage's state in shared
//                   memory, interpolates it and writes the next stage's records
//                   into the other record buffer, so one RK4 step is one
//                   interpolation and four flux launches.
//   k_flux_rec_dual : the JVP (dual numbers), reading the records directly.
//   k_face_records  : face records between REC and the packed exchange
//                     buffers of a partitioned residual.
#include <cstdint>
#include <mutex>
#include <type_traits>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "device_math.cuh"
#include "flux_rec.cuh"
#include "kargs.hpp"
#include "launch.hpp"

namespace sdrt {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr long long kWaitLimit = 1ll << 26;   // try_wait polls before giving up (seconds of waiting)

// ---- PTX helpers: mbarrier and bulk copies -------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < kWaitLimit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
// At most n non-blocking tests of the phase with the given parity; false if
// it has not completed by then.
__device__ __forceinline__ bool mbar_test_n(uint64_t* bar, uint32_t parity, int n) {
    const uint32_t a = smem_u32(bar);
    for (int it = 0; it < n; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// Global -> shared bulk copy completing on bar (16-byte aligned, size multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// Shared -> global bulk copy (bulk-group completion).
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_u32(src)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// 16-byte shared-memory load of data that is constant for the kernel's life
// (no memory clobber: the compiler may move it across other shared stores).
__device__ __forceinline__ float4 lds128_const(const float* p) {
    float4 r;
    asm("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "r"(smem_u32(p)));
    return r;
}

// 2D tensor copy (TMA) of one box at (x, y) of the tensor map into shared memory,
// completing on bar.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
// L2 prefetch of one box of a 2D tensor (no shared memory involved).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y)
                 : "memory");
}
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// Barrier among the first `count` threads of the block (id 1; id 0 is __syncthreads).
__device__ __forceinline__ void consumer_sync(int count) {
    asm volatile("bar.sync 1, %0;" ::"r"(count) : "memory");
}
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// ---- fluxes ----------------------------------------------------------------
template <int SYS, int RIE, int ND, typename S, typename T>
__device__ __forceinline__ void common_flux_f(const S* uL, const S* uR, const T* n, const KPhys<T>& P, S* F) {
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

template <int SYS, int ND, typename S, typename T>
__device__ __forceinline__ void internal_flux_f(const S* u, const T* Srow, const KPhys<T>& P, S* Ft) {
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
__device__ __forceinline__ void epi_store(const KEpi<T>& E, size_t idx, T r) {
    if (!isfinite(r)) atomicOr(E.flag, 1);
    switch (E.mode) {
        case EPI_STORE: E.out[idx] = r; break;
        case EPI_RK_FIRST: {
            const T u0 = E.u0[idx];
            E.uacc[idx] = fma(E.cacc, r, u0);
            E.unext[idx] = fma(E.cnext, r, u0);
            break;
        }
        case EPI_RK_MID:
            E.uacc[idx] = fma(E.cacc, r, E.uacc[idx]);
            E.unext[idx] = fma(E.cnext, r, E.u0[idx]);
            break;
        default: E.out[idx] = fma(E.cacc, r, E.uacc[idx]); break;
    }
}

// Stage update of the RS x V values R = inv * acc[i][v] owned by one thread
// (rows r0 + i < nrows, variables v at base + (r * V + v) * ld).  All loads are
// issued before any store: the state arrays are distinct, but the compiler
// cannot prove it, and interleaved load/store pairs would serialise.
template <int RS, int V, typename T>
__device__ __forceinline__ void epi_block(const KEpi<T>& E, const T (&acc)[RS][V], T inv, size_t base, int ld,
                                          int r0, int nrows) {
    T a[RS][V], b[RS][V];
    const bool need_u0 = E.mode == EPI_RK_FIRST || E.mode == EPI_RK_MID;
    const bool need_acc = E.mode == EPI_RK_MID || E.mode == EPI_RK_LAST;
    #pragma unroll
    for (int i = 0; i < RS; ++i)
        #pragma unroll
        for (int v = 0; v < V; ++v) {
            const size_t idx = base + (size_t)((r0 + i) * V + v) * ld;
            const bool ok = r0 + i < nrows;
            a[i][v] = (ok && need_u0) ? __ldg(E.u0 + idx) : T(0);
            b[i][v] = (ok && need_acc) ? E.uacc[idx] : T(0);
        }
    bool bad = false;
    #pragma unroll
    for (int i = 0; i < RS; ++i) {
        if (r0 + i >= nrows) continue;
        #pragma unroll
        for (int v = 0; v < V; ++v) {
            const size_t idx = base + (size_t)((r0 + i) * V + v) * ld;
            const T r = acc[i][v] * inv;
            bad |= !isfinite(r);
            switch (E.mode) {
                case EPI_STORE: E.out[idx] = r; break;
                case EPI_RK_FIRST:
                    E.uacc[idx] = fma(E.cacc, r, a[i][v]);
                    E.unext[idx] = fma(E.cnext, r, a[i][v]);
                    break;
                case EPI_RK_MID:
                    E.uacc[idx] = fma(E.cacc, r, b[i][v]);
                    E.unext[idx] = fma(E.cnext, r, a[i][v]);
                    break;
                default: E.out[idx] = fma(E.cacc, r, b[i][v]); break;
            }
        }
    }
    if (bad) atomicOr(E.flag, 1);
}

// Stage update of stages 1-3 with the next stage's state kept on chip: uacc
// goes to global memory, u0 + cnext R into this element's shared-memory state
// tile ut ([NS][8]: solution point, variable).
template <int RS, int V, typename T>
__device__ __forceinline__ void epi_block_next(const KEpi<T>& E, const T (&acc)[RS][V], T inv, size_t base, int ld,
                                               int r0, int nrows, T* ut) {
    T a[RS][V], b[RS][V];
    const bool mid = E.mode == EPI_RK_MID;
    #pragma unroll
    for (int i = 0; i < RS; ++i)
        #pragma unroll
        for (int v = 0; v < V; ++v) {
            const size_t idx = base + (size_t)((r0 + i) * V + v) * ld;
            const bool ok = r0 + i < nrows;
            a[i][v] = ok ? __ldg(E.u0 + idx) : T(0);
            b[i][v] = (ok && mid) ? E.uacc[idx] : T(0);
        }
    bool bad = false;
    #pragma unroll
    for (int i = 0; i < RS; ++i) {
        if (r0 + i >= nrows) continue;
        #pragma unroll
        for (int v = 0; v < V; ++v) {
            const size_t idx = base + (size_t)((r0 + i) * V + v) * ld;
            const T r = acc[i][v] * inv;
            bad |= !isfinite(r);
            E.uacc[idx] = fma(E.cacc, r, mid ? b[i][v] : a[i][v]);
            ut[(r0 + i) * 8 + v] = fma(E.cnext, r, a[i][v]);
        }
    }
    if (bad) atomicOr(E.flag, 1);
}

// Rows j = h + G i (i < NRT) of [M0; M12] u for one element whose state tile
// ut ([NS][8]) is in shared memory; A is the row-major operator in global
// memory (rows of nsp values, read through the L1 cache).  Rows past MI are
// computed from row MI - 1 and not used.
template <int NRT, int NS, int V, int G>
__device__ __forceinline__ void interp_rows_tile(const float* __restrict__ A, int nsp, int h, int MI, const float* ut,
                                                 float (&res)[NRT][V]) {
    static_assert(NS % 4 == 0 && V == 5, "four solution points per operator load; five variables");
    #pragma unroll
    for (int i = 0; i < NRT; ++i)
        #pragma unroll
        for (int v = 0; v < V; ++v) res[i][v] = 0.f;
    #pragma unroll
    for (int r = 0; r < NS; r += 4) {
        float u[4][V];
        #pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float4 t = *reinterpret_cast<const float4*>(ut + (r + q) * 8);
            u[q][0] = t.x;
            u[q][1] = t.y;
            u[q][2] = t.z;
            u[q][3] = t.w;
            u[q][4] = ut[(r + q) * 8 + 4];
        }
        #pragma unroll
        for (int i = 0; i < NRT; ++i) {
            const int j = min(h + G * i, MI - 1);
            const float4 x = __ldg(reinterpret_cast<const float4*>(A + (size_t)j * nsp + r));
            const float xq[4] = {x.x, x.y, x.z, x.w};
            #pragma unroll
            for (int q = 0; q < 4; ++q)
                #pragma unroll
                for (int v = 0; v < V; ++v) res[i][v] = fmaf(xq[q], u[q][v], res[i][v]);
        }
    }
}

// Divergence accumulators of one thread: RS rows x V variables.
template <typename T, int RS, int V>
struct ScalarAcc {
    T a[RS][V];
    __device__ __forceinline__ void zero() {
        #pragma unroll
        for (int i = 0; i < RS; ++i)
            #pragma unroll
            for (int v = 0; v < V; ++v) a[i][v] = T(0);
    }
    // a[i][v] += x[i] F[v]
    __device__ __forceinline__ void add(const T* x, const T* F) {
        #pragma unroll
        for (int i = 0; i < RS; ++i)
            #pragma unroll
            for (int v = 0; v < V; ++v) a[i][v] = fma(x[i], F[v], a[i][v]);
    }
    __device__ __forceinline__ T get(int i, int v) const { return a[i][v]; }
};

// The same sums on the paired FP32 FMA of sm_100 and later (__ffma2_rn: two
// IEEE round-to-nearest fmas per instruction, so every sum is bit-identical to
// the scalar one).  Row pairs (r0, r1) = (2p, 2p+1) and variable pairs (v, v+1)
// are accumulated crosswise, D = (r0 v, r1 v+1) += (x_r0, x_r1) (F_v, F_v+1) and
// X = (r0 v+1, r1 v) += (x_r0, x_r1) (F_v+1, F_v), so that both operands are
// plain register pairs; an odd last variable or row takes a broadcast pair.
template <int RS, int V>
struct PairAcc {
    static constexpr int RP = RS / 2, VP = V / 2;
    static constexpr bool ODD_R = RS % 2 != 0, ODD_V = V % 2 != 0;
    static constexpr int RPX = RP > 0 ? RP : 1, VPX = VP > 0 ? VP : 1;
    float2 d[RPX][VPX], x[RPX][VPX];
    float2 dl[RPX];      // odd V: (r0 V-1, r1 V-1)
    float2 rl[VPX];      // odd RS: (RS-1 v, RS-1 v+1)
    float rll;           // odd RS and odd V
    __device__ __forceinline__ void zero() {
        const float2 z = make_float2(0.f, 0.f);
        #pragma unroll
        for (int p = 0; p < RPX; ++p) {
            dl[p] = z;
            #pragma unroll
            for (int w = 0; w < VPX; ++w) d[p][w] = x[p][w] = z;
        }
        #pragma unroll
        for (int w = 0; w < VPX; ++w) rl[w] = z;
        rll = 0.f;
    }
    __device__ __forceinline__ void add(const float* xr, const float* F) {
        float2 P[VPX], Q[VPX];
        #pragma unroll
        for (int w = 0; w < VP; ++w) {
            P[w] = make_float2(F[2 * w], F[2 * w + 1]);
            Q[w] = make_float2(F[2 * w + 1], F[2 * w]);
        }
        #pragma unroll
        for (int p = 0; p < RP; ++p) {
            const float2 X = make_float2(xr[2 * p], xr[2 * p + 1]);
            #pragma unroll
            for (int w = 0; w < VP; ++w) {
                d[p][w] = __ffma2_rn(X, P[w], d[p][w]);
                x[p][w] = __ffma2_rn(X, Q[w], x[p][w]);
            }
            if constexpr (ODD_V) dl[p] = __ffma2_rn(X, make_float2(F[V - 1], F[V - 1]), dl[p]);
        }
        if constexpr (ODD_R) {
            const float2 X = make_float2(xr[RS - 1], xr[RS - 1]);
            #pragma unroll
            for (int w = 0; w < VP; ++w) rl[w] = __ffma2_rn(X, P[w], rl[w]);
            if constexpr (ODD_V) rll = fmaf(xr[RS - 1], F[V - 1], rll);
        }
    }
    // Called with indices known at compile time (fully unrolled loops).
    __device__ __forceinline__ float get(int i, int v) const {
        if (i < 2 * RP) {
            const int p = i >> 1;
            const bool r0 = (i & 1) == 0;
            if (v < 2 * VP) {
                const int w = v >> 1;
                if ((v & 1) == 0) return r0 ? d[p][w].x : x[p][w].y;
                return r0 ? x[p][w].x : d[p][w].y;
            }
            return r0 ? dl[p].x : dl[p].y;
        }
        if (v < 2 * VP) return (v & 1) == 0 ? rl[v >> 1].x : rl[v >> 1].y;
        return rll;
    }
};

template <typename T, int RS, int V> struct DivAcc { using type = ScalarAcc<T, RS, V>; };
template <int RS, int V> struct DivAcc<float, RS, V> { using type = PairAcc<RS, V>; };

// 16-byte shared-memory vector of T.
template <typename T> struct Vec16;
template <> struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
    __device__ static void get(const type& x, float* o) { o[0] = x.x; o[1] = x.y; o[2] = x.z; o[3] = x.w; }
};
template <> struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
    __device__ static void get(const type& x, double* o) { o[0] = x.x; o[1] = x.y; }
};

__device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

}  // namespace

// ---------------------------------------------------------------------------
// Interpolation to the external and internal flux points, written as records.
// 2 * TE threads, TE elements per tile, thread pair (h = 0, 1) per element.
template <typename T, int NS, int V, int NFE, int NFIU, int TE>
__global__ void __launch_bounds__(2 * TE) k_interp_rec(KBlock<T> B, const T* __restrict__ U, T* __restrict__ REC,
                                                    T* __restrict__ FIUR, int* __restrict__ err) {
    constexpr int NSP = (NS + 7) / 8 * 8;                 // equals B.Md_pad
    constexpr int MI = NFE + NFIU;
    constexpr int VB = 400 / (NS * (int)sizeof(T));
    constexpr int VG = (V <= VB) ? V : (VB > 0 ? VB : 1);
    using VT = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::n;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* As = reinterpret_cast<T*>(smem_raw);                                   // [Mir][NSP]
    T* Rs = reinterpret_cast<T*>(smem_raw + align16((size_t)B.Mir * NSP * sizeof(T)));   // [TE][ers]
    T* Fs = Rs + (size_t)TE * B.ers;                                          // [TE][frs]
    int* roff = reinterpret_cast<int*>(Fs + (size_t)TE * B.frs);             // [NFE]
    for (int i = threadIdx.x; i < B.Mir * NSP; i += blockDim.x) As[i] = B.Air[i];
    for (int i = threadIdx.x; i < NFE; i += blockDim.x) roff[i] = B.recoff[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int el = (threadIdx.x >> 5) * 16 + (lane & 15);
    const int h = lane >> 4;
    const int ntiles = (B.nelem + TE - 1) / TE;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int e0 = tile * TE;
        const int n = min(TE, B.nelem - e0);
        if (el < n) {
            const T* Ue = U + B.u_off + e0 + el;
            #pragma unroll 1
            for (int v0 = 0; v0 < V; v0 += VG) {
                T u[VG][NS];
                #pragma unroll
                for (int w = 0; w < VG; ++w) {
                    const int v = (v0 + w < V) ? v0 + w : V - 1;
                    #pragma unroll
                    for (int r = 0; r < NS; ++r) u[w][r] = __ldg(Ue + (size_t)(r * V + v) * B.ld);
                }
                // rows j = h, h + 2, ... in pairs (j, j + 2)
                #pragma unroll 1
                for (int jb = h; jb < MI; jb += 4) {
                    T acc[2][VG];
                    #pragma unroll
                    for (int i = 0; i < 2; ++i)
                        #pragma unroll
                        for (int w = 0; w < VG; ++w) acc[i][w] = T(0);
                    const VT* a0 = reinterpret_cast<const VT*>(As + jb * NSP);
                    const VT* a1 = reinterpret_cast<const VT*>(As + (jb + 2) * NSP);
                    #pragma unroll
                    for (int r = 0; r < NSP; r += VN) {
                        T x0[VN], x1[VN];
                        Vec16<T>::get(a0[r / VN], x0);
                        Vec16<T>::get(a1[r / VN], x1);
                        #pragma unroll
                        for (int q = 0; q < VN; ++q)
                            if (r + q < NS) {
                                #pragma unroll
                                for (int w = 0; w < VG; ++w) {
                                    acc[0][w] = fma(x0[q], u[w][r + q], acc[0][w]);
                                    acc[1][w] = fma(x1[q], u[w][r + q], acc[1][w]);
                                }
                            }
                    }
                    #pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const int j = jb + 2 * i;
                        #pragma unroll
                        for (int w = 0; w < VG; ++w) {
                            const int v = v0 + w;
                            if (v < V) {
                                if (j < NFE) Rs[(size_t)el * B.ers + roff[j] + v] = acc[i][w];
                                else if (j < MI) Fs[(size_t)el * B.frs + (j - NFE) * V + v] = acc[i][w];
                            }
                        }
                    }
                }
            }
        }
        fence_proxy_async();         // every writer orders its staging stores before the bulk store
        __syncthreads();
        if (threadIdx.x == 0) {
            bulk_s2g(REC + B.rec_base + (size_t)e0 * B.ers, Rs, (uint32_t)(n * B.ers * sizeof(T)));
            bulk_s2g(FIUR + B.fiur_base + (size_t)e0 * B.frs, Fs, (uint32_t)(n * B.frs * sizeof(T)));
            bulk_commit();
            bulk_wait_read0();     // the tile buffers may be reused once the copies have read them
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) bulk_wait0();   // writes visible before the kernel completes
    (void)err;
}

// ---------------------------------------------------------------------------
// Interpolation to the flux points as a producer / consumer pipeline (FP32).
//
// Warp NC / 32 (the last one) is the producer: for each of the CTA's tiles one
// lane streams the tile's solution values U[rho][v][e0 .. e0+TE) (one 2D tensor
// copy) into a two-stage shared-memory ring, completing on full[s].
// Consumer thread (e, v, g) copies the NS values of variable v of element e
// to registers, releases the stage (empty[s]) and computes the rows
// j = g, g + GR, ... of [u_fe; u_fiu] = [M0; M12] U (Eqs.
// "interpolation_procedure"), with every lane of a warp reading the same
// operator rows from shared memory (broadcast).  With ALLV a thread (e, g)
// takes all V variables (V times the FMAs per operator load); its warp holds 8
// elements x 4 row groups, so that the staging stores of a warp fall on 32
// distinct banks (record stride = 4 mod 8 words apart per element).  The results
// are assembled into one of two record staging buffers that a single thread
// writes out with bulk stores while the next tile is computed.  Persistent:
// one CTA per SM, two for tiles of at most 32 elements.
template <int NS, int V, int NFE, int NFIU, int TE, int GR, bool ALLV>
__global__ void __launch_bounds__((ALLV ? 1 : V) * TE * GR + 32, TE <= 32 ? 2 : 1) k_interp_pipe(KBlock<float> B,
                                                                     const __grid_constant__ CUtensorMap umap,
                                                                     float* __restrict__ REC,
                                                                     float* __restrict__ FIUR, int* __restrict__ err) {
    constexpr int NROW = NS * V;                      // rows (rho, v) of a U tile
    constexpr int MI = NFE + NFIU;
    constexpr int NSP = (NS + 7) / 8 * 8;             // operator row stride (= B.Md_pad)
    constexpr int NC = (ALLV ? 1 : V) * TE * GR;      // consumer threads
    static_assert(NC % 32 == 0 && TE % 32 == 0, "tile layout");
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* As = reinterpret_cast<float*>(smem_raw);                            // [Mir][NSP]
    size_t off = align16((size_t)B.Mir * NSP * sizeof(float));
    off = (off + 127) & ~size_t(127);
    float* Ub = reinterpret_cast<float*>(smem_raw + off);                      // [2][NROW][TE], 128-byte aligned
    off = align16(off + 2 * (size_t)NROW * TE * sizeof(float));
    const size_t st_elems = (size_t)TE * (B.ers + B.frs);
    float* St = reinterpret_cast<float*>(smem_raw + off);                      // [2][TE][ers + frs]
    off = align16(off + 2 * st_elems * sizeof(float));
    int* roff = reinterpret_cast<int*>(smem_raw + off);                        // [NFE]
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + align16(off + NFE * sizeof(int)));   // full[2], empty[2]

    const int tid = threadIdx.x;
    for (int i = tid; i < B.Mir * NSP; i += blockDim.x) As[i] = B.Air[i];
    for (int i = tid; i < NFE; i += blockDim.x) roff[i] = B.recoff[i];
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        mbar_init(&bar[2], NC / 32);
        mbar_init(&bar[3], NC / 32);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int ntiles = (B.nelem + TE - 1) / TE;
    const int lane = tid & 31;

    if (tid >= NC) {
        // Producer: one 2D tensor copy per tile, the box (TE elements x NROW
        // rows) of the block's state matrix at element e0 (a multiple of TE, so
        // 16-byte aligned); columns past the matrix's padded width read zeros.
        if (lane == 0) {
            int k = 0;
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
                const int s = k & 1;
                if (k >= 2 && !mbar_wait(&bar[2 + s], ((k >> 1) - 1) & 1)) atomicOr(err, 2);
                mbar_arrive_expect_tx(&bar[s], (uint32_t)(NROW * TE * sizeof(float)));
                fence_proxy_async();
                tma_load_2d(Ub + (size_t)s * NROW * TE, &umap, t * TE, 0, &bar[s]);
            }
        }
        return;
    }

    // Consumers.
    int el, v, g;
    if constexpr (ALLV) {
        static_assert(GR == 4, "8 elements x 4 row groups per warp");
        el = (tid >> 5) * 8 + (lane >> 2);
        v = 0;
        g = lane & 3;
    } else {
        el = tid % TE;
        v = (tid / TE) % V;
        g = tid / (TE * V);
    }
    int k = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
        const int s = k & 1;
        const int e0 = t * TE;
        const int n = min(TE, B.nelem - e0);
        if (!mbar_wait(&bar[s], (k >> 1) & 1)) atomicOr(err, 2);
        constexpr int UV = ALLV ? V : 1;          // variables held by a thread
        float u[UV][NS];
        const float* us = Ub + (size_t)s * NROW * TE + (size_t)v * TE + el;
        #pragma unroll
        for (int w = 0; w < UV; ++w)
            #pragma unroll
            for (int r = 0; r < NS; ++r) u[w][r] = us[(size_t)(r * V + w) * TE];
        fence_proxy_async();            // these reads precede the producer's next copies into the stage
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar[2 + s]);
        float* rs = St + (size_t)s * st_elems;
        float* fs = rs + (size_t)TE * B.ers;
        // The staging buffer s was last read by the bulk stores of tile k - 2.
        if (tid == 0) bulk_wait_read1();
        consumer_sync(NC);
        const bool store = el < n;
        if constexpr (ALLV) {
            // Rows j = g + GR i two at a time, stored right away (the operator
            // loads are free to move across the stores).
            #pragma unroll 1
            for (int j = g; j < MI; j += 2 * GR) {
                const int j2 = j + GR;
                const int jb = j2 < MI ? j2 : j;
                float acc[2][UV];
                #pragma unroll
                for (int w = 0; w < UV; ++w) acc[0][w] = acc[1][w] = 0.f;
                #pragma unroll
                for (int r = 0; r < NS; r += 4) {
                    const float4 x0 = lds128_const(As + (size_t)j * NSP + r);
                    const float4 x1 = lds128_const(As + (size_t)jb * NSP + r);
                    const float xa[4] = {x0.x, x0.y, x0.z, x0.w};
                    const float xb[4] = {x1.x, x1.y, x1.z, x1.w};
                    #pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (r + q < NS) {
                            #pragma unroll
                            for (int w = 0; w < UV; ++w) {
                                acc[0][w] = fmaf(xa[q], u[w][r + q], acc[0][w]);
                                acc[1][w] = fmaf(xb[q], u[w][r + q], acc[1][w]);
                            }
                        }
                }
                if (store) {
                    #pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const int jj = i == 0 ? j : j2;
                        if (jj >= MI) break;
                        float* dst = jj < NFE ? rs + (size_t)el * B.ers + roff[jj]
                                              : fs + (size_t)el * B.frs + (jj - NFE) * V;
                        #pragma unroll
                        for (int w = 0; w < UV; ++w) dst[w] = acc[i][w];
                    }
                }
            }
        } else {
            // All of this thread's rows j = g + i GR are accumulated in registers
            // first and stored afterwards.
            constexpr int NR = (MI + GR - 1) / GR;   // rows per thread (some past MI for g > 0)
            constexpr int RB = 4;                    // rows per pass: independent accumulation chains
            float acc[NR];
            #pragma unroll
            for (int i0 = 0; i0 < NR; i0 += RB) {
                #pragma unroll
                for (int i = i0; i < i0 + RB && i < NR; ++i) acc[i] = 0.f;
                #pragma unroll
                for (int r = 0; r < NS; r += 4) {
                    float4 x[RB];
                    #pragma unroll
                    for (int i = 0; i < RB; ++i) {
                        const int j = min(g + (i0 + i) * GR, MI - 1);   // rows past the end: computed, not stored
                        x[i] = lds128_const(As + (size_t)j * NSP + r);
                    }
                    #pragma unroll
                    for (int i = 0; i < RB; ++i) {
                        if (i0 + i >= NR) break;
                        const float xa[4] = {x[i].x, x[i].y, x[i].z, x[i].w};
                        #pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (r + q < NS) acc[i0 + i] = fmaf(xa[q], u[0][r + q], acc[i0 + i]);
                    }
                }
            }
            if (store) {
                #pragma unroll
                for (int i = 0; i < NR; ++i) {
                    const int j = g + i * GR;
                    if (j < NFE) rs[(size_t)el * B.ers + roff[j] + v] = acc[i];
                    else if (j < MI) fs[(size_t)el * B.frs + (j - NFE) * V + v] = acc[i];
                }
            }
        }
        fence_proxy_async();         // every writer orders its staging stores before the bulk stores
        consumer_sync(NC);
        if (tid == 0) {
            bulk_s2g(REC + B.rec_base + (size_t)e0 * B.ers, rs, (uint32_t)(n * B.ers * sizeof(float)));
            bulk_s2g(FIUR + B.fiur_base + (size_t)e0 * B.frs, fs, (uint32_t)(n * B.frs * sizeof(float)));
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait0();      // writes complete before the kernel ends
}

// ---------------------------------------------------------------------------
// Flux and divergence of one tile staged in shared memory (value path).
template <typename T, int V, int ND, int SYS, int RIE, int NS, int G, int NFE, int NFIU, int NW, bool FUSE = false>
__global__ void __launch_bounds__(32 * NW, FUSE ? 3 : 1) k_flux_rec(KBlock<T> B, const T* __restrict__ REC,
                                                      const T* __restrict__ FIUR, KPhys<T> P, KEpi<T> E,
                                                      const __grid_constant__ CUtensorMap u0map,
                                                      const __grid_constant__ CUtensorMap accmap, int prefetch) {
    static_assert(NFE % G == 0, "external points must split evenly across the G threads");
    constexpr int EPW = 32 / G;
    constexpr int TE = NW * EPW;
    constexpr int RS = (NS + G - 1) / G;
    constexpr int RSP = (RS + 3) / 4 * 4;
    constexpr int NDOF = ND;                  // DOFs per internal point (tetrahedra)
    constexpr int K2 = NFE + NDOF * NFIU;
    constexpr int NFACE = ND + 1;
    constexpr int ND2 = ND * ND;
    using VT = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::n;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw);
    size_t off = 16;
    T* As = reinterpret_cast<T*>(smem_raw + off);                 // [K2][G][RSP]
    off = align16(off + (size_t)K2 * G * RSP * sizeof(T));
    T* own = reinterpret_cast<T*>(smem_raw + off);                // [TE][ers]
    off = align16(off + (size_t)TE * B.ers * sizeof(T));
    T* part = reinterpret_cast<T*>(smem_raw + off);               // [TE][ers]: partner face records
    off = align16(off + (size_t)TE * B.ers * sizeof(T));
    T* fiu = reinterpret_cast<T*>(smem_raw + off);                // [TE][frs]
    off = align16(off + (size_t)TE * B.frs * sizeof(T));
    T* met = reinterpret_cast<T*>(smem_raw + off);                // [TE][nmp]
    off = align16(off + (size_t)TE * B.nmp * sizeof(T));
    unsigned char* prm = smem_raw + off;                          // [TE][pstride]
    off = align16(off + (size_t)TE * B.pstride);
    int* roff = reinterpret_cast<int*>(smem_raw + off);           // [NFE]
    int* fface = roff + NFE;                                      // [NFE]

    for (int i = threadIdx.x; i < K2 * G * RSP; i += blockDim.x) {
        const int j = i / (G * RSP);
        const int hh = (i / RSP) % G;
        const int r = hh * RS + i % RSP;
        As[i] = (i % RSP < RS && r < NS) ? B.Ad[(size_t)j * B.Md_pad + r] : T(0);
    }
    for (int i = threadIdx.x; i < NFE; i += blockDim.x) {
        roff[i] = B.recoff[i];
        fface[i] = B.fe_face[i];
    }
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int h = lane / EPW;
    const int el = warp * EPW + lane % EPW;
    const int ntiles = (B.nelem + TE - 1) / TE;
    uint32_t parity = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, parity ^= 1u) {
        const int e0 = tile * TE;
        const int n = min(TE, B.nelem - e0);
        // Stage the tile.
        if (threadIdx.x == 0) {
            // own records + partner face records + internal records + metric rows + permutations
            const uint32_t bytes =
                (uint32_t)((size_t)n * (B.ers + NFACE * B.frec + B.frs + B.nmp) * sizeof(T) + (size_t)n * B.pstride);
            mbar_arrive_expect_tx(bar, bytes);
            fence_proxy_async();
            bulk_g2s(own, REC + B.rec_base + (size_t)e0 * B.ers, (uint32_t)(n * B.ers * sizeof(T)), bar);
            bulk_g2s(fiu, FIUR + B.fiur_base + (size_t)e0 * B.frs, (uint32_t)(n * B.frs * sizeof(T)), bar);
            bulk_g2s(met, B.maos + (size_t)e0 * B.nmp, (uint32_t)(n * B.nmp * sizeof(T)), bar);
            bulk_g2s(prm, B.perm + (size_t)e0 * B.pstride, (uint32_t)(n * B.pstride), bar);
            // The stage-update inputs of this tile's epilogue, into L2 while the fluxes are computed.
            if (prefetch & 1) tma_prefetch_2d(&u0map, e0, 0);
            if (prefetch & 2) tma_prefetch_2d(&accmap, e0, 0);
        }
        for (int t = threadIdx.x; t < n * NFACE; t += blockDim.x) {
            const int le = t / NFACE, f = t % NFACE;
            const int src = __ldg(B.pfr + (size_t)(e0 + le) * NFACE + f);
            fence_proxy_async();
            bulk_g2s(part + (size_t)le * B.ers + f * B.frec, REC + src, (uint32_t)(B.frec * sizeof(T)), bar);
        }
        // The copies' wait, bounded (E.wait_polls > 0: that many non-blocking
        // polls); when it runs out the timeout bit is set and the kernel waits
        // again, with the normal bound, for its own copies in flight before it
        // reads the buffers.
        if (!(E.wait_polls > 0 ? mbar_test_n(bar, parity, E.wait_polls) : mbar_wait(bar, parity))) {
            atomicOr(E.flag, 2);
            mbar_wait(bar, parity);
        }

        const bool valid = el < n;
        const int le = valid ? el : 0;
        const T* own_e = own + (size_t)le * B.ers;
        const T* part_e = part + (size_t)le * B.ers;
        const T* met_e = met + (size_t)le * B.nmp;
        const unsigned char* prm_e = prm + (size_t)le * B.pstride;
        typename DivAcc<T, RS, V>::type acc;
        acc.zero();
        auto accumulate = [&](int j, const T* F) {
            const VT* a = reinterpret_cast<const VT*>(As + ((size_t)j * G + h) * RSP);
            T x[RSP];
            #pragma unroll
            for (int r = 0; r < RSP; r += VN) Vec16<T>::get(a[r / VN], x + r);
            acc.add(x, F);
        };
        // Accumulate the G fluxes of one round: thread h holds the flux of point
        // base + h; the value of thread h ^ m arrives with one xor-shuffle and
        // belongs to point base + (h ^ m).
        auto accumulate_round = [&](int base, const T* F) {
            accumulate(base + h, F);
            #pragma unroll
            for (int m = 1; m < G; ++m) {
                T Fm[V];
                #pragma unroll
                for (int v = 0; v < V; ++v) Fm[v] = __shfl_xor_sync(FULL, F[v], m * EPW);
                accumulate(base + (h ^ m), Fm);
            }
        };
        // External points j = q * G + h.
        #pragma unroll 1
        for (int q = 0; q < NFE / G; ++q) {
            const int j = q * G + h;
            const int f = fface[j];
            const int mrow = 1 + ND2 + f * (ND + 1);
            T nrm[ND];
            #pragma unroll
            for (int c = 0; c < ND; ++c) nrm[c] = met_e[mrow + c];
            const T s = met_e[mrow + ND];
            const T* uo_p = own_e + roff[j];
            const T* un_p = part_e + f * B.frec + (int)prm_e[j] * V;
            T uo[V], un[V], F[V];
            #pragma unroll
            for (int v = 0; v < V; ++v) {
                uo[v] = uo_p[v];
                un[v] = un_p[v];
            }
            T uL[V], uR[V];
            orient<V>(s > T(0), uo, un, uL, uR);
            if constexpr (SYS == SYS_EULER && RIE == RIE_RUSANOV) {
                rusanov_rec<T, ND>(uL, uR, nrm, P.gamma, s, F);
            } else {
                common_flux_f<SYS, RIE, ND>(uL, uR, nrm, P, F);
                #pragma unroll
                for (int v = 0; v < V; ++v) F[v] *= s;
            }
            accumulate_round(q * G, F);
        }
        // Internal points: every axis is a DOF (nu = axis * NFIU + k).
        T Srow[NDOF][ND];
        #pragma unroll
        for (int d = 0; d < NDOF; ++d)
            #pragma unroll
            for (int i = 0; i < ND; ++i) Srow[d][i] = met_e[1 + d * ND + i];
        #pragma unroll 1
        for (int q = 0; q < (NFIU + G - 1) / G; ++q) {
            const int k = q * G + h;
            const int kc = k < NFIU ? k : NFIU - 1;   // past the last point: computed, never accumulated
            T u[V];
            #pragma unroll
            for (int v = 0; v < V; ++v) u[v] = fiu[(size_t)le * B.frs + kc * V + v];
            // Euler: primitive state once per point, then S_axis . f for each axis.
            T pinv, pv[ND], pp;
            if constexpr (SYS == SYS_EULER) prim_rec<T, ND>(u, P.gamma, pinv, pv, pp);
            #pragma unroll
            for (int d = 0; d < NDOF; ++d) {
                T Ft[V];
                if constexpr (SYS == SYS_EULER) {
                    T sv = pv[0] * Srow[d][0];
                    #pragma unroll
                    for (int i = 1; i < ND; ++i) sv = fma(pv[i], Srow[d][i], sv);
                    Ft[0] = u[0] * sv;
                    #pragma unroll
                    for (int i = 0; i < ND; ++i) Ft[1 + i] = fma(u[1 + i], sv, pp * Srow[d][i]);
                    Ft[V - 1] = (u[V - 1] + pp) * sv;
                } else {
                    internal_flux_f<SYS, ND>(u, Srow[d], P, Ft);
                }
                if (k >= NFIU) {
                    #pragma unroll
                    for (int v = 0; v < V; ++v) Ft[v] = T(0);   // past the last point: contributes nothing
                }
                // Points past the last one hold zero fluxes; their operator
                // column index is clamped to a real column.
                const int base = NFE + d * NFIU + q * G;
                accumulate(min(base + h, NFE + d * NFIU + NFIU - 1), Ft);
                #pragma unroll
                for (int m = 1; m < G; ++m) {
                    T Fm[V];
                    #pragma unroll
                    for (int v = 0; v < V; ++v) Fm[v] = __shfl_xor_sync(FULL, Ft[v], m * EPW);
                    accumulate(min(base + (h ^ m), NFE + d * NFIU + NFIU - 1), Fm);
                }
            }
        }
        if constexpr (FUSE) {
            // Stages 1-3 of RK4: the next stage's state goes to this element's
            // own-record slot (read by this warp only), its interpolation to the
            // element's partner-record and internal-record slots, and the tile's
            // new records out with two bulk stores.
            static_assert(std::is_same<T, float>::value && V == 5 && G == 4, "fused interpolation: FP32 Euler");
            constexpr int MI = NFE + NFIU;
            constexpr int NRT = (MI + G - 1) / G;
            float* ut = own + (size_t)le * B.ers;
            __syncwarp();         // the warp's reads of its own records are complete
            if (valid) {
                const T inv = -met_e[0];
                T out[RS][V];
                #pragma unroll
                for (int i = 0; i < RS; ++i)
                    #pragma unroll
                    for (int v = 0; v < V; ++v) out[i][v] = acc.get(i, v);
                epi_block_next<RS, V>(E, out, inv, (size_t)B.u_off + e0 + el, B.ld, h * RS, NS, ut);
            }
            __syncwarp();         // the element's state tile is complete
            if (valid) {
                float res[NRT][V];
                interp_rows_tile<NRT, NS, V, G>(B.Air, B.Md_pad, h, MI, ut, res);
                float* rs = part + (size_t)le * B.ers;
                float* fs = fiu + (size_t)le * B.frs;
                #pragma unroll
                for (int i = 0; i < NRT; ++i) {
                    const int j = h + G * i;
                    if (j >= MI) break;
                    float* dst = j < NFE ? rs + roff[j] : fs + (j - NFE) * V;
                    #pragma unroll
                    for (int v = 0; v < V; ++v) dst[v] = res[i][v];
                }
            }
            fence_proxy_async();  // staging writes (and this thread's reads) before the bulk copies
            __syncthreads();
            if (threadIdx.x == 0) {
                bulk_s2g(E.rec_next + B.rec_base + (size_t)e0 * B.ers, part, (uint32_t)(n * B.ers * sizeof(T)));
                bulk_s2g(E.fiur_next + B.fiur_base + (size_t)e0 * B.frs, fiu, (uint32_t)(n * B.frs * sizeof(T)));
                bulk_commit();
                bulk_wait_read0();    // the staging slots may be refilled once the stores have read them
            }
            __syncthreads();
        } else {
            if (valid) {
                const int e = e0 + el;
                const T inv = -met_e[0];
                T out[RS][V];
                #pragma unroll
                for (int i = 0; i < RS; ++i)
                    #pragma unroll
                    for (int v = 0; v < V; ++v) out[i][v] = acc.get(i, v);
                epi_block<RS, V>(E, out, inv, (size_t)B.u_off + e, B.ld, h * RS, NS);
            }
            fence_proxy_async();  // this thread's reads of the tile precede the next tile's async copies
            __syncthreads();      // the tile buffers are free for the next tile's copies
        }
    }
    if constexpr (FUSE) {
        if (threadIdx.x == 0) bulk_wait0();   // record stores complete before the kernel ends
    }
}

// ---------------------------------------------------------------------------
// JVP: the residual with dual numbers, records read directly from global memory.
template <typename T, int V, int ND, int SYS, int RIE, int NS>
__global__ void __launch_bounds__(32 * V, 4) k_flux_rec_dual(KBlock<T> B, const T* __restrict__ REC,
                                                             const T* __restrict__ dREC, const T* __restrict__ FIUR,
                                                             const T* __restrict__ dFIUR, KPhys<T> P, KEpi<T> E) {
    using S = Dual<T>;
    constexpr int TE = 32;
    constexpr int NCOL = V * TE;
    constexpr int ND2 = ND * ND;
    constexpr int NFACE = ND + 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int NSP = B.Md_pad;
    const int K2 = B.nfe + B.nfi;
    T* As = reinterpret_cast<T*>(smem_raw);                                   // [K2][NSP]
    S* Fs = reinterpret_cast<S*>(smem_raw + (size_t)K2 * NSP * sizeof(T));    // [K2][V * TE]
    for (int i = threadIdx.x; i < K2 * NSP; i += blockDim.x) As[i] = B.Ad[i];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int ntiles = (B.nelem + TE - 1) / TE;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int e = tile * TE + lane;
        const bool valid = e < B.nelem;
        const int ec = valid ? e : B.nelem - 1;
        const size_t rec_e = (size_t)B.rec_base + (size_t)ec * B.ers;
        __syncthreads();
        for (int sg = warp; sg < B.nfe; sg += V) {
            const int f = __ldg(B.fe_face + sg);
            const int mrow = 1 + ND2 + f * (ND + 1);
            T n[ND];
            #pragma unroll
            for (int c = 0; c < ND; ++c) n[c] = __ldg(B.metric + (size_t)(mrow + c) * B.ld + ec);
            const T s = __ldg(B.metric + (size_t)(mrow + ND) * B.ld + ec);
            const size_t po = (size_t)__ldg(B.pfr + (size_t)ec * NFACE + f) +
                              (size_t)__ldg(B.perm + (size_t)ec * B.pstride + sg) * V;
            const size_t oo = rec_e + __ldg(B.recoff + sg);
            S uo[V], un[V], F[V];
            #pragma unroll
            for (int v = 0; v < V; ++v) {
                uo[v] = {__ldg(REC + oo + v), __ldg(dREC + oo + v)};
                un[v] = {__ldg(REC + po + v), __ldg(dREC + po + v)};
            }
            S uL[V], uR[V];
            orient<V>(s > T(0), uo, un, uL, uR);
            common_flux_f<SYS, RIE, ND>(uL, uR, n, P, F);
            #pragma unroll
            for (int v = 0; v < V; ++v) Fs[(size_t)sg * NCOL + v * TE + lane] = s * F[v];
        }
        for (int k = warp; k < B.nfiu; k += V) {
            S u[V];
            const size_t fo = (size_t)B.fiur_base + (size_t)ec * B.frs + (size_t)k * V;
            #pragma unroll
            for (int v = 0; v < V; ++v) u[v] = {__ldg(FIUR + fo + v), __ldg(dFIUR + fo + v)};
            const int4 tab = __ldg(reinterpret_cast<const int4*>(B.fi_tab) + k);
            const int dofs[3] = {tab.y, tab.z, tab.w};
            for (int q = 0; q < tab.x; ++q) {
                const int nu = dofs[q] & 0xffff;
                const int ax = dofs[q] >> 16;
                T Srow[ND];
                #pragma unroll
                for (int i = 0; i < ND; ++i) Srow[i] = __ldg(B.metric + (size_t)(1 + ax * ND + i) * B.ld + ec);
                S Ft[V];
                internal_flux_f<SYS, ND>(u, Srow, P, Ft);
                #pragma unroll
                for (int v = 0; v < V; ++v) Fs[(size_t)(B.nfe + nu) * NCOL + v * TE + lane] = Ft[v];
            }
        }
        __syncthreads();
        {
            const int v = warp;
            S acc[NS];
            #pragma unroll
            for (int r = 0; r < NS; ++r) acc[r] = szero<S>();
            const S* fcol = Fs + v * TE + lane;
            #pragma unroll 2
            for (int j = 0; j < K2; ++j) {
                const S b = fcol[(size_t)j * NCOL];
                const T* a = As + j * NSP;
                #pragma unroll
                for (int r = 0; r < NS; ++r) mac(acc[r], a[r], b);
            }
            if (valid) {
                const T inv = -__ldg(B.metric + e);
                #pragma unroll
                for (int r = 0; r < NS; ++r) {
                    const T d = acc[r].d * inv;
                    if (!isfinite(d)) atomicOr(E.flag, 1);
                    E.out[(size_t)B.u_off + (size_t)(r * V + v) * B.ld + e] = d;
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Host launchers.

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// dependency on the driver library).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// Tensor map of one block's state matrix: rows (rho, v), columns the padded
// elements (ld); boxes of te x nrow.
template <typename T>
static bool encode_state_map(CUtensorMap* map, const T* base, uint64_t ld, uint64_t nrow, uint32_t te) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || !base || (reinterpret_cast<uintptr_t>(base) & 15) != 0 || (ld * sizeof(T)) % 16 != 0 || nrow > 256 ||
        te > 256 || (te * sizeof(T)) % 16 != 0)
        return false;
    const cuuint64_t dims[2] = {ld, nrow};
    const cuuint64_t strides[1] = {ld * sizeof(T)};
    const cuuint32_t box[2] = {te, (cuuint32_t)nrow};
    const cuuint32_t estr[2] = {1, 1};
    const CUtensorMapDataType dt =
        sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    return enc(map, dt, 2, const_cast<T*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename K>
int blocks_per_sm(K kernel, int threads, int smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) n = 1;
    return n;
}

template <typename T, int NS, int V, int NFE, int NFIU, int TE>
void interp_rec_tile(const KBlock<T>& B, const T* U, T* REC, T* FIUR, int* err, int nsm, cudaStream_t st,
                     size_t smem) {
    auto k = k_interp_rec<T, NS, V, NFE, NFIU, TE>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int per = blocks_per_sm(k, 2 * TE, (int)smem);
    const int need = (B.nelem + TE - 1) / TE;
    const int grid = need < nsm * per ? need : nsm * per;
    k<<<grid, 2 * TE, smem, st>>>(B, U, REC, FIUR, err);
}

template <typename T, int NS, int V, int NFE, int NFIU>
void interp_rec_impl(const KBlock<T>& B, const T* U, T* REC, T* FIUR, int* err, int nsm, cudaStream_t st) {
    auto smem_of = [&](int TE) {
        return ((size_t)B.Mir * B.Md_pad * sizeof(T) + 15) / 16 * 16 + (size_t)TE * (B.ers + B.frs) * sizeof(T) +
               NFE * sizeof(int);
    };
    // 64-element tiles unless their records exceed ~150 KB of shared memory.
    if (smem_of(64) <= 150 * 1024) interp_rec_tile<T, NS, V, NFE, NFIU, 64>(B, U, REC, FIUR, err, nsm, st, smem_of(64));
    else interp_rec_tile<T, NS, V, NFE, NFIU, 32>(B, U, REC, FIUR, err, nsm, st, smem_of(32));
}

template <typename T, int V, int SYS, int RIE, int NS, int G, int NFE, int NFIU, int NW, bool FUSE = false>
void flux_rec_impl(const KBlock<T>& B, const T* REC, const T* FIUR, const KPhys<T>& P, const KEpi<T>& E, int nsm,
                   cudaStream_t st) {
    auto k = k_flux_rec<T, V, 3, SYS, RIE, NS, G, NFE, NFIU, NW, FUSE>;
    constexpr int TE = NW * (32 / G);
    constexpr int RSP = ((NS + G - 1) / G + 3) / 4 * 4;
    auto a16 = [](size_t x) { return (x + 15) / 16 * 16; };
    size_t smem = 16;
    smem = a16(smem + (size_t)(NFE + 3 * NFIU) * G * RSP * sizeof(T));
    smem = a16(smem + (size_t)TE * B.ers * sizeof(T));
    smem = a16(smem + (size_t)TE * B.ers * sizeof(T));
    smem = a16(smem + (size_t)TE * B.frs * sizeof(T));
    smem = a16(smem + (size_t)TE * B.nmp * sizeof(T));
    smem = a16(smem + (size_t)TE * B.pstride);
    smem += 2 * NFE * sizeof(int);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int per = blocks_per_sm(k, 32 * NW, (int)smem);
    const int need = (B.nelem + TE - 1) / TE;
    const int grid = need < nsm * per ? need : nsm * per;
    // L2 prefetch maps of the epilogue's stage inputs (u0 in stages 1-3, uacc in 2-4).
    CUtensorMap u0map{}, accmap{};
    int prefetch = 0;
    const uint64_t nrow = (uint64_t)NS * V;
    if ((E.mode == EPI_RK_FIRST || E.mode == EPI_RK_MID) && encode_state_map(&u0map, E.u0 + B.u_off, B.ld, nrow, TE))
        prefetch |= 1;
    if ((E.mode == EPI_RK_MID || E.mode == EPI_RK_LAST) &&
        encode_state_map(&accmap, (const T*)E.uacc + B.u_off, B.ld, nrow, TE))
        prefetch |= 2;
    k<<<grid, 32 * NW, smem, st>>>(B, REC, FIUR, P, E, u0map, accmap, prefetch);
}

template <typename T>
int flux_rec_dual_smem(const KBlock<T>& B, int V) {
    const int K2 = B.nfe + B.nfi;
    return K2 * B.Md_pad * (int)sizeof(T) + K2 * V * 32 * (int)sizeof(Dual<T>);
}

template <typename T, int V, int SYS, int RIE, int NS>
void flux_rec_dual_impl(const KBlock<T>& B, const T* REC, const T* dREC, const T* FIUR, const T* dFIUR,
                        const KPhys<T>& P, const KEpi<T>& E, int nsm, cudaStream_t st) {
    auto k = k_flux_rec_dual<T, V, 3, SYS, RIE, NS>;
    const int smem = flux_rec_dual_smem(B, V);
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const int per = blocks_per_sm(k, 32 * V, smem);
    const int need = (B.nelem + 31) / 32;
    const int grid = need < nsm * per ? need : nsm * per;
    k<<<grid, 32 * V, smem, st>>>(B, REC, dREC, FIUR, dFIUR, P, E);
}

}  // namespace

template <typename T>
bool fast_jvp_available(const KBlock<T>& B, int V) {
    return flux_rec_dual_smem(B, V) <= 227 * 1024;
}
template bool fast_jvp_available<float>(const KBlock<float>&, int);
template bool fast_jvp_available<double>(const KBlock<double>&, int);

bool fast_path_available(int shape, int nsol, int nd, int system, int riemann) {
    if (nd != 3 || shape != 2 /* tetrahedron */) return false;
    if (nsol != 20 && nsol != 35) return false;
    if (system == SYS_ADVECTION) return true;
    return system == SYS_EULER && riemann == RIE_RUSANOV;
}

template <int NS, int V, int NFE, int NFIU, int TE, int GR, bool ALLV>
static bool interp_pipe_impl(const KBlock<float>& B, const float* U, float* REC, float* FIUR, int* err, int nsm,
                             cudaStream_t st) {
    constexpr int NSP = (NS + 7) / 8 * 8;
    static_assert(NS * V <= 256 && TE <= 256, "tensor copy box");
    if (B.Md_pad != NSP) return false;
    CUtensorMap umap;
    if (!encode_state_map(&umap, U + B.u_off, (uint64_t)B.ld, (uint64_t)NS * V, TE)) return false;
    auto a16 = [](size_t x) { return (x + 15) / 16 * 16; };
    size_t smem = (a16((size_t)B.Mir * NSP * 4) + 127) / 128 * 128;
    smem = a16(smem + 2 * (size_t)NS * V * TE * 4);
    smem = a16(smem + 2 * (size_t)TE * (B.ers + B.frs) * 4);
    smem = a16(smem + NFE * 4) + 4 * 8;
    if (smem > 227 * 1024) return false;
    auto k = k_interp_pipe<NS, V, NFE, NFIU, TE, GR, ALLV>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int need = (B.nelem + TE - 1) / TE;
    const int slots = (TE <= 32 ? 2 : 1) * nsm;     // CTAs resident per SM (shared memory)
    const int grid = need < slots ? need : slots;
    k<<<grid, (ALLV ? 1 : V) * TE * GR + 32, smem, st>>>(B, umap, REC, FIUR, err);
    return true;
}

template <typename T>
int launch_interp_rec(const KBlock<T>& B, int V, const T* U, T* REC, T* FIUR, int* err, int nsm, cudaStream_t st) {
    if constexpr (std::is_same<T, float>::value) {
        if (V == 5 && B.nsol == 20 &&
            interp_pipe_impl<20, 5, 40, 10, 32, 4, true>(B, U, REC, FIUR, err, nsm, st))
            return 0;
        if (V == 5 && B.nsol == 35 &&
            interp_pipe_impl<35, 5, 60, 20, 32, 4, false>(B, U, REC, FIUR, err, nsm, st))
            return 0;
        if (V == 1 && B.nsol == 20 &&
            interp_pipe_impl<20, 1, 40, 10, 64, 4, false>(B, U, REC, FIUR, err, nsm, st))
            return 0;
        if (V == 1 && B.nsol == 35 &&
            interp_pipe_impl<35, 1, 60, 20, 64, 4, false>(B, U, REC, FIUR, err, nsm, st))
            return 0;
    }
    if (V == 5 && B.nsol == 20) interp_rec_impl<T, 20, 5, 40, 10>(B, U, REC, FIUR, err, nsm, st);
    else if (V == 5 && B.nsol == 35) interp_rec_impl<T, 35, 5, 60, 20>(B, U, REC, FIUR, err, nsm, st);
    else if (V == 1 && B.nsol == 20) interp_rec_impl<T, 20, 1, 40, 10>(B, U, REC, FIUR, err, nsm, st);
    else if (V == 1 && B.nsol == 35) interp_rec_impl<T, 35, 1, 60, 20>(B, U, REC, FIUR, err, nsm, st);
    else return -1;
    return 0;
}

// Face records between the record array and a packed exchange buffer (one
// thread per value, records of len values; consecutive threads walk a record).
template <typename T>
__global__ void k_face_records(const T* __restrict__ src, T* __restrict__ dst, const int* __restrict__ off,
                               int64_t n, int len, int scatter) {
    const int64_t total = n * len;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / len;
        const int k = (int)(i - r * len);
        if (scatter) dst[(int64_t)off[r] + k] = src[i];
        else dst[i] = src[(int64_t)off[r] + k];
    }
}

template <typename T>
void launch_face_records(const T* src, T* dst, const int* off, int64_t n, int len, bool scatter, int nsm,
                         cudaStream_t st) {
    const int64_t total = n * len;
    if (total <= 0) return;
    int64_t grid = (total + 255) / 256;
    if (grid > 8 * (int64_t)nsm) grid = 8 * (int64_t)nsm;
    k_face_records<T><<<(int)grid, 256, 0, st>>>(src, dst, off, n, len, scatter ? 1 : 0);
}
template void launch_face_records<float>(const float*, float*, const int*, int64_t, int, bool, int, cudaStream_t);
template void launch_face_records<double>(const double*, double*, const int*, int64_t, int, bool, int, cudaStream_t);

bool flux_rec_fusable(const KBlock<float>& B, int V, int system) {
    return system == SYS_EULER && V == 5 && B.nsol == 20 && B.Air != nullptr && B.Md_pad % 4 == 0 &&
           B.Mir >= 50 && B.ers >= 20 * 8;
}

template <typename T>
int launch_flux_rec(const KBlock<T>& B, int system, const T* REC, const T* dREC, const T* FIUR, const T* dFIUR,
                    const KPhys<T>& P, const KEpi<T>& E, int nsm, cudaStream_t st) {
    const bool dual = dREC != nullptr;
    if (system == SYS_EULER) {
        if (B.nsol == 20) {
            if (dual) flux_rec_dual_impl<T, 5, SYS_EULER, RIE_RUSANOV, 20>(B, REC, dREC, FIUR, dFIUR, P, E, nsm, st);
            else if constexpr (std::is_same<T, float>::value) {
                if (E.rec_next)
                    flux_rec_impl<T, 5, SYS_EULER, RIE_RUSANOV, 20, 4, 40, 10, 4, true>(B, REC, FIUR, P, E, nsm, st);
                else
                    flux_rec_impl<T, 5, SYS_EULER, RIE_RUSANOV, 20, 4, 40, 10, 4>(B, REC, FIUR, P, E, nsm, st);
            } else flux_rec_impl<T, 5, SYS_EULER, RIE_RUSANOV, 20, 4, 40, 10, 4>(B, REC, FIUR, P, E, nsm, st);
        } else {
            if (dual) flux_rec_dual_impl<T, 5, SYS_EULER, RIE_RUSANOV, 35>(B, REC, dREC, FIUR, dFIUR, P, E, nsm, st);
            else flux_rec_impl<T, 5, SYS_EULER, RIE_RUSANOV, 35, 4, 60, 20, 2>(B, REC, FIUR, P, E, nsm, st);
        }
    } else {
        if (B.nsol == 20) {
            if (dual) flux_rec_dual_impl<T, 1, SYS_ADVECTION, RIE_UPWIND, 20>(B, REC, dREC, FIUR, dFIUR, P, E, nsm, st);
            else flux_rec_impl<T, 1, SYS_ADVECTION, RIE_UPWIND, 20, 2, 40, 10, 4>(B, REC, FIUR, P, E, nsm, st);
        } else {
            if (dual) flux_rec_dual_impl<T, 1, SYS_ADVECTION, RIE_UPWIND, 35>(B, REC, dREC, FIUR, dFIUR, P, E, nsm, st);
            else flux_rec_impl<T, 1, SYS_ADVECTION, RIE_UPWIND, 35, 4, 60, 20, 4>(B, REC, FIUR, P, E, nsm, st);
        }
    }
    return 0;
}

template int launch_interp_rec<float>(const KBlock<float>&, int, const float*, float*, float*, int*, int,
                                      cudaStream_t);
template int launch_interp_rec<double>(const KBlock<double>&, int, const double*, double*, double*, int*, int,
                                       cudaStream_t);
template int launch_flux_rec<float>(const KBlock<float>&, int, const float*, const float*, const float*,
                                    const float*, const KPhys<float>&, const KEpi<float>&, int, cudaStream_t);
template int launch_flux_rec<double>(const KBlock<double>&, int, const double*, const double*, const double*,
                                     const double*, const KPhys<double>&, const KEpi<double>&, int, cudaStream_t);

}  // namespace sdrt
