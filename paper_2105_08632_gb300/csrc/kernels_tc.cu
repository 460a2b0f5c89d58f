// Tensor-core (tcgen05) interpolation to the flux points for tetrahedra of
// degree 3, FP32 states via a 3xTF32 split (sm_103a).
//
// [u_fe; u_fiu] = [M0; M12] U  (paper App. B, Eqs. "interpolation_procedure")
// is, per variable v, the GEMM  D_v (128 elements x N) = A_v (128 x K) B^T
// with A_v = U[:, v, tile] (K = N_s = 20, padded to 24), B = [M0; M12]
// (N = N_fe + N_fiu = 50, padded to 64).  One CTA of 128 threads owns one SM:
// the 128 elements of a tile sit on the 128 TMEM lanes, D_v occupies columns
// [64 v, 64 v + 64).  Each thread loads its element's 20 values of variable v
// (coalesced along the element index), splits them into TF32 hi + lo parts and
// writes row e of A_v in the no-swizzle K-major core-matrix layout; one thread
// issues D_v = Ah Bh + Ah Bl + Al Bh (3 x 3 tcgen05.mma of M128 N64 K8) and
// commits them to an mbarrier.  A_v is double-buffered so that the next
// variable's operand is written while the tensor core works.  After the last
// variable each thread reads its TMEM lane (tcgen05.ld) into the tile's record
// staging in shared memory, which one bulk copy writes to the record arrays
// (the same layout as k_interp_rec).
#include <cstdint>

#include "device_math.cuh"
#include "flux_rec.cuh"
#include "kargs.hpp"
#include "launch.hpp"
#include "tc_util.cuh"

namespace sdrt {

using namespace tc;

template <int NS, int V, int NFE, int NFIU>
__global__ void __launch_bounds__(128, 1) k_interp_tc(KBlock<float> B, const float* __restrict__ U,
                                                      float* __restrict__ REC, float* __restrict__ FIUR,
                                                      int* __restrict__ err) {
    constexpr int TE = 128;                          // elements per tile = TMEM lanes
    constexpr int KP = (NS + 7) / 8 * 8;             // K padded to the K8 MMA step
    constexpr int MI = NFE + NFIU;
    constexpr int NP = (MI + 15) / 16 * 16;          // N padded to a multiple of 16 (M = 128)
    constexpr uint32_t kCols = 512;
    static_assert(V * NP <= (int)kCols, "TMEM columns");
    constexpr uint32_t SBO = (KP / 4) * 128;         // 8-row groups
    constexpr uint32_t LBO = 128;                    // K-adjacent core matrices
    constexpr int A_BYTES = TE * KP * 4;
    constexpr int B_BYTES = NP * KP * 4;
    constexpr uint32_t IDESC = idesc_tf32(128, NP);

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* Bh = smem_raw;                    // [NP][KP] hi
    unsigned char* Bl = Bh + B_BYTES;                // lo
    unsigned char* Ah = Bl + B_BYTES;                // 2 buffers of [TE][KP] hi
    unsigned char* Al = Ah + 2 * A_BYTES;            // 2 buffers lo
    float* Rs = reinterpret_cast<float*>(Al + 2 * A_BYTES);       // [TE][ers]
    float* Fs = Rs + (size_t)TE * B.ers;                           // [TE][frs]
    int* roff = reinterpret_cast<int*>(Fs + (size_t)TE * B.frs);   // [NFE]
    uint64_t* bar = reinterpret_cast<uint64_t*>(roff + NFE + (NFE & 1));   // [2], 8-byte aligned
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    if (warp == 0) tmem_alloc(tslot, kCols);
    // Operator B = [M0; M12] (rows n < MI, K = rho), split into TF32 hi + lo.
    for (int i = tid; i < NP * KP; i += blockDim.x) {
        const int n = i / KP, k = i % KP;
        const float x = (n < MI && k < NS) ? B.Air[n * B.Md_pad + k] : 0.f;
        const float h = to_tf32(x);
        *reinterpret_cast<float*>(Bh + core_off(n, k, KP)) = h;
        *reinterpret_cast<float*>(Bl + core_off(n, k, KP)) = to_tf32(x - h);
    }
    // K padding columns of the A buffers stay zero.
    for (int i = tid; i < 4 * A_BYTES / 4; i += blockDim.x) reinterpret_cast<float*>(Ah)[i] = 0.f;
    for (int i = tid; i < NFE; i += blockDim.x) roff[i] = B.recoff[i];
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    uint32_t ph[2] = {0u, 0u};
    const int ntiles = (B.nelem + TE - 1) / TE;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int e0 = tile * TE;
        const int n = min(TE, B.nelem - e0);
        const int e = e0 + tid;
        const bool valid = tid < n;
        // All of the element's solution values first (they overlap the previous
        // tile's bulk store).
        float u[V][NS];
        #pragma unroll
        for (int v = 0; v < V; ++v)
            #pragma unroll
            for (int r = 0; r < NS; ++r) u[v][r] = valid ? __ldg(U + B.u_off + (size_t)(r * V + v) * B.ld + e) : 0.f;
        #pragma unroll
        for (int v = 0; v < V; ++v) {
            const int b = v & 1;
            if (v >= 2) {                            // buffer b was read by the MMAs of variable v - 2
                if (!mbar_wait(&bar[b], ph[b])) atomicOr(err, 2);
                ph[b] ^= 1u;
            }
            unsigned char* ah = Ah + b * A_BYTES;
            unsigned char* al = Al + b * A_BYTES;
            // Row tid, 4 K values per 16-byte store (8 lanes cover one 128-byte core matrix).
            #pragma unroll
            for (int r = 0; r < NS; r += 4) {
                float4 h, l;
                float* hp = &h.x;
                float* lp = &l.x;
                #pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float x = (r + q < NS) ? u[v][r + q] : 0.f;
                    hp[q] = to_tf32(x);
                    lp[q] = to_tf32(x - hp[q]);
                }
                *reinterpret_cast<float4*>(ah + core_off(tid, r, KP)) = h;
                *reinterpret_cast<float4*>(al + core_off(tid, r, KP)) = l;
            }
            fence_proxy_async();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(v * NP);
                #pragma unroll
                for (int kk = 0; kk < KP / 8; ++kk) {
                    const uint32_t koff = (uint32_t)kk * 2 * LBO;
                    const uint64_t dah = smem_desc(ah + koff, LBO, SBO), dal = smem_desc(al + koff, LBO, SBO);
                    const uint64_t dbh = smem_desc(Bh + koff, LBO, SBO), dbl = smem_desc(Bl + koff, LBO, SBO);
                    mma_tf32(d, dah, dbh, IDESC, kk > 0 ? 1u : 0u);
                    mma_tf32(d, dah, dbl, IDESC, 1u);
                    mma_tf32(d, dal, dbh, IDESC, 1u);
                }
                mma_commit(&bar[b]);
            }
        }
        // Wait for the last MMAs on both buffers, and for the previous tile's
        // bulk store to have read the staging buffers.
        #pragma unroll
        for (int b = 0; b < 2; ++b) {
            if (!mbar_wait(&bar[b], ph[b])) atomicOr(err, 2);
            ph[b] ^= 1u;
        }
        if (tid == 0) bulk_wait_read0();
        __syncthreads();
        tc_fence_after();
        // TMEM lane tid -> records of element e.  tcgen05.ld is warp-collective:
        // every lane executes it, only lanes with an element store.
        {
            float* rs = Rs + (size_t)tid * B.ers;
            float* fs = Fs + (size_t)tid * B.frs;
            #pragma unroll 1
            for (int v = 0; v < V; ++v) {
                #pragma unroll
                for (int c = 0; c < NP / 16; ++c) {
                    float x[16];
                    tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(v * NP + c * 16), x);
                    if (valid) {
                        #pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const int j = c * 16 + i;
                            if (j < NFE) rs[roff[j] + v] = x[i];
                            else if (j < MI) fs[(j - NFE) * V + v] = x[i];
                        }
                    }
                }
            }
        }
        fence_proxy_async();         // every writer orders its staging stores before the bulk store
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            bulk_s2g(REC + B.rec_base + (size_t)e0 * B.ers, Rs, (uint32_t)(n * B.ers * sizeof(float)));
            bulk_s2g(FIUR + B.fiur_base + (size_t)e0 * B.frs, Fs, (uint32_t)(n * B.frs * sizeof(float)));
            bulk_commit();
        }
    }
    if (tid == 0) bulk_wait0();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kCols);
}

// ---------------------------------------------------------------------------
// Euler fluxes on the CUDA cores, divergence on the tensor cores: tetrahedra of
// degree 3, FP32 states, 3xTF32 products with FP32 accumulation.
//
// Per tile of TE = 24 elements the divergence R~_v = [M14 | M13] F~_v of every
// variable v (paper App. B, Eq. "residual_sdrt_matrices") is one GEMM
//   D (128 x 32, FP32 in TMEM) = A (128 x K) B^T (32 x K)
// with rows v * 24 + e of A holding element e's transformed fluxes of variable
// v (rows 120..127 stay zero) and B the operator (N = 32 rows for the 20
// solution points).  K runs in two phases over one 40-column A buffer:
//   phase 1: the 40 external points; thread h (0..9) of an element owns points
//            4h .. 4h+3 and writes them with one 16-byte store per variable;
//   phase 2: the 10 internal points, point h with its 3 axis DOFs in columns
//            4h .. 4h+2 (column 4h+3 zero); the operator's internal columns are
//            reordered to this layout when it is staged.
// The tensor core thus replaces the per-element FMA accumulation and the
// exchange of fluxes between threads.  Each thread finally reads 10 rows of one
// TMEM lane (v, e) and applies dU/dt = -R~ / det J with the RK stage update.
// Records are staged as in k_flux_rec (bulk copies completing on an mbarrier).
template <int NS, int NFE, int NFIU>
__global__ void __launch_bounds__(256, 2) k_flux_tc(KBlock<float> B, const float* __restrict__ REC,
                                                    const float* __restrict__ FIUR, KPhys<float> P,
                                                    KEpi<float> E) {
    constexpr int V = 5, ND = 3, NFACE = 4, ND2 = 9;
    constexpr int TE = 24;                           // elements per tile
    constexpr int G = 10;                            // threads per element
    constexpr int KA = 40;                           // K columns per phase
    constexpr int KB = 2 * KA;                       // operator K columns
    constexpr int NP = 32;                           // N: solution points padded
    static_assert(NFE == KA && 4 * NFIU == KA && NFE == 4 * G && NFIU == G && NS <= NP, "tetrahedra of degree 3");
    constexpr uint32_t LBO = 128;
    constexpr uint32_t SBO_A = (KA / 4) * 128;
    constexpr uint32_t SBO_B = (KB / 4) * 128;
    constexpr int A_BYTES = 128 * KA * 4;
    constexpr int B_BYTES = NP * KB * 4;
    constexpr uint32_t IDESC = idesc_tf32(128, NP);
    constexpr uint32_t kCols = 32;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* Bh = smem_raw;                    // operator [NP][KB], TF32 hi / lo
    unsigned char* Bl = Bh + B_BYTES;
    unsigned char* Ah = Bl + B_BYTES;                // fluxes [128][KA], TF32 hi / lo
    unsigned char* Al = Ah + A_BYTES;
    float* own = reinterpret_cast<float*>(Al + A_BYTES);          // [TE][ers]
    float* part = own + (size_t)TE * B.ers;                        // [TE][ers]
    float* fiu = part + (size_t)TE * B.ers;                        // [TE][frs]
    float* met = fiu + (size_t)TE * B.frs;                         // [TE][nmp]
    unsigned char* prm = reinterpret_cast<unsigned char*>(met + (size_t)TE * B.nmp);   // [TE][pstride]
    int* roff = reinterpret_cast<int*>(prm + (size_t)TE * B.pstride);                 // [NFE]
    int* fface = roff + NFE;                                                           // [NFE]
    uint64_t* bar = reinterpret_cast<uint64_t*>(fface + NFE);                          // [2]: loads, MMAs
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);

    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    if (warp == 0) tmem_alloc(tslot, kCols);
    // Operator B[r][k]: k < 40 external point k; k = 40 + 4 q + d internal
    // point q, axis d (< 3), i.e. operator column NFE + d NFIU + q.
    for (int i = tid; i < NP * KB; i += blockDim.x) {
        const int r = i / KB, k = i % KB;
        float x = 0.f;
        if (r < NS) {
            if (k < NFE) {
                x = B.Ad[(size_t)k * B.Md_pad + r];
            } else {
                const int q = (k - NFE) >> 2, d = (k - NFE) & 3;
                if (d < ND) x = B.Ad[(size_t)(NFE + d * NFIU + q) * B.Md_pad + r];
            }
        }
        const float h = to_tf32(x);
        *reinterpret_cast<float*>(Bh + core_off(r, k, KB)) = h;
        *reinterpret_cast<float*>(Bl + core_off(r, k, KB)) = to_tf32(x - h);
    }
    for (int i = tid; i < 2 * A_BYTES / 4; i += blockDim.x) reinterpret_cast<float*>(Ah)[i] = 0.f;
    for (int i = tid; i < NFE; i += blockDim.x) {
        roff[i] = B.recoff[i];
        fface[i] = B.fe_face[i];
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    // Flux work: thread (e, h) with e = tid % TE, h = tid / TE (tid < TE * G).
    const bool worker = tid < TE * G;
    const int fe_ = tid % TE;
    const int h = worker ? tid / TE : 0;
    // Epilogue: TMEM lane L = 32 (warp % 4) + lane holds row (v, e) = (L / TE, L % TE);
    // warps 0-3 apply solution rows 0..9, warps 4-7 rows 10..19.
    const int lrow = 32 * (warp & 3) + (tid & 31);
    const int r0 = (warp >> 2) * 10;

    uint32_t ph_ld = 0, ph_mma = 0;
    int* err = E.flag;
    const int ntiles = (B.nelem + TE - 1) / TE;
    // Bulk copies of one tile's records (own external-point records, internal-
    // point records, metric rows, permutations, and the four partner face
    // records of every element), all completing on bar[0].
    auto issue_loads = [&](int t_) {
        const int e0_ = t_ * TE;
        const int n_ = min(TE, B.nelem - e0_);
        if (tid == 0) {
            const uint32_t bytes = (uint32_t)((size_t)n_ * (B.ers + NFACE * B.frec + B.frs + B.nmp) * sizeof(float) +
                                              (size_t)n_ * B.pstride);
            mbar_arrive_expect_tx(&bar[0], bytes);
            fence_proxy_async();
            bulk_g2s(own, REC + B.rec_base + (size_t)e0_ * B.ers, (uint32_t)(n_ * B.ers * sizeof(float)), &bar[0]);
            bulk_g2s(fiu, FIUR + B.fiur_base + (size_t)e0_ * B.frs, (uint32_t)(n_ * B.frs * sizeof(float)), &bar[0]);
            bulk_g2s(met, B.maos + (size_t)e0_ * B.nmp, (uint32_t)(n_ * B.nmp * sizeof(float)), &bar[0]);
            bulk_g2s(prm, B.perm + (size_t)e0_ * B.pstride, (uint32_t)(n_ * B.pstride), &bar[0]);
        }
        for (int t = tid; t < n_ * NFACE; t += blockDim.x) {
            const int le_ = t / NFACE, f = t % NFACE;
            const int src = __ldg(B.pfr + (size_t)(e0_ + le_) * NFACE + f);
            fence_proxy_async();
            bulk_g2s(part + (size_t)le_ * B.ers + f * B.frec, REC + src, (uint32_t)(B.frec * sizeof(float)), &bar[0]);
        }
    };
    if (blockIdx.x < ntiles) issue_loads(blockIdx.x);
    const bool need_u0 = E.mode == EPI_RK_FIRST || E.mode == EPI_RK_MID;
    const bool need_acc = E.mode == EPI_RK_MID || E.mode == EPI_RK_LAST;
    const int ev = lrow / TE, ee = lrow % TE;      // epilogue row (v, e) of this thread's TMEM lane
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int e0 = tile * TE;
        const int n = min(TE, B.nelem - e0);
        const bool epi = lrow < V * TE && ee < n;
        const size_t ebase = (size_t)B.u_off + (size_t)ev * B.ld + e0 + ee;
        const size_t ers_ = (size_t)V * B.ld;
        // Stage-update inputs of the epilogue, loaded early (independent of the fluxes).
        float a[10], b[10];
        #pragma unroll
        for (int i = 0; i < 10; ++i) {
            const size_t idx = ebase + (size_t)(r0 + i) * ers_;
            a[i] = (epi && need_u0) ? __ldg(E.u0 + idx) : 0.f;
            b[i] = (epi && need_acc) ? E.uacc[idx] : 0.f;
        }
        if (!mbar_wait(&bar[0], ph_ld)) {
            atomicOr(err, 2);
            mbar_wait(&bar[0], ph_ld);
        }
        ph_ld ^= 1u;

        const int le = fe_ < n ? fe_ : 0;     // past the tile's end: a real element, never stored
        const float* own_e = own + (size_t)le * B.ers;
        const float* part_e = part + (size_t)le * B.ers;
        const float* met_e = met + (size_t)le * B.nmp;
        const unsigned char* prm_e = prm + (size_t)le * B.pstride;
        // Phase 1: external points 4h .. 4h+3.
        if (worker) {
            float F[4][V];
            #pragma unroll
            for (int jj = 0; jj < 4; ++jj) {
                const int j = 4 * h + jj;
                const int f = fface[j];
                const int mrow = 1 + ND2 + f * (ND + 1);
                float nrm[ND];
                #pragma unroll
                for (int c = 0; c < ND; ++c) nrm[c] = met_e[mrow + c];
                const float s = met_e[mrow + ND];
                const float* uo_p = own_e + roff[j];
                const float* un_p = part_e + f * B.frec + (int)prm_e[j] * V;
                float uo[V], un[V];
                #pragma unroll
                for (int v = 0; v < V; ++v) {
                    uo[v] = uo_p[v];
                    un[v] = un_p[v];
                }
                float uL[V], uR[V];
                orient<V>(s > 0.f, uo, un, uL, uR);
                rusanov_rec<float, ND>(uL, uR, nrm, P.gamma, s, F[jj]);
            }
            #pragma unroll
            for (int v = 0; v < V; ++v) {
                float4 hi, lo;
                float* hp = &hi.x;
                float* lp = &lo.x;
                #pragma unroll
                for (int q = 0; q < 4; ++q) {
                    hp[q] = to_tf32(F[q][v]);
                    lp[q] = to_tf32(F[q][v] - hp[q]);
                }
                const uint32_t o = core_off(v * TE + fe_, 4 * h, KA);
                *reinterpret_cast<float4*>(Ah + o) = hi;
                *reinterpret_cast<float4*>(Al + o) = lo;
            }
        }
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            #pragma unroll
            for (int kk = 0; kk < KA / 8; ++kk) {
                const uint32_t ko = (uint32_t)kk * 2 * LBO;
                const uint64_t dah = smem_desc(Ah + ko, LBO, SBO_A), dal = smem_desc(Al + ko, LBO, SBO_A);
                const uint64_t dbh = smem_desc(Bh + ko, LBO, SBO_B), dbl = smem_desc(Bl + ko, LBO, SBO_B);
                mma_tf32(tmem, dah, dbh, IDESC, kk > 0 ? 1u : 0u);
                mma_tf32(tmem, dah, dbl, IDESC, 1u);
                mma_tf32(tmem, dal, dbh, IDESC, 1u);
            }
            mma_commit(&bar[1]);
        }
        // Phase 2 fluxes (registers) while the tensor core works: internal point h.
        float Ft[ND][V];
        if (worker) {
            float u[V];
            #pragma unroll
            for (int v = 0; v < V; ++v) u[v] = fiu[(size_t)le * B.frs + h * V + v];
            float pinv, pv[ND], pp;
            prim_rec<float, ND>(u, P.gamma, pinv, pv, pp);
            #pragma unroll
            for (int d = 0; d < ND; ++d) {
                const float* S = met_e + 1 + d * ND;
                float sv = pv[0] * S[0];
                #pragma unroll
                for (int i = 1; i < ND; ++i) sv = fmaf(pv[i], S[i], sv);
                Ft[d][0] = u[0] * sv;
                #pragma unroll
                for (int i = 0; i < ND; ++i) Ft[d][1 + i] = fmaf(u[1 + i], sv, pp * S[i]);
                Ft[d][V - 1] = (u[V - 1] + pp) * sv;
            }
        }
        const float inv = epi ? -met[(size_t)ee * B.nmp] : 0.f;   // -1 / det J of the epilogue's element
        if (!mbar_wait(&bar[1], ph_mma)) {       // phase 1 MMAs have read A
            atomicOr(err, 2);
            mbar_wait(&bar[1], ph_mma);
        }
        ph_mma ^= 1u;
        tc_fence_after();
        if (worker) {
            #pragma unroll
            for (int v = 0; v < V; ++v) {
                float4 hi, lo;
                float* hp = &hi.x;
                float* lp = &lo.x;
                #pragma unroll
                for (int d = 0; d < ND; ++d) {
                    hp[d] = to_tf32(Ft[d][v]);
                    lp[d] = to_tf32(Ft[d][v] - hp[d]);
                }
                hp[3] = 0.f;
                lp[3] = 0.f;
                const uint32_t o = core_off(v * TE + fe_, 4 * h, KA);
                *reinterpret_cast<float4*>(Ah + o) = hi;
                *reinterpret_cast<float4*>(Al + o) = lo;
            }
        }
        fence_proxy_async();     // A stores before the MMAs; record reads before the next tile's copies
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            #pragma unroll
            for (int kk = 0; kk < KA / 8; ++kk) {
                const uint32_t ko = (uint32_t)kk * 2 * LBO;
                const uint32_t kob = (uint32_t)(KA / 8 + kk) * 2 * LBO;
                const uint64_t dah = smem_desc(Ah + ko, LBO, SBO_A), dal = smem_desc(Al + ko, LBO, SBO_A);
                const uint64_t dbh = smem_desc(Bh + kob, LBO, SBO_B), dbl = smem_desc(Bl + kob, LBO, SBO_B);
                mma_tf32(tmem, dah, dbh, IDESC, 1u);
                mma_tf32(tmem, dah, dbl, IDESC, 1u);
                mma_tf32(tmem, dal, dbh, IDESC, 1u);
            }
            mma_commit(&bar[1]);
        }
        // The records of this tile are consumed: the next tile's copies overlap
        // the MMAs and the epilogue.
        if (tile + (int)gridDim.x < ntiles) issue_loads(tile + gridDim.x);
        if (!mbar_wait(&bar[1], ph_mma)) {
            atomicOr(err, 2);
            mbar_wait(&bar[1], ph_mma);
        }
        ph_mma ^= 1u;
        tc_fence_after();
        // Epilogue: rows r0 .. r0+9 of TMEM lane lrow (warp-collective loads).
        {
            float x[32];
            const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
            tmem_ld16(ta, x);
            tmem_ld16(ta + 16, x + 16);
            if (epi) {
                bool bad = false;
                #pragma unroll
                for (int i = 0; i < 10; ++i) {
                    const size_t idx = ebase + (size_t)(r0 + i) * ers_;
                    const float r = (r0 == 0 ? x[i] : x[10 + i]) * inv;
                    bad |= !isfinite(r);
                    switch (E.mode) {
                        case EPI_STORE: E.out[idx] = r; break;
                        case EPI_RK_FIRST:
                            E.uacc[idx] = fmaf(E.cacc, r, a[i]);
                            E.unext[idx] = fmaf(E.cnext, r, a[i]);
                            break;
                        case EPI_RK_MID:
                            E.uacc[idx] = fmaf(E.cacc, r, b[i]);
                            E.unext[idx] = fmaf(E.cnext, r, a[i]);
                            break;
                        default: E.out[idx] = fmaf(E.cacc, r, b[i]); break;
                    }
                }
                if (bad) atomicOr(err, 1);
            }
        }
        tc_fence_before();       // this thread's TMEM loads precede the next tile's MMAs
        __syncthreads();
    }
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kCols);
}

bool tc_flux_available(int shape, int nsol, int nvar, int system, int riemann) {
    return shape == 2 && nsol == 20 && nvar == 5 && system == SYS_EULER && riemann == RIE_RUSANOV;
}

int launch_flux_tc(const KBlock<float>& B, const float* REC, const float* FIUR, const KPhys<float>& P,
                   const KEpi<float>& E, int nsm, cudaStream_t st) {
    if (!(B.nsol == 20 && B.nfe == 40 && B.nfiu == 10 && B.nfaces == 4)) return -1;
    auto k = k_flux_tc<20, 40, 10>;
    constexpr int TE = 24;
    const size_t smem = 2 * (size_t)32 * 80 * 4 + 2 * (size_t)128 * 40 * 4 +
                        (size_t)TE * (2 * B.ers + B.frs + B.nmp) * 4 + (size_t)TE * B.pstride + 2 * 40 * 4 + 2 * 8 + 16;
    if (smem > 227 * 1024) return -1;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int need = (B.nelem + TE - 1) / TE;
    const int grid = need < 2 * nsm ? need : 2 * nsm;
    k<<<grid, 256, smem, st>>>(B, REC, FIUR, P, E);
    return 0;
}

// ---------------------------------------------------------------------------
bool tc_interp_available(int shape, int nsol, int nvar) { return shape == 2 && nsol == 20 && nvar == 5; }

int launch_interp_tc(const KBlock<float>& B, int V, const float* U, float* REC, float* FIUR, int* err, int nsm,
                     cudaStream_t st) {
    if (!(V == 5 && B.nsol == 20 && B.nfe == 40 && B.nfiu == 10)) return -1;
    auto k = k_interp_tc<20, 5, 40, 10>;
    constexpr int KP = 24, NP = 64;
    const size_t smem = 2 * (size_t)NP * KP * 4 + 4 * (size_t)128 * KP * 4 + (size_t)128 * (B.ers + B.frs) * 4 +
                        (40 + 2) * 4 + 2 * 8 + 16;
    if (smem > 227 * 1024) return -1;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int need = (B.nelem + 127) / 128;
    const int grid = need < nsm ? need : nsm;
    k<<<grid, 128, smem, st>>>(B, U, REC, FIUR, err);
    return 0;
}

}  // namespace sdrt
