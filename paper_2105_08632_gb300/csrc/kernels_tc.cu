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

#include "kargs.hpp"
#include "launch.hpp"

namespace sdrt {

namespace {

constexpr long long kWaitLimit = 1ll << 26;

__device__ __forceinline__ uint32_t s32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    const uint32_t a = s32(bar);
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
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void bulk_s2g(void* dst, const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(s32(src)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// TF32 rounding (round to nearest, ties away) of an FP32 value.
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// ---- tcgen05 -----------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s32(slot)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle, K-major: core matrices of 8 rows
// x 16 bytes; lbo = byte distance between K-adjacent core matrices, sbo =
// between row-adjacent groups of 8 rows; bits 46-48 = 0b001.
__device__ __forceinline__ uint64_t smem_desc(const void* p, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((s32(p) & 0x3FFFF) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::tf32: D F32, A and B TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(s32(bar))
                 : "memory");
}
// 16 consecutive 32-bit TMEM columns of this thread's lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* o) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    #pragma unroll
    for (int i = 0; i < 16; ++i) o[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row r, k) in a K-major core-matrix operand with
// kp K values per row (kp multiple of 4): [r / 8][k / 4][r % 8][k % 4].
__device__ __forceinline__ uint32_t core_off(int r, int k, int kp) {
    return (uint32_t)(((r >> 3) * (kp >> 2) + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

}  // namespace

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
                if (!mbar_wait(&bar[b], ph[b])) *err = 2;
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
            if (!mbar_wait(&bar[b], ph[b])) *err = 2;
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
