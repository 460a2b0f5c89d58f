// Tensor-core (tcgen05) LDG gradient chain of the Navier-Stokes residual, FP32
// states, 3xTF32 products with FP32 accumulation (sm_103a).
//
// For every variable v of a tile of 128 elements (one per TMEM lane):
//   GEMM 1  q~ = [M16 | M15 P M12] [C; U]   (paper Sec. 2.1: the transformed
//           gradient from the common value C of Eq. "common_var_for_grad" at
//           the external points and the internal-point states; App. B):
//           D1 (128 x ND N_s) = A1 (128 x (N_fe + N_s)) B1^T, row e of A1 the
//           element's [C_v; U_v];
//   q = J^{-T} q~ per solution point, on the CUDA cores from the TMEM row;
//   GEMM 2  [q_fe; q_fiu] = [M0; M12] q  for each gradient component i:
//           D2_i (128 x (N_fe + N_fiu)) = A2_i (128 x N_s) B2^T;
// and the rows of D2 go to the flux-point gradient arrays (QFE / QFIU layouts
// of kargs.hpp) that the residual kernel reads.  Each product is split into
// hi + lo TF32 parts, D = Ah Bh + Ah Bl + Al Bh.  The operators are staged
// once per CTA (K-major core-matrix layout, no swizzle); the A operands are
// written row by row by the threads, four threads per element (every fourth
// 4-column chunk), from values gathered one variable ahead.  One CTA of 512 threads per SM.  Every wait for the tensor
// core is bounded (2^22 polls, far above an MMA's microseconds); when one runs
// out the kernel records bit 1 of the error flag, the whole CTA stops and frees
// its tensor memory, and the caller's sdrt_sync reports SDRT_ERR_TIMEOUT.
#include <cstdint>

#include <cuda_runtime.h>

#include "kargs.hpp"
#include "launch.hpp"
#include "tc_util.cuh"

namespace sdrt {

using namespace tc;

namespace {

template <int NS, int NFE, int NFIU>
struct GradTC {
    static constexpr int V = 5, ND = 3, TE = 128, NT = 512, NH = NT / TE;   // NH threads per row
    static constexpr int NSP = (NS + 3) / 4 * 4;                        // D1 columns (d, s) at d * NSP + s
    static constexpr int N1 = ND * NSP, N1P = (N1 + 15) / 16 * 16;     // GEMM 1 N (M = 128 needs N % 16 == 0)
    static constexpr int K1 = NFE + NS, K1P = (K1 + 7) / 8 * 8;         // GEMM 1 K (K8 steps)
    static constexpr int N2 = NFE + NFIU, N2P = (N2 + 15) / 16 * 16;
    static constexpr int K2P = (NS + 7) / 8 * 8;
    static constexpr int B1_BYTES = N1P * K1P * 4, B2_BYTES = N2P * K2P * 4;
    static constexpr int A1_BYTES = TE * K1P * 4, A2_BYTES = TE * K2P * 4;
    // A region: A1 hi + lo, or two A2 buffers of hi + lo
    static constexpr int AREG = 2 * A1_BYTES > 4 * A2_BYTES ? 2 * A1_BYTES : 4 * A2_BYTES;
    static constexpr int SMEM = 2 * B1_BYTES + 2 * B2_BYTES + AREG + 64;
    static constexpr uint32_t COLS = 512;
    static_assert(N1P <= 256 && N2P <= 256 && N1P + 3 * N2P <= (int)COLS, "TMEM columns");
    static_assert(SMEM <= 227 * 1024, "shared memory");
};

// hi + lo TF32 parts of 4 values into the K-major core-matrix operand.
__device__ __forceinline__ void put4(unsigned char* hi, unsigned char* lo, int r, int k, int kp, const float (&x)[4]) {
    float4 h, l;
    float* hp = &h.x;
    float* lp = &l.x;
    #pragma unroll
    for (int q = 0; q < 4; ++q) {
        hp[q] = to_tf32(x[q]);
        lp[q] = to_tf32(x[q] - hp[q]);
    }
    *reinterpret_cast<float4*>(hi + core_off(r, k, kp)) = h;
    *reinterpret_cast<float4*>(lo + core_off(r, k, kp)) = l;
}

__device__ __forceinline__ void mma3(uint32_t d, const unsigned char* ah, const unsigned char* al,
                                     const unsigned char* bh, const unsigned char* bl, int kp, uint32_t idesc) {
    constexpr uint32_t LBO = 128;
    const uint32_t sbo = (uint32_t)(kp / 4) * 128;
    for (int kk = 0; kk < kp / 8; ++kk) {
        const uint32_t koff = (uint32_t)kk * 2 * LBO;
        const uint64_t dah = smem_desc(ah + koff, LBO, sbo), dal = smem_desc(al + koff, LBO, sbo);
        const uint64_t dbh = smem_desc(bh + koff, LBO, sbo), dbl = smem_desc(bl + koff, LBO, sbo);
        mma_tf32(d, dah, dbh, idesc, kk > 0 ? 1u : 0u);
        mma_tf32(d, dah, dbl, idesc, 1u);
        mma_tf32(d, dal, dbh, idesc, 1u);
    }
}

}  // namespace

template <int NS, int NFE, int NFIU>
__global__ void __launch_bounds__(512, 1) k_grad_tc(KBlock<float> B, const float* __restrict__ U,
                                                    const float* __restrict__ UFE, int64_t Ftot, float beta,
                                                    float* __restrict__ QFE, float* __restrict__ QFIU,
                                                    int* __restrict__ err) {
    using G = GradTC<NS, NFE, NFIU>;
    constexpr int V = G::V, ND = G::ND, TE = G::TE;
    constexpr int N1P = G::N1P, K1 = G::K1, K1P = G::K1P, N2 = G::N2, N2P = G::N2P, K2P = G::K2P;
    constexpr uint32_t ID1 = idesc_tf32(128, N1P), ID2 = idesc_tf32(128, N2P);
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* B1h = smem_raw;
    unsigned char* B1l = B1h + G::B1_BYTES;
    unsigned char* B2h = B1l + G::B1_BYTES;
    unsigned char* B2l = B2h + G::B2_BYTES;
    unsigned char* AR = B2l + G::B2_BYTES;
    uint64_t* bar = reinterpret_cast<uint64_t*>(AR + G::AREG);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);

    const int tid = threadIdx.x, warp = tid >> 5;
    constexpr int NH = G::NH;
    const int L = tid & (TE - 1), h = tid >> 7;           // element lane, quarter of the columns
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
    if (warp == 0) tmem_alloc(tslot, G::COLS);
    // B1[n][k] = [M16 | M15 P M12][(d, s)][k] with n = d * NSP + s (16-byte aligned
    // column groups per d): Ag holds it transposed, [k][Mg_pad], column d * NS + s.
    constexpr int NSP = G::NSP;
    for (int i = tid; i < N1P * K1P; i += G::NT) {
        const int n = i / K1P, k = i - n * K1P;
        const int d = n / NSP, sp = n - d * NSP;
        const float x = (d < ND && sp < NS && k < K1) ? B.Ag[(size_t)k * B.Mg_pad + d * NS + sp] : 0.f;
        const float hx = to_tf32(x);
        *reinterpret_cast<float*>(B1h + core_off(n, k, K1P)) = hx;
        *reinterpret_cast<float*>(B1l + core_off(n, k, K1P)) = to_tf32(x - hx);
    }
    // B2[n][k] = [M0; M12][n][k], row-major in Air.
    for (int i = tid; i < N2P * K2P; i += G::NT) {
        const int n = i / K2P, k = i - n * K2P;
        const float x = (n < N2 && k < NS) ? B.Air[(size_t)n * B.Md_pad + k] : 0.f;
        const float hx = to_tf32(x);
        *reinterpret_cast<float*>(B2h + core_off(n, k, K2P)) = hx;
        *reinterpret_cast<float*>(B2l + core_off(n, k, K2P)) = to_tf32(x - hx);
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
    unsigned char* A1h = AR;
    unsigned char* A1l = AR + G::A1_BYTES;

    uint32_t ph[2] = {0u, 0u};
    // true when the MMAs committed to bar[b] have completed
    auto wait = [&](int b) -> bool {
        const bool ok = mbar_wait(&bar[b], ph[b], 1ll << 22);
        if (!ok) atomicOr(err, 2);
        ph[b] ^= 1u;
        return ok;
    };
    bool aborted = false;
    const int ntiles = (B.nelem + TE - 1) / TE;
    // This thread's chunks of A1 row L for variable v of element e: [C_v at the
    // external points; U_v at the solution points], gathered into registers one
    // variable ahead (the loads run during the previous variable's stores).
    constexpr int NCH1 = (K1P / 4 + NH - 1) / NH;
    auto gather = [&](int v, int e, float (&pre)[NCH1][4]) {
        #pragma unroll
        for (int j = 0; j < NCH1; ++j) {
            const int c = h + j * NH;
            #pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = 4 * c + q;
                float val = 0.f;
                if (k < NFE) {
                    const int f = __ldg(B.fe_face + k);
                    const float s = __ldg(B.metric + (size_t)(B.mr_f + f * B.mr_ff + k * B.mr_fp + ND) * B.ld + e);
                    const float wo = s > 0.f ? 0.5f - beta : 0.5f + beta;   // own side is L when s > 0
                    const float own = __ldg(UFE + (size_t)v * Ftot + B.fe_base + (size_t)k * B.ld + e);
                    const float nbr = __ldg(UFE + (size_t)v * Ftot + __ldg(B.map + (size_t)k * B.ld + e));
                    val = wo * own + (1.f - wo) * nbr;
                } else if (k < K1) {
                    val = __ldg(U + B.u_off + (size_t)((k - NFE) * V + v) * B.ld + e);
                }
                pre[j][q] = val;
            }
        }
    };
    float pre[NCH1][4];
    if (blockIdx.x < ntiles) {
        const int e = min((int)blockIdx.x * TE + L, B.nelem - 1);
        gather(0, e, pre);
    }
    for (int tile = blockIdx.x; tile < ntiles && !aborted; tile += gridDim.x) {
        const int e0 = tile * TE;
        const bool valid = e0 + L < B.nelem;
        const int e = valid ? e0 + L : B.nelem - 1;       // lanes past the end repeat the last element
        const int tn = tile + gridDim.x;                  // next tile of this CTA
        const int en = min(tn * TE + L, B.nelem - 1);
        // J^{-1}_{di} = S_di / det J (affine block: one set per element)
        float Ji[ND * ND];
        {
            const float inv = __ldg(B.metric + e);
            #pragma unroll
            for (int k = 0; k < ND * ND; ++k) Ji[k] = __ldg(B.metric + (size_t)(1 + k) * B.ld + e) * inv;
        }
        #pragma unroll 1
        for (int v = 0; v < V && !aborted; ++v) {
            // A1 row L from the gathered values
            #pragma unroll
            for (int j = 0; j < NCH1; ++j) {
                const int c = h + j * NH;
                if (c < K1P / 4) put4(A1h, A1l, L, 4 * c, K1P, pre[j]);
            }
            fence_proxy_async();
            __syncthreads();
            if (tid == 0) {
                tc_fence_after();
                mma3(tmem, A1h, A1l, B1h, B1l, K1P, ID1);
                mma_commit(&bar[0]);
            }
            if (__syncthreads_or(!wait(0))) {
                aborted = true;
                break;
            }
            tc_fence_after();
            // q~ of this element at the solution points of this thread's chunks of
            // A2 (columns d * NSP + s of TMEM row L, groups of 4), loaded once for the 3 components
            constexpr int NCH = (K2P / 4 + NH - 1) / NH;      // chunks per thread
            float qt[NCH][ND][4];
            #pragma unroll
            for (int j = 0; j < NCH; ++j) {
                const int c = h + j * NH;
                #pragma unroll
                for (int d = 0; d < ND; ++d) {
                    uint32_t r[4] = {0u, 0u, 0u, 0u};
                    if (4 * c < NS) tmem_ld4_nowait(tmem + lane_base + (uint32_t)(d * NSP + 4 * c), r);
                    #pragma unroll
                    for (int q = 0; q < 4; ++q) qt[j][d][q] = __uint_as_float(r[q]);
                }
            }
            tmem_ld_wait();
            // GEMM 2 per gradient component i: A2_i = q_i(s) = sum_d J^{-1}_{di} q~(d, s)
            #pragma unroll
            for (int i = 0; i < ND; ++i) {
                const int b = i & 1;
                if (i == 2 && __syncthreads_or(!wait(0))) {   // buffer 0 read by the MMAs of component 0
                    aborted = true;
                    break;
                }
                unsigned char* ah = AR + b * 2 * G::A2_BYTES;
                unsigned char* al = ah + G::A2_BYTES;
                #pragma unroll
                for (int j = 0; j < NCH; ++j) {
                    const int c = h + j * NH;
                    if (c >= K2P / 4) continue;
                    float x[4];
                    #pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float val = 0.f;
                        if (4 * c + q < NS) {
                            val = Ji[0 * ND + i] * qt[j][0][q];
                            #pragma unroll
                            for (int d = 1; d < ND; ++d) val = fmaf(Ji[d * ND + i], qt[j][d][q], val);
                        }
                        x[q] = val;
                    }
                    put4(ah, al, L, 4 * c, K2P, x);
                }
                fence_proxy_async();
                __syncthreads();
                if (tid == 0) {
                    tc_fence_after();
                    mma3(tmem + (uint32_t)(N1P + i * N2P), ah, al, B2h, B2l, K2P, ID2);
                    mma_commit(&bar[b]);
                }
            }
            if (aborted) break;
            {
                const bool ok1 = wait(1), ok0 = wait(0);
                if (__syncthreads_or(!(ok1 && ok0))) {
                    aborted = true;
                    break;
                }
            }
            tc_fence_after();
            // the next variable's (or the next tile's first) A1 values, in flight during the stores
            if (v + 1 < V) gather(v + 1, e, pre);
            else if (tn < ntiles) gather(0, en, pre);
            // rows of D2 -> QFE / QFIU (component i, variable v)
            #pragma unroll 1
            for (int i = 0; i < ND; ++i) {
                const size_t dv = (size_t)(i * V + v);
                #pragma unroll 1
                for (int c = h; c < N2P / 16; c += NH) {
                    float x[16];
                    tmem_ld16(tmem + lane_base + (uint32_t)(N1P + i * N2P + c * 16), x);
                    if (valid) {
                        #pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int n = c * 16 + j;
                            if (n < NFE)
                                QFE[dv * Ftot + B.fe_base + (size_t)n * B.ld + e] = x[j];
                            else if (n < N2)
                                QFIU[(size_t)B.qfiu_off + ((size_t)(n - NFE) * (ND * V) + dv) * B.ld + e] = x[j];
                        }
                    }
                }
            }
            tc_fence_before();
            __syncthreads();                                  // TMEM rows read, A region free
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, G::COLS);
}

namespace {

template <int NS, int NFE, int NFIU>
int launch_grad_tc_impl(const KBlock<float>& B, const float* U, const float* UFE, int64_t Ftot, float beta,
                        float* QFE, float* QFIU, int* err, int nsm, cudaStream_t st) {
    using G = GradTC<NS, NFE, NFIU>;
    auto k = k_grad_tc<NS, NFE, NFIU>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    const int tiles = (B.nelem + G::TE - 1) / G::TE;
    k<<<tiles < nsm ? tiles : nsm, G::NT, G::SMEM, st>>>(B, U, UFE, Ftot, beta, QFE, QFIU, err);
    return 0;
}

}  // namespace

// Element types instantiated: tetrahedra of degree 3 and 4, hexahedra of
// degree 2, prisms of degree 2 (N_s, N_fe, N_fiu).
bool grad_tc_available(const KBlock<float>& B, int V, int nd) {
    if (V != 5 || nd != 3 || B.mr_inv != 0) return false;   // 3D Navier-Stokes, affine blocks
    const int s = B.nsol, f = B.nfe, u = B.nfiu;
    return (s == 20 && f == 40 && u == 10) || (s == 35 && f == 60 && u == 20) || (s == 27 && f == 54 && u == 54) ||
           (s == 18 && f == 39 && u == 21);
}

int launch_grad_tc(const KBlock<float>& B, int V, int nd, const float* U, const float* UFE, int64_t Ftot,
                   const KPhys<float>& P, float* QFE, float* QFIU, int* err, int nsm, cudaStream_t st) {
    if (!grad_tc_available(B, V, nd)) return -1;
    const int s = B.nsol, f = B.nfe;
    if (s == 20 && f == 40) return launch_grad_tc_impl<20, 40, 10>(B, U, UFE, Ftot, P.beta, QFE, QFIU, err, nsm, st);
    if (s == 35 && f == 60) return launch_grad_tc_impl<35, 60, 20>(B, U, UFE, Ftot, P.beta, QFE, QFIU, err, nsm, st);
    if (s == 27 && f == 54) return launch_grad_tc_impl<27, 54, 54>(B, U, UFE, Ftot, P.beta, QFE, QFIU, err, nsm, st);
    return launch_grad_tc_impl<18, 39, 21>(B, U, UFE, Ftot, P.beta, QFE, QFIU, err, nsm, st);
}

}  // namespace sdrt
