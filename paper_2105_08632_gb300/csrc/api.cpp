// C ABI of the SDRT library: contexts, element types, meshes and the residual,
// RK4, JVP / VJP entry points (declared in include/sdrt.h).
#include "sdrt.h"

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <array>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <vector>

#include "kargs.hpp"
#include "gen_api.hpp"
#include "launch.hpp"
#include "mapping.hpp"
#include "refel.hpp"
#include "internal.hpp"

using namespace sdrt;

namespace {

// Owned device allocation.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    cudaError_t alloc(size_t n) {
        release();
        bytes = n;
        if (n == 0) return cudaSuccess;
        return cudaMalloc(&p, n);
    }
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

template <typename T>
cudaError_t upload(DevBuf& b, const std::vector<T>& h) {
    cudaError_t e = b.alloc(h.size() * sizeof(T));
    if (e != cudaSuccess || h.empty()) return e;
    return cudaMemcpy(b.p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
}

struct EType {
    sdrt_etype_desc desc{};
    RefElement R;
    int Mi = 0, Mi_pad = 0, Md_pad = 0, Mg_pad = 0, Mir = 0, Mdt_pad = 0, Agr_pad = 0;
    DevBuf Ai[2], Ad[2], Air[2], Ag[2], Adt[2], Agr[2];  // [0] double, [1] float
    DevBuf Mq[2], wq[2];              // element quadrature: nodal basis at the points, weights
    DevBuf fe_face, fi_tab;
};

struct MBlock {
    int etype = 0, nelem = 0, ld = 0;
    int64_t u_off = 0, fe_base = 0, canon_base = 0;
    DevBuf metric, map;
    // Metric rows (kargs.hpp): one value set per element (affine) or per
    // point (curved: quadratic map, sdrt_setup_mesh_curved).
    bool curved = false;
    int nmetric = 0;
    int mr_inv = 0, mr_ss = 1, mr_ssk = 0, mr_si = 1, mr_sik = 0, mr_f = 0, mr_ff = 0, mr_fp = 0;
    int tile = 32;                // elements per CTA tile
    int tile_dual = 32;
    int gtile = 0, gtile_dual = 0;  // gradient kernel (viscous systems)
    int vtile = 0;                // VJP kernels (0: not available for this block)
    int64_t qfiu_off = 0;         // element offset of the block in QFIU
    // Record layout of the register-blocked path (kernels_fast.cu).
    int ers = 0, frs = 0, frec = 0, nmp = 0, pstride = 0;
    int64_t rec_base = 0, fiur_base = 0;
    DevBuf maos, pfr, perm, recoff;
    // Operator-specialised path (gen_stage.cuh): launcher of the element
    // type and the face-record index of every external point's partner,
    // [nfe][ld] (gen_api.hpp layout).
    GenLauncher gen = nullptr;
    DevBuf pmap;
};

struct Mesh {
    sdrt_physics phys{};
    int nvar = 0, nd = 0;
    std::vector<std::unique_ptr<MBlock>> blocks;
    int64_t state_len = 0, Ftot = 0, ndof = 0, nfe_total = 0;
    bool fast = false;                // every block on the register-blocked record path
    bool curved = false;              // some block has curved elements (generic kernels only)
    bool tc3 = false;                 // SDRT_TF32X3: tensor-core contractions where instantiated
    int64_t rec_total = 0, fiur_total = 0;
    int64_t qfiu_total = 0;           // viscous: length of QFIU
    std::vector<int32_t> partner;     // canonical face map
    std::vector<uint8_t> is_left;
    std::vector<double> sol_xyz;
    DevBuf ufe, dufe, ustage, uacc, uhost_dev, rec, drec, fiur, dfiur;
    DevBuf rec2, fiur2;          // second record buffers of the fused RK4 stages
    DevBuf qfe, dqfe, qfiu, dqfiu;    // viscous: flux-point gradients (kargs.hpp layout)
    DevBuf cbar;                      // viscous VJP: adjoint of the common value (UFE layout)
    DevBuf rk_r, rk_du, rk_err, rk_u0, rk_part;   // RK54: residual, second register, estimate, step start
    DevBuf qsol, diag_sums;           // Taylor-Green diagnostics: solution-point gradients, integrals
    double pi_err_prev = 1.0;         // RK54 PI controller: error norm of the last accepted step
    // Block tables of the generic kernels (one launch per kernel kind walks
    // every block): host copies and the device array, in the mesh precision.
    std::vector<KBlock<float>> kb_f;
    std::vector<KBlock<double>> kb_d;
    DevBuf kb_dev;
    // RK4 graph cache
    cudaGraphExec_t graph = nullptr;
    const void* graph_u = nullptr;
    double graph_dt = 0;
    std::vector<int> graph_slots;     // timing slots recorded inside the graph
    int64_t graph_launches = 0;       // kernel launches in one replay
    bool warmed = false;
    // Partition (sdrt_setup_partition): ghost blocks are copies of other
    // partitions' elements that share faces with this one; only their face
    // records are used, filled from the received exchange buffer.
    bool partition = false;
    std::vector<std::unique_ptr<MBlock>> ghosts;
    int xfrec = 0;                    // values per exchanged face record
    int64_t nsend = -1, nrecv = -1;   // -1: no exchange lists yet
    DevBuf xsend_off, xrecv_off;      // record path: REC offsets of the sent / received face records
    DevBuf xsend_idx, xrecv_idx;      // generic path: UFE index of every record value (-1: padding)
    const void* part_u = nullptr;     // generic path: the state of the last sdrt_residual_begin
    // Viscous partitions: gradient records (flux-point gradients of the face's
    // points, QFE indices) exchanged between sdrt_residual_gradients and _end.
    int xgrec = 0;
    DevBuf xsend_gidx, xrecv_gidx;
    bool part_grad = false;           // sdrt_residual_gradients ran since the last begin
    // Operator-specialised path: every block has a generated kernel (FP32
    // 3D Euler / Rusanov, SDRT scheme, whole mesh); two face-record arrays
    // (F_tot points x nvar, point-major) alternate between RK stages; the blocks run as
    // concurrent branches (one stream each, forked from and joined to the
    // context's stream).
    bool gen = false;
    DevBuf fr[2];
    std::vector<cudaStream_t> br;
    std::vector<cudaEvent_t> brev;
    cudaEvent_t fork_ev = nullptr;
    ~Mesh() {
        if (graph) cudaGraphExecDestroy(graph);
        for (cudaStream_t st : br) cudaStreamDestroy(st);
        for (cudaEvent_t ev : brev) cudaEventDestroy(ev);
        if (fork_ev) cudaEventDestroy(fork_ev);
    }
};

}  // namespace

struct sdrt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int nsm = 1;
    bool host_only = false;       // device == -1: host-side setup only, no compute
    bool use_tc = false;          // tensor-core interpolation where instantiated (SDRT_OPT_TENSOR_CORES)
    bool use_tc_div = false;      // tensor-core divergence where instantiated (SDRT_OPT_TC_DIVERGENCE)
    bool fuse_rk = true;          // next-stage interpolation in the RK4 stage update (SDRT_OPT_FUSED_RK)
    int use_gen = 1;              // operator-specialised kernels where generated (SDRT_OPT_GENERATED)
    int wait_polls = 0;           // first copy wait of the record flux kernel (SDRT_OPT_WAIT_POLLS)
    bool nvtx = false;            // NVTX ranges around entry points and kernel launches (SDRT_OPT_NVTX)
    bool use_tc_grad = true;      // tensor-core gradient chain where instantiated (SDRT_OPT_TC_GRADIENT)
    void* noalloc_scratch = nullptr;   // device address of sdrt_residual_noalloc's static buffer
    std::string err;
    std::vector<std::unique_ptr<EType>> etypes;
    std::vector<std::unique_ptr<Mesh>> meshes;
    DevBuf flag;
    int64_t launches = 0;
    // Per-launch timing: slot s owns events ev[2s], ev[2s+1] and a kernel kind.
    bool prof = false;
    std::vector<cudaEvent_t> ev;
    std::vector<int> slot_kind;
    std::vector<int> eager_slots;        // reusable slots for launches outside graphs
    int eager_next = 0;
    std::vector<int>* capture_slots = nullptr;   // slots of the graph being captured
    std::vector<int> pending;            // slots recorded since the last collect
    ~sdrt_ctx() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

namespace {

enum { KIND_INTERP = 0, KIND_RESIDUAL = 1, KIND_JVP = 2, KIND_GRAD = 3, KIND_COUNT = 4 };

int new_slot(sdrt_ctx* ctx, int kind) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return -1;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return -1;
    }
    ctx->ev.push_back(a);
    ctx->ev.push_back(b);
    ctx->slot_kind.push_back(kind);
    return (int)ctx->slot_kind.size() - 1;
}

// Start timing one launch: returns the slot (or -1 when profiling is off).
const char* kind_name(int kind) {
    static const char* names[KIND_COUNT] = {"interpolation", "residual", "residual_jvp", "gradient"};
    const int k = kind & 0xff;
    return k >= 0 && k < KIND_COUNT ? names[k] : "kernel";
}

// An NVTX range for the lifetime of an entry point's call (SDRT_OPT_NVTX).
struct NvtxScope {
    bool on;
    NvtxScope(const sdrt_ctx* ctx, const char* name) : on(ctx && ctx->nvtx) {
        if (on) nvtxRangePushA(name);
    }
    ~NvtxScope() {
        if (on) nvtxRangePop();
    }
};

int prof_begin(sdrt_ctx* ctx, int kind, cudaStream_t st = nullptr) {
    if (!st) st = ctx->stream;
    if (ctx->nvtx) nvtxRangePushA(kind_name(kind));
    if (!ctx->prof) return -1;
    int s;
    if (ctx->capture_slots) {
        s = new_slot(ctx, kind);
        if (s < 0) return -1;
        ctx->capture_slots->push_back(s);
    } else {
        if (ctx->eager_next == (int)ctx->eager_slots.size()) {
            int n = new_slot(ctx, kind);
            if (n < 0) return -1;
            ctx->eager_slots.push_back(n);
        }
        s = ctx->eager_slots[ctx->eager_next++];
        ctx->slot_kind[s] = kind;
        ctx->pending.push_back(s);
    }
    // Inside a stream capture a plain record is only a dependency marker: an
    // external record becomes an event-record node that replays record.
    if (ctx->capture_slots) cudaEventRecordWithFlags(ctx->ev[2 * s], st, cudaEventRecordExternal);
    else cudaEventRecord(ctx->ev[2 * s], st);
    return s;
}

void prof_end(sdrt_ctx* ctx, int s, cudaStream_t st = nullptr) {
    if (ctx->nvtx) nvtxRangePop();
    if (s < 0) return;
    if (!st) st = ctx->stream;
    if (ctx->capture_slots) cudaEventRecordWithFlags(ctx->ev[2 * s + 1], st, cudaEventRecordExternal);
    else cudaEventRecord(ctx->ev[2 * s + 1], st);
}

bool viscous(const Mesh& m) {
    return m.phys.system == SDRT_ADVDIFF || m.phys.system == SDRT_NAVIER_STOKES;
}

int fail(sdrt_ctx* c, int code, const std::string& msg) {
    if (c) c->err = msg;
    return code;
}

#define SDRT_CUDA(call)                                                                            \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess)                                                                     \
            return fail(ctx, SDRT_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)

int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Affine map of one element: x = x0 + J (x~ - x~0); J columns from vertex edges.
bool element_jacobian(int shape, const double* X, int nd, double* J) {
    int cols[3];
    switch (shape) {
        case TRI: cols[0] = 1; cols[1] = 2; break;
        case QUAD: cols[0] = 1; cols[1] = 3; break;
        case TET: cols[0] = 1; cols[1] = 2; cols[2] = 3; break;
        case PRI: cols[0] = 1; cols[1] = 2; cols[2] = 3; break;
        default: cols[0] = 1; cols[1] = 3; cols[2] = 4; break;
    }
    for (int d = 0; d < nd; ++d)
        for (int i = 0; i < nd; ++i) J[i * nd + d] = 0.5 * (X[cols[d] * nd + i] - X[i]);
    // affinity check on every vertex
    const auto& ref = ref_vertices(shape);
    const int nv = shape_nverts(shape);
    double scale = 0;
    for (int k = 0; k < nd * nd; ++k) scale = std::max(scale, std::fabs(J[k]));
    for (int v = 0; v < nv; ++v)
        for (int i = 0; i < nd; ++i) {
            double x = X[i];
            for (int d = 0; d < nd; ++d) x += J[i * nd + d] * (ref[v * nd + d] - ref[d]);
            if (std::fabs(x - X[v * nd + i]) > 1e-10 * (scale + std::fabs(X[v * nd + i]))) return false;
        }
    return true;
}

double det_inv(const double* J, int nd, double* Ji) {
    if (nd == 2) {
        double d = J[0] * J[3] - J[1] * J[2];
        Ji[0] = J[3] / d;
        Ji[1] = -J[1] / d;
        Ji[2] = -J[2] / d;
        Ji[3] = J[0] / d;
        return d;
    }
    double d = J[0] * (J[4] * J[8] - J[5] * J[7]) - J[1] * (J[3] * J[8] - J[5] * J[6]) +
               J[2] * (J[3] * J[7] - J[4] * J[6]);
    Ji[0] = (J[4] * J[8] - J[5] * J[7]) / d;
    Ji[1] = (J[2] * J[7] - J[1] * J[8]) / d;
    Ji[2] = (J[1] * J[5] - J[2] * J[4]) / d;
    Ji[3] = (J[5] * J[6] - J[3] * J[8]) / d;
    Ji[4] = (J[0] * J[8] - J[2] * J[6]) / d;
    Ji[5] = (J[2] * J[3] - J[0] * J[5]) / d;
    Ji[6] = (J[3] * J[7] - J[4] * J[6]) / d;
    Ji[7] = (J[1] * J[6] - J[0] * J[7]) / d;
    Ji[8] = (J[0] * J[4] - J[1] * J[3]) / d;
    return d;
}

template <typename T>
KBlock<T> make_kblock(const EType& et, const MBlock& b) {
    const int pi = std::is_same<T, float>::value ? 1 : 0;
    KBlock<T> K{};
    K.nsol = et.R.nsol;
    K.nfe = et.R.nfe;
    K.nfi = et.R.nfi;
    K.nfiu = et.R.nfiu;
    K.nfaces = et.R.nfaces;
    K.nelem = b.nelem;
    K.ld = b.ld;
    K.u_off = b.u_off;
    K.fe_base = b.fe_base;
    K.Ai = et.Ai[pi].as<T>();
    K.Mi = et.Mi;
    K.Mi_pad = et.Mi_pad;
    K.Ad = et.Ad[pi].as<T>();
    K.Md_pad = et.Md_pad;
    K.Ag = et.Ag[pi].as<T>();
    K.Adt = et.Adt[pi].as<T>();
    K.Mdt_pad = et.Mdt_pad;
    K.Mg_pad = et.Mg_pad;
    K.Agr = et.Agr[pi].as<T>();
    K.Agr_pad = et.Agr_pad;
    K.qfiu_off = b.qfiu_off;
    K.fe_face = et.fe_face.as<int>();
    K.fi_tab = et.fi_tab.as<int>();
    K.metric = b.metric.as<T>();
    K.mr_inv = b.mr_inv;
    K.mr_ss = b.mr_ss;
    K.mr_ssk = b.mr_ssk;
    K.mr_si = b.mr_si;
    K.mr_sik = b.mr_sik;
    K.mr_f = b.mr_f;
    K.mr_ff = b.mr_ff;
    K.mr_fp = b.mr_fp;
    K.map = b.map.as<int>();
    K.Air = et.Air[pi].as<T>();
    K.Mir = et.Mir;
    K.ers = b.ers;
    K.frs = b.frs;
    K.frec = b.frec;
    K.nmp = b.nmp;
    K.pstride = b.pstride;
    K.rec_base = b.rec_base;
    K.fiur_base = b.fiur_base;
    K.maos = b.maos.as<T>();
    K.pfr = b.pfr.as<int>();
    K.perm = b.perm.as<unsigned char>();
    K.recoff = b.recoff.as<int>();
    K.te_interp = 32;
    K.te_res = b.tile;
    K.te_res_dual = b.tile_dual;
    K.te_grad = b.gtile;
    K.te_grad_dual = b.gtile_dual;
    K.te_vjp = b.vtile;
    return K;
}

template <typename T>
KSet<T> kset(const Mesh& m);
template <>
KSet<float> kset<float>(const Mesh& m) {
    return {m.kb_f.data(), m.kb_dev.as<KBlock<float>>(), (int)m.kb_f.size()};
}
template <>
KSet<double> kset<double>(const Mesh& m) {
    return {m.kb_d.data(), m.kb_dev.as<KBlock<double>>(), (int)m.kb_d.size()};
}

template <typename T>
KPhys<T> make_phys(const sdrt_physics& p) {
    KPhys<T> P{};
    for (int d = 0; d < 3; ++d) P.a[d] = (T)p.a[d];
    P.gamma = (T)p.gamma;
    P.mu = (T)p.mu;
    P.prandtl = (T)p.prandtl;
    P.beta = (T)p.beta;
    P.eta = (T)p.eta;
    return P;
}

// Operator-specialised path: one launch of `kind` (0 interpolation into the
// face records FRout, 1 fused stage) per block; with several blocks each
// block is a branch of its own stream, forked from and joined to the
// context's stream (concurrent kernels; inside a graph capture, parallel
// graph branches), except while per-launch timing is on.
int gen_launch_blocks(sdrt_ctx* ctx, Mesh& m, int kind, const float* U, const float* FRin, float* FRout,
                      const KEpi<float>& E) {
    const KPhys<float> P = make_phys<float>(m.phys);
    const int nb = (int)m.blocks.size();
    // With per-launch timing on, the branches run one after the other on the
    // context's stream, so that each launch's events time that launch alone.
    const bool fork = nb > 1 && !ctx->prof;
    if (fork) SDRT_CUDA(cudaEventRecord(m.fork_ev, ctx->stream));
    for (int b = 0; b < nb; ++b) {
        MBlock& mb = *m.blocks[b];
        cudaStream_t st = fork ? m.br[b] : ctx->stream;
        if (fork) SDRT_CUDA(cudaStreamWaitEvent(st, m.fork_ev, 0));
        GenArgs a{};
        a.nelem = mb.nelem;
        a.ld = mb.ld;
        a.u_off = mb.u_off;
        a.fr_base = mb.fe_base * m.nvar;
        a.metric = mb.metric.as<float>();
        a.pmap = mb.pmap.as<int>();
        a.U = U;
        a.FRin = FRin;
        a.FRout = FRout;
        a.P = P;
        a.E = E;
        // timing slot of this block's launch (kind | (block + 1) << 8: sdrt_profile_collect_blocks)
        const int s = prof_begin(ctx, (kind == 0 ? KIND_INTERP : KIND_RESIDUAL) | ((b + 1) << 8), st);
        const int r = mb.gen(kind, a, m.nvar, m.phys.system, m.phys.riemann, ctx->nsm, st);
        prof_end(ctx, s, st);
        if (r != 0) return fail(ctx, SDRT_ERR_UNSUPPORTED, "generated kernel not instantiated for this system");
        ++ctx->launches;
        if (fork) {
            SDRT_CUDA(cudaEventRecord(m.brev[b], st));
            SDRT_CUDA(cudaStreamWaitEvent(ctx->stream, m.brev[b], 0));
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SDRT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return SDRT_OK;
}

// Residual-type evaluation of the whole mesh: interpolation of every block,
// then the residual kernel of every block with epilogue E.
template <typename T>
int run_residual(sdrt_ctx* ctx, Mesh& m, const T* U, const T* dU, const KEpi<T>& E) {
    if constexpr (std::is_same<T, float>::value) {
        if (!dU && m.gen && ctx->use_gen) {
            // Operator-specialised kernels: face records of U, then the fused stage.
            int r = gen_launch_blocks(ctx, m, 0, U, nullptr, m.fr[0].as<float>(), E);
            if (r) return r;
            return gen_launch_blocks(ctx, m, 1, U, m.fr[0].as<float>(), nullptr, E);
        }
    }
    const KPhys<T> P = make_phys<T>(m.phys);
    T* ufe = m.ufe.as<T>();
    T* dufe = m.dufe.as<T>();
    const int sys = m.phys.system;   // sdrt_system and System share their values
    bool fast = m.fast;
    if (fast && dU)
        for (auto& bp : m.blocks)
            if (!fast_jvp_available<T>(make_kblock<T>(*ctx->etypes[bp->etype], *bp), m.nvar)) fast = false;
    if (fast) {
        // Register-blocked record path: interpolation of every block, then fluxes + divergence.
        T* rec = m.rec.as<T>();
        T* drec = m.drec.as<T>();
        T* fiur = m.fiur.as<T>();
        T* dfiur = m.dfiur.as<T>();
        for (auto& bp : m.blocks) {
            const EType& et = *ctx->etypes[bp->etype];
            KBlock<T> K = make_kblock<T>(et, *bp);
            // Interpolation: tensor cores (tcgen05, 3xTF32) where instantiated, else CUDA cores.
            auto interp = [&](const T* X, T* rec_out, T* fiur_out) {
                int r = -1;
                if constexpr (std::is_same<T, float>::value) {
                    if ((ctx->use_tc || m.tc3) && tc_interp_available(et.R.shape, et.R.nsol, m.nvar))
                        r = launch_interp_tc(K, m.nvar, X, rec_out, fiur_out, ctx->flag.as<int>(), ctx->nsm,
                                             ctx->stream);
                }
                if (r != 0)
                    r = launch_interp_rec<T>(K, m.nvar, X, rec_out, fiur_out, ctx->flag.as<int>(), ctx->nsm,
                                             ctx->stream);
                return r;
            };
            int s = prof_begin(ctx, KIND_INTERP);
            int r = interp(U, rec, fiur);
            prof_end(ctx, s);
            if (r != 0) return fail(ctx, SDRT_ERR_UNSUPPORTED, "record path not instantiated");
            ++ctx->launches;
            if (dU) {
                s = prof_begin(ctx, KIND_INTERP);
                interp(dU, drec, dfiur);
                prof_end(ctx, s);
                ++ctx->launches;
            }
        }
        KEpi<T> Ew = E;
        Ew.wait_polls = ctx->wait_polls;
        for (auto& bp : m.blocks) {
            const EType& et = *ctx->etypes[bp->etype];
            KBlock<T> K = make_kblock<T>(et, *bp);
            const int s = prof_begin(ctx, dU ? KIND_JVP : KIND_RESIDUAL);
            int r = -1;
            if constexpr (std::is_same<T, float>::value) {
                if (!dU && (ctx->use_tc_div || m.tc3) &&
                    tc_flux_available(et.R.shape, et.R.nsol, m.nvar, sys, m.phys.riemann))
                    r = launch_flux_tc(K, rec, fiur, P, E, ctx->nsm, ctx->stream);
            }
            if (r != 0)
                launch_flux_rec<T>(K, sys, rec, dU ? drec : nullptr, fiur, dU ? dfiur : nullptr, P, Ew, ctx->nsm,
                                   ctx->stream);
            prof_end(ctx, s);
            ++ctx->launches;
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(ctx, SDRT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
        return SDRT_OK;
    }
    // Generic path: one launch per kernel kind, each walking the tiles of every block.
    const KSet<T> ks = kset<T>(m);
    int s = prof_begin(ctx, KIND_INTERP);
    launch_interp_ext<T>(ks, m.nvar, U, ufe, m.Ftot, ctx->nsm, ctx->stream);
    prof_end(ctx, s);
    ++ctx->launches;
    if (dU) {
        s = prof_begin(ctx, KIND_INTERP);
        launch_interp_ext<T>(ks, m.nvar, dU, dufe, m.Ftot, ctx->nsm, ctx->stream);
        prof_end(ctx, s);
        ++ctx->launches;
    }
    KVisc<T> Q{};
    if (viscous(m)) {
        // Flux-point gradients of every block (they read every block's u_fe).
        Q = {m.qfe.as<T>(), dU ? m.dqfe.as<T>() : nullptr, m.qfiu.as<T>(), dU ? m.dqfiu.as<T>() : nullptr};
        bool tc_grad = false;
        if constexpr (std::is_same<T, float>::value) {
            // Tensor-core gradient chain where every block is of an instantiated kind.
            tc_grad = !dU && ctx->use_tc_grad;
            for (auto& bp : m.blocks)
                tc_grad = tc_grad && grad_tc_available(make_kblock<float>(*ctx->etypes[bp->etype], *bp), m.nvar, m.nd);
            if (tc_grad)
                for (auto& bp : m.blocks) {
                    s = prof_begin(ctx, KIND_GRAD);
                    launch_grad_tc(make_kblock<float>(*ctx->etypes[bp->etype], *bp), m.nvar, m.nd, U, ufe, m.Ftot, P,
                                   m.qfe.as<float>(), m.qfiu.as<float>(), ctx->flag.as<int>(), ctx->nsm, ctx->stream);
                    prof_end(ctx, s);
                    ++ctx->launches;
                }
        }
        if (!tc_grad) {
            s = prof_begin(ctx, KIND_GRAD);
            int r = launch_grad<T>(ks, sys, m.nd, U, dU, ufe, dU ? dufe : nullptr, m.Ftot, P, m.qfe.as<T>(),
                                   dU ? m.dqfe.as<T>() : nullptr, m.qfiu.as<T>(), dU ? m.dqfiu.as<T>() : nullptr,
                                   ctx->nsm, ctx->stream);
            prof_end(ctx, s);
            if (r == -2)
                return fail(ctx, SDRT_ERR_UNSUPPORTED, "JVP tile does not fit in shared memory for this element type");
            if (r != 0) return fail(ctx, SDRT_ERR_UNSUPPORTED, "system not supported by the gradient kernel");
            ++ctx->launches;
        }
    }
    s = prof_begin(ctx, dU ? KIND_JVP : KIND_RESIDUAL);
    int r = launch_residual<T>(ks, sys, m.phys.riemann, m.nd, U, dU, ufe, dU ? dufe : nullptr, m.Ftot, P, E, Q, ctx->nsm,
                               ctx->stream);
    prof_end(ctx, s);
    if (r == -2) return fail(ctx, SDRT_ERR_UNSUPPORTED, "JVP tile does not fit in shared memory for this element type");
    if (r != 0) return fail(ctx, SDRT_ERR_UNSUPPORTED, "system / flux combination not supported");
    ++ctx->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SDRT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return SDRT_OK;
}

// W^T dR/dU: forward interpolation of every block, the face adjoints GS of
// every block (in the tangent face-state buffer), then the element pass.
template <typename T>
int run_vjp(sdrt_ctx* ctx, Mesh& m, const T* U, const T* W, T* out) {
    const KPhys<T> P = make_phys<T>(m.phys);
    T* ufe = m.ufe.as<T>();
    T* gs = m.dufe.as<T>();
    const KSet<T> ks = kset<T>(m);
    if (!ks.all_tiled(TK_VJP))
        return fail(ctx, SDRT_ERR_UNSUPPORTED, "VJP tile does not fit in shared memory for this element type");
    int s = prof_begin(ctx, KIND_INTERP);
    launch_interp_ext<T>(ks, m.nvar, U, ufe, m.Ftot, ctx->nsm, ctx->stream);
    prof_end(ctx, s);
    ++ctx->launches;
    if (viscous(m)) {
        // Forward gradients at the flux points, then the three adjoint passes.
        s = prof_begin(ctx, KIND_GRAD);
        int r = launch_grad<T>(ks, m.phys.system, m.nd, U, nullptr, ufe, nullptr, m.Ftot, P, m.qfe.as<T>(), nullptr,
                               m.qfiu.as<T>(), nullptr, ctx->nsm, ctx->stream);
        prof_end(ctx, s);
        if (r != 0) return fail(ctx, SDRT_ERR_UNSUPPORTED, "system not supported by the gradient kernel");
        ++ctx->launches;
        for (int pass = 0; pass < 3; ++pass) {
            s = prof_begin(ctx, KIND_JVP);
            r = launch_vjp_visc<T>(ks, pass, m.phys.system, m.phys.riemann, m.nd, U, W, ufe, m.qfe.as<T>(),
                                   m.qfiu.as<T>(), gs, m.cbar.as<T>(), m.Ftot, P, out, ctx->flag.as<int>(), ctx->nsm,
                                   ctx->stream);
            prof_end(ctx, s);
            if (r != 0) return fail(ctx, SDRT_ERR_UNSUPPORTED, "system / flux combination not supported by the VJP");
            ++ctx->launches;
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(ctx, SDRT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
        return SDRT_OK;
    }
    for (int pass = 0; pass < 2; ++pass) {
        s = prof_begin(ctx, KIND_JVP);
        int r = launch_vjp<T>(ks, pass, m.phys.system, m.phys.riemann, m.nd, U, W, ufe, gs, m.Ftot, P, out,
                              ctx->flag.as<int>(), ctx->nsm, ctx->stream);
        prof_end(ctx, s);
        if (r != 0) return fail(ctx, SDRT_ERR_UNSUPPORTED, "system / flux combination not supported by the VJP");
        ++ctx->launches;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SDRT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return SDRT_OK;
}

// Whether stages 1-3 of RK4 can interpolate the next stage's state in their
// epilogue (record path, FP32 Euler on tetrahedra of degree 3, CUDA-core kernels).
bool rk_fusable(sdrt_ctx* ctx, const Mesh& m) {
    if (!m.fast || m.phys.precision != SDRT_FP32 || ctx->use_tc || ctx->use_tc_div || m.tc3 || !m.rec2.p ||
        !m.fiur2.p)
        return false;
    for (auto& bp : m.blocks)
        if (!flux_rec_fusable(make_kblock<float>(*ctx->etypes[bp->etype], *bp), m.nvar, m.phys.system)) return false;
    return true;
}

// RK4 with one interpolation per step: the state U is interpolated into the
// records once, and the epilogues of stages 1-3 interpolate the next stage's
// state into the other record buffer (the two alternate), so the stage state
// never goes to global memory.  Stage 4 writes the new U.
int rk4_stages_fused(sdrt_ctx* ctx, Mesh& m, float* U, double dt) {
    const KPhys<float> P = make_phys<float>(m.phys);
    float* recs[2] = {m.rec.as<float>(), m.rec2.as<float>()};
    float* fiurs[2] = {m.fiur.as<float>(), m.fiur2.as<float>()};
    for (auto& bp : m.blocks) {
        KBlock<float> K = make_kblock<float>(*ctx->etypes[bp->etype], *bp);
        const int s = prof_begin(ctx, KIND_INTERP);
        const int r = launch_interp_rec<float>(K, m.nvar, U, recs[0], fiurs[0], ctx->flag.as<int>(), ctx->nsm,
                                               ctx->stream);
        prof_end(ctx, s);
        if (r != 0) return fail(ctx, SDRT_ERR_UNSUPPORTED, "record path not instantiated");
        ++ctx->launches;
    }
    KEpi<float> E{};
    E.flag = ctx->flag.as<int>();
    E.wait_polls = ctx->wait_polls;
    E.u0 = U;
    E.uacc = m.uacc.as<float>();
    E.unext = m.ustage.as<float>();
    const float c6 = (float)(dt / 6.0), c3 = (float)(dt / 3.0), c2 = (float)(dt / 2.0), c1 = (float)dt;
    const int modes[4] = {EPI_RK_FIRST, EPI_RK_MID, EPI_RK_MID, EPI_RK_LAST};
    const float cacc[4] = {c6, c3, c3, c6};
    const float cnext[4] = {c2, c2, c1, 0.0f};
    for (int stage = 0; stage < 4; ++stage) {
        E.mode = modes[stage];
        E.cacc = cacc[stage];
        E.cnext = cnext[stage];
        E.out = stage == 3 ? U : nullptr;
        E.rec_next = stage < 3 ? recs[(stage + 1) & 1] : nullptr;
        E.fiur_next = stage < 3 ? fiurs[(stage + 1) & 1] : nullptr;
        for (auto& bp : m.blocks) {
            KBlock<float> K = make_kblock<float>(*ctx->etypes[bp->etype], *bp);
            const int s = prof_begin(ctx, KIND_RESIDUAL);
            launch_flux_rec<float>(K, m.phys.system, recs[stage & 1], nullptr, fiurs[stage & 1], nullptr, P, E,
                                   ctx->nsm, ctx->stream);
            prof_end(ctx, s);
            ++ctx->launches;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SDRT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return SDRT_OK;
}

// RK4 on the operator-specialised path: the face records of U, then four
// fused stages; stages 1-3 write the face records of the next stage's state
// (the two record arrays alternate), so each stage reads its partners' states
// without a separate interpolation launch.
int rk4_stages_gen(sdrt_ctx* ctx, Mesh& m, float* U, double dt) {
    float* fr[2] = {m.fr[0].as<float>(), m.fr[1].as<float>()};
    float* us = m.ustage.as<float>();
    KEpi<float> E{};
    E.flag = ctx->flag.as<int>();
    E.u0 = U;
    E.uacc = m.uacc.as<float>();
    E.unext = us;
    int r = gen_launch_blocks(ctx, m, 0, U, nullptr, fr[0], E);
    if (r) return r;
    const float c6 = (float)(dt / 6.0), c3 = (float)(dt / 3.0), c2 = (float)(dt / 2.0), c1 = (float)dt;
    const int modes[4] = {EPI_RK_FIRST, EPI_RK_MID, EPI_RK_MID, EPI_RK_LAST};
    const float cacc[4] = {c6, c3, c3, c6};
    const float cnext[4] = {c2, c2, c1, 0.0f};
    for (int stage = 0; stage < 4; ++stage) {
        E.mode = modes[stage];
        E.cacc = cacc[stage];
        E.cnext = cnext[stage];
        E.out = stage == 3 ? U : nullptr;
        r = gen_launch_blocks(ctx, m, 1, stage == 0 ? U : us, fr[stage & 1], stage < 3 ? fr[(stage + 1) & 1] : nullptr,
                              E);
        if (r) return r;
    }
    return SDRT_OK;
}

template <typename T>
int rk4_stages(sdrt_ctx* ctx, Mesh& m, T* U, double dt) {
    if constexpr (std::is_same<T, float>::value) {
        if (m.gen && ctx->use_gen) return rk4_stages_gen(ctx, m, U, dt);
        if (ctx->fuse_rk && rk_fusable(ctx, m)) return rk4_stages_fused(ctx, m, U, dt);
    }
    KEpi<T> E{};
    E.flag = ctx->flag.as<int>();
    T* us = m.ustage.as<T>();
    T* ua = m.uacc.as<T>();
    const T c6 = (T)(dt / 6.0), c3 = (T)(dt / 3.0), c2 = (T)(dt / 2.0), c1 = (T)dt;
    E.u0 = U;
    E.uacc = ua;
    E.unext = us;
    E.mode = EPI_RK_FIRST;
    E.cacc = c6;
    E.cnext = c2;
    int r = run_residual<T>(ctx, m, U, nullptr, E);
    if (r) return r;
    E.mode = EPI_RK_MID;
    E.cacc = c3;
    E.cnext = c2;
    if ((r = run_residual<T>(ctx, m, us, nullptr, E))) return r;
    E.cnext = c1;
    if ((r = run_residual<T>(ctx, m, us, nullptr, E))) return r;
    E.mode = EPI_RK_LAST;
    E.cacc = c6;
    E.out = U;
    return run_residual<T>(ctx, m, us, nullptr, E);
}

// ---------------------------------------------------------------------------
// RK54: the five-stage fourth-order two-register scheme of Carpenter & Kennedy
// (1994, NASA TM-109112), published rationals.  Its linear stability
// polynomial is the one of the paper's Eq. "rk_exponential".
const double kRK54A[5] = {0.0, -567301805773.0 / 1357537059087.0, -2404267990393.0 / 2016746695238.0,
                          -3550918686646.0 / 2091501179385.0, -1275806237668.0 / 842570457699.0};
const double kRK54B[5] = {1432997174477.0 / 9575080441755.0, 5161836677717.0 / 13612068292357.0,
                          1720146321549.0 / 2090206949498.0, 3134564353537.0 / 4481467310338.0,
                          2277821191437.0 / 14882151754819.0};

// The embedded estimate's weights n = b - b^: the unit null vector (last
// component positive) of the four conditions of order <= 3 on the stages,
// sum n = 0, n.c = 0, n.c^2 = 0, n.(a c) = 0, so U - U^ = sum_j n_j k_j with
// U^ third order.  Computed from the Butcher form of the two-register scheme;
// the null vector from the 4 x 4 minors (cofactor expansion).
std::array<double, 5> rk54_estimate_weights() {
    double a[5][5] = {}, D[5] = {}, W[5] = {};
    for (int i = 0; i < 5; ++i) {
        for (int j = 0; j < 5; ++j) a[i][j] = W[j];
        for (int j = 0; j < 5; ++j) D[j] = kRK54A[i] * D[j] + (j == i ? 1.0 : 0.0);
        for (int j = 0; j < 5; ++j) W[j] += kRK54B[i] * D[j];
    }
    double c[5], ac[5];
    for (int i = 0; i < 5; ++i) {
        c[i] = 0;
        for (int j = 0; j < 5; ++j) c[i] += a[i][j];
    }
    for (int i = 0; i < 5; ++i) {
        ac[i] = 0;
        for (int j = 0; j < 5; ++j) ac[i] += a[i][j] * c[j];
    }
    double M[4][5];
    for (int j = 0; j < 5; ++j) {
        M[0][j] = 1.0;
        M[1][j] = c[j];
        M[2][j] = c[j] * c[j];
        M[3][j] = ac[j];
    }
    auto det4 = [](double m[4][4]) {
        double d = 0;
        for (int c0 = 0; c0 < 4; ++c0) {
            double s[3][3];
            for (int r = 1; r < 4; ++r)
                for (int cc = 0, k = 0; cc < 4; ++cc)
                    if (cc != c0) s[r - 1][k++] = m[r][cc];
            const double d3 = s[0][0] * (s[1][1] * s[2][2] - s[1][2] * s[2][1]) -
                              s[0][1] * (s[1][0] * s[2][2] - s[1][2] * s[2][0]) +
                              s[0][2] * (s[1][0] * s[2][1] - s[1][1] * s[2][0]);
            d += (c0 % 2 ? -1.0 : 1.0) * m[0][c0] * d3;
        }
        return d;
    };
    std::array<double, 5> n{};
    double nn = 0;
    for (int j = 0; j < 5; ++j) {
        double m[4][4];
        for (int r = 0; r < 4; ++r)
            for (int cc = 0, k = 0; cc < 5; ++cc)
                if (cc != j) m[r][k++] = M[r][cc];
        n[j] = (j % 2 ? -1.0 : 1.0) * det4(m);
        nn += n[j] * n[j];
    }
    const double sgn = n[4] < 0 ? -1.0 : 1.0;
    for (double& x : n) x *= sgn / std::sqrt(nn);
    return n;
}

// PI step-size factor (the reading stated with the oracle): accepted steps
// 0.9 err^(-0.7/k) err_prev^(0.4/k), rejected ones 0.9 err^(-0.7/k), k = 4
// (third-order estimate), clipped to [0.2, 5].
double pi_factor(double err, double err_prev, bool accepted) {
    const double k = 4.0;
    err = std::max(err, 1e-16);
    err_prev = std::max(err_prev, 1e-16);
    double f = 0.9 * std::pow(err, -0.7 / k) * (accepted ? std::pow(err_prev, 0.4 / k) : 1.0);
    return std::min(5.0, std::max(0.2, f));
}

int check_mesh(sdrt_ctx* ctx, int mesh_id) {
    if (!ctx) return SDRT_ERR_ARG;
    if (mesh_id < 0 || mesh_id >= (int)ctx->meshes.size() || !ctx->meshes[mesh_id])
        return fail(ctx, SDRT_ERR_ARG, "invalid mesh id");
    return SDRT_OK;
}

int check_compute(sdrt_ctx* ctx, int mesh_id) {
    int r = check_mesh(ctx, mesh_id);
    if (r) return r;
    if (ctx->host_only) return fail(ctx, SDRT_ERR_STATE, "host-only context: no device computation");
    return SDRT_OK;
}

// Whole-mesh computations: not on a partition (its ghost records come from the exchange).
int check_whole(sdrt_ctx* ctx, int mesh_id) {
    int r = check_compute(ctx, mesh_id);
    if (r) return r;
    if (ctx->meshes[mesh_id]->partition)
        return fail(ctx, SDRT_ERR_STATE, "partition mesh: use sdrt_residual_begin / sdrt_residual_end");
    return SDRT_OK;
}

// (Re)builds the block tables of the generic kernels from the mesh blocks.
int refresh_tables(sdrt_ctx* ctx, Mesh& m) {
    m.kb_f.clear();
    m.kb_d.clear();
    const bool f32 = m.phys.precision == SDRT_FP32;
    for (auto& bp : m.blocks) {
        const EType& et = *ctx->etypes[bp->etype];
        if (f32) m.kb_f.push_back(make_kblock<float>(et, *bp));
        else m.kb_d.push_back(make_kblock<double>(et, *bp));
    }
    if (!ctx->host_only) {
        if (f32) SDRT_CUDA(upload(m.kb_dev, m.kb_f));
        else SDRT_CUDA(upload(m.kb_dev, m.kb_d));
    }
    return SDRT_OK;
}

int ensure_workspace(sdrt_ctx* ctx, Mesh& m, bool need_dual, bool need_rk) {
    const size_t es = m.phys.precision == SDRT_FP32 ? 4 : 8;
    if (!m.ufe.p) SDRT_CUDA(m.ufe.alloc((size_t)m.nvar * m.Ftot * es));
    if (need_dual && !m.dufe.p) SDRT_CUDA(m.dufe.alloc((size_t)m.nvar * m.Ftot * es));
    if (viscous(m)) {
        const size_t nq = (size_t)m.nd * m.nvar * m.Ftot;
        if (!m.qfe.p) SDRT_CUDA(m.qfe.alloc(nq * es));
        if (!m.qfiu.p) SDRT_CUDA(m.qfiu.alloc((size_t)m.qfiu_total * es));
        if (need_dual && !m.dqfe.p) SDRT_CUDA(m.dqfe.alloc(nq * es));
        if (need_dual && !m.dqfiu.p) SDRT_CUDA(m.dqfiu.alloc((size_t)m.qfiu_total * es));
    }
    if (m.fast) {
        if (!m.rec.p) SDRT_CUDA(m.rec.alloc((size_t)m.rec_total * es));
        if (!m.fiur.p) SDRT_CUDA(m.fiur.alloc((size_t)m.fiur_total * es));
        if (need_dual && !m.drec.p) SDRT_CUDA(m.drec.alloc((size_t)m.rec_total * es));
        if (need_dual && !m.dfiur.p) SDRT_CUDA(m.dfiur.alloc((size_t)m.fiur_total * es));
    }
    if (need_rk && m.fast && m.phys.precision == SDRT_FP32) {
        if (!m.rec2.p) SDRT_CUDA(m.rec2.alloc((size_t)m.rec_total * es));
        if (!m.fiur2.p) SDRT_CUDA(m.fiur2.alloc((size_t)m.fiur_total * es));
    }
    if (m.gen) {
        const size_t nfr = (size_t)m.Ftot * m.nvar * sizeof(float);
        if (!m.fr[0].p) SDRT_CUDA(m.fr[0].alloc(nfr));
        if (need_rk && !m.fr[1].p) SDRT_CUDA(m.fr[1].alloc(nfr));
    }
    if (need_rk && !m.ustage.p) {
        SDRT_CUDA(m.ustage.alloc((size_t)m.state_len * es));
        SDRT_CUDA(m.uacc.alloc((size_t)m.state_len * es));
        SDRT_CUDA(cudaMemset(m.ustage.p, 0, m.ustage.bytes));
        SDRT_CUDA(cudaMemset(m.uacc.p, 0, m.uacc.bytes));
    }
    return SDRT_OK;
}

// Partitioned residual, first half: interpolation of the owned blocks into
// the records, then the packed face records to send.
template <typename T>
int residual_begin_impl(sdrt_ctx* ctx, Mesh& m, const T* U, T* send) {
    if (!m.fast) {
        // Generic path: the owned blocks' external-point states into UFE, then the
        // send buffer gathered from it.
        T* ufe = m.ufe.as<T>();
        const KSet<T> ks = kset<T>(m);
        const int s = prof_begin(ctx, KIND_INTERP);
        launch_interp_ext<T>(ks, m.nvar, U, ufe, m.Ftot, ctx->nsm, ctx->stream);
        prof_end(ctx, s);
        ++ctx->launches;
        if (m.nsend > 0) {
            launch_gather_values<T>(ufe, send, m.xsend_idx.as<int>(), m.nsend * m.xfrec, false, ctx->nsm, ctx->stream);
            ++ctx->launches;
        }
        m.part_u = U;
        m.part_grad = false;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(ctx, SDRT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
        return SDRT_OK;
    }
    T* rec = m.rec.as<T>();
    T* fiur = m.fiur.as<T>();
    for (auto& bp : m.blocks) {
        KBlock<T> K = make_kblock<T>(*ctx->etypes[bp->etype], *bp);
        const int s = prof_begin(ctx, KIND_INTERP);
        const int r = launch_interp_rec<T>(K, m.nvar, U, rec, fiur, ctx->flag.as<int>(), ctx->nsm, ctx->stream);
        prof_end(ctx, s);
        if (r != 0) return fail(ctx, SDRT_ERR_UNSUPPORTED, "record path not instantiated");
        ++ctx->launches;
    }
    if (m.nsend > 0) {
        launch_face_records<T>(rec, send, m.xsend_off.as<int>(), m.nsend, m.xfrec, false, ctx->nsm, ctx->stream);
        ++ctx->launches;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SDRT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return SDRT_OK;
}

// Second half: the received face records into the ghost slots, then fluxes
// and divergence of the owned blocks.
template <typename T>
int residual_end_impl(sdrt_ctx* ctx, Mesh& m, const T* recv, T* R) {
    if (!m.fast) {
        T* ufe = m.ufe.as<T>();
        if (!m.part_u) return fail(ctx, SDRT_ERR_STATE, "sdrt_residual_end before sdrt_residual_begin");
        KVisc<T> Q{};
        if (viscous(m)) {
            // recv holds gradient records: into the ghost faces' flux-point gradients
            // (the face states arrived with sdrt_residual_gradients).
            if (!m.part_grad) return fail(ctx, SDRT_ERR_STATE, "viscous partition: sdrt_residual_gradients first");
            if (m.nrecv > 0) {
                launch_gather_values<T>(recv, m.qfe.as<T>(), m.xrecv_gidx.as<int>(), m.nrecv * m.xgrec, true,
                                        ctx->nsm, ctx->stream);
                ++ctx->launches;
            }
            Q = {m.qfe.as<T>(), nullptr, m.qfiu.as<T>(), nullptr};
        } else if (m.nrecv > 0) {
            launch_gather_values<T>(recv, ufe, m.xrecv_idx.as<int>(), m.nrecv * m.xfrec, true, ctx->nsm, ctx->stream);
            ++ctx->launches;
        }
        const KPhys<T> P = make_phys<T>(m.phys);
        KEpi<T> E{};
        E.mode = EPI_STORE;
        E.out = R;
        E.flag = ctx->flag.as<int>();
        const KSet<T> ks = kset<T>(m);
        const int s = prof_begin(ctx, KIND_RESIDUAL);
        const int r = launch_residual<T>(ks, m.phys.system, m.phys.riemann, m.nd, static_cast<const T*>(m.part_u),
                                         nullptr, ufe, nullptr, m.Ftot, P, E, Q, ctx->nsm, ctx->stream);
        prof_end(ctx, s);
        if (r != 0) return fail(ctx, SDRT_ERR_UNSUPPORTED, "system / flux combination not supported");
        ++ctx->launches;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(ctx, SDRT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
        return SDRT_OK;
    }
    T* rec = m.rec.as<T>();
    T* fiur = m.fiur.as<T>();
    if (m.nrecv > 0) {
        launch_face_records<T>(recv, rec, m.xrecv_off.as<int>(), m.nrecv, m.xfrec, true, ctx->nsm, ctx->stream);
        ++ctx->launches;
    }
    const KPhys<T> P = make_phys<T>(m.phys);
    KEpi<T> E{};
    E.mode = EPI_STORE;
    E.out = R;
    E.flag = ctx->flag.as<int>();
    for (auto& bp : m.blocks) {
        KBlock<T> K = make_kblock<T>(*ctx->etypes[bp->etype], *bp);
        const int s = prof_begin(ctx, KIND_RESIDUAL);
        launch_flux_rec<T>(K, m.phys.system, rec, nullptr, fiur, nullptr, P, E, ctx->nsm, ctx->stream);
        prof_end(ctx, s);
        ++ctx->launches;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SDRT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return SDRT_OK;
}

// Viscous partitions, middle step: the received face states into the ghost
// faces, the flux-point gradients of the owned elements, then the packed
// gradient records to send.
template <typename T>
int residual_gradients_impl(sdrt_ctx* ctx, Mesh& m, const T* recv, T* send_grad) {
    T* ufe = m.ufe.as<T>();
    if (m.nrecv > 0) {
        launch_gather_values<T>(recv, ufe, m.xrecv_idx.as<int>(), m.nrecv * m.xfrec, true, ctx->nsm, ctx->stream);
        ++ctx->launches;
    }
    const KPhys<T> P = make_phys<T>(m.phys);
    const KSet<T> ks = kset<T>(m);
    const int s = prof_begin(ctx, KIND_GRAD);
    const int r = launch_grad<T>(ks, m.phys.system, m.nd, static_cast<const T*>(m.part_u), nullptr, ufe, nullptr,
                                 m.Ftot, P, m.qfe.as<T>(), nullptr, m.qfiu.as<T>(), nullptr, ctx->nsm, ctx->stream);
    prof_end(ctx, s);
    if (r != 0) return fail(ctx, SDRT_ERR_UNSUPPORTED, "system not supported by the gradient kernel");
    ++ctx->launches;
    if (m.nsend > 0) {
        launch_gather_values<T>(m.qfe.as<T>(), send_grad, m.xsend_gidx.as<int>(), m.nsend * m.xgrec, false, ctx->nsm,
                                ctx->stream);
        ++ctx->launches;
    }
    m.part_grad = true;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SDRT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return SDRT_OK;
}

// FR-SDRT operators from the SDRT ones (Sec. 2.3): internal DOFs at the
// solution points, nu = r nd + d (point r, reference axis d), M12 = I,
// M13_FR[s, nu] = (M15 P M12)[(d, s), r], and M15_FR with M15_FR P_FR = M15 P M12
// (the same viscous gradient operator; the axis-0 DOF of each point carries it).
RefElement fr_variant(const RefElement& S) {
    RefElement R = S;
    const int nd = S.nd, ns = S.nsol;
    std::vector<double> G((size_t)nd * ns * ns, 0.0);      // M15 P M12: (nd ns) x ns
    for (int m = 0; m < nd * ns; ++m)
        for (int mu = 0; mu < S.nfi; ++mu) {
            const double a = S.M15[(size_t)m * S.nfi + mu];
            if (a == 0.0) continue;
            const double* row = &S.M12[(size_t)S.fi_point[mu] * ns];
            for (int r = 0; r < ns; ++r) G[(size_t)m * ns + r] += a * row[r];
        }
    R.nfiu = ns;
    R.nfi = nd * ns;
    R.xfiu = S.xs;
    R.fi_point.resize(R.nfi);
    R.fi_axis.resize(R.nfi);
    for (int r = 0; r < ns; ++r)
        for (int d = 0; d < nd; ++d) {
            R.fi_point[r * nd + d] = r;
            R.fi_axis[r * nd + d] = d;
        }
    R.M12.assign((size_t)ns * ns, 0.0);
    for (int r = 0; r < ns; ++r) R.M12[(size_t)r * ns + r] = 1.0;
    R.M13.assign((size_t)ns * R.nfi, 0.0);
    R.M15.assign((size_t)nd * ns * R.nfi, 0.0);
    for (int s = 0; s < ns; ++s)
        for (int r = 0; r < ns; ++r)
            for (int d = 0; d < nd; ++d) R.M13[(size_t)s * R.nfi + r * nd + d] = G[((size_t)d * ns + s) * ns + r];
    for (int m = 0; m < nd * ns; ++m)
        for (int r = 0; r < ns; ++r) R.M15[(size_t)m * R.nfi + r * nd] = G[(size_t)m * ns + r];
    return R;
}

}  // namespace

extern "C" {

int sdrt_create(sdrt_ctx** out, int device, void* stream) {
    if (!out) return SDRT_ERR_ARG;
    *out = nullptr;
    auto ctx = std::make_unique<sdrt_ctx>();
    if (device == -1) {
        ctx->host_only = true;
        *out = ctx.release();
        return SDRT_OK;
    }
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) return SDRT_ERR_CUDA;
    if (device < 0 || device >= n) return SDRT_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return SDRT_ERR_CUDA;
    ctx->device = device;
    ctx->stream = static_cast<cudaStream_t>(stream);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return SDRT_ERR_CUDA;
    ctx->nsm = prop.multiProcessorCount;
    if (ctx->flag.alloc(sizeof(int)) != cudaSuccess) return SDRT_ERR_CUDA;
    if (cudaMemset(ctx->flag.p, 0, sizeof(int)) != cudaSuccess) return SDRT_ERR_CUDA;
    // The static buffer of sdrt_residual_noalloc: looking up its address loads
    // the module that holds it (lazy module loading), so the device memory it
    // takes is taken here and not in the allocation-free call.
    if (sdrt::internal_noalloc_scratch_address(&ctx->noalloc_scratch) != cudaSuccess) return SDRT_ERR_CUDA;
    *out = ctx.release();
    return SDRT_OK;
}

void sdrt_destroy(sdrt_ctx* ctx) {
    if (!ctx) return;
    if (!ctx->host_only) cudaSetDevice(ctx->device);
    delete ctx;
}

const char* sdrt_last_error(const sdrt_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int sdrt_set_stream(sdrt_ctx* ctx, void* stream) {
    if (!ctx) return SDRT_ERR_ARG;
    ctx->stream = static_cast<cudaStream_t>(stream);
    for (auto& m : ctx->meshes)
        if (m && m->graph) {
            cudaGraphExecDestroy(m->graph);
            m->graph = nullptr;
        }
    return SDRT_OK;
}

int sdrt_setup_element_type(sdrt_ctx* ctx, const sdrt_etype_desc* d, int* etype_id) {
    if (!ctx || !d || !etype_id) return fail(ctx, SDRT_ERR_ARG, "null argument");
    if (d->shape < 0 || d->shape > 4) return fail(ctx, SDRT_ERR_ARG, "unknown shape");
    if (d->degree < 1 || d->degree > 6) return fail(ctx, SDRT_ERR_UNSUPPORTED, "degree must be in 1..6");
    if (d->scheme != SDRT_SCHEME_SDRT && d->scheme != SDRT_SCHEME_FR) return fail(ctx, SDRT_ERR_ARG, "unknown scheme");
    for (size_t i = 0; i < ctx->etypes.size(); ++i)
        if (ctx->etypes[i]->desc.shape == d->shape && ctx->etypes[i]->desc.degree == d->degree &&
            ctx->etypes[i]->desc.scheme == d->scheme) {
            *etype_id = (int)i;
            return SDRT_OK;
        }
    auto et = std::make_unique<EType>();
    et->desc = *d;
    try {
        et->R = build_ref_element(d->shape, d->degree);
        if (d->scheme == SDRT_SCHEME_FR) et->R = fr_variant(et->R);
    } catch (const std::exception& ex) {
        return fail(ctx, SDRT_ERR_UNSUPPORTED, ex.what());
    }
    const RefElement& R = et->R;
    et->Mi = R.nfe + R.nfiu;
    et->Mi_pad = round_up(et->Mi, 8);
    et->Md_pad = round_up(R.nsol, 8);
    et->Mg_pad = round_up(R.nd * R.nsol, 8);
    // Ai has kMR (8) trailing zeros: a GEMM over its M12 columns alone reads up to
    // 8 rows past the last one.
    std::vector<double> Ai((size_t)R.nsol * et->Mi_pad + 8, 0.0), Ad((size_t)(R.nfe + R.nfi) * et->Md_pad, 0.0);
    const int nfe_pad = round_up(R.nfe, 8);
    et->Mdt_pad = nfe_pad + round_up(R.nfi, 8);
    std::vector<double> Adt((size_t)R.nsol * et->Mdt_pad, 0.0);
    for (int r = 0; r < R.nsol; ++r) {
        for (int j = 0; j < R.nfe; ++j) Ai[(size_t)r * et->Mi_pad + j] = R.M0[(size_t)j * R.nsol + r];
        for (int j = 0; j < R.nfiu; ++j) Ai[(size_t)r * et->Mi_pad + R.nfe + j] = R.M12[(size_t)j * R.nsol + r];
        for (int k = 0; k < R.nfe; ++k) Ad[(size_t)k * et->Md_pad + r] = R.M14[(size_t)r * R.nfe + k];
        for (int k = 0; k < R.nfi; ++k) Ad[(size_t)(R.nfe + k) * et->Md_pad + r] = R.M13[(size_t)r * R.nfi + k];
        for (int k = 0; k < R.nfe; ++k) Adt[(size_t)r * et->Mdt_pad + k] = R.M14[(size_t)r * R.nfe + k];
        for (int k = 0; k < R.nfi; ++k) Adt[(size_t)r * et->Mdt_pad + nfe_pad + k] = R.M13[(size_t)r * R.nfi + k];
    }
    std::vector<float> Adtf(Adt.begin(), Adt.end());
    std::vector<float> Aif(Ai.begin(), Ai.end()), Adf(Ad.begin(), Ad.end());
    // Gradient operator [M16 | M15 P M12] transposed: row k < nfe is column k of
    // M16, row nfe + r is column r of M15 P M12 (P: internal DOF -> its point).
    std::vector<double> Ag((size_t)(R.nfe + R.nsol) * et->Mg_pad, 0.0);
    for (int m = 0; m < R.nd * R.nsol; ++m) {
        for (int k = 0; k < R.nfe; ++k) Ag[(size_t)k * et->Mg_pad + m] = R.M16[(size_t)m * R.nfe + k];
        for (int nu = 0; nu < R.nfi; ++nu) {
            const double a = R.M15[(size_t)m * R.nfi + nu];
            const double* row = &R.M12[(size_t)R.fi_point[nu] * R.nsol];
            for (int r = 0; r < R.nsol; ++r) Ag[(size_t)(R.nfe + r) * et->Mg_pad + m] += a * row[r];
        }
    }
    std::vector<float> Agf(Ag.begin(), Ag.end());
    // The same operator row-major with rows (rho, d), for its transpose in the
    // viscous VJP: Agr[(rho ND + d)][k] = [M16 | M15 P M12][d nsol + rho][k].
    et->Agr_pad = round_up(R.nfe + R.nsol, 8);
    std::vector<double> Agr((size_t)R.nd * R.nsol * et->Agr_pad, 0.0);
    for (int d = 0; d < R.nd; ++d)
        for (int r = 0; r < R.nsol; ++r)
            for (int k = 0; k < R.nfe + R.nsol; ++k)
                Agr[((size_t)r * R.nd + d) * et->Agr_pad + k] = Ag[(size_t)k * et->Mg_pad + d * R.nsol + r];
    std::vector<float> Agrf(Agr.begin(), Agr.end());
    // Row-major interpolation operator for the register-blocked kernels.
    et->Mir = round_up(et->Mi + 2, 4);   // zero rows past Mi: row pairs (j, j + 2) stay in bounds
    std::vector<double> Air((size_t)et->Mir * et->Md_pad, 0.0);
    for (int j = 0; j < et->Mi; ++j)
        for (int r = 0; r < R.nsol; ++r)
            Air[(size_t)j * et->Md_pad + r] =
                j < R.nfe ? R.M0[(size_t)j * R.nsol + r] : R.M12[(size_t)(j - R.nfe) * R.nsol + r];
    std::vector<float> Airf(Air.begin(), Air.end());
    std::vector<int> tab((size_t)R.nfiu * 4, 0);
    for (int nu = 0; nu < R.nfi; ++nu) {
        int k = R.fi_point[nu];
        int& cnt = tab[(size_t)k * 4];
        if (cnt >= 3) return fail(ctx, SDRT_ERR_UNSUPPORTED, "more than 3 DOFs at an internal point");
        tab[(size_t)k * 4 + 1 + cnt] = nu | (R.fi_axis[nu] << 16);
        ++cnt;
    }
    if (!ctx->host_only) {
        SDRT_CUDA(upload(et->Ai[0], Ai));
        SDRT_CUDA(upload(et->Ad[0], Ad));
        SDRT_CUDA(upload(et->Ai[1], Aif));
        SDRT_CUDA(upload(et->Ad[1], Adf));
        SDRT_CUDA(upload(et->fe_face, R.fe_face));
        SDRT_CUDA(upload(et->fi_tab, tab));
        SDRT_CUDA(upload(et->Air[0], Air));
        SDRT_CUDA(upload(et->Air[1], Airf));
        SDRT_CUDA(upload(et->Ag[0], Ag));
        SDRT_CUDA(upload(et->Ag[1], Agf));
        SDRT_CUDA(upload(et->Adt[0], Adt));
        SDRT_CUDA(upload(et->Adt[1], Adtf));
        SDRT_CUDA(upload(et->Agr[0], Agr));
        SDRT_CUDA(upload(et->Agr[1], Agrf));
        SDRT_CUDA(upload(et->Mq[0], R.Mq));
        SDRT_CUDA(upload(et->Mq[1], std::vector<float>(R.Mq.begin(), R.Mq.end())));
        SDRT_CUDA(upload(et->wq[0], R.wq));
        SDRT_CUDA(upload(et->wq[1], std::vector<float>(R.wq.begin(), R.wq.end())));
    }
    ctx->etypes.push_back(std::move(et));
    *etype_id = (int)ctx->etypes.size() - 1;
    return SDRT_OK;
}

int sdrt_get_etype_info(sdrt_ctx* ctx, int id, sdrt_etype_info* out) {
    if (!ctx || !out) return SDRT_ERR_ARG;
    if (id < 0 || id >= (int)ctx->etypes.size()) return fail(ctx, SDRT_ERR_ARG, "invalid element type id");
    const RefElement& R = ctx->etypes[id]->R;
    *out = {R.nd, R.nsol, R.nfe, R.nfi, R.nfiu, R.nfaces};
    return SDRT_OK;
}

int sdrt_get_operator(sdrt_ctx* ctx, int id, int which, double* out, int64_t n) {
    if (!ctx || !out) return SDRT_ERR_ARG;
    if (id < 0 || id >= (int)ctx->etypes.size()) return fail(ctx, SDRT_ERR_ARG, "invalid element type id");
    const RefElement& R = ctx->etypes[id]->R;
    const std::vector<double>* src = nullptr;
    switch (which) {
        case 0: src = &R.M0; break;
        case 1: src = &R.M12; break;
        case 2: src = &R.M13; break;
        case 3: src = &R.M14; break;
        case 4: src = &R.M15; break;
        case 5: src = &R.M16; break;
        case 6: src = &R.xs; break;
        case 7: src = &R.xfe; break;
        default: return fail(ctx, SDRT_ERR_ARG, "unknown operator");
    }
    if ((int64_t)src->size() != n) return fail(ctx, SDRT_ERR_ARG, "size mismatch");
    std::memcpy(out, src->data(), src->size() * sizeof(double));
    return SDRT_OK;
}

static int setup_mesh_impl(sdrt_ctx* ctx, const sdrt_physics* phys, int nblocks, const sdrt_block* blocks,
                           const double* const* nodes, const uint8_t* ghost, int64_t nfaces, const sdrt_face* faces,
                           int* mesh_id);

int sdrt_setup_mesh(sdrt_ctx* ctx, const sdrt_physics* phys, int nblocks, const sdrt_block* blocks, int64_t nfaces,
                    const sdrt_face* faces, int* mesh_id) {
    return setup_mesh_impl(ctx, phys, nblocks, blocks, nullptr, nullptr, nfaces, faces, mesh_id);
}

int sdrt_setup_mesh_curved(sdrt_ctx* ctx, const sdrt_physics* phys, int nblocks, const sdrt_block* blocks,
                           const double* const* nodes, int64_t nfaces, const sdrt_face* faces, int* mesh_id) {
    if (!nodes) return fail(ctx, SDRT_ERR_ARG, "null node array list");
    return setup_mesh_impl(ctx, phys, nblocks, blocks, nodes, nullptr, nfaces, faces, mesh_id);
}

int sdrt_setup_partition(sdrt_ctx* ctx, const sdrt_physics* phys, int nblocks, const sdrt_block* blocks,
                         const uint8_t* ghost, int64_t nfaces, const sdrt_face* faces, int* mesh_id) {
    if (!ghost) return fail(ctx, SDRT_ERR_ARG, "null ghost flags");
    return setup_mesh_impl(ctx, phys, nblocks, blocks, nullptr, ghost, nfaces, faces, mesh_id);
}

static int setup_mesh_impl(sdrt_ctx* ctx, const sdrt_physics* phys, int nblocks, const sdrt_block* blocks,
                           const double* const* nodes, const uint8_t* ghost, int64_t nfaces, const sdrt_face* faces,
                           int* mesh_id) {
    if (!ctx || !phys || !blocks || !mesh_id || nblocks <= 0 || (nfaces > 0 && !faces))
        return fail(ctx, SDRT_ERR_ARG, "null or empty argument");
    int nown = nblocks;
    if (ghost) {
        nown = 0;
        while (nown < nblocks && !ghost[nown]) ++nown;
        for (int b = nown; b < nblocks; ++b)
            if (!ghost[b]) return fail(ctx, SDRT_ERR_ARG, "ghost blocks must follow the owned blocks");
        if (nown == 0) return fail(ctx, SDRT_ERR_ARG, "a partition needs an owned block");
    }
    if (phys->ndim != 2 && phys->ndim != 3) return fail(ctx, SDRT_ERR_ARG, "ndim must be 2 or 3");
    if (phys->precision != SDRT_FP32 && phys->precision != SDRT_FP64 && phys->precision != SDRT_TF32X3)
        return fail(ctx, SDRT_ERR_ARG, "bad precision");
    if (phys->system < SDRT_ADVECTION || phys->system > SDRT_NAVIER_STOKES) return fail(ctx, SDRT_ERR_ARG, "bad system");
    const bool scalar = phys->system == SDRT_ADVECTION || phys->system == SDRT_ADVDIFF;
    if (scalar && phys->riemann == SDRT_ROE) return fail(ctx, SDRT_ERR_ARG, "Roe flux needs the Euler or Navier-Stokes system");
    auto m = std::make_unique<Mesh>();
    m->phys = *phys;
    if (phys->precision == SDRT_TF32X3) {
        // FP32 states; the record path's contractions on the tensor cores
        m->tc3 = true;
        m->phys.precision = SDRT_FP32;
    }
    const int nd = phys->ndim;
    m->nd = nd;
    m->nvar = (phys->system == SDRT_ADVECTION || phys->system == SDRT_ADVDIFF) ? 1 : nd + 2;
    const bool f32 = m->phys.precision == SDRT_FP32;

    // Layout.
    int64_t canon = 0;
    m->fast = true;
    for (int b = 0; b < nblocks; ++b) {
        const sdrt_block& B = blocks[b];
        const bool curved = nodes && nodes[b];
        if (B.etype < 0 || B.etype >= (int)ctx->etypes.size()) return fail(ctx, SDRT_ERR_ARG, "bad etype id");
        if (B.nelem <= 0 || (!B.verts && !curved)) return fail(ctx, SDRT_ERR_ARG, "empty block");
        const RefElement& R = ctx->etypes[B.etype]->R;
        if (R.nd != nd) return fail(ctx, SDRT_ERR_ARG, "element dimension does not match physics");
        auto mb = std::make_unique<MBlock>();
        if (curved) {
            if (ctx->etypes[B.etype]->desc.scheme != SDRT_SCHEME_SDRT)
                return fail(ctx, SDRT_ERR_UNSUPPORTED, "curved elements take the SDRT scheme");
            // per point: 1/det J and S at the solution points, S at the unique
            // internal points, normal and scale at the external points
            mb->curved = true;
            mb->mr_inv = 1;
            mb->mr_ss = R.nsol;
            mb->mr_ssk = nd * nd;
            mb->mr_si = R.nsol * (1 + nd * nd);
            mb->mr_sik = nd * nd;
            mb->mr_f = mb->mr_si + R.nfiu * nd * nd;
            mb->mr_ff = 0;
            mb->mr_fp = nd + 1;
            mb->nmetric = mb->mr_f + R.nfe * (nd + 1);
            m->curved = true;
        } else {
            mb->mr_f = 1 + nd * nd;
            mb->mr_ff = nd + 1;
            mb->nmetric = 1 + nd * nd + R.nfaces * (nd + 1);
        }
        mb->etype = B.etype;
        mb->nelem = B.nelem;
        mb->ld = round_up(B.nelem, 32);
        mb->u_off = m->state_len;
        mb->fe_base = m->Ftot;
        mb->canon_base = canon;
        m->state_len += (int64_t)R.nsol * m->nvar * mb->ld;
        m->Ftot += (int64_t)R.nfe * mb->ld;
        m->ndof += (int64_t)R.nsol * m->nvar * B.nelem;
        canon += (int64_t)R.nfe * B.nelem;
        if (ctx->etypes[B.etype]->desc.scheme != SDRT_SCHEME_SDRT || curved ||
            !fast_path_available(R.shape, R.nsol, nd, phys->system, phys->riemann))
            m->fast = false;
        if (phys->system == SDRT_ADVDIFF || phys->system == SDRT_NAVIER_STOKES) {
            mb->qfiu_off = m->qfiu_total;
            m->qfiu_total += (int64_t)R.nfiu * nd * m->nvar * mb->ld;
        }
        m->blocks.push_back(std::move(mb));
    }
    m->nfe_total = canon;
    if (m->fast && ctx->use_gen == 2 && !ghost && f32 && !m->tc3 && phys->system == SDRT_EULER && nd == 3 &&
        phys->riemann == SDRT_RUSANOV) {
        // SDRT_OPT_GENERATED = 2: the operator-specialised kernels replace the record path.
        bool all = true;
        for (auto& bp : m->blocks) {
            const RefElement& R = ctx->etypes[bp->etype]->R;
            all = all && gen_launcher(R.shape, R.p) != nullptr;
        }
        if (all) m->fast = false;
    }
    if (m->fast) {
        // Record strides: multiples of 4 values (16-byte bulk copies), odd multiples
        // of 4 for conflict-free shared-memory rows.
        auto odd4 = [](int x) {
            x = round_up(x, 4);
            return ((x / 4) % 2 == 1) ? x : x + 4;
        };
        for (int b = 0; b < nblocks; ++b) {
            MBlock& mb = *m->blocks[b];
            const RefElement& R = ctx->etypes[mb.etype]->R;
            const int npf = R.nfe / R.nfaces;
            mb.frec = round_up(npf * m->nvar, 4);
            mb.ers = odd4(R.nfaces * mb.frec);
            mb.frs = odd4(R.nfiu * m->nvar);
            mb.nmp = odd4(1 + nd * nd + R.nfaces * (nd + 1));
            mb.pstride = round_up(R.nfe, 16);
            if ((mb.pstride / 16) % 2 == 0) mb.pstride += 16;
            mb.rec_base = m->rec_total;
            mb.fiur_base = m->fiur_total;
            m->rec_total += (int64_t)mb.nelem * mb.ers;
            m->fiur_total += (int64_t)mb.nelem * mb.frs;
        }
    }
    if (canon >= INT32_MAX || m->Ftot >= INT32_MAX) return fail(ctx, SDRT_ERR_UNSUPPORTED, "mesh too large for int32 maps");
    if (ghost) {
        if (m->fast) {
            for (int b = 1; b < nblocks; ++b)
                if (m->blocks[b]->frec != m->blocks[0]->frec)
                    return fail(ctx, SDRT_ERR_UNSUPPORTED, "partitions need one face-record size");
        } else if ((int64_t)nd * m->nvar * m->Ftot >= INT32_MAX) {
            return fail(ctx, SDRT_ERR_UNSUPPORTED, "partition too large for int32 face-state indices");
        }
    }

    // Metrics and physical points (paper Sec. 2: mapping, Jacobian and its
    // inverse, evaluated analytically): affine blocks one value set per
    // element, curved blocks (quadratic map, mapping.hpp) one per point where
    // the method uses it (Sec. 2.1): 1/det J and S = det J J^{-1} at the
    // solution points, S at the unique internal points, the normal and scale at
    // the external points.
    struct HostBlk {
        std::vector<double> Ji, det;           // affine: per element J^{-1}, det J
        std::vector<double> h;                 // per element: largest |J_ij| (pairing tolerance)
        std::vector<double> xfe;               // physical external points
        std::vector<double> pn, pmag;          // curved: unit J^{-T} n~ and det J |J^{-T} n~| per external point
        std::vector<double> metric;            // [NM][ld]
        std::vector<uint8_t> glued;            // per (e, f)
    };
    std::vector<HostBlk> hb(nblocks);
    for (int b = 0; b < nblocks; ++b) {
        const sdrt_block& B = blocks[b];
        const RefElement& R = ctx->etypes[B.etype]->R;
        MBlock& mb = *m->blocks[b];
        const int nv = shape_nverts(R.shape);
        HostBlk& H = hb[b];
        H.h.resize(B.nelem);
        H.xfe.resize((size_t)B.nelem * R.nfe * nd);
        H.metric.assign((size_t)mb.nmetric * mb.ld, 0.0);
        H.glued.assign((size_t)B.nelem * R.nfaces, 0);
        auto row = [&](int k, int e) -> double& { return H.metric[(size_t)k * mb.ld + e]; };
        if (mb.curved) {
            const int NN = map_nnodes(R.shape);
            // shape functions and gradients at a reference point set
            auto table = [&](const std::vector<double>& X, std::vector<double>& N, std::vector<double>& dN) {
                const size_t np = X.size() / nd;
                N.resize(np * NN);
                dN.resize(np * NN * nd);
                for (size_t q = 0; q < np; ++q) map_shape(R.shape, &X[q * nd], &N[q * NN], &dN[q * NN * nd]);
            };
            std::vector<double> Ns, dNs, Nk, dNk, Nf, dNf;
            table(R.xs, Ns, dNs);
            table(R.xfiu, Nk, dNk);
            table(R.xfe, Nf, dNf);
            H.pn.resize((size_t)B.nelem * R.nfe * nd);
            H.pmag.resize((size_t)B.nelem * R.nfe);
            for (int e = 0; e < B.nelem; ++e) {
                const double* Xn = nodes[b] + (size_t)e * NN * nd;
                // x and J (J[i * nd + d] = dx_i / dx~_d) at point q of a table; det and J^{-1}
                double x[3], J[9], Ji[9];
                auto at = [&](const std::vector<double>& N, const std::vector<double>& dN, int q) {
                    for (int i = 0; i < nd; ++i) {
                        x[i] = 0;
                        for (int d = 0; d < nd; ++d) J[i * nd + d] = 0;
                        for (int k = 0; k < NN; ++k) {
                            const double X = Xn[(size_t)k * nd + i];
                            x[i] += X * N[(size_t)q * NN + k];
                            for (int d = 0; d < nd; ++d) J[i * nd + d] += X * dN[((size_t)q * NN + k) * nd + d];
                        }
                    }
                    for (int k = 0; k < nd * nd; ++k) H.h[e] = std::max(H.h[e], std::fabs(J[k]));
                    return det_inv(J, nd, Ji);
                };
                H.h[e] = 0;
                for (int sp = 0; sp < R.nsol; ++sp) {
                    const double det = at(Ns, dNs, sp);
                    if (!(det > 0)) return fail(ctx, SDRT_ERR_MESH, "inverted or degenerate element");
                    row(sp * mb.mr_inv, e) = 1.0 / det;
                    for (int k = 0; k < nd * nd; ++k) row(mb.mr_ss + sp * mb.mr_ssk + k, e) = det * Ji[k];
                    for (int i = 0; i < nd; ++i) m->sol_xyz.push_back(x[i]);
                }
                for (int q = 0; q < R.nfiu; ++q) {
                    const double det = at(Nk, dNk, q);
                    if (!(det > 0)) return fail(ctx, SDRT_ERR_MESH, "inverted or degenerate element");
                    for (int k = 0; k < nd * nd; ++k) row(mb.mr_si + q * mb.mr_sik + k, e) = det * Ji[k];
                }
                for (int sg = 0; sg < R.nfe; ++sg) {
                    const double det = at(Nf, dNf, sg);
                    if (!(det > 0)) return fail(ctx, SDRT_ERR_MESH, "inverted or degenerate element");
                    const size_t pt = (size_t)e * R.nfe + sg;
                    const int f = R.fe_face[sg];
                    double nrm = 0;
                    for (int i = 0; i < nd; ++i) {
                        double c = 0;
                        for (int d = 0; d < nd; ++d) c += Ji[d * nd + i] * R.face_nrm[f * nd + d];
                        H.pn[pt * nd + i] = c;
                        nrm += c * c;
                        H.xfe[pt * nd + i] = x[i];
                    }
                    nrm = std::sqrt(nrm);
                    for (int i = 0; i < nd; ++i) H.pn[pt * nd + i] /= nrm;
                    H.pmag[pt] = det * nrm;
                }
            }
            continue;
        }
        H.Ji.resize((size_t)B.nelem * nd * nd);
        H.det.resize(B.nelem);
        const auto& ref = ref_vertices(R.shape);
        for (int e = 0; e < B.nelem; ++e) {
            const double* X = B.verts + (size_t)e * nv * nd;
            double J[9];
            double* Ji = &H.Ji[(size_t)e * nd * nd];
            if (!element_jacobian(R.shape, X, nd, J))
                return fail(ctx, SDRT_ERR_UNSUPPORTED, "element " + std::to_string(e) + " of block " +
                                                           std::to_string(b) +
                                                           " is not affine (curved elements: sdrt_setup_mesh_curved)");
            double det = det_inv(J, nd, Ji);
            if (!(det > 0)) return fail(ctx, SDRT_ERR_MESH, "inverted or degenerate element");
            H.det[e] = det;
            H.h[e] = 0;
            for (int k = 0; k < nd * nd; ++k) H.h[e] = std::max(H.h[e], std::fabs(J[k]));
            row(0, e) = 1.0 / det;
            for (int d = 0; d < nd; ++d)
                for (int i = 0; i < nd; ++i) row(1 + d * nd + i, e) = det * Ji[d * nd + i];
            for (int sg = 0; sg < R.nfe; ++sg)
                for (int i = 0; i < nd; ++i) {
                    double x = X[i];
                    for (int d = 0; d < nd; ++d) x += J[i * nd + d] * (R.xfe[sg * nd + d] - ref[d]);
                    H.xfe[((size_t)e * R.nfe + sg) * nd + i] = x;
                }
            for (int sp = 0; sp < R.nsol; ++sp)
                for (int i = 0; i < nd; ++i) {
                    double x = X[i];
                    for (int d = 0; d < nd; ++d) x += J[i * nd + d] * (R.xs[sp * nd + d] - ref[d]);
                    m->sol_xyz.push_back(x);
                }
        }
    }

    // Face pairing.
    m->partner.assign(m->nfe_total, -1);
    m->is_left.assign(m->nfe_total, 0);
    // Unit physical normal J^{-T} n~ / |J^{-T} n~| and scale det J |J^{-T} n~|
    // at external point sg of element e of block b.
    auto point_normal = [&](int b, int e, int sg, double* n, double& mag) {
        const RefElement& R = ctx->etypes[blocks[b].etype]->R;
        const HostBlk& H = hb[b];
        if (m->blocks[b]->curved) {
            const size_t pt = (size_t)e * R.nfe + sg;
            for (int i = 0; i < nd; ++i) n[i] = H.pn[pt * nd + i];
            mag = H.pmag[pt];
            return;
        }
        const int f = R.fe_face[sg];
        const double* Ji = &H.Ji[(size_t)e * nd * nd];
        double s = 0;
        for (int i = 0; i < nd; ++i) {
            n[i] = 0;
            for (int d = 0; d < nd; ++d) n[i] += Ji[d * nd + i] * R.face_nrm[f * nd + d];
            s += n[i] * n[i];
        }
        s = std::sqrt(s);
        for (int i = 0; i < nd; ++i) n[i] /= s;
        mag = H.det[e] * s;
    };
    for (int64_t fi = 0; fi < nfaces; ++fi) {
        const sdrt_face& F = faces[fi];
        int bs[2] = {F.blk_l, F.blk_r}, es[2] = {F.elem_l, F.elem_r}, fs[2] = {F.face_l, F.face_r};
        for (int s = 0; s < 2; ++s) {
            if (bs[s] < 0 || bs[s] >= nblocks || es[s] < 0 || es[s] >= blocks[bs[s]].nelem)
                return fail(ctx, SDRT_ERR_ARG, "face references a missing element");
            const RefElement& R = ctx->etypes[blocks[bs[s]].etype]->R;
            if (fs[s] < 0 || fs[s] >= R.nfaces) return fail(ctx, SDRT_ERR_ARG, "bad local face index");
            uint8_t& g = hb[bs[s]].glued[(size_t)es[s] * R.nfaces + fs[s]];
            if (g) return fail(ctx, SDRT_ERR_MESH, "a face is glued twice");
            g = 1;
        }
        const RefElement& RL = ctx->etypes[blocks[F.blk_l].etype]->R;
        const RefElement& RR = ctx->etypes[blocks[F.blk_r].etype]->R;
        std::vector<int> iL, iR;
        for (int s = 0; s < RL.nfe; ++s)
            if (RL.fe_face[s] == F.face_l) iL.push_back(s);
        for (int s = 0; s < RR.nfe; ++s)
            if (RR.fe_face[s] == F.face_r) iR.push_back(s);
        if (iL.size() != iR.size()) return fail(ctx, SDRT_ERR_MESH, "glued faces have different point counts");
        const double tol = 1e-8 * hb[F.blk_l].h[F.elem_l];
        std::vector<char> used(iR.size(), 0);
        const MBlock& bl = *m->blocks[F.blk_l];
        const MBlock& br = *m->blocks[F.blk_r];
        for (size_t a = 0; a < iL.size(); ++a) {
            const double* xl = &hb[F.blk_l].xfe[((size_t)F.elem_l * RL.nfe + iL[a]) * nd];
            int hit = -1;
            for (size_t c = 0; c < iR.size(); ++c) {
                if (used[c]) continue;
                const double* xr = &hb[F.blk_r].xfe[((size_t)F.elem_r * RR.nfe + iR[c]) * nd];
                double dd = 0;
                for (int i = 0; i < nd; ++i) dd = std::max(dd, std::fabs(xr[i] + F.shift[i] - xl[i]));
                if (dd <= tol) {
                    hit = (int)c;
                    break;
                }
            }
            if (hit < 0) return fail(ctx, SDRT_ERR_MESH, "face flux points do not coincide (face " + std::to_string(fi) + ")");
            used[hit] = 1;
            const int sL = iL[a], sR = iR[hit];
            int64_t gL = bl.canon_base + (int64_t)F.elem_l * RL.nfe + sL;
            int64_t gR = br.canon_base + (int64_t)F.elem_r * RR.nfe + sR;
            m->partner[gL] = (int32_t)gR;
            m->partner[gR] = (int32_t)gL;
            m->is_left[gL] = 1;
            // Face metric: the L side's unit normal on both sides; each side's
            // own scale, signed (+ on the L side).
            double nL[3], nR[3], magL, magR;
            point_normal(F.blk_l, F.elem_l, sL, nL, magL);
            point_normal(F.blk_r, F.elem_r, sR, nR, magR);
            const int rl = bl.mr_f + F.face_l * bl.mr_ff + sL * bl.mr_fp;
            const int rr = br.mr_f + F.face_r * br.mr_ff + sR * br.mr_fp;
            for (int c = 0; c < nd; ++c) {
                hb[F.blk_l].metric[(size_t)(rl + c) * bl.ld + F.elem_l] = nL[c];
                hb[F.blk_r].metric[(size_t)(rr + c) * br.ld + F.elem_r] = nL[c];
            }
            hb[F.blk_l].metric[(size_t)(rl + nd) * bl.ld + F.elem_l] = magL;
            hb[F.blk_r].metric[(size_t)(rr + nd) * br.ld + F.elem_r] = -magR;
        }
    }
    for (int b = 0; b < nown; ++b)     // ghost elements keep their other faces unglued
        for (uint8_t g : hb[b].glued)
            if (!g) return fail(ctx, SDRT_ERR_MESH, "mesh has an unglued face (only closed / periodic meshes)");

    // Device copies (ghost blocks need none: only their face records are read).
    for (int b = 0; b < nown; ++b) {
        MBlock& mb = *m->blocks[b];
        const RefElement& R = ctx->etypes[mb.etype]->R;
        std::vector<int> dmap((size_t)R.nfe * mb.ld, 0);
        for (int e = 0; e < mb.nelem; ++e)
            for (int s = 0; s < R.nfe; ++s) {
                int64_t g = m->partner[mb.canon_base + (int64_t)e * R.nfe + s];
                int pb = nblocks - 1;
                while (m->blocks[pb]->canon_base > g) --pb;
                const MBlock& q = *m->blocks[pb];
                const int qnfe = ctx->etypes[q.etype]->R.nfe;
                const int64_t rel = g - q.canon_base;
                const int pe = (int)(rel / qnfe), ps = (int)(rel % qnfe);
                dmap[(size_t)s * mb.ld + e] = (int)(q.fe_base + (int64_t)ps * q.ld + pe);
            }
        if (!ctx->host_only) {
            SDRT_CUDA(upload(mb.map, dmap));
            if (f32) {
                std::vector<float> mf(hb[b].metric.begin(), hb[b].metric.end());
                SDRT_CUDA(upload(mb.metric, mf));
            } else {
                SDRT_CUDA(upload(mb.metric, hb[b].metric));
            }
        }
        if (m->fast) {
            // Record-path tables: metric rows per element, partner face-record
            // offsets, partner permutations, point offsets inside a record.
            const int NM = mb.nmetric;
            std::vector<double> maos((size_t)mb.nelem * mb.nmp, 0.0);
            for (int e = 0; e < mb.nelem; ++e)
                for (int k = 0; k < NM; ++k) maos[(size_t)e * mb.nmp + k] = hb[b].metric[(size_t)k * mb.ld + e];
            std::vector<int> first(R.nfaces, -1);
            for (int s = 0; s < R.nfe; ++s)
                if (first[R.fe_face[s]] < 0) first[R.fe_face[s]] = s;
            std::vector<int> recoff(R.nfe);
            for (int s = 0; s < R.nfe; ++s)
                recoff[s] = R.fe_face[s] * mb.frec + (s - first[R.fe_face[s]]) * m->nvar;
            std::vector<int> pfr((size_t)mb.nelem * R.nfaces, 0);
            std::vector<uint8_t> perm((size_t)mb.nelem * mb.pstride, 0);
            for (int e = 0; e < mb.nelem; ++e)
                for (int s = 0; s < R.nfe; ++s) {
                    int64_t g = m->partner[mb.canon_base + (int64_t)e * R.nfe + s];
                    int pb = nblocks - 1;
                    while (m->blocks[pb]->canon_base > g) --pb;
                    const MBlock& q = *m->blocks[pb];
                    const RefElement& RQ = ctx->etypes[q.etype]->R;
                    const int64_t rel = g - q.canon_base;
                    const int pe = (int)(rel / RQ.nfe), ps = (int)(rel % RQ.nfe);
                    const int pf = RQ.fe_face[ps];
                    int pfirst = 0;
                    while (RQ.fe_face[pfirst] != pf) ++pfirst;
                    pfr[(size_t)e * R.nfaces + R.fe_face[s]] = (int)(q.rec_base + (int64_t)pe * q.ers + pf * q.frec);
                    perm[(size_t)e * mb.pstride + s] = (uint8_t)(ps - pfirst);
                }
            if (m->rec_total >= INT32_MAX) return fail(ctx, SDRT_ERR_UNSUPPORTED, "mesh too large for int32 record offsets");
            if (!ctx->host_only) {
                if (f32) {
                    std::vector<float> mf(maos.begin(), maos.end());
                    SDRT_CUDA(upload(mb.maos, mf));
                } else {
                    SDRT_CUDA(upload(mb.maos, maos));
                }
                SDRT_CUDA(upload(mb.pfr, pfr));
                SDRT_CUDA(upload(mb.perm, perm));
                SDRT_CUDA(upload(mb.recoff, recoff));
            }
        }
        // Tile widths: keep the residual kernel's shared memory within ~100 KB
        // (two CTAs per SM), down to 8 elements per tile for large element types.
        const EType& et = *ctx->etypes[mb.etype];
        auto smem_of = [&](int TE, bool dual) {
            int ra = std::max(R.nsol, R.nfi);
            return (ra + et.Mi) * m->nvar * TE * (f32 ? 4 : 8) * (dual ? 2 : 1);
        };
        for (int dual = 0; dual < 2; ++dual) {
            int TE = 32;
            while (TE > 4 && smem_of(TE, dual) > 100 * 1024) TE /= 2;
            if (smem_of(TE, dual) > 220 * 1024) {
                if (!dual) return fail(ctx, SDRT_ERR_UNSUPPORTED, "element type too large for the shared-memory tile");
                TE = 0;   // JVP unavailable for this block
            }
            (dual ? mb.tile_dual : mb.tile) = TE;
        }
        if (phys->system == SDRT_ADVDIFF || phys->system == SDRT_NAVIER_STOKES) {
            auto gsmem_of = [&](int TE, bool dual) {
                return (R.nsol + R.nfe + nd * R.nsol) * m->nvar * TE * (f32 ? 4 : 8) * (dual ? 2 : 1);
            };
            for (int dual = 0; dual < 2; ++dual) {
                int TE = 32;
                while (TE > 4 && gsmem_of(TE, dual) > 100 * 1024) TE /= 2;
                while (TE > 1 && gsmem_of(TE, dual) > 220 * 1024) TE /= 2;
                if (gsmem_of(TE, dual) > 220 * 1024) {
                    if (!dual) return fail(ctx, SDRT_ERR_UNSUPPORTED, "element type too large for the gradient tile");
                    TE = 0;
                }
                (dual ? mb.gtile_dual : mb.gtile) = TE;
            }
        }
        {
            const bool visc = phys->system == SDRT_ADVDIFF || phys->system == SDRT_NAVIER_STOKES;
            auto vsmem_of = [&](int TE) {
                const int rows = R.nsol + R.nfiu + R.nfi + R.nfe + (visc ? nd * (R.nfe + R.nfiu + R.nsol) : 0);
                return rows * m->nvar * TE * (f32 ? 4 : 8);
            };
            int TE = 32;
            while (TE > 1 && vsmem_of(TE) > 100 * 1024) TE /= 2;
            mb.vtile = vsmem_of(TE) <= 220 * 1024 ? TE : 0;
        }
    }
    if (ghost) {
        // The state arrays and every kernel cover the owned blocks; the ghost
        // blocks keep their face-record slots (after the owned records).
        int64_t gsol = 0;
        for (int b = nown; b < nblocks; ++b) {
            MBlock& g = *m->blocks[b];
            const RefElement& R = ctx->etypes[g.etype]->R;
            m->ndof -= (int64_t)R.nsol * m->nvar * g.nelem;
            gsol += (int64_t)g.nelem * R.nsol * nd;
        }
        if (nown < nblocks) m->state_len = m->blocks[nown]->u_off;   // no ghost blocks: one partition
        m->sol_xyz.resize(m->sol_xyz.size() - (size_t)gsol);
        for (int b = nown; b < nblocks; ++b) m->ghosts.push_back(std::move(m->blocks[b]));
        m->blocks.resize(nown);
        m->partition = true;
        if (m->fast) {
            m->xfrec = m->blocks[0]->frec;
        } else {
            // Generic path: records of (points per face) x nvar values, padded to the
            // largest face of the mesh's element types and to a multiple of 4.
            int npf = 0;
            for (int b = 0; b < nblocks; ++b) {
                const MBlock& q = b < nown ? *m->blocks[b] : *m->ghosts[b - nown];
                const RefElement& R = ctx->etypes[q.etype]->R;
                std::vector<int> cnt(R.nfaces, 0);
                for (int k = 0; k < R.nfe; ++k) npf = std::max(npf, ++cnt[R.fe_face[k]]);
            }
            m->xfrec = round_up(npf * m->nvar, 4);
            if (viscous(*m)) m->xgrec = round_up(npf * nd * m->nvar, 4);
        }
    }
    // Operator-specialised path: FP32 3D Euler / Rusanov on whole meshes of
    // SDRT element types that have generated kernels and are not on the
    // record path.
    if (!ghost && !m->fast && !m->curved && f32 && phys->system == SDRT_EULER && nd == 3 &&
        phys->riemann == SDRT_RUSANOV && (int64_t)m->Ftot * m->nvar < INT32_MAX) {
        bool all = true;
        for (auto& bp : m->blocks) {
            const EType& et = *ctx->etypes[bp->etype];
            bp->gen = et.desc.scheme == SDRT_SCHEME_SDRT ? gen_launcher(et.R.shape, et.R.p) : nullptr;
            all = all && bp->gen != nullptr;
        }
        m->gen = all;
    }
    if (m->gen && !ctx->host_only) {
        for (auto& bp : m->blocks) {
            MBlock& mb = *bp;
            const int nfe = ctx->etypes[mb.etype]->R.nfe;
            std::vector<int> pm((size_t)nfe * mb.ld, 0);
            for (int e = 0; e < mb.nelem; ++e)
                for (int sg = 0; sg < nfe; ++sg) {
                    // partner (block q, element pe, point ps) of canonical index g
                    const int64_t g = m->partner[mb.canon_base + (int64_t)e * nfe + sg];
                    int pb = (int)m->blocks.size() - 1;
                    while (m->blocks[pb]->canon_base > g) --pb;
                    const MBlock& q = *m->blocks[pb];
                    const int qnfe = ctx->etypes[q.etype]->R.nfe;
                    const int64_t pe = (g - q.canon_base) / qnfe, ps = (g - q.canon_base) % qnfe;
                    pm[(size_t)sg * mb.ld + e] =
                        (int)((q.fe_base + (pe / 32) * 32 * qnfe + ps * 32 + pe % 32) * m->nvar);
                }
            SDRT_CUDA(upload(mb.pmap, pm));
        }
        if (m->blocks.size() > 1) {
            SDRT_CUDA(cudaEventCreateWithFlags(&m->fork_ev, cudaEventDisableTiming));
            for (size_t b = 0; b < m->blocks.size(); ++b) {
                cudaStream_t st;
                cudaEvent_t ev;
                SDRT_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
                m->br.push_back(st);
                SDRT_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
                m->brev.push_back(ev);
            }
        }
    }
    // Block tables of the generic kernels (tile widths are final here).
    if (int rt = refresh_tables(ctx, *m)) return rt;
    ctx->meshes.push_back(std::move(m));
    *mesh_id = (int)ctx->meshes.size() - 1;
    return SDRT_OK;
}

int sdrt_get_mesh_info(sdrt_ctx* ctx, int mesh_id, sdrt_mesh_info* out) {
    int r = check_mesh(ctx, mesh_id);
    if (r) return r;
    if (!out) return fail(ctx, SDRT_ERR_ARG, "null output");
    const Mesh& m = *ctx->meshes[mesh_id];
    out->nvar = m.nvar;
    out->nblocks = (int)m.blocks.size();
    out->ndim = m.nd;
    out->precision = m.tc3 ? SDRT_TF32X3 : m.phys.precision;
    out->state_len = m.state_len;
    out->ndof = m.ndof;
    out->nfe_total = m.nfe_total;
    out->path = m.fast ? SDRT_PATH_RECORD : (m.gen && ctx->use_gen) ? SDRT_PATH_GENERATED : SDRT_PATH_GENERIC;
    out->curved = m.curved ? 1 : 0;
    return SDRT_OK;
}

int sdrt_get_block_layout(sdrt_ctx* ctx, int mesh_id, int block, sdrt_block_layout* out) {
    int r = check_mesh(ctx, mesh_id);
    if (r) return r;
    const Mesh& m = *ctx->meshes[mesh_id];
    if (!out || block < 0 || block >= (int)m.blocks.size()) return fail(ctx, SDRT_ERR_ARG, "bad block");
    const MBlock& b = *m.blocks[block];
    const RefElement& R = ctx->etypes[b.etype]->R;
    *out = {b.etype, R.nsol, m.nvar, b.nelem, b.ld, R.nfe, b.u_off};
    return SDRT_OK;
}

int sdrt_get_sol_points(sdrt_ctx* ctx, int mesh_id, double* out, int64_t n) {
    int r = check_mesh(ctx, mesh_id);
    if (r) return r;
    const Mesh& m = *ctx->meshes[mesh_id];
    if (!out || n != (int64_t)m.sol_xyz.size()) return fail(ctx, SDRT_ERR_ARG, "size mismatch");
    std::memcpy(out, m.sol_xyz.data(), m.sol_xyz.size() * sizeof(double));
    return SDRT_OK;
}

int sdrt_get_face_map(sdrt_ctx* ctx, int mesh_id, int32_t* partner, uint8_t* is_left, int64_t n) {
    int r = check_mesh(ctx, mesh_id);
    if (r) return r;
    const Mesh& m = *ctx->meshes[mesh_id];
    if (!partner || n != m.nfe_total) return fail(ctx, SDRT_ERR_ARG, "size mismatch");
    std::memcpy(partner, m.partner.data(), m.partner.size() * sizeof(int32_t));
    if (is_left) std::memcpy(is_left, m.is_left.data(), m.is_left.size());
    return SDRT_OK;
}

int sdrt_residual(sdrt_ctx* ctx, int mesh_id, const void* U, void* R) {
    NvtxScope nvtx_scope(ctx, "sdrt_residual");
    int r = check_whole(ctx, mesh_id);
    if (r) return r;
    if (!U || !R || U == R) return fail(ctx, SDRT_ERR_ARG, "U and R must be distinct device arrays");
    Mesh& m = *ctx->meshes[mesh_id];
    if ((r = ensure_workspace(ctx, m, false, false))) return r;
    if (m.phys.precision == SDRT_FP32) {
        KEpi<float> E{};
        E.mode = EPI_STORE;
        E.out = static_cast<float*>(R);
        E.flag = ctx->flag.as<int>();
        return run_residual<float>(ctx, m, static_cast<const float*>(U), nullptr, E);
    }
    KEpi<double> E{};
    E.mode = EPI_STORE;
    E.out = static_cast<double*>(R);
    E.flag = ctx->flag.as<int>();
    return run_residual<double>(ctx, m, static_cast<const double*>(U), nullptr, E);
}

int sdrt_set_exchange(sdrt_ctx* ctx, int mesh_id, int64_t nsend, const int32_t* send, int64_t nrecv,
                      const int32_t* recv) {
    int r = check_mesh(ctx, mesh_id);
    if (r) return r;
    Mesh& m = *ctx->meshes[mesh_id];
    if (!m.partition) return fail(ctx, SDRT_ERR_STATE, "not a partition mesh");
    if (nsend < 0 || nrecv < 0 || (nsend > 0 && !send) || (nrecv > 0 && !recv))
        return fail(ctx, SDRT_ERR_ARG, "bad exchange lists");
    const int nown = (int)m.blocks.size();
    auto offsets = [&](int64_t n, const int32_t* t, bool ghosts, std::vector<int>& out) -> bool {
        out.resize(n);
        for (int64_t i = 0; i < n; ++i) {
            const int b = t[3 * i], e = t[3 * i + 1], f = t[3 * i + 2];
            const MBlock* q = nullptr;
            if (!ghosts && b >= 0 && b < nown) q = m.blocks[b].get();
            if (ghosts && b >= nown && b < nown + (int)m.ghosts.size()) q = m.ghosts[b - nown].get();
            if (!q || e < 0 || e >= q->nelem || f < 0 || f >= ctx->etypes[q->etype]->R.nfaces) return false;
            out[i] = (int)(q->rec_base + (int64_t)e * q->ers + (int64_t)f * q->frec);
        }
        return true;
    };
    std::vector<int> so, ro;
    if (!offsets(nsend, send, false, so)) return fail(ctx, SDRT_ERR_ARG, "send list: not an owned (block, element, face)");
    if (!offsets(nrecv, recv, true, ro)) return fail(ctx, SDRT_ERR_ARG, "receive list: not a ghost (block, element, face)");
    if (m.fast) {
        if (!ctx->host_only) {
            if (nsend > 0) SDRT_CUDA(upload(m.xsend_off, so));
            if (nrecv > 0) SDRT_CUDA(upload(m.xrecv_off, ro));
        }
    } else {
        // Generic path: value k * nvar + v of a record is variable v of the face's
        // k-th point (local point order) in the face-state array UFE.
        auto indices = [&](int64_t n, const int32_t* t, std::vector<int>& out) {
            out.assign((size_t)n * m.xfrec, -1);
            for (int64_t i = 0; i < n; ++i) {
                const int b = t[3 * i], e = t[3 * i + 1], f = t[3 * i + 2];
                const MBlock& q = b < nown ? *m.blocks[b] : *m.ghosts[b - nown];
                const RefElement& R = ctx->etypes[q.etype]->R;
                int k = 0;
                for (int sg = 0; sg < R.nfe; ++sg) {
                    if (R.fe_face[sg] != f) continue;
                    for (int v = 0; v < m.nvar; ++v)
                        out[(size_t)i * m.xfrec + k * m.nvar + v] =
                            (int)((int64_t)v * m.Ftot + q.fe_base + (int64_t)sg * q.ld + e);
                    ++k;
                }
            }
        };
        std::vector<int> si, ri;
        indices(nsend, send, si);
        indices(nrecv, recv, ri);
        if (!ctx->host_only) {
            if (nsend > 0) SDRT_CUDA(upload(m.xsend_idx, si));
            if (nrecv > 0) SDRT_CUDA(upload(m.xrecv_idx, ri));
        }
        if (m.xgrec > 0) {
            // Gradient records: value k * nd * nvar + dv is component dv = d * nvar + v
            // of the face's k-th point in QFE ([nd][nvar][F_tot]).
            const int ndv = m.nd * m.nvar;
            auto gindices = [&](int64_t n, const int32_t* t, std::vector<int>& out) {
                out.assign((size_t)n * m.xgrec, -1);
                for (int64_t i = 0; i < n; ++i) {
                    const int b = t[3 * i], e = t[3 * i + 1], f = t[3 * i + 2];
                    const MBlock& q = b < nown ? *m.blocks[b] : *m.ghosts[b - nown];
                    const RefElement& R = ctx->etypes[q.etype]->R;
                    int k = 0;
                    for (int sg = 0; sg < R.nfe; ++sg) {
                        if (R.fe_face[sg] != f) continue;
                        for (int dv = 0; dv < ndv; ++dv)
                            out[(size_t)i * m.xgrec + k * ndv + dv] =
                                (int)((int64_t)dv * m.Ftot + q.fe_base + (int64_t)sg * q.ld + e);
                        ++k;
                    }
                }
            };
            std::vector<int> gs, gr;
            gindices(nsend, send, gs);
            gindices(nrecv, recv, gr);
            if (!ctx->host_only) {
                if (nsend > 0) SDRT_CUDA(upload(m.xsend_gidx, gs));
                if (nrecv > 0) SDRT_CUDA(upload(m.xrecv_gidx, gr));
            }
        }
    }
    m.nsend = nsend;
    m.nrecv = nrecv;
    return SDRT_OK;
}

int sdrt_get_exchange_info(sdrt_ctx* ctx, int mesh_id, int64_t* nsend, int64_t* nrecv, int32_t* face_record,
                           int32_t* grad_record) {
    int r = check_mesh(ctx, mesh_id);
    if (r) return r;
    const Mesh& m = *ctx->meshes[mesh_id];
    if (!m.partition) return fail(ctx, SDRT_ERR_STATE, "not a partition mesh");
    if (nsend) *nsend = m.nsend;
    if (nrecv) *nrecv = m.nrecv;
    if (face_record) *face_record = m.xfrec;
    if (grad_record) *grad_record = m.xgrec;
    return SDRT_OK;
}


static int check_partition(sdrt_ctx* ctx, int mesh_id) {
    int r = check_compute(ctx, mesh_id);
    if (r) return r;
    const Mesh& m = *ctx->meshes[mesh_id];
    if (!m.partition) return fail(ctx, SDRT_ERR_STATE, "not a partition mesh");
    if (m.nsend < 0) return fail(ctx, SDRT_ERR_STATE, "no exchange lists (sdrt_set_exchange)");
    return SDRT_OK;
}

int sdrt_residual_gradients(sdrt_ctx* ctx, int mesh_id, const void* recv, void* send_grad) {
    NvtxScope nvtx_scope(ctx, "sdrt_residual_gradients");
    int r = check_partition(ctx, mesh_id);
    if (r) return r;
    Mesh& m = *ctx->meshes[mesh_id];
    if (!viscous(m)) return fail(ctx, SDRT_ERR_STATE, "gradients are exchanged for the viscous systems only");
    if (!m.part_u) return fail(ctx, SDRT_ERR_STATE, "sdrt_residual_gradients before sdrt_residual_begin");
    if ((m.nrecv > 0 && !recv) || (m.nsend > 0 && !send_grad)) return fail(ctx, SDRT_ERR_ARG, "null array");
    if ((r = ensure_workspace(ctx, m, false, false))) return r;
    if (m.phys.precision == SDRT_FP32)
        return residual_gradients_impl<float>(ctx, m, static_cast<const float*>(recv), static_cast<float*>(send_grad));
    return residual_gradients_impl<double>(ctx, m, static_cast<const double*>(recv), static_cast<double*>(send_grad));
}

int sdrt_residual_begin(sdrt_ctx* ctx, int mesh_id, const void* U, void* send) {
    NvtxScope nvtx_scope(ctx, "sdrt_residual_begin");
    int r = check_partition(ctx, mesh_id);
    if (r) return r;
    Mesh& m = *ctx->meshes[mesh_id];
    if (!U || (m.nsend > 0 && !send)) return fail(ctx, SDRT_ERR_ARG, "null array");
    if ((r = ensure_workspace(ctx, m, false, false))) return r;
    if (m.phys.precision == SDRT_FP32)
        return residual_begin_impl<float>(ctx, m, static_cast<const float*>(U), static_cast<float*>(send));
    return residual_begin_impl<double>(ctx, m, static_cast<const double*>(U), static_cast<double*>(send));
}

int sdrt_residual_end(sdrt_ctx* ctx, int mesh_id, const void* recv, void* R) {
    NvtxScope nvtx_scope(ctx, "sdrt_residual_end");
    int r = check_partition(ctx, mesh_id);
    if (r) return r;
    Mesh& m = *ctx->meshes[mesh_id];
    if (!R || (m.nrecv > 0 && !recv)) return fail(ctx, SDRT_ERR_ARG, "null array");
    if ((r = ensure_workspace(ctx, m, false, false))) return r;
    if (m.phys.precision == SDRT_FP32)
        return residual_end_impl<float>(ctx, m, static_cast<const float*>(recv), static_cast<float*>(R));
    return residual_end_impl<double>(ctx, m, static_cast<const double*>(recv), static_cast<double*>(R));
}

static int rk4_eager(sdrt_ctx* ctx, Mesh& m, void* U, double dt) {
    if (m.phys.precision == SDRT_FP32) return rk4_stages<float>(ctx, m, static_cast<float*>(U), dt);
    return rk4_stages<double>(ctx, m, static_cast<double*>(U), dt);
}

int sdrt_rk4_step(sdrt_ctx* ctx, int mesh_id, void* U, double dt, int nsteps) {
    NvtxScope nvtx_scope(ctx, "sdrt_rk4_step");
    int r = check_whole(ctx, mesh_id);
    if (r) return r;
    if (!U || nsteps < 0 || !(std::isfinite(dt))) return fail(ctx, SDRT_ERR_ARG, "bad argument");
    Mesh& m = *ctx->meshes[mesh_id];
    if ((r = ensure_workspace(ctx, m, false, true))) return r;
    int s = 0;
    if (!m.warmed && nsteps > 0) {
        // First step runs eagerly (loads the kernels) before any graph capture.
        if ((r = rk4_eager(ctx, m, U, dt))) return r;
        m.warmed = true;
        s = 1;
    }
    if (s >= nsteps) return SDRT_OK;
    if (!m.graph || m.graph_u != U || m.graph_dt != dt) {
        if (m.graph) {
            cudaGraphExecDestroy(m.graph);
            m.graph = nullptr;
        }
        if (ctx->stream == nullptr) {
            // Capture needs a non-default stream: run eagerly.
            for (; s < nsteps; ++s)
                if ((r = rk4_eager(ctx, m, U, dt))) return r;
            return SDRT_OK;
        }
        cudaGraph_t g;
        const int64_t before = ctx->launches;
        m.graph_slots.clear();
        SDRT_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        ctx->capture_slots = &m.graph_slots;
        r = rk4_eager(ctx, m, U, dt);
        ctx->capture_slots = nullptr;
        cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
        m.graph_launches = ctx->launches - before;   // kernel nodes of one RK4 step
        ctx->launches = before;
        if (r) return r;
        if (ce != cudaSuccess) return fail(ctx, SDRT_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&m.graph, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) return fail(ctx, SDRT_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ce));
        m.graph_u = U;
        m.graph_dt = dt;
    }
    for (; s < nsteps; ++s) {
        SDRT_CUDA(cudaGraphLaunch(m.graph, ctx->stream));
        ctx->launches += m.graph_launches;
    }
    // Events inside the graph hold the timings of its last replay.
    if (ctx->prof) ctx->pending.insert(ctx->pending.end(), m.graph_slots.begin(), m.graph_slots.end());
    return SDRT_OK;
}

}  // extern "C"

namespace {

// One RK54 step of U (device), five residuals and stage updates; with
// estimate, the embedded estimate accumulates in m.rk_err.
template <typename T>
int rk54_stages(sdrt_ctx* ctx, Mesh& m, T* U, double dt, bool estimate) {
    static const std::array<double, 5> ne = rk54_estimate_weights();
    T* R = m.rk_r.as<T>();
    for (int i = 0; i < 5; ++i) {
        KEpi<T> E{};
        E.mode = EPI_STORE;
        E.out = R;
        E.flag = ctx->flag.as<int>();
        int r = run_residual<T>(ctx, m, U, nullptr, E);
        if (r) return r;
        launch_rk2n<T>(m.state_len, U, m.rk_du.as<T>(), R, estimate ? m.rk_err.as<T>() : nullptr, kRK54A[i],
                       kRK54B[i], ne[i], dt, i == 0, ctx->nsm, ctx->stream);
        ++ctx->launches;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SDRT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return SDRT_OK;
}

int rk54_workspace(sdrt_ctx* ctx, Mesh& m, bool adaptive) {
    const size_t bytes = (size_t)m.state_len * (m.phys.precision == SDRT_FP32 ? 4 : 8);
    if (!m.rk_r.p) SDRT_CUDA(m.rk_r.alloc(bytes));
    if (!m.rk_du.p) SDRT_CUDA(m.rk_du.alloc(bytes));
    if (adaptive) {
        if (!m.rk_err.p) SDRT_CUDA(m.rk_err.alloc(bytes));
        if (!m.rk_u0.p) SDRT_CUDA(m.rk_u0.alloc(bytes));
        if (!m.rk_part.p) SDRT_CUDA(m.rk_part.alloc(256 * sizeof(double)));
    }
    return SDRT_OK;
}

// One attempted adaptive step: on acceptance U holds the new state, on
// rejection the old one; *err = the L-infinity error norm.
template <typename T>
int rk54_attempt(sdrt_ctx* ctx, Mesh& m, T* U, double dt, double atol, double rtol, double* err) {
    const size_t bytes = (size_t)m.state_len * sizeof(T);
    SDRT_CUDA(cudaMemcpyAsync(m.rk_u0.p, U, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    int r = rk54_stages<T>(ctx, m, U, dt, true);
    if (r) return r;
    const int nparts = 256;
    launch_err_linf<T>(m.state_len, m.rk_err.as<T>(), m.rk_u0.as<T>(), U, atol, rtol, m.rk_part.as<double>(), nparts,
                       ctx->stream);
    ++ctx->launches;
    double part[256];
    SDRT_CUDA(cudaMemcpyAsync(part, m.rk_part.p, nparts * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    SDRT_CUDA(cudaStreamSynchronize(ctx->stream));
    double e = 0;
    for (int i = 0; i < nparts; ++i) e = (part[i] > e || part[i] != part[i]) ? part[i] : e;
    *err = e;
    if (!(e <= 1.0)) SDRT_CUDA(cudaMemcpyAsync(U, m.rk_u0.p, bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    return SDRT_OK;
}

}  // namespace

extern "C" {

int sdrt_rk54_step(sdrt_ctx* ctx, int mesh_id, void* U, double dt, int nsteps) {
    NvtxScope nvtx_scope(ctx, "sdrt_rk54_step");
    int r = check_whole(ctx, mesh_id);
    if (r) return r;
    if (!U || nsteps < 0 || !(std::isfinite(dt))) return fail(ctx, SDRT_ERR_ARG, "bad argument");
    Mesh& m = *ctx->meshes[mesh_id];
    if ((r = ensure_workspace(ctx, m, false, false))) return r;
    if ((r = rk54_workspace(ctx, m, false))) return r;
    for (int s = 0; s < nsteps; ++s) {
        r = m.phys.precision == SDRT_FP32 ? rk54_stages<float>(ctx, m, static_cast<float*>(U), dt, false)
                                           : rk54_stages<double>(ctx, m, static_cast<double*>(U), dt, false);
        if (r) return r;
    }
    return SDRT_OK;
}

int sdrt_rk54_adaptive_step(sdrt_ctx* ctx, int mesh_id, void* U, double dt, double atol, double rtol, double* err,
                            double* dt_next, int* accepted) {
    NvtxScope nvtx_scope(ctx, "sdrt_rk54_adaptive_step");
    int r = check_whole(ctx, mesh_id);
    if (r) return r;
    if (!U || !err || !dt_next || !accepted || !(dt > 0) || !(atol > 0) || !(rtol >= 0))
        return fail(ctx, SDRT_ERR_ARG, "bad argument");
    Mesh& m = *ctx->meshes[mesh_id];
    if ((r = ensure_workspace(ctx, m, false, false))) return r;
    if ((r = rk54_workspace(ctx, m, true))) return r;
    double e = 0;
    r = m.phys.precision == SDRT_FP32 ? rk54_attempt<float>(ctx, m, static_cast<float*>(U), dt, atol, rtol, &e)
                                       : rk54_attempt<double>(ctx, m, static_cast<double*>(U), dt, atol, rtol, &e);
    if (r) return r;
    *err = e;
    if (!(e == e)) return fail(ctx, SDRT_ERR_NONFINITE, "non-finite RK54 error estimate");
    *accepted = e <= 1.0;
    *dt_next = dt * pi_factor(e, m.pi_err_prev, *accepted != 0);
    if (*accepted) m.pi_err_prev = e;
    return SDRT_OK;
}

int sdrt_rk54_integrate(sdrt_ctx* ctx, int mesh_id, void* U, double t_span, double* dt_inout, double atol,
                        double rtol, int max_steps, int* n_accepted, int* n_rejected) {
    NvtxScope nvtx_scope(ctx, "sdrt_rk54_integrate");
    if (!dt_inout || !n_accepted || !n_rejected || !(t_span >= 0) || max_steps < 1)
        return fail(ctx, SDRT_ERR_ARG, "bad argument");
    *n_accepted = *n_rejected = 0;
    double t = 0, dt = *dt_inout;
    while (t < t_span) {
        if (*n_accepted + *n_rejected >= max_steps)
            return fail(ctx, SDRT_ERR_STATE, "RK54 integration did not reach the end within max_steps");
        const double h = std::min(dt, t_span - t);
        double err = 0, dn = 0;
        int acc = 0;
        int r = sdrt_rk54_adaptive_step(ctx, mesh_id, U, h, atol, rtol, &err, &dn, &acc);
        if (r) return r;
        if (acc) {
            t += h;
            ++*n_accepted;
        } else {
            ++*n_rejected;
        }
        dt = dn;
    }
    *dt_inout = dt;
    return SDRT_OK;
}

}  // extern "C"

namespace {

template <typename T>
int tgv_diagnostics(sdrt_ctx* ctx, Mesh& m, const T* U, double* sums) {
    T* R = m.rk_r.as<T>();
    KEpi<T> E{};
    E.mode = EPI_STORE;
    E.out = R;
    E.flag = ctx->flag.as<int>();
    int r = run_residual<T>(ctx, m, U, nullptr, E);
    if (r) return r;
    const KPhys<T> P = make_phys<T>(m.phys);
    const KSet<T> ks = kset<T>(m);
    launch_interp_ext<T>(ks, m.nvar, U, m.ufe.as<T>(), m.Ftot, ctx->nsm, ctx->stream);
    ++ctx->launches;
    r = launch_grad<T>(ks, m.phys.system, m.nd, U, nullptr, m.ufe.as<T>(), nullptr, m.Ftot, P, m.qfe.as<T>(), nullptr,
                       m.qfiu.as<T>(), nullptr, ctx->nsm, ctx->stream, m.qsol.as<T>());
    if (r) return fail(ctx, SDRT_ERR_UNSUPPORTED, "gradient kernel not available");
    ++ctx->launches;
    SDRT_CUDA(cudaMemsetAsync(m.diag_sums.p, 0, 5 * sizeof(double), ctx->stream));
    const int pi = std::is_same<T, float>::value ? 1 : 0;
    for (auto& bp : m.blocks) {
        const EType& et = *ctx->etypes[bp->etype];
        launch_tgv_diag<T>(make_kblock<T>(et, *bp), U, m.qsol.as<T>(), R, et.Mq[pi].as<T>(), et.wq[pi].as<T>(),
                           (int)et.R.wq.size(), (T)m.phys.gamma, m.diag_sums.as<double>(), ctx->nsm, ctx->stream);
        ++ctx->launches;
    }
    SDRT_CUDA(cudaMemcpyAsync(sums, m.diag_sums.p, 5 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    SDRT_CUDA(cudaStreamSynchronize(ctx->stream));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SDRT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return SDRT_OK;
}

}  // namespace

extern "C" {

int sdrt_tgv_diagnostics(sdrt_ctx* ctx, int mesh_id, const void* U, double rho_inf, double v_inf, double length,
                         double* out) {
    NvtxScope nvtx_scope(ctx, "sdrt_tgv_diagnostics");
    int r = check_whole(ctx, mesh_id);
    if (r) return r;
    if (!U || !out || !(rho_inf > 0) || !(v_inf > 0) || !(length > 0)) return fail(ctx, SDRT_ERR_ARG, "bad argument");
    Mesh& m = *ctx->meshes[mesh_id];
    if (m.phys.system != SDRT_NAVIER_STOKES || m.nd != 3)
        return fail(ctx, SDRT_ERR_UNSUPPORTED, "the Taylor-Green diagnostics need a 3D Navier-Stokes mesh");
    if (m.curved)
        return fail(ctx, SDRT_ERR_UNSUPPORTED, "the Taylor-Green diagnostics take affine elements (one det J each)");
    if ((r = ensure_workspace(ctx, m, false, false))) return r;
    if ((r = rk54_workspace(ctx, m, false))) return r;
    const size_t es = m.phys.precision == SDRT_FP32 ? 4 : 8;
    if (!m.qsol.p) SDRT_CUDA(m.qsol.alloc((size_t)m.nd * m.state_len * es));
    if (!m.diag_sums.p) SDRT_CUDA(m.diag_sums.alloc(5 * sizeof(double)));
    double s[5];
    r = m.phys.precision == SDRT_FP32 ? tgv_diagnostics<float>(ctx, m, static_cast<const float*>(U), s)
                                       : tgv_diagnostics<double>(ctx, m, static_cast<const double*>(U), s);
    if (r) return r;
    const double scale = rho_inf * v_inf * v_inf, tc = length / v_inf, vol = s[0];
    out[0] = s[1] / vol / scale;                                   // <E*>
    out[1] = -tc * s[2] / vol / scale;                             // eps1 = -d<E*>/dt*
    out[2] = 2.0 * m.phys.mu * tc * s[3] / vol / scale;            // eps2
    out[3] = -tc * s[4] / vol / scale;                             // eps3
    return SDRT_OK;
}

int sdrt_set_option(sdrt_ctx* ctx, int option, int value) {
    if (!ctx) return SDRT_ERR_ARG;
    if (option == SDRT_OPT_TENSOR_CORES) ctx->use_tc = value != 0;
    else if (option == SDRT_OPT_TC_DIVERGENCE) ctx->use_tc_div = value != 0;
    else if (option == SDRT_OPT_FUSED_RK) ctx->fuse_rk = value != 0;
    else if (option == SDRT_OPT_GENERATED) ctx->use_gen = value < 0 ? 0 : value > 2 ? 2 : value;
    else if (option == SDRT_OPT_WAIT_POLLS) ctx->wait_polls = value < 0 ? 0 : value;
    else if (option == SDRT_OPT_NVTX) ctx->nvtx = value != 0;
    else if (option == SDRT_OPT_TC_GRADIENT) ctx->use_tc_grad = value != 0;
    else return fail(ctx, SDRT_ERR_ARG, "unknown option");
    for (auto& m : ctx->meshes)
        if (m && m->graph) {
            cudaGraphExecDestroy(m->graph);
            m->graph = nullptr;
        }
    return SDRT_OK;
}

int sdrt_profile_enable(sdrt_ctx* ctx, int enable) {
    if (!ctx) return SDRT_ERR_ARG;
    if (ctx->host_only) return fail(ctx, SDRT_ERR_STATE, "host-only context");
    ctx->prof = enable != 0;
    ctx->pending.clear();
    ctx->eager_next = 0;
    for (auto& m : ctx->meshes)
        if (m && m->graph) {
            cudaGraphExecDestroy(m->graph);
            m->graph = nullptr;
        }
    return SDRT_OK;
}

int sdrt_profile_collect_blocks(sdrt_ctx* ctx, int max_blocks, double* ms_out, int64_t* count_out) {
    if (!ctx || !ms_out || !count_out || max_blocks < 0) return SDRT_ERR_ARG;
    if (ctx->host_only) return fail(ctx, SDRT_ERR_STATE, "host-only context");
    SDRT_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int s : ctx->pending) {
        float t = 0;
        SDRT_CUDA(cudaEventElapsedTime(&t, ctx->ev[2 * s], ctx->ev[2 * s + 1]));
        const int kind = ctx->slot_kind[s] & 0xff;
        int row = ctx->slot_kind[s] >> 8;         // 0: launch over all blocks, b + 1: block b only
        if (row > max_blocks) row = 0;
        ms_out[row * KIND_COUNT + kind] += t;
        count_out[row * KIND_COUNT + kind] += 1;
    }
    ctx->pending.clear();
    ctx->eager_next = 0;
    return SDRT_OK;
}

int sdrt_profile_collect(sdrt_ctx* ctx, double* ms_out, int64_t* count_out) {
    if (!ctx || !ms_out || !count_out) return SDRT_ERR_ARG;
    if (ctx->host_only) return fail(ctx, SDRT_ERR_STATE, "host-only context");
    SDRT_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int s : ctx->pending) {
        float t = 0;
        SDRT_CUDA(cudaEventElapsedTime(&t, ctx->ev[2 * s], ctx->ev[2 * s + 1]));
        ms_out[ctx->slot_kind[s] & 0xff] += t;
        count_out[ctx->slot_kind[s] & 0xff] += 1;
    }
    ctx->pending.clear();
    ctx->eager_next = 0;
    return SDRT_OK;
}

int sdrt_rk4_step_host(sdrt_ctx* ctx, int mesh_id, const void* Uin, void* Uout, double dt, int nsteps) {
    NvtxScope nvtx_scope(ctx, "sdrt_rk4_step_host");
    int r = check_whole(ctx, mesh_id);
    if (r) return r;
    if (!Uin || !Uout) return fail(ctx, SDRT_ERR_ARG, "null host buffer");
    Mesh& m = *ctx->meshes[mesh_id];
    const size_t bytes = (size_t)m.state_len * (m.phys.precision == SDRT_FP32 ? 4 : 8);
    if (!m.uhost_dev.p) SDRT_CUDA(m.uhost_dev.alloc(bytes));
    SDRT_CUDA(cudaMemcpyAsync(m.uhost_dev.p, Uin, bytes, cudaMemcpyHostToDevice, ctx->stream));
    if ((r = sdrt_rk4_step(ctx, mesh_id, m.uhost_dev.p, dt, nsteps))) return r;
    SDRT_CUDA(cudaMemcpyAsync(Uout, m.uhost_dev.p, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    SDRT_CUDA(cudaStreamSynchronize(ctx->stream));
    return SDRT_OK;
}

int sdrt_jvp(sdrt_ctx* ctx, int mesh_id, const void* U, const void* V, void* JV) {
    NvtxScope nvtx_scope(ctx, "sdrt_jvp");
    int r = check_whole(ctx, mesh_id);
    if (r) return r;
    if (!U || !V || !JV || JV == U || JV == V) return fail(ctx, SDRT_ERR_ARG, "bad device arrays");
    Mesh& m = *ctx->meshes[mesh_id];
    if ((r = ensure_workspace(ctx, m, true, false))) return r;
    if (m.phys.precision == SDRT_FP32) {
        KEpi<float> E{};
        E.mode = EPI_STORE;
        E.out = static_cast<float*>(JV);
        E.flag = ctx->flag.as<int>();
        return run_residual<float>(ctx, m, static_cast<const float*>(U), static_cast<const float*>(V), E);
    }
    KEpi<double> E{};
    E.mode = EPI_STORE;
    E.out = static_cast<double*>(JV);
    E.flag = ctx->flag.as<int>();
    return run_residual<double>(ctx, m, static_cast<const double*>(U), static_cast<const double*>(V), E);
}

int sdrt_vjp(sdrt_ctx* ctx, int mesh_id, const void* U, const void* W, void* JTW) {
    NvtxScope nvtx_scope(ctx, "sdrt_vjp");
    int r = check_whole(ctx, mesh_id);
    if (r) return r;
    if (!U || !W || !JTW || JTW == U || JTW == W) return fail(ctx, SDRT_ERR_ARG, "bad device arrays");
    Mesh& m = *ctx->meshes[mesh_id];
    if ((r = ensure_workspace(ctx, m, true, false))) return r;
    if (viscous(m) && !m.cbar.p)
        SDRT_CUDA(m.cbar.alloc((size_t)m.nvar * m.Ftot * (m.phys.precision == SDRT_FP32 ? 4 : 8)));
    if (m.phys.precision == SDRT_FP32)
        return run_vjp<float>(ctx, m, static_cast<const float*>(U), static_cast<const float*>(W),
                              static_cast<float*>(JTW));
    return run_vjp<double>(ctx, m, static_cast<const double*>(U), static_cast<const double*>(W),
                           static_cast<double*>(JTW));
}

int sdrt_autotune(sdrt_ctx* ctx, int mesh_id, const void* U, int reps) {
    NvtxScope nvtx_scope(ctx, "sdrt_autotune");
    int r = check_whole(ctx, mesh_id);
    if (r) return r;
    if (!U || reps < 1) return fail(ctx, SDRT_ERR_ARG, "null state or reps < 1");
    Mesh& m = *ctx->meshes[mesh_id];
    if (m.fast) return SDRT_OK;                 // the record-path kernels have fixed tiles
    // The operator-specialised kernels have fixed tiles too: on their meshes
    // the generic kernels' tiles are tuned with those kernels switched off
    // (they run with SDRT_OPT_GENERATED = 0).
    if ((r = ensure_workspace(ctx, m, false, false))) return r;
    const size_t es = m.phys.precision == SDRT_FP32 ? 4 : 8;
    DevBuf R;
    SDRT_CUDA(R.alloc((size_t)m.state_len * es));
    cudaEvent_t a, b;
    SDRT_CUDA(cudaEventCreate(&a));
    SDRT_CUDA(cudaEventCreate(&b));
    const bool prof = ctx->prof;
    ctx->prof = false;
    const int use_gen = ctx->use_gen;
    ctx->use_gen = 0;
    // Time `reps` residual evaluations of the whole mesh (ms per evaluation).
    auto timed = [&](float* ms) -> int {
        int rr;
        if ((rr = sdrt_residual(ctx, mesh_id, U, R.p))) return rr;    // warm-up (and attribute setup)
        SDRT_CUDA(cudaEventRecord(a, ctx->stream));
        for (int i = 0; i < reps; ++i)
            if ((rr = sdrt_residual(ctx, mesh_id, U, R.p))) return rr;
        SDRT_CUDA(cudaEventRecord(b, ctx->stream));
        SDRT_CUDA(cudaEventSynchronize(b));
        SDRT_CUDA(cudaEventElapsedTime(ms, a, b));
        *ms /= reps;
        return SDRT_OK;
    };
    const bool visc = viscous(m);
    int rc = SDRT_OK;
    // Coordinate descent over the blocks: residual tile, then (viscous) gradient tile.
    for (auto& bp : m.blocks) {
        const RefElement& RE = ctx->etypes[bp->etype]->R;
        const EType& et = *ctx->etypes[bp->etype];
        for (int which = 0; which < (visc ? 2 : 1) && rc == SDRT_OK; ++which) {
            int& tile = which == 0 ? bp->tile : bp->gtile;
            const int keep = tile;
            int best = keep;
            float best_ms = 1e30f;
            // multiples of 4 (16-byte tile rows); the non-powers of two balance the
            // tile GEMMs' 8 x 4 thread blocks over the CTA's threads for some shapes
            for (int te : {4, 8, 12, 16, 20, 24, 28, 32, 40, 48, 64}) {
                const size_t smem = which == 0
                                        ? (size_t)(std::max(RE.nsol, RE.nfi) + et.Mi) * m.nvar * te * es
                                        : (size_t)(RE.nsol + RE.nfe + m.nd * RE.nsol) * m.nvar * te * es;
                if (smem > 220 * 1024) continue;
                tile = te;
                if ((rc = refresh_tables(ctx, m))) break;
                float ms = 0;
                if ((rc = timed(&ms))) break;
                if (ms < best_ms) {
                    best_ms = ms;
                    best = te;
                }
            }
            tile = rc == SDRT_OK ? best : keep;
            if (int rt = refresh_tables(ctx, m)) rc = rc ? rc : rt;
        }
        if (rc) break;
    }
    ctx->prof = prof;
    ctx->use_gen = use_gen;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (m.graph) {
        cudaGraphExecDestroy(m.graph);
        m.graph = nullptr;
    }
    // Non-finite values of the tuning state are not the caller's concern.
    cudaStreamSynchronize(ctx->stream);
    cudaMemset(ctx->flag.p, 0, sizeof(int));
    return rc;
}

int sdrt_get_tiles(sdrt_ctx* ctx, int mesh_id, int block, int32_t* out) {
    int r = check_mesh(ctx, mesh_id);
    if (r) return r;
    const Mesh& m = *ctx->meshes[mesh_id];
    if (!out || block < 0 || block >= (int)m.blocks.size()) return fail(ctx, SDRT_ERR_ARG, "bad block or output");
    const MBlock& b = *m.blocks[block];
    const int32_t v[6] = {32, b.tile, b.tile_dual, b.gtile, b.gtile_dual, b.vtile};
    for (int i = 0; i < 6; ++i) out[i] = v[i];
    return SDRT_OK;
}

int sdrt_sync(sdrt_ctx* ctx) {
    if (!ctx) return SDRT_ERR_ARG;
    if (ctx->host_only) return SDRT_OK;
    SDRT_CUDA(cudaStreamSynchronize(ctx->stream));
    int h = 0;
    SDRT_CUDA(cudaMemcpy(&h, ctx->flag.p, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
        SDRT_CUDA(cudaMemset(ctx->flag.p, 0, sizeof(int)));
        if (h & 2) return fail(ctx, SDRT_ERR_TIMEOUT, "a kernel's bounded wait for its copies ran out");
        return fail(ctx, SDRT_ERR_NONFINITE, "a kernel produced a non-finite value");
    }
    return SDRT_OK;
}

int64_t sdrt_launch_count(const sdrt_ctx* ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"

// ---------------------------------------------------------------------------
// Internal hooks (internal.hpp) used by the allocation-free entry point.

namespace {

// The value-residual launches of run_residual, with the face states in `ufe`.
template <typename T>
int residual_into(sdrt_ctx* ctx, Mesh& m, const T* U, T* R, T* ufe) {
    const KPhys<T> P = make_phys<T>(m.phys);
    KEpi<T> E{};
    E.mode = EPI_STORE;
    E.out = R;
    E.flag = ctx->flag.as<int>();
    const KSet<T> ks = kset<T>(m);
    launch_interp_ext<T>(ks, m.nvar, U, ufe, m.Ftot, ctx->nsm, ctx->stream);
    ++ctx->launches;
    int r = launch_residual<T>(ks, m.phys.system, m.phys.riemann, m.nd, U, nullptr, ufe, nullptr, m.Ftot, P, E,
                               KVisc<T>{}, ctx->nsm, ctx->stream);
    if (r != 0) return fail(ctx, SDRT_ERR_UNSUPPORTED, "system / flux combination not supported");
    ++ctx->launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(ctx, SDRT_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return SDRT_OK;
}

}  // namespace

namespace sdrt {

int internal_device(const sdrt_ctx* ctx) { return (!ctx || ctx->host_only) ? -1 : ctx->device; }

int internal_fail(sdrt_ctx* ctx, int code, const char* msg) { return fail(ctx, code, msg); }

void* internal_noalloc_scratch(const sdrt_ctx* ctx) { return ctx->noalloc_scratch; }

int internal_residual_with_scratch(sdrt_ctx* ctx, int mesh_id, const void* U, void* R, void* scratch,
                                   size_t scratch_bytes) {
    int r = check_whole(ctx, mesh_id);
    if (r) return r;
    if (!U || !R || U == R || !scratch) return fail(ctx, SDRT_ERR_ARG, "U and R must be distinct device arrays");
    Mesh& m = *ctx->meshes[mesh_id];
    if (viscous(m))
        return fail(ctx, SDRT_ERR_UNSUPPORTED, "the allocation-free entry point covers the inviscid systems only");
    const size_t es = m.phys.precision == SDRT_FP32 ? 4 : 8;
    const size_t need = (size_t)m.nvar * (size_t)m.Ftot * es;
    if (need > scratch_bytes)
        return fail(ctx, SDRT_ERR_UNSUPPORTED,
                    "mesh needs " + std::to_string(need) + " bytes of face-state scratch, more than the " +
                        std::to_string(scratch_bytes) + "-byte static buffer of the allocation-free entry point");
    if (m.phys.precision == SDRT_FP32)
        return residual_into<float>(ctx, m, static_cast<const float*>(U), static_cast<float*>(R),
                                    static_cast<float*>(scratch));
    return residual_into<double>(ctx, m, static_cast<const double*>(U), static_cast<double*>(R),
                                 static_cast<double*>(scratch));
}

}  // namespace sdrt
