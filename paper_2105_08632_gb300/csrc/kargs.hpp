// Argument blocks shared by the host launch code and the CUDA kernels.
#pragma once

#include <cstdint>

namespace sdrt {

enum System { SYS_ADVECTION = 0, SYS_ADVDIFF = 1, SYS_EULER = 2, SYS_NS = 3 };
enum Riemann { RIE_UPWIND = 0, RIE_RUSANOV = 1, RIE_ROE = 2 };

// Per-block device data of one mesh block (element type + its elements).
//
// State arrays: value (rho, v, e) of the block at u_off + (rho * V + v) * ld + e.
// External-point arrays ("face states", UFE): value (sigma, v, e) at
//   v * F_tot + fe_base + sigma * ld + e   (F_tot = sum of nfe * ld over blocks).
// Metric rows (k, e) at metric[k * ld + e] hold, at the points where the
// method evaluates them (paper Sec. 2.1):
//   1 / det J at each solution point,
//   S_di = det J * (J^{-1})_di = det J dx~_d / dx_i at each solution point
//        (physical gradients) and each unique internal flux point (fluxes),
//   the unit normal n_L of the face's L side (c < ND) and the signed scale
//        s = +-det J |J^{-T} n~| (+ on the L side) at each external point.
// Affine elements have one value of each per element (rows: 1/det J at 0,
// S_di at 1 + d * ND + i, face f at 1 + ND^2 + f (ND + 1) + c), curved ones
// one per point; the row of each quantity is given by the mr_* fields.
template <typename T>
struct KBlock {
    int nsol, nfe, nfi, nfiu, nfaces;
    int nelem, ld;
    int64_t u_off;       // element offset of the block in a state array
    int64_t fe_base;     // offset of the block's first external point in UFE
    const T* Ai;         // interpolation operator, transposed: [nsol][Mi_pad], rows [M0; M12]
    int Mi, Mi_pad;      // Mi = nfe + nfiu
    const T* Ad;         // divergence operator, transposed: [nfe + nfi][Md_pad], columns [M14 | M13]
    int Md_pad;
    const T* Adt;        // VJP: [M14 | M13] row-major: [nsol][Mdt_pad], M13 from column round_up(nfe, 8)
    int Mdt_pad;
    const T* Ag;         // viscous: [M16 | M15 P M12] transposed: [nfe + nsol][Mg_pad], columns (d, rho)
    int Mg_pad;          // ND * nsol rounded up to 8
    const T* Agr;        // viscous VJP: [M16 | M15 P M12] row-major with rows (rho, d): [ND * nsol][Agr_pad]
    int Agr_pad;         // nfe + nsol rounded up to 8
    int64_t qfiu_off;    // viscous: element offset of the block in QFIU
    const int* fe_face;  // [nfe] local face of each external point
    const int* fi_tab;   // [nfiu][4]: count, then (nu | axis << 16) per internal DOF of the point
    const T* metric;     // [NM][ld]
    // Metric row addressing (affine: strides 0, curved: one row set per point):
    int mr_inv;          // 1/det J at solution point s: row s * mr_inv
    int mr_ss, mr_ssk;   // S_di at solution point s: row mr_ss + s * mr_ssk + d * ND + i
    int mr_si, mr_sik;   // S_di at unique internal point k: row mr_si + k * mr_sik + d * ND + i
    int mr_f, mr_ff, mr_fp;  // normal / scale of external point sigma on face f: mr_f + f * mr_ff + sigma * mr_fp + c
    const int* map;      // [nfe][ld] UFE index (without the v * F_tot term) of the paired point
    const T* Air;        // interpolation operator row-major: [Mir][Md_pad], rows [M0; M12], Mir = Mi rounded to 4
    int Mir;
    // Record layout of the register-blocked path (kernels_fast.cu): every
    // element owns one contiguous record of its external-point states, face by
    // face (face f at frecoff[f], point l of the face at + l * V, variable v at
    // + v), and one record of its internal-point states (point k at k * V + v).
    // Strides are multiples of 4 values (16-byte aligned bulk copies) and odd
    // multiples of 4 where possible (conflict-free shared-memory rows).
    int ers;             // element record stride in REC (values)
    int frs;             // internal-point record stride in FIUR (values)
    int frec;            // face record size (values): points per face * V rounded up to 4
    int nmp;             // metric record stride in MAOS (values)
    int pstride;         // permutation row stride (bytes)
    int64_t rec_base;    // offset of element 0's record in REC
    int64_t fiur_base;   // offset of element 0's record in FIUR
    const T* maos;       // [nelem][nmp] metric rows (same content as `metric`)
    const int* pfr;      // [nelem][nfaces] REC offset of the partner's face record
    const unsigned char* perm;  // [nelem][pstride] local index, in the partner's face record, of each external point
    const int* recoff;   // [nfe] offset of external point j in the element record
    // Tile widths (elements per tile) of the generic kernels for this block.
    int te_interp, te_res, te_res_dual, te_grad, te_grad_dual, te_vjp;
};

// The blocks of a mesh as one work table for the generic kernels: global tile
// g belongs to the first block b whose tile count (ceil(nelem / TE_b), TE_b
// the kernel's tile width) exceeds g minus the tiles of the blocks before it.
// One launch walks the tiles of every block (blocks: device array).
template <typename T>
struct KTable {
    const KBlock<T>* blocks;
    int nblocks;
};

// Which tile width a generic kernel uses.
enum TileKind { TK_INTERP = 0, TK_RES = 1, TK_RES_DUAL = 2, TK_GRAD = 3, TK_GRAD_DUAL = 4, TK_VJP = 5 };

template <typename T>
__host__ __device__ inline int tile_width(const KBlock<T>& B, int kind) {
    switch (kind) {
        case TK_INTERP: return B.te_interp;
        case TK_RES: return B.te_res;
        case TK_RES_DUAL: return B.te_res_dual;
        case TK_GRAD: return B.te_grad;
        case TK_GRAD_DUAL: return B.te_grad_dual;
        default: return B.te_vjp;
    }
}

// Physical gradients of the viscous systems at the flux points.
//   QFE  [ND][V][F_tot]: gradient at external points (UFE indexing), component d
//        of variable v at (d * V + v) * F_tot + fe_base + sigma * ld + e;
//   QFIU per block: (k, d, v, e) at qfiu_off + ((k * ND + d) * V + v) * ld + e.
// d-prefixed arrays: tangents (JVP).
template <typename T>
struct KVisc {
    const T* qfe;
    const T* dqfe;
    const T* qfiu;
    const T* dqfiu;
};

template <typename T>
struct KPhys {
    T a[3];
    T gamma, mu, prandtl, beta, eta;
};

// Stage update fused into the divergence epilogue (R = dU/dt of the tile):
//   EPI_STORE  out = R
//   EPI_RK_FIRST   uacc = u0 + cacc R ; unext = u0 + cnext R
//   EPI_RK_MID     uacc = uacc + cacc R ; unext = u0 + cnext R
//   EPI_RK_LAST    out = uacc + cacc R
enum EpiMode { EPI_STORE = 0, EPI_RK_FIRST = 1, EPI_RK_MID = 2, EPI_RK_LAST = 3 };

template <typename T>
struct KEpi {
    int mode;
    T* out;
    const T* u0;
    T* uacc;
    T* unext;
    T cacc, cnext;
    int* flag;           // bit 0: a non-finite value was produced; bit 1: a bounded wait ran out
    int wait_polls;      // record flux kernel: polls of its first copy wait (0: the normal bound)
    // Non-null (record path, stages 1-3 of RK4): the next stage's state
    // u0 + cnext R is not stored but interpolated right away into these record
    // buffers (the layouts of REC and FIUR).
    T* rec_next;
    T* fiur_next;
};

}  // namespace sdrt
