/*
 * sdrt.h -- C ABI of the GB300 (sm_103a) Spectral Difference Raviart-Thomas
 * residual library (arXiv 2105.08632).
 *
 * The library evaluates the SDRT semi-discrete residual dU/dt = R(U) (paper
 * Sec. 2.1, Eqs. "interpolate_sol_to_flux" .. "divergence_sdrt" and the
 * semi-discrete form after it; matrix form App. B, Eq. "residual_sdrt_matrices")
 * for meshes of triangles, quadrilaterals, tetrahedra, prisms and hexahedra,
 * classical RK4 steps of it, and its Jacobian-vector / vector-Jacobian products.
 *
 * Conventions shared by every entry point
 *  - Return value: SDRT_OK (0) or a negative sdrt_status.  The message of the
 *    last failure of a context is available from sdrt_last_error().
 *  - Device calls are asynchronous and ordered on the context's CUDA stream.
 *    Argument / state errors are reported immediately; kernel launch errors
 *    are returned by the call that launched; the non-finite flag raised by a
 *    kernel, and the timeout flag of a bounded device wait, are reported by
 *    sdrt_sync().
 *  - Pointers named *_dev are device pointers owned by the caller; *_host are
 *    host pointers owned by the caller.  The library never frees caller memory.
 *  - State layout: the state of a mesh is one array holding its blocks one
 *    after the other.  Block b starts at element offset `offset` (see
 *    sdrt_block_layout) and stores value (rho, v, e) -- solution point rho,
 *    variable v, element e -- at offset + (rho * nvar + v) * ld + e, where
 *    ld >= nelem is a multiple of 32 (the paper's state matrix, App. B Eq.
 *    "state_matrices", with the element index fastest).  Padding entries
 *    (nelem <= e < ld) are never read as data and never written.
 *    The element type is double (SDRT_FP64) or float (SDRT_FP32, SDRT_TF32X3).
 *  - Ordering of solution / flux points and local faces: see sdrt_point_order
 *    in the package documentation; it is the same convention as the mesh
 *    faces' local numbering documented at sdrt_face.
 */
#ifndef SDRT_H
#define SDRT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdrt_ctx sdrt_ctx;

typedef enum {
    SDRT_OK = 0,
    SDRT_ERR_ARG = -1,          /* invalid argument (null pointer, bad id, size mismatch) */
    SDRT_ERR_UNSUPPORTED = -2,  /* valid request outside the implemented set */
    SDRT_ERR_CUDA = -3,         /* a CUDA runtime call failed */
    SDRT_ERR_STATE = -4,        /* call out of order (e.g. mesh used before setup) */
    SDRT_ERR_NONFINITE = -5,    /* a kernel produced NaN / Inf (reported by sdrt_sync) */
    SDRT_ERR_TIMEOUT = -6,      /* a bounded device wait gave up */
    SDRT_ERR_MESH = -7          /* faces do not match / inverted or non-affine element */
} sdrt_status;

typedef enum { SDRT_TRI = 0, SDRT_QUAD = 1, SDRT_TET = 2, SDRT_PRI = 3, SDRT_HEX = 4 } sdrt_shape;
typedef enum { SDRT_ADVECTION = 0, SDRT_ADVDIFF = 1, SDRT_EULER = 2, SDRT_NAVIER_STOKES = 3 } sdrt_system;
typedef enum { SDRT_UPWIND = 0, SDRT_RUSANOV = 1, SDRT_ROE = 2 } sdrt_riemann;
/* Arithmetic of a mesh.  SDRT_TF32X3: FP32 states and the FP32 accuracy
 * class, with the dense contractions of the record path (FP32 Euler /
 * Rusanov tetrahedra of degree 3: the interpolation [M0; M12] U and the
 * divergence [M14 | M13] F~) on the tensor cores, each product split into
 * three TF32 products (hi hi + hi lo + lo hi) with FP32 accumulation
 * (tcgen05); everything else runs the FP32 kernels.  It meets the same
 * bounds as SDRT_FP32.  Plain TF32 (10-bit mantissa, ~5e-4 relative per
 * product) would not, and is not offered. */
typedef enum { SDRT_FP64 = 0, SDRT_FP32 = 1, SDRT_TF32X3 = 2 } sdrt_precision;

/* Element type: reference element and degree p (paper App. A). */
typedef struct {
    int32_t shape;   /* sdrt_shape */
    int32_t degree;  /* p >= 1; p <= 4 validated (simplices are unstable for p >= 5, Sec. 3.1.1) */
    int32_t scheme;  /* SDRT_SCHEME_SDRT (0) or SDRT_SCHEME_FR (1) */
} sdrt_etype_desc;

/* Schemes of an element type.
 *   SDRT_SCHEME_SDRT: the spectral difference Raviart-Thomas residual (Sec. 2.1).
 *   SDRT_SCHEME_FR:   FR-SDRT (Sec. 2.3, Eq. "divergence_fr" with the correction
 *     field's divergence taken from the RT external-point functions): the
 *     transformed flux at the solution points, differentiated there, plus
 *     M14 (F~_fe - (M0 f~) . n~).  It runs on the same kernels as SDRT with the
 *     internal DOFs at the solution points ((r, d) for solution point r and axis
 *     d; M12 = I) and the divergence operator M13_FR[s, (r, d)] = (M15 P M12)[(d, s), r],
 *     which the identities D = M16 M0 + M15 P M12 (exact reference gradient of
 *     the solution space) and M16[(d, s), j] = n~_jd M14[s, j] turn the FR
 *     correction into; the viscous gradient operator is the same as SDRT's.
 *     Generic kernels only (no record path). */
#define SDRT_SCHEME_SDRT 0
#define SDRT_SCHEME_FR 1

/* Counts of one element type (paper App. A, Tables "nsolpts_nfpts", "nfpts_extra"). */
typedef struct {
    int32_t ndim, nsol, nfe, nfi, nfiu, nfaces;
} sdrt_etype_info;

/* Physics of a mesh.  Fluxes (Sec. 2.1, 3, 5): advection f = a u; advection-
 * diffusion f = a u - mu grad u; Euler; Navier-Stokes with dynamic viscosity
 * mu, Prandtl number, ratio of specific heats gamma.  Common fluxes: upwind
 * (Eq. "flux_advection"), Rusanov (wave speed max(|v.n|+c) per side), Roe;
 * viscous terms use the LDG common value / flux with parameters beta, eta
 * (Eq. "common_var_for_grad" and the common viscous flux of Sec. 2.1). */
typedef struct {
    int32_t system;      /* sdrt_system */
    int32_t riemann;     /* sdrt_riemann */
    int32_t precision;   /* sdrt_precision of the state arrays */
    int32_t ndim;        /* 2 or 3, must match every block's element type */
    double a[3];         /* advection velocity */
    double mu, gamma, prandtl, beta, eta;
} sdrt_physics;

/* One block of elements of a single type.  verts: host, FP64,
 * nelem x nvert x ndim, vertices in the reference order of the type:
 *   tri (-1,-1),(1,-1),(-1,1); quad (-1,-1),(1,-1),(1,1),(-1,1);
 *   tet (-1,-1,-1),(1,-1,-1),(-1,1,-1),(-1,-1,1);
 *   pri tri x {-1} then tri x {+1}; hex quad x {-1} then quad x {+1}.
 * With sdrt_setup_mesh the elements must be affine images of the reference
 * element (else SDRT_ERR_UNSUPPORTED); curved elements are set up with
 * sdrt_setup_mesh_curved.  Copied at setup. */
typedef struct {
    int32_t etype;
    int32_t nelem;
    const double* verts;
} sdrt_block;

/* A glued pair of faces.  Local face numbering (vertex subsets):
 *   tri  e0 (0,1) e1 (1,2) e2 (2,0)      quad e0 (0,1) e1 (1,2) e2 (3,2) e3 (0,3)
 *   tet  f0 (0,1,2) f1 (0,1,3) f2 (1,2,3) f3 (0,2,3)
 *   pri  f0 (0,1,2) f1 (0,1,4,3) f2 (1,2,5,4) f3 (0,2,5,3) f4 (3,4,5)
 *   hex  f0 (0,1,2,3) f1 (0,1,5,4) f2 (1,2,6,5) f3 (3,2,6,7) f4 (0,3,7,4) f5 (4,5,6,7)
 * The first element is the face's L side: the common value and common flux
 * of the face are evaluated once with (u_L, u_R, n_L).  shift: x_L = x_R + shift
 * for coincident points (periodic faces). */
typedef struct {
    int32_t blk_l, elem_l, face_l;
    int32_t blk_r, elem_r, face_r;
    double shift[3];
} sdrt_face;

typedef struct {
    int32_t nvar, nblocks, ndim, precision;
    int64_t state_len;   /* length of a state array in elements (with padding) */
    int64_t ndof;        /* sum over blocks of nsol * nvar * nelem */
    int64_t nfe_total;   /* number of external flux points of the mesh */
    int32_t path;        /* kernels of the residual and RK4 steps: SDRT_PATH_* */
    int32_t curved;      /* 1 if some block has curved elements (sdrt_setup_mesh_curved) */
} sdrt_mesh_info;
/* Kernel paths of a mesh (sdrt_mesh_info.path). */
#define SDRT_PATH_GENERIC 0      /* generic tile kernels, any element type / system */
#define SDRT_PATH_RECORD 1       /* register-blocked record kernels (tetrahedra of degree 3 / 4) */
#define SDRT_PATH_GENERATED 2    /* operator-specialised kernels (SDRT_OPT_GENERATED) */

typedef struct {
    int32_t etype, nsol, nvar, nelem, ld, nfe;
    int64_t offset;      /* element offset of the block in a state array */
} sdrt_block_layout;

/* Create a context on CUDA device `device` issuing work on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  The stream is borrowed:
 * it must outlive the context.  device = -1 creates a host-only context:
 * element types and meshes are built on the host (operators, metrics, face
 * maps can be queried) but every device computation returns SDRT_ERR_STATE.
 * A device context also looks up the address of sdrt_residual_noalloc's
 * static buffer, which takes its SDRT_NOALLOC_SCRATCH_BYTES of device memory
 * (once per device and process) if no earlier context did. */
int sdrt_create(sdrt_ctx** ctx, int device, void* cuda_stream);
/* Destroy a context and every device buffer it owns. NULL is ignored. */
void sdrt_destroy(sdrt_ctx* ctx);
/* Message of the last failure of ctx (static storage of the context). */
const char* sdrt_last_error(const sdrt_ctx* ctx);
/* Replace the stream of later calls (borrowed). */
int sdrt_set_stream(sdrt_ctx* ctx, void* cuda_stream);

/* Build one element type: point sets, Vandermonde inverses and the matrix
 * operators M0, M12, M13, M14, M15, M16 in FP64 on the host (paper Sec. 2.1
 * Vandermonde equations, App. A bases, App. B operators), then upload them.
 * Identical descriptors return the existing id. */
int sdrt_setup_element_type(sdrt_ctx* ctx, const sdrt_etype_desc* desc, int* etype_id);
int sdrt_get_etype_info(sdrt_ctx* ctx, int etype_id, sdrt_etype_info* out);

/* Export an FP64 operator of an element type to host memory, row-major.
 * which: 0 = M0 (nfe x nsol), 1 = M12 (nfiu x nsol), 2 = M13 (nsol x nfi),
 *        3 = M14 (nsol x nfe), 4 = M15 (ndim*nsol x nfi), 5 = M16 (ndim*nsol x nfe),
 *        6 = solution points (nsol x ndim), 7 = external flux points (nfe x ndim).
 * n must equal the operator's size. */
int sdrt_get_operator(sdrt_ctx* ctx, int etype_id, int which, double* host_out, int64_t n);

/* Build a mesh: affine metrics per element (Eqs. "mapping_jacobian",
 * "inverse_mapping_jacobian"), physical unit normals and det J |J^{-T} n~| at
 * external flux points, and the int32 map pairing every external flux point
 * with the coincident point of the glued face (matched by physical
 * coordinates after the periodic shift).  Every external face must be glued
 * exactly once (periodic / closed meshes).  Host inputs are copied. */
int sdrt_setup_mesh(sdrt_ctx* ctx, const sdrt_physics* phys, int nblocks, const sdrt_block* blocks,
                    int64_t nfaces, const sdrt_face* faces, int* mesh_id);

/* Build a mesh whose blocks may hold curved elements.  The paper maps every
 * element by a mapping function and evaluates its Jacobian, determinant and
 * inverse analytically (Sec. 2, Eqs. "mapping_function", "mapping_jacobian",
 * "inverse_mapping_jacobian", "transformed_quantities"); a curved element
 * here is the second-order Lagrange map x(x~) = sum_k X_k N_k(x~) of its
 * nodes.
 *   nodes[b] = NULL: block b is affine, as for sdrt_setup_mesh.
 *   nodes[b] != NULL: host FP64 array nelem x nnode x ndim of node positions.
 *     The nodes are the reference points whose coordinates all lie in
 *     {-1, 0, 1}, in lexicographic order with x~ fastest (tri 6, quad 9,
 *     tet 10, pri 18, hex 27 nodes; the vertices are among them), and N_k
 *     spans polynomials of total degree <= 2 (tri, tet), of degree <= 2 per
 *     coordinate (quad, hex), or their product (pri: triangle x z).
 *     blocks[b].verts is not read (may be NULL).  Glued faces must coincide
 *     point by point (conforming curved faces; periodic shifts as usual).
 * The metrics are evaluated in FP64 at every point where the method uses
 * them (Sec. 2.1): J^{-T} at the solution points (physical gradients),
 * det J J^{-1} at the internal flux points (Eq. "normal_transformed_flux"),
 * the unit normal and det J |J^{-T} n~| at the external flux points (the
 * transformed common flux; the L side's normal on both sides, each side's
 * own scale), 1 / det J at the solution points (the semi-discrete form), and
 * stored in the mesh precision.  A uniform state is preserved exactly when
 * the transformed flux space holds the cofactors det J J^{-1} (quadratic
 * polynomials; e.g. tetrahedra of degree >= 2, triangles of degree >= 1).
 * Meshes with curved blocks run on the generic kernels (residual, RK
 * steps, JVP, VJP, viscous systems); SDRT_ERR_UNSUPPORTED for the FR-SDRT
 * scheme on curved blocks; sdrt_tgv_diagnostics refuses them.
 * SDRT_ERR_MESH for a non-positive det J at any of those points.  Host
 * inputs are copied. */
int sdrt_setup_mesh_curved(sdrt_ctx* ctx, const sdrt_physics* phys, int nblocks, const sdrt_block* blocks,
                           const double* const* nodes, int64_t nfaces, const sdrt_face* faces, int* mesh_id);
int sdrt_get_mesh_info(sdrt_ctx* ctx, int mesh_id, sdrt_mesh_info* out);

/* One partition of a mesh whose residual is distributed over processes or
 * devices.  Elements couple only through the common flux at shared faces
 * (paper Sec. 2.1, Eq. "flux_advection" and the common fluxes), so a
 * partition needs, once per residual evaluation, the external-point states of
 * the faces it shares with other partitions, and nothing else.
 * blocks / faces as for sdrt_setup_mesh; ghost[b] = 1 marks blocks that hold
 * copies of OTHER partitions' elements sharing a face with this partition's
 * elements (their vertices pair the face points; their other faces stay
 * unglued; no residual is computed for them).  Ghost blocks come after the
 * owned ones; faces keep the L / R order of the whole mesh.  The state arrays
 * of the partition hold the owned blocks only.  Inviscid systems (advection,
 * Euler) and, with a second exchange of the face points' gradients, the
 * viscous ones; any element types: the record path (tetrahedra of degree 3 /
 * 4) exchanges whole face records of its record layout, the generic path the
 * face points' states gathered from its face-state array.  Whole-mesh calls (sdrt_residual,
 * sdrt_rk4_step, sdrt_jvp, sdrt_vjp, ...) return SDRT_ERR_STATE on a
 * partition.  Host inputs are copied. */
int sdrt_setup_partition(sdrt_ctx* ctx, const sdrt_physics* phys, int nblocks, const sdrt_block* blocks,
                         const uint8_t* ghost, int64_t nfaces, const sdrt_face* faces, int* mesh_id);

/* Exchange lists of a partition, host int32 triplets (block, element, local
 * face) in the numbering of sdrt_setup_partition: send[i] names the i-th
 * face record this partition packs (an owned element's face), recv[i] the
 * ghost face that the i-th received record fills.  Partition q's send list
 * towards p must list the faces in the order of p's receive list from q.
 * SDRT_ERR_ARG for a triplet outside the owned (send) or ghost (recv) blocks. */
int sdrt_set_exchange(sdrt_ctx* ctx, int mesh_id, int64_t nsend, const int32_t* send, int64_t nrecv,
                      const int32_t* recv);
/* Counts of the exchange lists (-1 before sdrt_set_exchange) and the values per
 * face record (points per face x nvar, padded to a multiple of 4; on meshes whose
 * faces differ in point count, sized for the largest face, the rest zero) and per
 * gradient record of the viscous systems (points per face x ndim x nvar, padded
 * the same way; 0 for the inviscid ones).  Null outputs are skipped. */
int sdrt_get_exchange_info(sdrt_ctx* ctx, int mesh_id, int64_t* nsend, int64_t* nrecv, int32_t* face_record,
                           int32_t* grad_record);

/* Partitioned residual, first half: interpolation of the owned blocks to
 * their flux points (Eq. "interpolation_procedure"), then the send buffer
 * send_dev (device, nsend x face_record values, caller owned) packed in the
 * order of the send list.  Asynchronous on the context's stream. */
int sdrt_residual_begin(sdrt_ctx* ctx, int mesh_id, const void* U_dev, void* send_dev);
/* Viscous systems (advection-diffusion, Navier-Stokes; generic path): the
 * gradient needs the common value at the faces (Sec. 2.1, LDG), so the
 * partitioned residual takes a second exchange.  After the face states have
 * moved: recv_dev (nrecv x face_record) fills the ghost faces, the flux-point
 * gradients of the owned elements follow (q~ = M16 C + M15 P M12 U, q = J^-T q~),
 * and send_grad_dev (nsend x grad_record values, the face points' gradients,
 * component d * nvar + v) is packed.  sdrt_residual_end then takes the received
 * gradient records.  SDRT_ERR_STATE on an inviscid partition or before begin. */
int sdrt_residual_gradients(sdrt_ctx* ctx, int mesh_id, const void* recv_dev, void* send_grad_dev);
/* Second half, after the caller has moved every partition's send buffer
 * segments into the receive buffers (NCCL, device copies, ...): recv_dev
 * (device, nrecv x face_record values) fills the ghost faces, then the common
 * and internal fluxes and the divergence of the owned blocks give R_dev =
 * dU/dt (owned state layout).  Same values as sdrt_residual on the whole
 * mesh, element by element.  The generic path reads the state passed to
 * sdrt_residual_begin again here: it must stay valid and unchanged in between.
 * Viscous systems: recv_dev holds the gradient records (nrecv x grad_record)
 * of the exchange after sdrt_residual_gradients. */
int sdrt_residual_end(sdrt_ctx* ctx, int mesh_id, const void* recv_dev, void* R_dev);
int sdrt_get_block_layout(sdrt_ctx* ctx, int mesh_id, int block, sdrt_block_layout* out);

/* Physical coordinates of the solution points, host FP64, blocks in order,
 * each block nelem x nsol x ndim (no padding). n = total length. */
int sdrt_get_sol_points(sdrt_ctx* ctx, int mesh_id, double* host_out, int64_t n);

/* Face map in canonical numbering g = base[b] + e * nfe[b] + sigma (no padding;
 * base = running sum of nelem * nfe): partner_out[g] = canonical index of the
 * paired point, is_left_out[g] = 1 on the L side of the face.  n = nfe_total.
 * Bit-exact contract of the mesh setup. */
int sdrt_get_face_map(sdrt_ctx* ctx, int mesh_id, int32_t* partner_out, uint8_t* is_left_out, int64_t n);

/* R = dU/dt for the whole mesh.  U_dev, R_dev: device state arrays (layout
 * above, precision of the mesh); may not alias. */
int sdrt_residual(sdrt_ctx* ctx, int mesh_id, const void* U_dev, void* R_dev);

/* Size in bytes of the fixed face-state buffer used by sdrt_residual_noalloc. */
#define SDRT_NOALLOC_SCRATCH_BYTES (32u << 20)

/* The residual of sdrt_residual, for callers that cannot allocate device
 * memory (for example a solver running as a plugin inside a framework whose
 * memory pool owns the whole device, or a time-critical loop that cannot take
 * cudaMalloc's implicit device synchronisation).  The paper has no
 * counterpart: this is a property of the library, not of the method.
 *  - Allocates nothing: the face states exchanged between elements go to a
 *    fixed SDRT_NOALLOC_SCRATCH_BYTES buffer that is part of the library image
 *    (a file-scope __device__ array).  Its device memory is taken when a
 *    context is created on a device (sdrt_create looks up the buffer's
 *    address, which loads the code module holding it) and held until process
 *    exit; the address is kept per context, so a context created after a
 *    device reset looks it up again.  The caller passes U_dev and R_dev as
 *    for sdrt_residual.
 *  - Kernel code: the CUDA runtime loads a kernel's code at its first launch
 *    (lazy loading, the default); a caller that must see no change of free
 *    device memory during its loop makes one call (or one sdrt_residual of
 *    the same mesh) during set-up.
 *  - Runs the generic kernels (interpolation to the external points, then the
 *    residual kernel) for every mesh, so on meshes that sdrt_residual runs on
 *    the record path (FP32 Euler / advection tetrahedra of degree 3 or 4) the
 *    two results agree to FP32 rounding, not bit for bit.
 *  - Inviscid systems only (advection, Euler): the viscous systems need
 *    flux-point gradients that do not fit a fixed buffer of this size;
 *    they return SDRT_ERR_UNSUPPORTED.
 *  - The mesh must need at most SDRT_NOALLOC_SCRATCH_BYTES of face states
 *    (nvar * external flux points (rows padded to 32 elements) * 4 or 8
 *    bytes); larger meshes are rejected with SDRT_ERR_UNSUPPORTED and a
 *    message giving both sizes.  Example: Euler on 40,000 tetrahedra of degree
 *    3 in FP32 needs 40,000 x 40 points x 5 x 4 B = 32,000,000 B and fits
 *    (limit 33,554,432 B).
 *  - All calls share the one buffer: calls whose kernels can overlap on the
 *    GPU (different streams, other contexts) race and give wrong results;
 *    serialise them.  Nothing needs clearing between calls: each call writes
 *    every entry it reads. */
int sdrt_residual_noalloc(sdrt_ctx* ctx, int mesh_id, const void* U_dev, void* R_dev);

/* nsteps classical RK4 steps of size dt, in place on U_dev (device).  Each
 * stage is one residual evaluation fused with its stage update (paper Sec. 2.1
 * explicit RK; RK4 stability polynomial Eq. "rk_exponential").  With
 * SDRT_OPT_FUSED_RK on (default) and an FP32 Euler mesh of degree-3
 * tetrahedra, stages 1-3 also interpolate the next stage's state to the flux
 * points in their epilogue, so one step is one interpolation and four flux
 * kernels and the stage states stay on chip. */
int sdrt_rk4_step(sdrt_ctx* ctx, int mesh_id, void* U_dev, double dt, int nsteps);

/* nsteps RK54 steps of size dt, in place on U_dev (device): the five-stage
 * fourth-order two-register scheme of Carpenter & Kennedy (1994) that the
 * paper cites for its Taylor-Green runs (Sec. 5.3; its stability polynomial
 * is Eq. "rk_exponential"), published coefficients.  Each stage is one
 * residual evaluation and an update of the two registers
 * dU <- A_i dU + dt R(U), U <- U + B_i dU.  Uses mesh workspaces (allocated
 * on first use). */
int sdrt_rk54_step(sdrt_ctx* ctx, int mesh_id, void* U_dev, double dt, int nsteps);

/* One adaptive RK54 step attempt of size dt with the embedded third-order
 * estimate (U - U^ = sum_j n_j k_j over the stage slopes, n the unit null
 * vector of the order <= 3 conditions) and a PI step-size controller (the
 * paper pairs RK54 with one, Sec. 5.3, citing Butcher; it prints neither the
 * estimator nor the gains):
 *   err = max |U - U^| / (atol + rtol max(|U_start|, |U|))   (L-infinity, as
 *         in the paper's runs);
 *   accepted (err <= 1): U holds the new state, dt_next = dt * clip(0.9
 *         err^(-0.7/4) err_prev^(0.4/4), 0.2, 5), err_prev <- err (kept per mesh,
 *         initially 1);
 *   rejected: U is restored, dt_next = dt * clip(0.9 err^(-0.7/4), 0.2, 5).
 * Synchronises the stream (the error norm is read on the host). */
int sdrt_rk54_adaptive_step(sdrt_ctx* ctx, int mesh_id, void* U_dev, double dt, double atol, double rtol,
                            double* err, double* dt_next, int* accepted);

/* Adaptive RK54 over a time span t_span from the step size *dt_inout (the
 * last step is shortened to end exactly at t_span); *dt_inout returns the
 * controller's next step size.  SDRT_ERR_STATE after max_steps attempts. */
int sdrt_rk54_integrate(sdrt_ctx* ctx, int mesh_id, void* U_dev, double t_span, double* dt_inout, double atol,
                        double rtol, int max_steps, int* n_accepted, int* n_rejected);

/* Taylor-Green vortex diagnostics of the state U_dev (paper Sec. 5.3; 3D
 * Navier-Stokes meshes), ensemble averages <.> = (1/|Omega|) int_Omega . with
 * an element quadrature exact for degree 10 (7 Gauss-Legendre points per
 * direction, collapsed on simplices), velocity gradients from the LDG
 * gradients of the scheme (Sec. 2.1), t_c = length / v_inf:
 *   out[0] = <E*>, E* = (1/2) rho v.v / (rho_inf v_inf^2);
 *   out[1] = eps1 = -d<E*>/dt*, from the residual: -t_c <v . R_m - |v|^2 R_rho / 2>
 *            / (rho_inf v_inf^2);
 *   out[2] = eps2 = 2 mu t_c <S^d : S^d> / (rho_inf v_inf^2);
 *   out[3] = eps3 = -t_c <p div v> / (rho_inf v_inf^2).
 * eps1 - eps2 - eps3 estimates the numerical dissipation.  Synchronises the
 * stream. */
int sdrt_tgv_diagnostics(sdrt_ctx* ctx, int mesh_id, const void* U_dev, double rho_inf, double v_inf, double length,
                         double* out4);

/* Same as sdrt_rk4_step with host buffers: copies U_in_host to the device,
 * steps, copies the result to U_out_host and synchronises the stream.
 * U_in_host / U_out_host: state_len values (may be the same buffer; pinned
 * memory gives the fastest copies). */
int sdrt_rk4_step_host(sdrt_ctx* ctx, int mesh_id, const void* U_in_host, void* U_out_host,
                       double dt, int nsteps);

/* Jacobian-vector product JV = (dR/dU)(U) . V (device arrays, state layout).
 * At ties of |.| and max() the derivative of the first / non-negative branch
 * is taken. */
int sdrt_jvp(sdrt_ctx* ctx, int mesh_id, const void* U_dev, const void* V_dev, void* JV_dev);

/* Vector-Jacobian product JTW = (dR/dU)(U)^T . W (device arrays, state
 * layout; the adjoint of the discrete operator of Sec. 2.1 / App. B, which the
 * paper does not spell out: W is carried back through the divergence
 * [M14 | M13]^T, the transposed Jacobians of the common and internal fluxes,
 * and the interpolation [M0; M12]^T).  Viscous systems (advection-diffusion,
 * Navier-Stokes: LDG, Sec. 2.1) also carry W back through the flux-point
 * gradients: [M0; M12]^T at the solution points, J^{-1}, [M16 | M15 P M12]^T,
 * and the common value C(u_L, u_R) of the two sides of each face.  Same branch
 * convention at ties as sdrt_jvp, so <W, J V> = <J^T W, V> up to rounding.
 * Uses the mesh's face-state and gradient buffers (allocated on first use). */
int sdrt_vjp(sdrt_ctx* ctx, int mesh_id, const void* U_dev, const void* W_dev, void* JTW_dev);

/* Tile autotuner of the generic kernels (every element type other than the
 * register-blocked tetrahedra of degree 3 and 4, which have fixed tiles): for
 * each block in turn, times `reps` residual evaluations of the whole mesh at
 * U_dev (device state, not modified) for tile widths of 4, 8, 12, 16, 20, 24,
 * 28, 32, 40, 48 and 64 elements (multiples of 4: 16-byte tile rows) that
 * fit in shared memory, and keeps the fastest (the residual kernel's tile,
 * and for the viscous systems the gradient kernel's).  Results are bit-for-bit
 * the same for every tile width (tiles only partition the elements).  Drops
 * the mesh's captured RK4 graph.  Synchronises the stream; allocates a
 * temporary residual array. */
int sdrt_autotune(sdrt_ctx* ctx, int mesh_id, const void* U_dev, int reps);

/* Tile widths (elements per CTA tile) of one block's generic kernels:
 * out[6] = {interpolation, residual, residual JVP, gradient, gradient JVP,
 * VJP}; 0 = not available for this block. */
int sdrt_get_tiles(sdrt_ctx* ctx, int mesh_id, int block, int32_t* out);

/* Synchronise the context's stream; returns SDRT_ERR_TIMEOUT if a kernel's
 * bounded wait for its asynchronous copies ran out, else SDRT_ERR_NONFINITE if
 * a kernel wrote NaN / Inf into a residual, since the last sync (and clears
 * the flags). */
int sdrt_sync(sdrt_ctx* ctx);

/* Number of kernel launches issued by the context since creation (for
 * accounting). */
int64_t sdrt_launch_count(const sdrt_ctx* ctx);

/* Options of a context.
 *   SDRT_OPT_TENSOR_CORES (default 0): 1 = run the interpolation of FP32
 *     tetrahedra of degree 3 on the tensor cores (tcgen05, products split
 *     into three TF32 products, FP32 accumulation); 0 = CUDA-core FMA kernels
 *     only (currently the faster of the two for that kernel).  Results agree
 *     to FP32 rounding. */
#define SDRT_OPT_TENSOR_CORES 0
/*   SDRT_OPT_TC_DIVERGENCE (default 0): 1 = for FP32 Euler / Rusanov on
 *     tetrahedra of degree 3, compute the fluxes on the CUDA cores and the
 *     divergence [M14 | M13] F~ on the tensor cores (tcgen05, 3xTF32, FP32
 *     accumulation in tensor memory); 0 = CUDA-core FMA accumulation. */
#define SDRT_OPT_TC_DIVERGENCE 1
/*   SDRT_OPT_FUSED_RK (default 1): 1 = RK4 steps on FP32 Euler meshes of
 *     degree-3 tetrahedra (CUDA-core kernels) interpolate each next stage's
 *     state inside the previous stage's update; 0 = one interpolation kernel
 *     per stage.  Same operations either way: the results are bit-identical. */
#define SDRT_OPT_FUSED_RK 2
/*   SDRT_OPT_GENERATED (default 1): 1 = residuals and RK4 steps of FP32 3D
 *     Euler / Rusanov meshes whose element types all have operator-specialised
 *     kernels (hexahedra of degree 1-3, prisms and tetrahedra of degree 1-4,
 *     SDRT scheme; meshes of degree-3 / 4 tetrahedra only keep the record path)
 *     run them: the structural non-zeros of [M0; M12] and [M14 | M13] compiled
 *     in, one fused stage kernel per element type and RK stage writing the
 *     next stage's face records, the element types as concurrent branches;
 *     0 = the generic kernels; 2 = as 1, and meshes set up afterwards take the
 *     operator-specialised kernels also where the record path would run.
 *     Results agree to FP32 rounding. */
#define SDRT_OPT_GENERATED 3
/*   SDRT_OPT_WAIT_POLLS (default 0): > 0 = the record-path flux kernel (FP32 /
 *     FP64 tetrahedra of degree 3 / 4) checks its first wait for its copies
 *     that many times without blocking; when that runs out it records a
 *     timeout, which sdrt_sync reports as SDRT_ERR_TIMEOUT, and then waits for
 *     its copies with the normal bound, so its results stay correct.  A test
 *     hook for the timeout path; 0 = the normal bound (about 2^26 polls).
 *     Changing it drops captured RK4 graphs. */
#define SDRT_OPT_WAIT_POLLS 4
/*   SDRT_OPT_NVTX (default 0): 1 = NVTX ranges (host-side markers for
 *     profilers such as Nsight Compute's --nvtx filters) around the main entry
 *     points (sdrt_residual, sdrt_rk4_step, sdrt_jvp, sdrt_vjp, the RK54 and
 *     partitioned-residual calls, ...) and around every kernel launch, named by
 *     the kernel's kind (interpolation, residual, residual_jvp, gradient).  No
 *     effect on results; without an attached tool the markers cost a branch. */
#define SDRT_OPT_NVTX 5
/*   SDRT_OPT_TC_GRADIENT (default 1): 1 = residuals and RK steps of FP32 3D
 *     Navier-Stokes meshes whose blocks are all affine tetrahedra of degree
 *     3 / 4, hexahedra of degree 2 or prisms of degree 2 compute the LDG
 *     gradient chain (q~ = [M16 | M15 P M12] [C; U], q = J^-T q~, q at the
 *     flux points = [M0; M12] q; Sec. 2.1) on the tensor cores (tcgen05,
 *     products split into three TF32 products, FP32 accumulation in tensor
 *     memory); 0 = the CUDA-core gradient kernel.  Results agree to FP32
 *     rounding.  The JVP, VJP and diagnostics keep the CUDA-core kernel. */
#define SDRT_OPT_TC_GRADIENT 6
int sdrt_set_option(sdrt_ctx* ctx, int option, int value);

/* Per-launch device timing with CUDA events recorded on the context's stream
 * around every kernel the context launches, including inside the captured
 * RK4 graphs (enabling or disabling drops captured graphs, which are then
 * re-captured).  Costs two event records per launch.  While it is on, the
 * element types' kernels of the operator-specialised path run one after the
 * other instead of as concurrent branches, so that each launch is timed
 * alone. */
int sdrt_profile_enable(sdrt_ctx* ctx, int enable);

/* Synchronise the stream, then ADD to ms_out[kind] the device milliseconds and
 * to count_out[kind] the number of launches recorded since the last collect.
 * kind: 0 = interpolation to external points, 1 = residual / divergence
 * kernel, 2 = its JVP variant, 3 = flux-point gradients (viscous systems).  Arrays of 4 entries, caller
 * owned.  A graph replayed several times between two collects keeps only its
 * last replay's timings: collect after every sdrt_rk4_step call. */
int sdrt_profile_collect(sdrt_ctx* ctx, double* ms_out, int64_t* count_out);

/* The same timings split by mesh block: ADD to ms_out[row * 4 + kind] and
 * count_out[row * 4 + kind], row 0 for launches that cover every block of a
 * mesh (generic and record kernels), row b + 1 for launches of block b alone
 * (the operator-specialised kernels, one launch per block; blocks past
 * max_blocks count in row 0).  Arrays of 4 (max_blocks + 1) entries, caller
 * owned.  Consumes the recorded timings like sdrt_profile_collect. */
int sdrt_profile_collect_blocks(sdrt_ctx* ctx, int max_blocks, double* ms_out, int64_t* count_out);

#ifdef __cplusplus
}
#endif

#endif /* SDRT_H */
