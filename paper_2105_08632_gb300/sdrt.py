"""Thin ctypes binding of libsdrt (include/sdrt.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts Python /
NumPy / torch arguments to the C structs and pointers of the C ABI.  The
functions keep the C names (sdrt_create, sdrt_setup_element_type, ...).  The
Mesh class bundles them for convenience.  If libsdrt.so is missing or fails to
load, import of this module raises: there is no fallback implementation.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsdrt.so")

SHAPES = {"tri": 0, "quad": 1, "tet": 2, "pri": 3, "hex": 4}
SYSTEMS = {"advection": 0, "advdiff": 1, "euler": 2, "ns": 3}
RIEMANN = {"upwind": 0, "rusanov": 1, "roe": 2}
PRECISION = {"fp64": 0, "fp32": 1, "tf32x3": 2}
STATUS = {0: "SDRT_OK", -1: "SDRT_ERR_ARG", -2: "SDRT_ERR_UNSUPPORTED", -3: "SDRT_ERR_CUDA",
          -4: "SDRT_ERR_STATE", -5: "SDRT_ERR_NONFINITE", -6: "SDRT_ERR_TIMEOUT", -7: "SDRT_ERR_MESH"}

EXPORTED = ["sdrt_create", "sdrt_destroy", "sdrt_last_error", "sdrt_set_stream", "sdrt_setup_element_type",
            "sdrt_get_etype_info", "sdrt_get_operator", "sdrt_setup_mesh", "sdrt_get_mesh_info",
            "sdrt_get_block_layout", "sdrt_get_sol_points", "sdrt_get_face_map", "sdrt_residual",
            "sdrt_rk4_step", "sdrt_rk4_step_host", "sdrt_jvp", "sdrt_vjp", "sdrt_sync", "sdrt_launch_count",
            "sdrt_profile_enable", "sdrt_profile_collect", "sdrt_residual_noalloc", "sdrt_set_option",
            "sdrt_autotune", "sdrt_get_tiles", "sdrt_profile_collect_blocks", "sdrt_rk54_step",
            "sdrt_rk54_adaptive_step", "sdrt_rk54_integrate", "sdrt_tgv_diagnostics", "sdrt_setup_mesh_curved"]


class SdrtError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class EtypeDesc(ctypes.Structure):
    _fields_ = [("shape", ctypes.c_int32), ("degree", ctypes.c_int32), ("scheme", ctypes.c_int32)]


SCHEMES = {"sdrt": 0, "fr": 1}


class EtypeInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("ndim", "nsol", "nfe", "nfi", "nfiu", "nfaces")]


class Physics(ctypes.Structure):
    _fields_ = [("system", ctypes.c_int32), ("riemann", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("ndim", ctypes.c_int32), ("a", ctypes.c_double * 3), ("mu", ctypes.c_double),
                ("gamma", ctypes.c_double), ("prandtl", ctypes.c_double), ("beta", ctypes.c_double),
                ("eta", ctypes.c_double)]


class Block(ctypes.Structure):
    _fields_ = [("etype", ctypes.c_int32), ("nelem", ctypes.c_int32), ("verts", ctypes.POINTER(ctypes.c_double))]


class Face(ctypes.Structure):
    _fields_ = [("blk_l", ctypes.c_int32), ("elem_l", ctypes.c_int32), ("face_l", ctypes.c_int32),
                ("blk_r", ctypes.c_int32), ("elem_r", ctypes.c_int32), ("face_r", ctypes.c_int32),
                ("shift", ctypes.c_double * 3)]


class MeshInfo(ctypes.Structure):
    _fields_ = [("nvar", ctypes.c_int32), ("nblocks", ctypes.c_int32), ("ndim", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("state_len", ctypes.c_int64), ("ndof", ctypes.c_int64),
                ("nfe_total", ctypes.c_int64), ("path", ctypes.c_int32), ("curved", ctypes.c_int32)]


class BlockLayout(ctypes.Structure):
    _fields_ = [("etype", ctypes.c_int32), ("nsol", ctypes.c_int32), ("nvar", ctypes.c_int32),
                ("nelem", ctypes.c_int32), ("ld", ctypes.c_int32), ("nfe", ctypes.c_int32),
                ("offset", ctypes.c_int64)]


_lib = None


def lib():
    """Load libsdrt.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libsdrt.so not found at {LIB_PATH}; run paper_2105_08632_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "sdrt_create": (I, [ctypes.POINTER(P), I, P]),
        "sdrt_destroy": (None, [P]),
        "sdrt_last_error": (ctypes.c_char_p, [P]),
        "sdrt_set_stream": (I, [P, P]),
        "sdrt_setup_element_type": (I, [P, ctypes.POINTER(EtypeDesc), ctypes.POINTER(I)]),
        "sdrt_get_etype_info": (I, [P, I, ctypes.POINTER(EtypeInfo)]),
        "sdrt_get_operator": (I, [P, I, I, ctypes.POINTER(D), I64]),
        "sdrt_setup_mesh": (I, [P, ctypes.POINTER(Physics), I, ctypes.POINTER(Block), I64, ctypes.POINTER(Face),
                                ctypes.POINTER(I)]),
        "sdrt_setup_mesh_curved": (I, [P, ctypes.POINTER(Physics), I, ctypes.POINTER(Block),
                                       ctypes.POINTER(ctypes.POINTER(D)), I64, ctypes.POINTER(Face),
                                       ctypes.POINTER(I)]),
        "sdrt_get_mesh_info": (I, [P, I, ctypes.POINTER(MeshInfo)]),
        "sdrt_get_block_layout": (I, [P, I, I, ctypes.POINTER(BlockLayout)]),
        "sdrt_get_sol_points": (I, [P, I, ctypes.POINTER(D), I64]),
        "sdrt_get_face_map": (I, [P, I, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_uint8), I64]),
        "sdrt_residual": (I, [P, I, P, P]),
        "sdrt_rk4_step": (I, [P, I, P, D, I]),
        "sdrt_rk4_step_host": (I, [P, I, P, P, D, I]),
        "sdrt_rk54_step": (I, [P, I, P, D, I]),
        "sdrt_tgv_diagnostics": (I, [P, I, P, D, D, D, ctypes.POINTER(D)]),
        "sdrt_rk54_adaptive_step": (I, [P, I, P, D, D, D, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(I)]),
        "sdrt_rk54_integrate": (I, [P, I, P, D, ctypes.POINTER(D), D, D, I, ctypes.POINTER(I), ctypes.POINTER(I)]),
        "sdrt_jvp": (I, [P, I, P, P, P]),
        "sdrt_vjp": (I, [P, I, P, P, P]),
        "sdrt_sync": (I, [P]),
        "sdrt_launch_count": (I64, [P]),
        "sdrt_profile_enable": (I, [P, I]),
        "sdrt_profile_collect": (I, [P, ctypes.POINTER(D), ctypes.POINTER(I64)]),
        "sdrt_profile_collect_blocks": (I, [P, I, ctypes.POINTER(D), ctypes.POINTER(I64)]),
        "sdrt_residual_noalloc": (I, [P, I, P, P]),
        "sdrt_set_option": (I, [P, I, I]),
        "sdrt_autotune": (I, [P, I, P, I]),
        "sdrt_get_tiles": (I, [P, I, I, ctypes.POINTER(ctypes.c_int32)]),
        "sdrt_setup_partition": (I, [P, ctypes.POINTER(Physics), I, ctypes.POINTER(Block), ctypes.POINTER(ctypes.c_uint8),
                                     I64, ctypes.POINTER(Face), ctypes.POINTER(I)]),
        "sdrt_set_exchange": (I, [P, I, I64, ctypes.POINTER(ctypes.c_int32), I64, ctypes.POINTER(ctypes.c_int32)]),
        "sdrt_get_exchange_info": (I, [P, I, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(ctypes.c_int32),
                                       ctypes.POINTER(ctypes.c_int32)]),
        "sdrt_residual_gradients": (I, [P, I, P, P]),
        "sdrt_residual_begin": (I, [P, I, P, P]),
        "sdrt_residual_end": (I, [P, I, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(ctx, code):
    if code != 0:
        msg = lib().sdrt_last_error(ctx).decode() if ctx else ""
        raise SdrtError(code, msg)


def _ptr(x):
    """Device / host pointer of a torch tensor or NumPy array, or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


# ---------------------------------------------------------------------------
# C-ABI functions, same names.

def sdrt_create(device=0, stream=None):
    ctx = ctypes.c_void_p()
    _check(None, lib().sdrt_create(ctypes.byref(ctx), int(device), stream))
    return ctx


def sdrt_destroy(ctx):
    lib().sdrt_destroy(ctx)


def sdrt_set_stream(ctx, stream):
    _check(ctx, lib().sdrt_set_stream(ctx, stream))


def sdrt_setup_element_type(ctx, shape, degree, scheme="sdrt"):
    out = ctypes.c_int()
    d = EtypeDesc(SHAPES[shape] if isinstance(shape, str) else int(shape), int(degree),
                  SCHEMES[scheme] if isinstance(scheme, str) else int(scheme))
    _check(ctx, lib().sdrt_setup_element_type(ctx, ctypes.byref(d), ctypes.byref(out)))
    return out.value


def sdrt_get_etype_info(ctx, etype):
    info = EtypeInfo()
    _check(ctx, lib().sdrt_get_etype_info(ctx, int(etype), ctypes.byref(info)))
    return {n: getattr(info, n) for n, _ in EtypeInfo._fields_}


OPERATORS = {"M0": 0, "M12": 1, "M13": 2, "M14": 3, "M15": 4, "M16": 5, "xs": 6, "xfe": 7}


def sdrt_get_operator(ctx, etype, name):
    i = sdrt_get_etype_info(ctx, etype)
    nd, ns, nfe, nfi, nfiu = i["ndim"], i["nsol"], i["nfe"], i["nfi"], i["nfiu"]
    shapes = {"M0": (nfe, ns), "M12": (nfiu, ns), "M13": (ns, nfi), "M14": (ns, nfe),
              "M15": (nd * ns, nfi), "M16": (nd * ns, nfe), "xs": (ns, nd), "xfe": (nfe, nd)}
    out = np.empty(shapes[name], np.float64)
    _check(ctx, lib().sdrt_get_operator(ctx, int(etype), OPERATORS[name],
                                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.size))
    return out


def sdrt_setup_mesh(ctx, physics, blocks, faces, ghost=None, nodes=None):
    """physics: Physics struct; blocks: list of (etype_id, verts float64 (E, nv, ND));
    faces: int array (F, 6) and shift array (F, ND) as a tuple.  ghost: per-block
    flags (uint8) -> sdrt_setup_partition.  nodes: per-block None or the curved
    elements' quadratic-map nodes float64 (E, NN, ND) -> sdrt_setup_mesh_curved."""
    nb = len(blocks)
    barr = (Block * nb)()
    keep = []
    for i, (et, verts) in enumerate(blocks):
        v = np.ascontiguousarray(verts, np.float64)
        keep.append(v)
        barr[i] = Block(int(et), int(v.shape[0]), v.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if nodes is not None and any(x is not None for x in nodes):
        if ghost is not None:
            raise ValueError("partitions take affine elements")
        if len(nodes) != nb:
            raise ValueError("one node array (or None) per block")
        narr = (ctypes.POINTER(ctypes.c_double) * nb)()
        for i, x in enumerate(nodes):
            if x is None:
                continue
            x = np.ascontiguousarray(x, np.float64)
            if x.ndim != 3 or x.shape[0] != blocks[i][1].shape[0]:
                raise ValueError("nodes of block %d: (nelem, nnode, ndim) expected" % i)
            keep.append(x)
            narr[i] = x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    fidx, shift = faces
    nf = len(fidx)
    farr = (Face * max(nf, 1))()
    for i in range(nf):
        r = fidx[i]
        s = list(shift[i]) + [0.0] * (3 - len(shift[i]))
        farr[i] = Face(int(r[0]), int(r[1]), int(r[2]), int(r[3]), int(r[4]), int(r[5]), (ctypes.c_double * 3)(*s))
    out = ctypes.c_int()
    if nodes is not None and any(x is not None for x in nodes):
        _check(ctx, lib().sdrt_setup_mesh_curved(ctx, ctypes.byref(physics), nb, barr, narr, nf, farr,
                                                 ctypes.byref(out)))
    elif ghost is None:
        _check(ctx, lib().sdrt_setup_mesh(ctx, ctypes.byref(physics), nb, barr, nf, farr, ctypes.byref(out)))
    else:
        g = np.ascontiguousarray(ghost, np.uint8)
        if g.shape != (nb,):
            raise ValueError("one ghost flag per block")
        _check(ctx, lib().sdrt_setup_partition(ctx, ctypes.byref(physics), nb, barr,
                                               g.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), nf, farr,
                                               ctypes.byref(out)))
    return out.value


def sdrt_setup_partition(ctx, physics, blocks, ghost, faces):
    return sdrt_setup_mesh(ctx, physics, blocks, faces, ghost=ghost)


def sdrt_set_exchange(ctx, mesh, send, recv):
    """send / recv: int32 arrays (n, 3) of (block, element, face) triplets."""
    s = np.ascontiguousarray(np.asarray(send, np.int32).reshape(-1, 3))
    r = np.ascontiguousarray(np.asarray(recv, np.int32).reshape(-1, 3))
    P32 = ctypes.POINTER(ctypes.c_int32)
    _check(ctx, lib().sdrt_set_exchange(ctx, int(mesh), len(s), s.ctypes.data_as(P32), len(r), r.ctypes.data_as(P32)))


def sdrt_get_exchange_info(ctx, mesh):
    ns, nr, fr, gr = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int32()
    _check(ctx, lib().sdrt_get_exchange_info(ctx, int(mesh), ctypes.byref(ns), ctypes.byref(nr), ctypes.byref(fr),
                                             ctypes.byref(gr)))
    return {"nsend": ns.value, "nrecv": nr.value, "face_record": fr.value, "grad_record": gr.value}


def sdrt_residual_gradients(ctx, mesh, recv, send_grad):
    _check(ctx, lib().sdrt_residual_gradients(ctx, int(mesh), _ptr(recv), _ptr(send_grad)))


def sdrt_residual_begin(ctx, mesh, U, send):
    _check(ctx, lib().sdrt_residual_begin(ctx, int(mesh), _ptr(U), _ptr(send)))


def sdrt_residual_end(ctx, mesh, recv, R):
    _check(ctx, lib().sdrt_residual_end(ctx, int(mesh), _ptr(recv), _ptr(R)))


def sdrt_get_mesh_info(ctx, mesh):
    info = MeshInfo()
    _check(ctx, lib().sdrt_get_mesh_info(ctx, int(mesh), ctypes.byref(info)))
    return {n: getattr(info, n) for n, _ in MeshInfo._fields_}


def sdrt_get_block_layout(ctx, mesh, block):
    lay = BlockLayout()
    _check(ctx, lib().sdrt_get_block_layout(ctx, int(mesh), int(block), ctypes.byref(lay)))
    return {n: getattr(lay, n) for n, _ in BlockLayout._fields_}


def sdrt_get_sol_points(ctx, mesh, n):
    out = np.empty(n, np.float64)
    _check(ctx, lib().sdrt_get_sol_points(ctx, int(mesh), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), n))
    return out


def sdrt_get_face_map(ctx, mesh, n):
    part = np.empty(n, np.int32)
    left = np.empty(n, np.uint8)
    _check(ctx, lib().sdrt_get_face_map(ctx, int(mesh), part.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                        left.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)), n))
    return part, left


def sdrt_residual(ctx, mesh, U, R):
    _check(ctx, lib().sdrt_residual(ctx, int(mesh), _ptr(U), _ptr(R)))


def sdrt_residual_noalloc(ctx, mesh, U, R):
    """sdrt_residual without any device allocation (fixed library-image scratch;
    see include/sdrt.h for the size limit and the sharing rules)."""
    _check(ctx, lib().sdrt_residual_noalloc(ctx, int(mesh), _ptr(U), _ptr(R)))


def sdrt_rk4_step(ctx, mesh, U, dt, nsteps=1):
    _check(ctx, lib().sdrt_rk4_step(ctx, int(mesh), _ptr(U), float(dt), int(nsteps)))


def sdrt_rk54_step(ctx, mesh, U, dt, nsteps=1):
    _check(ctx, lib().sdrt_rk54_step(ctx, int(mesh), _ptr(U), float(dt), int(nsteps)))


def sdrt_rk54_adaptive_step(ctx, mesh, U, dt, atol, rtol):
    """(accepted, err, dt_next) of one adaptive RK54 step attempt."""
    err, dtn, acc = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(ctx, lib().sdrt_rk54_adaptive_step(ctx, int(mesh), _ptr(U), float(dt), float(atol), float(rtol),
                                              ctypes.byref(err), ctypes.byref(dtn), ctypes.byref(acc)))
    return bool(acc.value), err.value, dtn.value


def sdrt_rk54_integrate(ctx, mesh, U, t_span, dt, atol, rtol, max_steps=100000):
    """(dt_next, accepted steps, rejected steps) of an adaptive integration over t_span."""
    d, na, nr = ctypes.c_double(dt), ctypes.c_int(), ctypes.c_int()
    _check(ctx, lib().sdrt_rk54_integrate(ctx, int(mesh), _ptr(U), float(t_span), ctypes.byref(d), float(atol),
                                          float(rtol), int(max_steps), ctypes.byref(na), ctypes.byref(nr)))
    return d.value, na.value, nr.value


def sdrt_tgv_diagnostics(ctx, mesh, U, rho_inf=1.0, v_inf=1.0, length=1.0):
    """Dict <E*>, eps1, eps2, eps3 of the Taylor-Green diagnostics."""
    out = (ctypes.c_double * 4)()
    _check(ctx, lib().sdrt_tgv_diagnostics(ctx, int(mesh), _ptr(U), float(rho_inf), float(v_inf), float(length), out))
    return {"E": out[0], "eps1": out[1], "eps2": out[2], "eps3": out[3]}


def sdrt_rk4_step_host(ctx, mesh, U_in, U_out, dt, nsteps=1):
    _check(ctx, lib().sdrt_rk4_step_host(ctx, int(mesh), _ptr(U_in), _ptr(U_out), float(dt), int(nsteps)))


def sdrt_jvp(ctx, mesh, U, V, JV):
    _check(ctx, lib().sdrt_jvp(ctx, int(mesh), _ptr(U), _ptr(V), _ptr(JV)))


def sdrt_vjp(ctx, mesh, U, W, JTW):
    _check(ctx, lib().sdrt_vjp(ctx, int(mesh), _ptr(U), _ptr(W), _ptr(JTW)))


def sdrt_sync(ctx):
    _check(ctx, lib().sdrt_sync(ctx))


def sdrt_launch_count(ctx):
    return int(lib().sdrt_launch_count(ctx))


SDRT_OPT_TENSOR_CORES = 0
SDRT_OPT_TC_DIVERGENCE = 1
SDRT_OPT_FUSED_RK = 2
SDRT_OPT_GENERATED = 3
SDRT_OPT_WAIT_POLLS = 4
SDRT_OPT_NVTX = 5
SDRT_OPT_TC_GRADIENT = 6
PATHS = {0: "generic", 1: "record", 2: "generated"}


def sdrt_autotune(ctx, mesh, U, reps=3):
    _check(ctx, lib().sdrt_autotune(ctx, int(mesh), _ptr(U), int(reps)))


TILE_KINDS = ("interp", "residual", "residual_jvp", "gradient", "gradient_jvp", "vjp")


def sdrt_get_tiles(ctx, mesh, block):
    out = (ctypes.c_int32 * 6)()
    _check(ctx, lib().sdrt_get_tiles(ctx, int(mesh), int(block), out))
    return dict(zip(TILE_KINDS, list(out)))


def sdrt_set_option(ctx, option, value):
    _check(ctx, lib().sdrt_set_option(ctx, int(option), int(value)))


def sdrt_profile_enable(ctx, enable=True):
    _check(ctx, lib().sdrt_profile_enable(ctx, 1 if enable else 0))


KERNEL_KINDS = ("interp_ext", "residual", "residual_jvp", "gradient")


def sdrt_profile_collect(ctx):
    """Dict kind -> (milliseconds, launches) recorded since the last collect."""
    ms = (ctypes.c_double * 4)()
    cnt = (ctypes.c_int64 * 4)()
    _check(ctx, lib().sdrt_profile_collect(ctx, ms, cnt))
    return {k: (ms[i], cnt[i]) for i, k in enumerate(KERNEL_KINDS)}


def sdrt_profile_collect_blocks(ctx, nblocks):
    """List of nblocks + 1 dicts kind -> (milliseconds, launches): entry 0 for
    launches over all blocks, entry b + 1 for launches of block b alone."""
    n = 4 * (nblocks + 1)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    _check(ctx, lib().sdrt_profile_collect_blocks(ctx, int(nblocks), ms, cnt))
    return [{k: (ms[4 * r + i], cnt[4 * r + i]) for i, k in enumerate(KERNEL_KINDS)} for r in range(nblocks + 1)]


# ---------------------------------------------------------------------------
# Convenience wrapper.

def make_physics(system, ndim, riemann="rusanov", precision="fp32", a=(1.0, 0.0, 0.0), mu=0.0, gamma=1.4,
                 prandtl=0.72, beta=0.5, eta=0.1):
    a = list(a) + [0.0] * (3 - len(a))
    return Physics(SYSTEMS[system], RIEMANN[riemann], PRECISION[precision], int(ndim),
                   (ctypes.c_double * 3)(*a[:3]), mu, gamma, prandtl, beta, eta)


class Context:
    """A library context on one CUDA device, bound to torch's current stream."""

    def __init__(self, device=0, stream=None):
        if stream is None and device >= 0:               # device -1: host-only context
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        self.device = device
        self.ptr = sdrt_create(device, stream)

    def close(self):
        if self.ptr:
            sdrt_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mesh:
    """A mesh set up in a Context: mesh dict from inputs.meshes plus physics.
    Blocks with a "nodes" array hold curved elements (sdrt_setup_mesh_curved)."""

    def __init__(self, ctx, mesh, degree, physics, ghost=None, scheme="sdrt"):
        self.ctx = ctx
        c = ctx.ptr
        blocks = []
        self.etypes = []
        for i, blk in enumerate(mesh["blocks"]):
            if isinstance(degree, int):
                p = degree
            elif isinstance(degree, (list, tuple)):
                p = degree[i]                  # one degree per block
            else:
                p = degree[blk["shape"]]       # one degree per element shape
            et = sdrt_setup_element_type(c, blk["shape"], p, scheme)
            self.etypes.append(et)
            blocks.append((et, blk["verts"]))
        nodes = [blk.get("nodes") for blk in mesh["blocks"]]
        self.id = sdrt_setup_mesh(c, physics, blocks, (mesh["faces"], mesh["shift"]), ghost=ghost, nodes=nodes)
        self.info = sdrt_get_mesh_info(c, self.id)
        self.layouts = [sdrt_get_block_layout(c, self.id, b) for b in range(self.info["nblocks"])]
        self.dtype_np = np.float64 if self.info["precision"] == 0 else np.float32   # fp32 / tf32x3: FP32 states

    @property
    def state_len(self):
        return self.info["state_len"]

    @property
    def nvar(self):
        return self.info["nvar"]

    def sol_points(self):
        """List per block of physical solution points (E, N_s, ND)."""
        nd = self.info["ndim"]
        n = sum(l["nelem"] * l["nsol"] * nd for l in self.layouts)
        flat = sdrt_get_sol_points(self.ctx.ptr, self.id, n)
        out, s = [], 0
        for l in self.layouts:
            k = l["nelem"] * l["nsol"] * nd
            out.append(flat[s:s + k].reshape(l["nelem"], l["nsol"], nd))
            s += k
        return out

    def pack(self, blocks):
        """List of (N_s, V, E) arrays -> flat state array (NumPy, padded layout)."""
        out = np.zeros(self.state_len, self.dtype_np)
        for l, a in zip(self.layouts, blocks):
            ns, V, E, ld, off = l["nsol"], l["nvar"], l["nelem"], l["ld"], l["offset"]
            view = out[off:off + ns * V * ld].reshape(ns, V, ld)
            view[:, :, :E] = a
        return out

    def unpack(self, flat):
        flat = np.asarray(flat)
        out = []
        for l in self.layouts:
            ns, V, E, ld, off = l["nsol"], l["nvar"], l["nelem"], l["ld"], l["offset"]
            out.append(np.array(flat[off:off + ns * V * ld].reshape(ns, V, ld)[:, :, :E]))
        return out

    def face_map(self):
        return sdrt_get_face_map(self.ctx.ptr, self.id, self.info["nfe_total"])

    def _check(self, *arrays, device=True):
        """The C ABI takes bare pointers: check length, dtype, contiguity and
        placement of every state array before a call reaches the device."""
        for a in arrays:
            if isinstance(a, int):
                continue                      # raw pointer: the caller vouches for it
            n = a.numel() if hasattr(a, "numel") else a.size
            if n != self.state_len:
                raise ValueError(f"state array has {n} values, the mesh needs {self.state_len}")
            if hasattr(a, "is_cuda"):
                if a.is_cuda != device:
                    raise ValueError("state array on the wrong device" if device else "host buffer expected")
                if device and a.device.index != self.ctx.device:
                    raise ValueError(f"state array on cuda:{a.device.index}, context on cuda:{self.ctx.device}")
                if not a.is_contiguous():
                    raise ValueError("state array must be contiguous")
                ok = str(a.dtype) == ("torch.float32" if self.dtype_np == np.float32 else "torch.float64")
            else:
                if device:
                    raise ValueError("device computation needs a CUDA tensor or a raw device pointer")
                if not a.flags["C_CONTIGUOUS"]:
                    raise ValueError("state array must be contiguous")
                ok = a.dtype == self.dtype_np
            if not ok:
                raise ValueError("state array dtype does not match the mesh precision")

    def residual(self, U, R):
        self._check(U, R)
        sdrt_residual(self.ctx.ptr, self.id, U, R)

    def rk4_step(self, U, dt, nsteps=1):
        self._check(U)
        sdrt_rk4_step(self.ctx.ptr, self.id, U, dt, nsteps)

    def rk54_step(self, U, dt, nsteps=1):
        self._check(U)
        sdrt_rk54_step(self.ctx.ptr, self.id, U, dt, nsteps)

    def rk54_adaptive_step(self, U, dt, atol, rtol):
        self._check(U)
        return sdrt_rk54_adaptive_step(self.ctx.ptr, self.id, U, dt, atol, rtol)

    def rk54_integrate(self, U, t_span, dt, atol, rtol, max_steps=100000):
        self._check(U)
        return sdrt_rk54_integrate(self.ctx.ptr, self.id, U, t_span, dt, atol, rtol, max_steps)

    def tgv_diagnostics(self, U, rho_inf=1.0, v_inf=1.0, length=1.0):
        self._check(U)
        return sdrt_tgv_diagnostics(self.ctx.ptr, self.id, U, rho_inf, v_inf, length)

    def rk4_step_host(self, U_in, U_out, dt, nsteps=1):
        self._check(U_in, U_out, device=False)
        sdrt_rk4_step_host(self.ctx.ptr, self.id, U_in, U_out, dt, nsteps)

    def jvp(self, U, V, JV):
        self._check(U, V, JV)
        sdrt_jvp(self.ctx.ptr, self.id, U, V, JV)

    def vjp(self, U, W, JTW):
        self._check(U, W, JTW)
        sdrt_vjp(self.ctx.ptr, self.id, U, W, JTW)

    def autotune(self, U, reps=3):
        self._check(U)
        sdrt_autotune(self.ctx.ptr, self.id, U, reps)

    def tiles(self):
        return [sdrt_get_tiles(self.ctx.ptr, self.id, b) for b in range(self.info["nblocks"])]

    def sync(self):
        sdrt_sync(self.ctx.ptr)
