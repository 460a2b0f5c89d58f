"""Element metrics, physical face normals and flux-point pairing across faces.

Oracle (test infrastructure only).
  * mapping x = M(x~) per element (paper Sec. 2, Eq. "mapping_function"; the
    paper evaluates the Jacobians analytically): affine when a block gives only
    vertices, the quadratic Lagrange map of oracle/mapping.py when it also gives
    "nodes" (curved elements).  J_ij = dx_i/dx~_j, det J, J^{-1} (Eqs.
    "mapping_jacobian", "inverse_mapping_jacobian"), evaluated where the
    method uses them (Sec. 2.1): J^{-T} at the solution points (physical
    gradients), det J J^{-1} at the internal flux points (Eq.
    "normal_transformed_flux"), det J |J^{-T} n~| at the external flux points
    (transformed common flux) and 1 / det J at the solution points (the
    semi-discrete form).  Affine elements have one value per element, which
    the per-point arrays repeat.
  * physical normal at an external flux point n = J^{-T} n~ (unnormalised); the
    transformed common flux is det J |n| F(u_L, u_R, n/|n|) (Eq. before
    "divergence_sdrt"; reading: |n| is the norm of J^{-T} n~).
  * external flux points of glued faces are paired by physical coordinates
    (after the periodic shift) to 1e-9 of the element size (Sec. 2.1: the common
    value / flux uses "the flux point adjacent to" each point).
Each glued face has one orientation, taken from the mesh's face list (L = first
element of the row): the common value C(u_L, u_R) and the common flux
F(u_L, u_R, n_L) are single-valued per face (Sec. 2.1: the same C for both
adjacent points, F of the R side = -F of the L side), which matters for the
LDG parameter beta != 0.
The face map is returned in canonical global numbering
    g = fe_base[b] + e * N_fe[b] + sigma,
the bit-exact contract shared with the library.

Parity: pinned by the involution / coincidence tests of the map, free-stream
preservation and conservation (tests/test_oracle_residual.py).
"""
from dataclasses import dataclass

import numpy as np

from . import mapping, operators, points


@dataclass
class BlockGeom:
    shape: str
    p: int
    ops: operators.ElementOps
    nelem: int
    J: np.ndarray          # (E, ND, ND)
    detJ: np.ndarray       # (E,)
    Jinv: np.ndarray       # (E, ND, ND)  dx~_i / dx_j
    xsol: np.ndarray       # (E, N_s, ND) physical solution points
    xfe: np.ndarray        # (E, N_fe, ND) physical external flux points
    nunit: np.ndarray      # (E, N_fe, ND) physical unit normal at external points
    nmag: np.ndarray       # (E, N_fe) det J |J^{-T} n~|
    dets: np.ndarray = None    # (E, N_s) det J at the solution points
    Jinvs: np.ndarray = None   # (E, N_s, ND, ND) J^{-1} at the solution points
    detf: np.ndarray = None    # (E, N_fiu) det J at the unique internal flux points
    Jinvf: np.ndarray = None   # (E, N_fiu, ND, ND) J^{-1} there
    size: np.ndarray = None    # (E,) largest |J_ij| of the element (pairing tolerance)
    curved: bool = False


@dataclass
class MeshGeom:
    blocks: list
    fe_base: np.ndarray    # canonical base of each block's external points
    partner: np.ndarray    # (total_fe,) canonical index of the paired point
    is_left: np.ndarray    # (total_fe,) True where the point's element is the face's L side
    nd: int


def affine_map(shape, verts):
    """Affine coefficients C ((ND+1) x ND) with x = [x~, 1] @ C, fitted to the vertices."""
    ref = points.VERTS[shape]
    A = np.column_stack([ref, np.ones(len(ref))])
    E = verts.shape[0]
    C = np.empty((E, A.shape[1], verts.shape[2]))
    for e in range(E):
        C[e], res, _, _ = np.linalg.lstsq(A, verts[e], rcond=None)
        if np.abs(A @ C[e] - verts[e]).max() > 1e-9 * (1 + np.abs(verts[e]).max()):
            raise ValueError("element is not affine")
    return C


def _curved_block(shape, p, ops, Xn):
    """Geometry of a block of quadratic elements with mapping nodes Xn (E, NN, ND)."""
    xs, Js = mapping.jacobians(shape, Xn, ops.xs)
    xfe, Jfe = mapping.jacobians(shape, Xn, ops.xfe)
    _, Jf = mapping.jacobians(shape, Xn, ops.xfiu)
    dets, detfe, detf = np.linalg.det(Js), np.linalg.det(Jfe), np.linalg.det(Jf)
    if min(dets.min(), detfe.min(), detf.min()) <= 0:
        raise ValueError("inverted element")
    Jinvfe = np.linalg.inv(Jfe)
    n_phys = np.einsum("epji,pj->epi", Jinvfe, ops.nrm_fe)   # J^{-T} n~ at each point
    nrm = np.linalg.norm(n_phys, axis=2)
    return BlockGeom(shape, p, ops, len(Xn), None, None, None, xs, xfe,
                     n_phys / nrm[:, :, None], detfe * nrm,
                     dets=dets, Jinvs=np.linalg.inv(Js), detf=detf, Jinvf=np.linalg.inv(Jf),
                     size=np.abs(Js).reshape(len(Xn), -1).max(axis=1), curved=True)


def build(mesh, degrees):
    """degrees: one int for every block, a list with one degree per block, or
    a dict shape -> p.  A block with a "nodes" array (E, NN, ND) holds curved
    elements (quadratic map, oracle/mapping.py); its "verts" are not used."""
    blocks = []
    nd = mesh["blocks"][0]["verts"].shape[2]
    for i, blk in enumerate(mesh["blocks"]):
        shape = blk["shape"]
        if isinstance(degrees, int):
            p = degrees
        elif isinstance(degrees, (list, tuple)):
            p = degrees[i]
        else:
            p = degrees[shape]
        ops = operators.get(shape, p)
        if "nodes" in blk:
            blocks.append(_curved_block(shape, p, ops, np.asarray(blk["nodes"], float)))
            continue
        C = affine_map(shape, blk["verts"])
        J = np.transpose(C[:, :nd, :], (0, 2, 1))          # J_ij = dx_i / dx~_j
        detJ = np.linalg.det(J)
        if np.any(detJ <= 0):
            raise ValueError("inverted element")
        Jinv = np.linalg.inv(J)
        def to_phys(Xr):
            return np.einsum("pk,ekd->epd", np.column_stack([Xr, np.ones(len(Xr))]), C)
        n_phys = np.einsum("eji,pj->epi", Jinv, ops.nrm_fe)   # J^{-T} n~
        nrm = np.linalg.norm(n_phys, axis=2)
        E, ns, nk = len(J), ops.n_sol, len(ops.xfiu)
        blocks.append(BlockGeom(shape, p, ops, E, J, detJ, Jinv,
                                to_phys(ops.xs), to_phys(ops.xfe),
                                n_phys / nrm[:, :, None], detJ[:, None] * nrm,
                                dets=np.repeat(detJ[:, None], ns, 1),
                                Jinvs=np.repeat(Jinv[:, None], ns, 1),
                                detf=np.repeat(detJ[:, None], nk, 1),
                                Jinvf=np.repeat(Jinv[:, None], nk, 1),
                                size=np.abs(J).reshape(E, -1).max(axis=1)))
    nfe = np.array([b.ops.n_fe for b in blocks])
    ne = np.array([b.nelem for b in blocks])
    fe_base = np.concatenate([[0], np.cumsum(nfe * ne)])[:-1]
    total = int((nfe * ne).sum())
    partner = np.full(total, -1, np.int64)
    is_left = np.zeros(total, bool)
    for (bL, eL, fL, bR, eR, fR), s in zip(mesh["faces"], mesh["shift"]):
        GL, GR = blocks[bL], blocks[bR]
        iL = np.nonzero(GL.ops.fe_face == fL)[0]
        iR = np.nonzero(GR.ops.fe_face == fR)[0]
        XL = GL.xfe[eL, iL]
        XR = GR.xfe[eR, iR] + s
        size = GL.size[eL]
        d = np.linalg.norm(XL[:, None, :] - XR[None, :, :], axis=2)
        j = np.argmin(d, axis=1)
        if len(iL) != len(iR) or d[np.arange(len(iL)), j].max() > 1e-9 * size \
                or len(set(j.tolist())) != len(iL):
            raise ValueError("face flux points do not match")
        gL = fe_base[bL] + eL * GL.ops.n_fe + iL
        gR = fe_base[bR] + eR * GR.ops.n_fe + iR[j]
        partner[gL] = gR
        partner[gR] = gL
        is_left[gL] = True
    if np.any(partner < 0):
        raise ValueError("unpaired external flux points")
    return MeshGeom(blocks, fe_base, partner, is_left, nd)
