"""Affine metrics, physical face normals and flux-point pairing across faces.

Oracle (test infrastructure only).
  * mapping x = M(x~) is affine per element (paper Sec. 2, Eq. "mapping_function";
    the paper assumes analytical Jacobians on uniform grids).  J_ij = dx_i/dx~_j,
    det J, J^{-1} (Eqs. "mapping_jacobian", "inverse_mapping_jacobian").
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

from . import operators, points


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


def build(mesh, degrees):
    """degrees: one int for every block, a list with one degree per block, or
    a dict shape -> p."""
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
        blocks.append(BlockGeom(shape, p, ops, len(J), J, detJ, Jinv,
                                to_phys(ops.xs), to_phys(ops.xfe),
                                n_phys / nrm[:, :, None], detJ[:, None] * nrm))
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
        size = np.abs(GL.J[eL]).max()
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
