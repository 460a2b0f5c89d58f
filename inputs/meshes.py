"""Structured periodic meshes built from subdivided boxes.

A mesh is a dict:
  blocks : list of {"shape": str, "verts": float64 (E, n_vertices, ND)}
           vertices in the reference-vertex order of the element type;
  faces  : int64 (F, 6)  rows (bL, eL, fL, bR, eR, fR): local face fL of element
           eL of block bL is glued to face fR of element eR of block bR;
  shift  : float64 (F, ND) with x_L = x_R + shift for coincident points
           (nonzero across periodic boundaries);
  box    : (lo, hi) float64 (ND,) each.

Local face numbering (vertex subsets per element type, the same convention the
library and the oracle use for their face point sets):
  tri  e0 (0,1) e1 (1,2) e2 (2,0)
  quad e0 (0,1) e1 (1,2) e2 (3,2) e3 (0,3)
  tet  f0 (0,1,2) f1 (0,1,3) f2 (1,2,3) f3 (0,2,3)
  pri  f0 (0,1,2) f1 (0,1,4,3) f2 (1,2,5,4) f3 (0,2,5,3) f4 (3,4,5)
  hex  f0 (0,1,2,3) f1 (0,1,5,4) f2 (1,2,6,5) f3 (3,2,6,7) f4 (0,3,7,4) f5 (4,5,6,7)

Subdivisions of one unit cell (paper Sec. 3: N_p = 1, 2, 6):
  tri : two triangles split along the (0,0)-(1,1) diagonal;
  tet : the six Kuhn (Freudenthal) tetrahedra around the (0,0,0)-(1,1,1)
        diagonal, conforming under translation;
  pri : the two triangles above extruded along z (their z-faces match the
        tetrahedra's);
  pri_x : the same prism pair extruded along x instead (quadrilateral faces on
        z = const planes), used to glue prisms to hexahedra;
  quad / hex : the cell itself.
"""
import itertools

import numpy as np

FACE_VERTS = {
    "tri": [(0, 1), (1, 2), (2, 0)],
    "quad": [(0, 1), (1, 2), (3, 2), (0, 3)],
    "tet": [(0, 1, 2), (0, 1, 3), (1, 2, 3), (0, 2, 3)],
    "pri": [(0, 1, 2), (0, 1, 4, 3), (1, 2, 5, 4), (0, 2, 5, 3), (3, 4, 5)],
    "hex": [(0, 1, 2, 3), (0, 1, 5, 4), (1, 2, 6, 5), (3, 2, 6, 7), (0, 3, 7, 4), (4, 5, 6, 7)],
}


def _cell_elements(kind):
    """Integer corner coordinates of the elements of one unit cell."""
    if kind == "quad":
        return "quad", [[(0, 0), (1, 0), (1, 1), (0, 1)]]
    if kind == "tri":
        return "tri", [[(0, 0), (1, 0), (1, 1)], [(0, 0), (1, 1), (0, 1)]]
    if kind == "hex":
        return "hex", [[(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
                        (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)]]
    if kind == "pri":
        out = []
        for t in ([(0, 0), (1, 0), (1, 1)], [(0, 0), (1, 1), (0, 1)]):
            out.append([(a, b, 0) for a, b in t] + [(a, b, 1) for a, b in t])
        return "pri", out
    if kind == "pri_x":
        # triangles in the (y, z) plane extruded along x
        out = []
        for t in ([(0, 0), (1, 0), (1, 1)], [(0, 0), (1, 1), (0, 1)]):
            out.append([(0, b, c) for b, c in t] + [(1, b, c) for b, c in t])
        return "pri", out
    if kind == "tet":
        out = []
        for perm in itertools.permutations(range(3)):
            v = [np.zeros(3, int)]
            for a in perm:
                nxt = v[-1].copy()
                nxt[a] += 1
                v.append(nxt)
            e1, e2, e3 = v[1] - v[0], v[2] - v[0], v[3] - v[0]
            if np.linalg.det(np.array([e1, e2, e3], float)) < 0:
                v[2], v[3] = v[3], v[2]
            out.append([tuple(int(c) for c in x) for x in v])
        return "tet", out
    raise ValueError(kind)


def _orient_ok(shape, corners):
    c = np.array(corners, float)
    if shape in ("tri", "quad"):
        e1 = c[1] - c[0]
        e2 = c[-1] - c[0] if shape == "quad" else c[2] - c[0]
        return e1[0] * e2[1] - e1[1] * e2[0] > 0
    if shape == "tet":
        return np.linalg.det(np.array([c[1] - c[0], c[2] - c[0], c[3] - c[0]])) > 0
    if shape == "pri":
        return np.linalg.det(np.array([c[1] - c[0], c[2] - c[0], c[3] - c[0]])) > 0
    if shape == "hex":
        return np.linalg.det(np.array([c[1] - c[0], c[3] - c[0], c[4] - c[0]])) > 0
    return True


def box_mesh(kinds, n, lo, hi):
    """Periodic box mesh.

    kinds : one cell kind ("tri", "quad", "tet", "pri", "pri_x", "hex") for the
            whole box, or a list of length n[-1] giving the kind of each slab of
            cells along the last axis (mixed meshes).
    n     : cells per axis (tuple of ND ints).
    """
    n = tuple(int(v) for v in n)
    nd = len(n)
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    h = (hi - lo) / np.array(n)
    if isinstance(kinds, str):
        kinds = [kinds] * n[-1]
    assert len(kinds) == n[-1]

    blocks = {}       # shape -> list of integer corner arrays
    order = []
    for cell in itertools.product(*[range(k) for k in n[::-1]]):
        cell = cell[::-1]                           # x fastest
        shape, elems = _cell_elements(kinds[cell[-1]])
        for corners in elems:
            assert _orient_ok(shape, corners), (shape, corners)
            if shape not in blocks:
                blocks[shape] = []
                order.append(shape)
            blocks[shape].append(np.array(corners, int) + np.array(cell, int))

    out_blocks = []
    int_blocks = []
    for shape in order:
        iv = np.array(blocks[shape])                # (E, nv, ND) integer
        int_blocks.append((shape, iv))
        out_blocks.append({"shape": shape, "verts": lo + iv * h})

    # Face adjacency through periodic integer keys.
    table = {}
    nn = np.array(n)
    for b, (shape, iv) in enumerate(int_blocks):
        for e in range(len(iv)):
            for f, fv in enumerate(FACE_VERTS[shape]):
                pts = iv[e, list(fv)]
                # vertex set modulo the box, plus the centroid modulo the box (the
                # vertex set alone aliases distinct faces when a box is 2 cells wide)
                csum = tuple(int(c) for c in (pts.sum(axis=0) % (len(fv) * nn)))
                key = (csum, tuple(sorted(tuple(int(c) for c in x) for x in (pts % nn))))
                table.setdefault(key, []).append((b, e, f, pts.mean(axis=0)))
    faces, shifts = [], []
    for key, lst in table.items():
        if len(lst) != 2:
            raise ValueError(f"non-manifold or unmatched face {key}: {len(lst)}")
        (bL, eL, fL, cL), (bR, eR, fR, cR) = lst
        faces.append((bL, eL, fL, bR, eR, fR))
        shifts.append(np.round((cL - cR) / nn) * nn * h)
    return {"blocks": out_blocks, "faces": np.array(faces, np.int64),
            "shift": np.array(shifts, float).reshape(-1, nd), "box": (lo, hi)}


def n_elements(mesh):
    return sum(len(b["verts"]) for b in mesh["blocks"])


def merge_meshes(parts):
    """Disconnected union of meshes (independent problems batched into one):
    blocks concatenated, face block indices offset, shifts kept."""
    blocks, faces, shifts = [], [], []
    nb = 0
    for m in parts:
        blocks.extend(m["blocks"])
        f = np.array(m["faces"], np.int64).copy()
        f[:, 0] += nb
        f[:, 3] += nb
        faces.append(f)
        shifts.append(m["shift"])
        nb += len(m["blocks"])
    return {"blocks": blocks, "faces": np.concatenate(faces), "shift": np.concatenate(shifts)}
