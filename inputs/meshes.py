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


# Reference vertices of each element type (the vertex order above).
_REF_VERTS = {
    "tri": [(-1, -1), (1, -1), (-1, 1)],
    "quad": [(-1, -1), (1, -1), (1, 1), (-1, 1)],
    "tet": [(-1, -1, -1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1)],
    "pri": [(-1, -1, -1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1), (1, -1, 1), (-1, 1, 1)],
    "hex": [(-1, -1, -1), (1, -1, -1), (1, 1, -1), (-1, 1, -1), (-1, -1, 1), (1, -1, 1), (1, 1, 1), (-1, 1, 1)],
}


def map_nodes(shape):
    """Reference positions of the nodes of a curved element's quadratic map:
    the points of the reference element with every coordinate in {-1, 0, 1},
    lexicographic with x fastest (tri 6, quad 9, tet 10, pri 18, hex 27)."""
    nd = len(_REF_VERTS[shape][0])
    out = []
    for c in itertools.product((-1, 0, 1), repeat=nd):
        x = c[::-1]
        s = sum(x[:2])
        if shape == "tet":
            s = sum(x) + 1
        if shape in ("quad", "hex") or s <= 0:
            out.append(x)
    return np.array(out, float)


def curved_mesh(mesh, amp, seed=None):
    """The mesh with every element curved: each block gains "nodes" (E, NN, ND),
    the nodes of its straight element moved by the smooth periodic displacement
      2D  d = amp L (sin(2 pi y~) , sin(2 pi x~)),
      3D  d = amp L (sin(2 pi y~) sin(2 pi z~), sin(2 pi z~) sin(2 pi x~), sin(2 pi x~) sin(2 pi y~)),
    x~ = (x - lo) / L per axis (L the box size along each axis; a phase drawn
    from seed shifts each sine when given).  Vertices move too ("verts" is
    updated), faces and periodic shifts are unchanged: the displacement is
    periodic, so glued faces keep coincident points."""
    lo, hi = (np.asarray(v, float) for v in mesh["box"])
    L = hi - lo
    nd = len(L)
    ph = np.zeros(nd) if seed is None else np.random.default_rng(seed).uniform(0, 2 * np.pi, nd)

    def disp(x):
        t = 2 * np.pi * (x - lo) / L + ph
        s = np.sin(t)
        if nd == 2:
            return amp * L * np.stack([s[..., 1], s[..., 0]], axis=-1)
        return amp * L * np.stack([s[..., 1] * s[..., 2], s[..., 2] * s[..., 0], s[..., 0] * s[..., 1]], axis=-1)

    blocks = []
    for blk in mesh["blocks"]:
        shape = blk["shape"]
        ref = np.array(_REF_VERTS[shape], float)
        A = np.column_stack([ref, np.ones(len(ref))])
        Xn = map_nodes(shape)
        An = np.column_stack([Xn, np.ones(len(Xn))])
        V = np.asarray(blk["verts"], float)
        nodes = np.empty((len(V), len(Xn), nd))
        for e in range(len(V)):
            C = np.linalg.lstsq(A, V[e], rcond=None)[0]
            nodes[e] = An @ C
        nodes = nodes + disp(nodes)
        vidx = [int(np.nonzero((Xn == r).all(axis=1))[0][0]) for r in ref]
        blocks.append({"shape": shape, "verts": nodes[:, vidx].copy(), "nodes": nodes})
    out = dict(mesh)
    out["blocks"] = blocks
    return out
