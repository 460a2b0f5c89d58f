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

    Elements: cells in lexicographic order (x fastest), within a cell in the
    order of its subdivision, grouped into one block per shape (blocks in the
    order the shapes first appear).  Faces: one row per glued pair, in the
    order of the first appearance of the face (blocks, elements, local faces
    in order); the first appearance is the L side.
    """
    n = tuple(int(v) for v in n)
    nd = len(n)
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    h = (hi - lo) / np.array(n)
    if isinstance(kinds, str):
        kinds = [kinds] * n[-1]
    assert len(kinds) == n[-1]

    # cells in order, x fastest
    grids = np.meshgrid(*[np.arange(k) for k in n], indexing="ij")
    cells = np.stack([g.transpose(tuple(range(nd))[::-1]).ravel() for g in grids], axis=1)   # (Ncell, ND)
    slab = cells[:, -1]
    # (shape -> list of (sort key, integer corners)) over the cells of every kind
    per_shape = {}
    for kind in dict.fromkeys(kinds):
        shape, elems = _cell_elements(kind)
        sel = np.nonzero(np.array([kinds[z] == kind for z in range(n[-1])])[slab])[0]
        for j, corners in enumerate(elems):
            assert _orient_ok(shape, corners), (shape, corners)
            iv = cells[sel][:, None, :] + np.asarray(corners, int)[None, :, :]
            per_shape.setdefault(shape, []).append((sel * 16 + j, iv))
    first = {s: min(int(k.min()) for k, _ in lst) for s, lst in per_shape.items()}
    order = sorted(per_shape, key=lambda s: first[s])
    int_blocks, out_blocks = [], []
    for shape in order:
        keys = np.concatenate([k for k, _ in per_shape[shape]])
        ivs = np.concatenate([v for _, v in per_shape[shape]])
        iv = ivs[np.argsort(keys, kind="stable")]
        int_blocks.append((shape, iv))
        out_blocks.append({"shape": shape, "verts": lo + iv * h})

    # Face adjacency through periodic integer keys: the vertex set modulo the
    # box plus the centroid sum modulo the box (the vertex set alone aliases
    # distinct faces when a box is 2 cells wide).
    nn = np.array(n)
    radix = np.cumprod(np.concatenate([[1], nn[:-1]]))
    recs = []          # (key rows, b, e, f, centroid)
    for b, (shape, iv) in enumerate(int_blocks):
        E = len(iv)
        for f, fv in enumerate(FACE_VERTS[shape]):
            k = len(fv)
            pts = iv[:, list(fv)]                                   # (E, k, ND)
            csum = pts.sum(axis=1) % (k * nn)
            codes = np.sort(((pts % nn) * radix).sum(axis=2), axis=1)
            key = np.full((E, 1 + nd + 4), -1, np.int64)
            key[:, 0] = k
            key[:, 1:1 + nd] = csum
            key[:, 1 + nd:1 + nd + k] = codes
            recs.append((key, np.full(E, b), np.arange(E), np.full(E, f), pts.mean(axis=1)))
    K = np.concatenate([r[0] for r in recs])
    B = np.concatenate([r[1] for r in recs])
    El = np.concatenate([r[2] for r in recs])
    F = np.concatenate([r[3] for r in recs])
    C = np.concatenate([r[4] for r in recs])
    # appearance order: blocks, elements, local faces
    seq = np.lexsort((F, El, B))
    rank = np.empty(len(seq), np.int64)
    rank[seq] = np.arange(len(seq))
    srt = np.lexsort((rank,) + tuple(K[:, c] for c in range(K.shape[1] - 1, -1, -1)))   # by key, then appearance
    Ks = K[srt]
    same_next = np.all(Ks[1:] == Ks[:-1], axis=1)
    starts = np.nonzero(np.concatenate([[True], ~same_next]))[0]
    counts = np.diff(np.concatenate([starts, [len(srt)]]))
    if np.any(counts != 2):
        bad = starts[counts != 2][0]
        raise ValueError(f"non-manifold or unmatched face {tuple(Ks[bad])}: {counts[counts != 2][0]}")
    iL, iR = srt[starts], srt[starts + 1]                       # L: first appearance
    pair_order = np.argsort(rank[iL], kind="stable")
    iL, iR = iL[pair_order], iR[pair_order]
    faces = np.stack([B[iL], El[iL], F[iL], B[iR], El[iR], F[iR]], axis=1).astype(np.int64)
    shifts = np.round((C[iL] - C[iR]) / nn) * nn * h
    return {"blocks": out_blocks, "faces": faces, "shift": np.asarray(shifts, float).reshape(-1, nd),
            "box": (lo, hi)}


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
