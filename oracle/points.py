"""Reference elements, solution points and flux points with their degrees of freedom.

Oracle (test infrastructure only).  Follows paper App. A:
  * reference triangle / tetrahedron: x_i >= -1 with the slanted facet through
    (1,-1[,-1]) (App. A, "Triangles and Tetrahedrons elements"; the printed
    inequality "sum x_i <= 0" is only right for the triangle; for the tetrahedron
    we take sum x_i <= -1, whose vertices are (-1,-1,-1), (1,-1,-1), (-1,1,-1),
    (-1,-1,1));
  * quadrilateral / hexahedron: [-1, 1]^ND (App. A, "Tensor-product elements");
  * prism: triangle x [-1, 1] (App. A, "Triangular prismatic elements").

Point sets (App. A):
  * tensor-product elements: Gauss-Legendre (GL) solution points, GL external
    flux points, internal flux points along axis d at the p-point GL rule in d
    times the (p+1)-point GL rule in the other axes, one DOF along e_d;
  * simplices: the paper places solution, internal and triangular-face points at
    Williams-Shunn quadrature points, whose coordinates are not printed in the
    paper.  We substitute a derivable, fully symmetric, unisolvent family: the
    barycentric lattice of degree q warped by the (q+1)-point GL rule,
        lambda_a = (1 + m v_{i_a} - sum_{b != a} v_{i_b}) / (m + 1),
    with multi-index i (|i| = q), v the GL nodes mapped to [0, 1] and m = 2
    (triangle) or 3 (tetrahedron).  For equispaced v this is the principal
    lattice; with GL nodes every point is strictly inside.  Counts are the
    paper's: (q+1)(q+2)/2 and (q+1)(q+2)(q+3)/6.
  * triangle: p+1 GL points per edge; internal flux points = triangle set of
    degree p-1 with DOFs along x and y.
  * tetrahedron: triangle set of degree p on every face; internal = tetrahedron
    set of degree p-1 with DOFs along x, y, z.
  * prism: triangle faces carry the triangle set of degree p, quadrilateral faces
    a (p+1)^2 GL grid; internal group 1 = triangle internal set x (p+1) GL levels
    in z with DOFs along x and y; group 2 = triangle face set x p GL levels in z
    with one DOF along z.

Ordering conventions (shared, as a written convention only, with the library):
  * GL nodes ascending; tensor grids with x fastest, then y, then z;
  * triangle set: multi-index (a, b, c), a + b + c = q, b outer, a inner,
    lambda_1 <- a, lambda_2 <- b, lambda_0 <- c, point = sum_k lambda_k V_k;
  * tetrahedron set: (a, b, c, d), c outer, b, a inner; lambda_1 <- a,
    lambda_2 <- b, lambda_3 <- c, lambda_0 <- d;
  * external flux points face by face (face order below), points inside a face
    in the order of that face's parametrisation;
  * internal DOFs: direction outer, unique point inner (simplices); axis blocks
    (tensor-product); prism: group-1 x, group-1 y, group-2 z.

Parity: pinned by the point-count tables (App. A Tables "nsolpts_nfpts",
"nfpts_extra"), symmetry and interiority tests, and unisolvence of the
Vandermonde matrices (tests/test_oracle_points.py).
"""
import numpy as np

SHAPES = ("tri", "quad", "tet", "pri", "hex")
NDIM = {"tri": 2, "quad": 2, "tet": 3, "pri": 3, "hex": 3}

# Reference vertices.
VERTS = {
    "tri": np.array([[-1, -1], [1, -1], [-1, 1]], float),
    "quad": np.array([[-1, -1], [1, -1], [1, 1], [-1, 1]], float),
    "tet": np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], float),
    "pri": np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1],
                     [-1, -1, 1], [1, -1, 1], [-1, 1, 1]], float),
    "hex": np.array([[-1, -1, -1], [1, -1, -1], [1, 1, -1], [-1, 1, -1],
                     [-1, -1, 1], [1, -1, 1], [1, 1, 1], [-1, 1, 1]], float),
}

# Faces: (vertex indices, outward reference normal before normalisation).
FACES = {
    "tri": [((0, 1), (0, -1)), ((1, 2), (1, 1)), ((2, 0), (-1, 0))],
    "quad": [((0, 1), (0, -1)), ((1, 2), (1, 0)), ((3, 2), (0, 1)), ((0, 3), (-1, 0))],
    "tet": [((0, 1, 2), (0, 0, -1)), ((0, 1, 3), (0, -1, 0)),
            ((1, 2, 3), (1, 1, 1)), ((0, 2, 3), (-1, 0, 0))],
    "hex": [((0, 1, 2, 3), (0, 0, -1)), ((0, 1, 5, 4), (0, -1, 0)),
            ((1, 2, 6, 5), (1, 0, 0)), ((3, 2, 6, 7), (0, 1, 0)),
            ((0, 3, 7, 4), (-1, 0, 0)), ((4, 5, 6, 7), (0, 0, 1))],
    "pri": [((0, 1, 2), (0, 0, -1)), ((0, 1, 4, 3), (0, -1, 0)),
            ((1, 2, 5, 4), (1, 1, 0)), ((0, 2, 5, 3), (-1, 0, 0)),
            ((3, 4, 5), (0, 0, 1))],
}


def gauss_legendre(n):
    """n-point Gauss-Legendre nodes on [-1, 1], ascending (library routine)."""
    x, _ = np.polynomial.legendre.leggauss(n)
    return np.sort(x)


def _unit_nodes(q):
    return (gauss_legendre(q + 1) + 1.0) / 2.0


def tri_bary(q):
    """Barycentric coordinates (l0, l1, l2) of the warped triangle lattice of degree q."""
    v = _unit_nodes(q)
    out = []
    for b in range(q + 1):
        for a in range(q + 1 - b):
            c = q - a - b
            l1 = (1 + 2 * v[a] - v[b] - v[c]) / 3
            l2 = (1 + 2 * v[b] - v[a] - v[c]) / 3
            l0 = (1 + 2 * v[c] - v[a] - v[b]) / 3
            out.append((l0, l1, l2))
    return np.array(out).reshape(-1, 3)


def tet_bary(q):
    """Barycentric coordinates (l0, l1, l2, l3) of the warped tetrahedron lattice of degree q."""
    v = _unit_nodes(q)
    out = []
    for c in range(q + 1):
        for b in range(q + 1 - c):
            for a in range(q + 1 - c - b):
                d = q - a - b - c
                idx = (d, a, b, c)
                lam = []
                for k in range(4):
                    others = sum(v[idx[j]] for j in range(4) if j != k)
                    lam.append((1 + 3 * v[idx[k]] - others) / 4)
                out.append(lam)
    return np.array(out).reshape(-1, 4)


def tri_set(q):
    """Triangle set of degree q in reference coordinates."""
    return tri_bary(q) @ VERTS["tri"]


def tet_set(q):
    return tet_bary(q) @ VERTS["tet"]


def _grid(axes):
    """Tensor grid with the first axis fastest. axes: list of 1D arrays."""
    mesh = np.meshgrid(*axes[::-1], indexing="ij")
    return np.stack([m.ravel() for m in mesh[::-1]], axis=1)


def sol_points(shape, p):
    g = gauss_legendre(p + 1)
    if shape == "tri":
        return tri_set(p)
    if shape == "tet":
        return tet_set(p)
    if shape == "quad":
        return _grid([g, g])
    if shape == "hex":
        return _grid([g, g, g])
    if shape == "pri":
        t = tri_set(p)
        return np.vstack([np.column_stack([t, np.full(len(t), z)]) for z in g])
    raise ValueError(shape)


def face_points(shape, p, f):
    """Reference coordinates of the external flux points of face f (paper App. A)."""
    vids, _ = FACES[shape][f]
    V = VERTS[shape]
    g = gauss_legendre(p + 1)
    if shape in ("tri",):
        A, B = V[vids[0]], V[vids[1]]
        return np.array([A + (B - A) * (1 + t) / 2 for t in g])
    if shape == "quad":
        A, B = V[vids[0]], V[vids[1]]
        return np.array([A + (B - A) * (1 + t) / 2 for t in g])
    if shape == "tet":
        return tri_bary(p) @ V[list(vids)]
    if shape == "hex":
        n = np.array(FACES[shape][f][1], float)
        fixed = int(np.argmax(np.abs(n)))
        free = [a for a in range(3) if a != fixed]
        pts = np.zeros(((p + 1) ** 2, 3))
        uv = _grid([g, g])
        pts[:, free[0]] = uv[:, 0]
        pts[:, free[1]] = uv[:, 1]
        pts[:, fixed] = n[fixed]
        return pts
    if shape == "pri":
        if len(vids) == 3:
            return tri_bary(p) @ V[list(vids)]
        # quadrilateral face: edge (first two vertices, bottom) fastest, z outer
        A, B = V[vids[0]][:2], V[vids[1]][:2]
        out = []
        for z in g:
            for t in g:
                xy = A + (B - A) * (1 + t) / 2
                out.append((xy[0], xy[1], z))
        return np.array(out)
    raise ValueError(shape)


def face_normal(shape, f):
    n = np.array(FACES[shape][f][1], float)
    return n / np.linalg.norm(n)


def ext_points(shape, p):
    """External flux points: coordinates (N_fe, ND), unit reference normals, face index."""
    xs, ns, fs = [], [], []
    for f in range(len(FACES[shape])):
        x = face_points(shape, p, f)
        xs.append(x)
        ns.append(np.tile(face_normal(shape, f), (len(x), 1)))
        fs.append(np.full(len(x), f))
    return np.vstack(xs), np.vstack(ns), np.concatenate(fs)


def internal_points(shape, p):
    """Unique internal flux points (N_fiu, ND) and internal DOFs.

    Returns (xu, dof_point, dof_dir): dof_point[nu] is the unique-point index of
    internal DOF nu and dof_dir[nu] its reference direction (a unit axis vector).
    """
    nd = NDIM[shape]
    eye = np.eye(nd)
    if shape in ("tri", "tet"):
        xu = tri_set(p - 1) if shape == "tri" else tet_set(p - 1)
        k = np.arange(len(xu))
        dof_point = np.concatenate([k] * nd)
        dof_dir = np.vstack([np.tile(eye[d], (len(xu), 1)) for d in range(nd)])
        return xu, dof_point, dof_dir
    if shape in ("quad", "hex"):
        gi = gauss_legendre(p)
        g = gauss_legendre(p + 1)
        blocks, dirs = [], []
        for d in range(nd):
            axes = [gi if a == d else g for a in range(nd)]
            pts = _grid(axes)
            blocks.append(pts)
            dirs.append(np.tile(eye[d], (len(pts), 1)))
        xu = np.vstack(blocks)
        return xu, np.arange(len(xu)), np.vstack(dirs)
    if shape == "pri":
        g = gauss_legendre(p + 1)
        gi = gauss_legendre(p)
        t1 = tri_set(p - 1)
        t2 = tri_set(p)
        g1 = np.vstack([np.column_stack([t1, np.full(len(t1), z)]) for z in g]).reshape(-1, 3)
        g2 = np.vstack([np.column_stack([t2, np.full(len(t2), z)]) for z in gi]).reshape(-1, 3)
        xu = np.vstack([g1, g2])
        n1, n2 = len(g1), len(g2)
        dof_point = np.concatenate([np.arange(n1), np.arange(n1), n1 + np.arange(n2)])
        dof_dir = np.vstack([np.tile(eye[0], (n1, 1)), np.tile(eye[1], (n1, 1)),
                             np.tile(eye[2], (n2, 1))])
        return xu, dof_point, dof_dir
    raise ValueError(shape)


def counts(shape, p):
    """(N_sol, N_fe, N_fi, N_fiu) built from the point sets themselves."""
    xu, dof_point, _ = internal_points(shape, p)
    return (len(sol_points(shape, p)), len(ext_points(shape, p)[0]), len(dof_point), len(xu))
