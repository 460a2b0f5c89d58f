"""Quadratic (curved) element mappings: shape functions and their derivatives.

Oracle (test infrastructure only).  The paper maps every element from its
reference element by a mapping function x = M(x~) with Jacobian
J_ij = dM_i / dx~_j, its determinant and inverse (Sec. 2, Eqs.
"mapping_function", "mapping_jacobian", "inverse_mapping_jacobian") and
evaluates the Jacobians analytically.  It does not fix the form of M; the
curved elements here use the second-order Lagrange mapping (reading):

  M(x~) = sum_k X_k N_k(x~),

with X_k the physical positions of the mapping nodes and N_k the Lagrange
basis of the element type's quadratic space on those nodes:
  tri / tet    polynomials of total degree <= 2,
  quad / hex   polynomials of degree <= 2 in each coordinate,
  pri          (total degree <= 2 in x~, y~) x (degree <= 2 in z~).
The mapping nodes are the points of the reference element whose coordinates
all lie in {-1, 0, 1}, in lexicographic order with x~ fastest (tri 6, quad 9,
tet 10, pri 18, hex 27 nodes); the element's vertices are among them.

Here the basis is built by inverting the Vandermonde matrix of the space's
monomials at the nodes (N = m(x) V^{-1}), and its gradient follows from the
monomials' exact derivatives.

Parity: pinned by the Kronecker property at the nodes, the reproduction of
every quadratic of the space, central finite differences of the
derivatives, and, through the geometry built on it, the exact volume of a
curved periodic box and free-stream preservation
(tests/test_oracle_curved.py).
"""
import itertools

import numpy as np

from . import points

ND = {"tri": 2, "quad": 2, "tet": 3, "pri": 3, "hex": 3}


def _inside(shape, x):
    if shape in ("quad", "hex"):
        return True
    if shape == "tri":
        return x[0] + x[1] <= 0
    if shape == "tet":
        return x[0] + x[1] + x[2] <= -1
    return x[0] + x[1] <= 0                    # prism: triangle cross-section


def nodes(shape):
    """Mapping nodes (NN, ND) of an element type, x~ fastest."""
    nd = ND[shape]
    out = []
    for c in itertools.product((-1.0, 0.0, 1.0), repeat=nd):
        x = c[::-1]                            # last index slowest -> x fastest
        if _inside(shape, x):
            out.append(x)
    return np.array(out)


def exponents(shape):
    """Monomial exponents spanning the element type's quadratic space."""
    nd = ND[shape]
    out = []
    for a in itertools.product(range(3), repeat=nd):
        if shape in ("tri", "tet") and sum(a) > 2:
            continue
        if shape == "pri" and a[0] + a[1] > 2:
            continue
        out.append(a)
    return np.array(out)


def _monomials(E, X):
    """m (npts, nm) and dm (npts, nm, ND)."""
    X = np.atleast_2d(X)
    npts, nd = X.shape
    m = np.ones((npts, len(E)))
    dm = np.zeros((npts, len(E), nd))
    for j, a in enumerate(E):
        for d in range(nd):
            m[:, j] *= X[:, d] ** a[d]
        for k in range(nd):
            if a[k] == 0:
                continue
            t = a[k] * X[:, k] ** (a[k] - 1)
            for d in range(nd):
                if d != k:
                    t = t * X[:, d] ** a[d]
            dm[:, j, k] = t
    return m, dm


def shape_functions(shape, X):
    """N (npts, NN) and dN (npts, NN, ND) = dN_k / dx~_d at reference points X."""
    E = exponents(shape)
    V, _ = _monomials(E, nodes(shape))         # V[i, j] = m_j(node_i)
    Vinv = np.linalg.inv(V)
    m, dm = _monomials(E, X)
    return m @ Vinv, np.einsum("pjd,jk->pkd", dm, Vinv)


def affine_nodes(shape, verts):
    """Nodes of the straight (affine) element with the given vertices (E, nv, ND):
    the affine image of the reference nodes."""
    ref = points.VERTS[shape]
    A = np.column_stack([ref, np.ones(len(ref))])
    Xn = nodes(shape)
    out = np.empty((verts.shape[0], len(Xn), verts.shape[2]))
    An = np.column_stack([Xn, np.ones(len(Xn))])
    for e in range(verts.shape[0]):
        C = np.linalg.lstsq(A, verts[e], rcond=None)[0]
        out[e] = An @ C
    return out


def jacobians(shape, Xnodes, X):
    """Physical positions (E, npts, ND) and Jacobians J_ij = dx_i / dx~_j
    (E, npts, ND, ND) of the quadratic map at reference points X."""
    N, dN = shape_functions(shape, X)
    x = np.einsum("pk,eki->epi", N, Xnodes)
    J = np.einsum("pkj,eki->epij", dN, Xnodes)
    return x, J
