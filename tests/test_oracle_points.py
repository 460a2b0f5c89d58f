"""Pins of the oracle's point sets: the paper's point-count tables, symmetry of
face point sets (needed for conforming pairing), interiority and unisolvence."""
import itertools
import os

import numpy as np
import pytest

from oracle import bases, operators, points

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "point_counts.txt")


def _table():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        s, p, *v = line.split()
        rows.append((s, int(p), tuple(int(x) for x in v)))
    return rows


@pytest.mark.parametrize("shape,p,vals", _table())
def test_counts_match_paper_tables(shape, p, vals):
    n_sol, n_flux, n_fe, n_fi, n_fiu = vals
    assert n_flux == n_fe + n_fi
    assert points.counts(shape, p) == (n_sol, n_fe, n_fi, n_fiu)
    # dim RT_p equals the number of flux DOFs (App. A)
    assert len(bases.rt_modes(shape, p)) == n_flux
    assert len(bases.sol_exponents(shape, p)) == n_sol


def _inside(shape, X, strict_tol=1e-12):
    if shape == "tri":
        return np.all(X >= -1 - strict_tol) and np.all(X.sum(1) <= strict_tol)
    if shape == "tet":
        return np.all(X >= -1 - strict_tol) and np.all(X.sum(1) <= -1 + strict_tol)
    if shape == "pri":
        return np.all(X >= -1 - strict_tol) and np.all(X[:, :2].sum(1) <= strict_tol) \
            and np.all(X[:, 2] <= 1 + strict_tol)
    return np.all(np.abs(X) <= 1 + strict_tol)


@pytest.mark.parametrize("shape", points.SHAPES)
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_points_inside_and_on_faces(shape, p):
    assert _inside(shape, points.sol_points(shape, p))
    xu, _, _ = points.internal_points(shape, p)
    assert _inside(shape, xu)
    xfe, nfe, face = points.ext_points(shape, p)
    # every external point lies on the plane of its face
    for f, (vids, _) in enumerate(points.FACES[shape]):
        V = points.VERTS[shape][list(vids)]
        n = points.face_normal(shape, f)
        d = (xfe[face == f] - V[0]) @ n
        assert np.abs(d).max() < 1e-14
        assert np.allclose(nfe[face == f], n)


def _tri_perms(q):
    lam = points.tri_bary(q)
    keyset = {tuple(np.round(l, 12)) for l in lam}
    for perm in itertools.permutations(range(3)):
        perm_set = {tuple(np.round(l[list(perm)], 12)) for l in lam}
        assert perm_set == keyset


@pytest.mark.parametrize("q", [0, 1, 2, 3, 4])
def test_triangle_set_symmetric(q):
    """Invariance under all 6 vertex permutations: any glued pair of triangular
    faces then sees coincident points whatever their relative orientation."""
    _tri_perms(q)


@pytest.mark.parametrize("q", [0, 1, 2, 3])
def test_tet_set_symmetric(q):
    lam = points.tet_bary(q)
    keyset = {tuple(np.round(l, 12)) for l in lam}
    for perm in itertools.permutations(range(4)):
        assert {tuple(np.round(l[list(perm)], 12)) for l in lam} == keyset


def test_equispaced_lattice_limit():
    """The warped lattice reduces to the principal lattice for equispaced nodes:
    check the construction formula on q = 1 (GL nodes of 2 points, barycentric
    coordinates of each point must be a convex combination summing to 1)."""
    for q in range(0, 6):
        lam = points.tri_bary(q)
        assert np.allclose(lam.sum(1), 1) and lam.min() > 0
        lam = points.tet_bary(q)
        assert np.allclose(lam.sum(1), 1) and lam.min() > 0


@pytest.mark.parametrize("shape", points.SHAPES)
@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_unisolvent(shape, p):
    op = operators.get(shape, p)
    assert op.cond_sol < 1e6
    assert op.cond_flux < 1e6
