"""Pins of the oracle's curved (quadratic isoparametric) elements against what
the mathematics fixes (paper Sec. 2: mapping, Jacobian, inverse Jacobian and
the transformed quantities, evaluated analytically at every point the method
uses them; Sec. 2.1 for where each metric enters):

  * the quadratic shape functions: Kronecker property at the mapping nodes,
    exact reproduction of the element type's quadratic space, derivatives
    against central differences;
  * straight elements given as nodes give the affine oracle's residual;
  * the mapped volume of a curved periodic box is the box volume (a periodic
    displacement moves no volume), element quadrature of degree 10;
  * free-stream preservation: the cofactor matrix det J J^{-1} of a quadratic
    map is a quadratic polynomial with divergence-free rows, so the RT
    interpolant of the transformed constant flux is exact for p >= 2 on
    tetrahedra (p >= 1 on triangles, where the cofactors are linear) and the
    residual of a uniform state vanishes; for p = 1 on curved tetrahedra it
    does not (the test can fail);
  * discrete conservation with the per-point det J;
  * the LDG gradient of a field linear in the physical coordinates is exact
    in elements none of whose faces is periodic (J^{-T} at each solution
    point; a transposed J fails);
  * convergence of linear advection on curved tetrahedra.
"""
import numpy as np
import pytest

from inputs import meshes
from oracle import mapping
from oracle import mesh as omesh
from oracle import operators
from oracle import physics as phx
from oracle import residual as ores
from tests import quadrature

SHAPES = ["tri", "quad", "tet", "pri", "hex"]
N2 = {"tri": (3, 3), "quad": (3, 3), "tet": (2, 2, 2), "pri": (2, 2, 2), "hex": (2, 2, 2)}
AMP = 0.04


def _curved(shape, n=None, amp=AMP, seed=None):
    n = n or N2[shape]
    nd = len(n)
    m = meshes.box_mesh(shape, n, [0.0] * nd, [1.0] * nd)
    return meshes.curved_mesh(m, amp, seed)


def _eval(geom, fn, nvar):
    out = []
    for g in geom.blocks:
        X = g.xsol.reshape(-1, g.xsol.shape[-1])
        v = fn(X).reshape(g.nelem, g.ops.n_sol, nvar)
        out.append(np.ascontiguousarray(np.transpose(v, (1, 2, 0))))
    return out


@pytest.mark.parametrize("shape", SHAPES)
def test_shape_functions(shape):
    Xn = mapping.nodes(shape)
    N, dN = mapping.shape_functions(shape, Xn)
    assert np.allclose(N, np.eye(len(Xn)), atol=1e-13)
    rng = np.random.default_rng(3)
    nd = Xn.shape[1]
    # random points inside the reference element
    X = rng.uniform(-1, 1, (40, nd))
    if shape in ("tri", "pri"):
        X = X[X[:, 0] + X[:, 1] <= 0]
    if shape == "tet":
        X = X[X.sum(axis=1) <= -1]
    N, dN = mapping.shape_functions(shape, X)
    for a in mapping.exponents(shape):
        f = lambda Y: np.prod(Y ** a, axis=1)             # noqa: E731
        assert np.allclose(N @ f(Xn), f(X), atol=1e-12)
    h = 1e-6
    for d in range(nd):
        e = np.zeros(nd)
        e[d] = h
        fd = (mapping.shape_functions(shape, X + e)[0] - mapping.shape_functions(shape, X - e)[0]) / (2 * h)
        assert np.allclose(dN[:, :, d], fd, atol=1e-8)


@pytest.mark.parametrize("shape", SHAPES)
def test_straight_nodes_give_the_affine_residual(shape):
    n = N2[shape]
    nd = len(n)
    m = meshes.box_mesh(shape, n, [0.0] * nd, [1.0] * nd)
    mc = meshes.curved_mesh(m, 0.0)
    p = 2
    ga, gc = omesh.build(m, p), omesh.build(mc, p)
    assert gc.blocks[0].curved and not ga.blocks[0].curved
    ph = phx.Physics("euler", nd, "rusanov")
    rng = np.random.default_rng(5)
    state = [1.2, 0.3, -0.2, 3.0] if nd == 2 else [1.2, 0.3, -0.2, 0.1, 3.0]
    U = [np.asarray(state)[None, :, None] * (1 + 0.05 * rng.uniform(-1, 1, (g.ops.n_sol, nd + 2, g.nelem)))
         for g in ga.blocks]
    Ra, Rc = ores.residual(ga, ph, U), ores.residual(gc, ph, U)
    for a, c in zip(Ra, Rc):
        assert np.abs(a - c).max() <= 1e-11 * np.abs(a).max()
    assert np.array_equal(ga.partner, gc.partner)


@pytest.mark.parametrize("shape", SHAPES)
def test_curved_box_volume(shape):
    mc = _curved(shape, seed=11)
    nd = len(N2[shape])
    Xq, Wq = quadrature.rule(shape, 10)
    vol = 0.0
    for blk in mc["blocks"]:
        _, J = mapping.jacobians(shape, blk["nodes"], Xq)
        det = np.linalg.det(J)
        assert det.min() > 0
        vol += np.einsum("q,eq->", Wq, det)
    assert vol == pytest.approx(1.0, abs=1e-12)
    # the displacement is not a rigid motion: det J varies within elements
    assert np.ptp(det, axis=1).max() > 1e-3


@pytest.mark.parametrize("shape,p,exact", [("tet", 2, True), ("tet", 3, True), ("tri", 1, True),
                                           ("tri", 2, True), ("tet", 1, False)])
def test_free_stream_on_curved_simplices(shape, p, exact):
    geom = omesh.build(_curved(shape), p)
    nd = geom.nd
    ph = phx.Physics("euler", nd, "rusanov")
    state = np.array([1.2, 0.3, -0.2, 3.0] if nd == 2 else [1.2, 0.3, -0.2, 0.1, 3.0])
    U = [np.repeat(state[None, :, None], g.nelem, 2).repeat(g.ops.n_sol, 0) for g in geom.blocks]
    R = ores.residual(geom, ph, U)
    err = max(np.abs(r).max() for r in R)
    if exact:
        assert err < 1e-11, err
    else:
        assert err > 1e-4, err


def _weights(g):
    Xq, Wq = quadrature.rule(g.shape, 10)
    return Wq @ operators.nodal_sol(g.shape, g.p, g.ops.xs, Xq)


@pytest.mark.parametrize("shape,p", [(s, p) for s in SHAPES for p in (1, 3)])
def test_conservation_on_curved_meshes(shape, p):
    """sum_e sum_s w_s det J_s dU/dt_s = -sum_e (boundary flux integrals) = 0:
    the common flux is single-valued per face and each side's det J |J^{-T} n~|
    is its own surface element."""
    geom = omesh.build(_curved(shape, seed=2), p)
    nd = geom.nd
    ph = phx.Physics("euler", nd, "rusanov")
    state = np.array([1.2, 0.3, -0.2, 3.0] if nd == 2 else [1.2, 0.3, -0.2, 0.1, 3.0])
    rng = np.random.default_rng(9)
    U = [state[None, :, None] * (1 + 0.1 * rng.uniform(-1, 1, (g.ops.n_sol, nd + 2, g.nelem))) for g in geom.blocks]
    R = ores.residual(geom, ph, U)
    tot = sum(np.einsum("s,sve,es->v", _weights(g), r, g.dets) for g, r in zip(geom.blocks, R))
    scale = max(np.abs(r).max() for r in R)
    assert np.abs(tot).max() < 1e-12 * scale, (tot, scale)


@pytest.mark.parametrize("shape,p", [("tet", 2), ("tet", 3), ("tri", 2), ("hex", 2), ("pri", 2)])
def test_linear_field_gradient_exact_away_from_periodic_faces(shape, p):
    n = (3, 3) if len(N2[shape]) == 2 else (3, 3, 3)
    mc = _curved(shape, n=n, seed=4)
    geom = omesh.build(mc, p)
    nd = geom.nd
    a = np.array([0.7, -1.3, 0.4][:nd])
    ph = phx.Physics("advdiff", nd, "upwind", a=(1.0, 0.5, 0.25), mu=0.1, beta=0.3, eta=0.1)
    U = _eval(geom, lambda X: (X @ a + 0.25)[:, None], 1)
    Q = ores.solution_gradients(geom, ph, U)
    # elements none of whose faces is periodic (both traces of every face are
    # the same continuous linear field)
    inner = [np.ones(g.nelem, bool) for g in geom.blocks]
    for (bL, eL, fL, bR, eR, fR), s in zip(mc["faces"], mc["shift"]):
        if np.abs(s).max() > 0:
            inner[bL][eL] = False
            inner[bR][eR] = False
    checked = 0
    for g, q, ok in zip(geom.blocks, Q, inner):
        got = q[:, :, 0, ok]                                    # (ND, N_s, E_inner)
        assert np.abs(got - a[:, None, None]).max() < 1e-11
        checked += ok.sum()
    assert checked > 0


def test_advection_converges_on_curved_tetrahedra():
    """dU/dt of u = sin(2 pi x) against -a . grad u at the solution points
    (p = 3): on curved tetrahedra the error falls by more than 3.5 from 2 to 4
    cells per axis (the affine mesh: 8.7) and stays within 2.5 times the affine
    mesh's error."""
    a = np.array([1.0, 0.5, 0.25])
    k = 2 * np.pi
    errs = {}
    for amp in (0.0, 0.03):
        for n in (2, 4):
            m = meshes.box_mesh("tet", (n, n, n), [0.0] * 3, [1.0] * 3)
            geom = omesh.build(meshes.curved_mesh(m, amp), 3)
            ph = phx.Physics("advection", 3, "upwind", a=tuple(a))
            U = _eval(geom, lambda X: np.sin(k * X[:, 0])[:, None], 1)
            exact = _eval(geom, lambda X: (-a[0] * k * np.cos(k * X[:, 0]))[:, None], 1)
            R = ores.residual(geom, ph, U)
            errs[amp, n] = max(np.abs(r - x).max() for r, x in zip(R, exact))
    assert errs[0.03, 2] / errs[0.03, 4] > 3.5, errs
    assert errs[0.03, 4] < 2.5 * errs[0.0, 4], errs
