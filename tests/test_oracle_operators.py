"""Pins of the oracle's operators against closed forms computed with sympy
(independent of the oracle's monomial bases) and an independent quadrature:
  * M0 / M12 reproduce every member of the solution space exactly;
  * [M14 M13] applied to the normal components of any RT_p field gives its exact
    divergence at the solution points (App. A: div RT_p = solution space);
  * M16 / M15 give the exact reference gradient of any solution-space member;
  * internal flux basis functions have zero net outflow (zero normal trace);
  * D_sol differentiates the solution space exactly.
"""
import numpy as np
import pytest
import sympy as sp

from oracle import operators, points
from tests import quadrature

X = sp.symbols("x0 x1 x2")


def _space_monos(shape, p, extra_axis=None):
    """Monomials of the solution space (extra_axis: that axis allows degree p+1,
    used for the tensor-product RT components)."""
    nd = points.NDIM[shape]
    xs = X[:nd]
    out = []
    rng = range(p + 2)
    import itertools
    for e in itertools.product(rng, repeat=nd):
        if shape in ("tri", "tet"):
            ok = sum(e) <= p
        elif shape in ("quad", "hex"):
            ok = all(k <= (p + 1 if a == extra_axis else p) for a, k in enumerate(e))
        else:  # prism
            ok = e[0] + e[1] <= p and e[2] <= (p + 1 if extra_axis == 2 else p)
        if ok:
            out.append(sp.Mul(*[x ** k for x, k in zip(xs, e)]))
    return out


def _random_poly(monos, rng):
    return sum(sp.Rational(int(rng.integers(-9, 10)), int(rng.integers(1, 5))) * m for m in monos)


def _random_rt(shape, p, rng):
    nd = points.NDIM[shape]
    xs = X[:nd]
    if shape in ("tri", "tet"):
        f = [_random_poly(_space_monos(shape, p), rng) for _ in range(nd)]
        hom = [m for m in _space_monos(shape, p) if sp.Poly(m, *xs).total_degree() == p]
        h = _random_poly(hom, rng)
        return [fi + xi * h for fi, xi in zip(f, xs)]
    if shape in ("quad", "hex"):
        return [_random_poly(_space_monos(shape, p, extra_axis=d), rng) for d in range(nd)]
    # prism: [P_p(x,y)^2 + (x,y) Pbar_p(x,y)] P_p(z)  x  P_p(x,y) P_{p+1}(z)
    base = _space_monos(shape, p)
    hom = [m for m in base if sp.Poly(m, X[0], X[1]).total_degree() == p]
    f0 = _random_poly(base, rng)
    f1 = _random_poly(base, rng)
    h = _random_poly(hom, rng)
    f2 = _random_poly(_space_monos(shape, p, extra_axis=2), rng)
    return [f0 + X[0] * h, f1 + X[1] * h, f2]


def _ev(expr, pts):
    nd = pts.shape[1]
    fn = sp.lambdify(X[:nd], expr, "numpy")
    return np.broadcast_to(np.asarray(fn(*pts.T), float), (len(pts),)).copy()


CASES = [(s, p) for s in points.SHAPES for p in (1, 2, 3, 4)]


@pytest.mark.parametrize("shape,p", CASES)
def test_interpolation_reproduces_solution_space(shape, p):
    op = operators.get(shape, p)
    rng = np.random.default_rng(1)
    u = _random_poly(_space_monos(shape, p), rng)
    us = _ev(u, op.xs)
    scale = np.abs(us).max()
    assert np.abs(op.M0 @ us - _ev(u, op.xfe)).max() < 1e-11 * scale
    assert np.abs(op.M12 @ us - _ev(u, op.xfiu)).max() < 1e-11 * scale
    for d in range(op.nd):
        g = _ev(sp.diff(u, X[d]), op.xs)
        assert np.abs(op.Dsol[d] @ us - g).max() < 1e-10 * scale


@pytest.mark.parametrize("shape,p", CASES)
def test_divergence_exact_on_rt_fields(shape, p):
    op = operators.get(shape, p)
    rng = np.random.default_rng(2)
    f = _random_rt(shape, p, rng)
    nd = op.nd
    xfi = op.xfiu[op.fi_point]
    fe = np.stack([_ev(c, op.xfe) for c in f], axis=1)
    fi = np.stack([_ev(c, xfi) for c in f], axis=1)
    Fn_fe = (fe * op.nrm_fe).sum(1)
    Fn_fi = (fi * op.fi_dir).sum(1)
    div = sum(sp.diff(c, X[d]) for d, c in enumerate(f))
    exact = _ev(div, op.xs)
    got = op.M14 @ Fn_fe + op.M13 @ Fn_fi
    assert np.abs(got - exact).max() < 1e-10 * max(1.0, np.abs(fe).max())


@pytest.mark.parametrize("shape,p", CASES)
def test_gradient_operators_exact(shape, p):
    """q~ = M16 u_fe + M15 P M12 u reproduces grad u for u in the solution space
    (App. B gradient equation with continuous common values)."""
    op = operators.get(shape, p)
    rng = np.random.default_rng(3)
    u = _random_poly(_space_monos(shape, p), rng)
    us = _ev(u, op.xs)
    qt = op.M16 @ _ev(u, op.xfe) + op.M15 @ (op.P @ (op.M12 @ us))
    qt = qt.reshape(op.nd, op.n_sol)
    for d in range(op.nd):
        g = _ev(sp.diff(u, X[d]), op.xs)
        assert np.abs(qt[d] - g).max() < 1e-9 * max(1.0, np.abs(us).max())


@pytest.mark.parametrize("shape,p", CASES)
def test_internal_basis_has_zero_outflow(shape, p):
    """int div l^fi = 0 (zero normal trace of internal RT functions, App. A) and
    int div l^fe_nu = face quadrature weight of nu, positive and summing to the
    face measure."""
    op = operators.get(shape, p)
    Xq, Wq = quadrature.rule(shape, 10)
    w = Wq @ operators.nodal_sol(shape, p, op.xs, Xq)   # weights of the nodal basis
    assert abs(w.sum() - Wq.sum()) < 1e-12
    assert np.abs(w @ op.M13).max() < 1e-11
    fw = w @ op.M14
    for f in range(len(points.FACES[shape])):
        sel = op.fe_face == f
        assert np.all(fw[sel] > 0)
    # total outflow of a constant unit normal field equals the boundary measure
    # weighted by n~: for f = e_d, sum_nu fw_nu n~_nu,d = int div e_d = 0
    for d in range(op.nd):
        assert abs(fw @ op.nrm_fe[:, d]) < 1e-11
