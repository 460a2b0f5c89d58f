"""Pins of the oracle's Taylor-Green diagnostics (oracle/tgv.py, paper Sec. 5.3):

* the element quadrature integrates every monomial of degree <= 10 exactly
  (closed forms on the reference simplex / prism / box);
* at the Taylor-Green initial state (Eq. "tgvInitCondition", Re 1600, Ma 0.1):
  <E*> = 1/8 up to the O(Ma^2) density variation; eps2 = 2 mu <S^d : S^d> =
  3 mu / 4 (t_c = 1: the initial strain rate of the divergence-free field);
  eps3 = 0 (div v = 0);
* eps1, evaluated from the residual, equals the finite-difference time
  derivative of <E*> along the oracle's own RK4 steps (the two formulas agree).
"""
from math import factorial

import numpy as np
import pytest

from inputs import fields, meshes
from oracle import mesh as omesh
from oracle import physics as ophx
from oracle import residual as ores
from oracle import tgv


def _simplex_monomial(a):
    """int over the unit simplex of prod xi_d^a_d = prod a_d! / (|a| + nd)!."""
    return np.prod([factorial(k) for k in a]) / factorial(sum(a) + len(a))


@pytest.mark.parametrize("shape", ["tri", "tet", "pri", "quad", "hex"])
def test_quadrature_is_exact_to_degree_10(shape):
    X, W = tgv.quadrature(shape)
    nd = X.shape[1]
    xi = (X + 1.0) / 2.0                                  # reference vertices -> unit simplex / cube
    rng = np.random.default_rng(5)
    for _ in range(40):
        a = rng.integers(0, 11, nd)
        while a.sum() > 10:
            a[rng.choice(np.flatnonzero(a))] -= 1
        got = np.sum(W * np.prod(xi ** a, axis=1)) / 2.0 ** nd
        if shape in ("tri", "tet"):
            want = _simplex_monomial(list(a))
        elif shape == "pri":
            want = _simplex_monomial(list(a[:2])) / (a[2] + 1)
        else:
            want = np.prod(1.0 / (a + 1))
        assert got == pytest.approx(want, rel=1e-12, abs=1e-15), (shape, a)


def _tgv_case(n, p):
    mesh = meshes.box_mesh("tet", (n,) * 3, [0.0] * 3, [2 * np.pi] * 3)
    geom = omesh.build(mesh, p)
    oph = ophx.Physics("ns", 3, "rusanov", mu=1 / 1600, Pr=0.71, beta=0.5, eta=0.1)
    U = [np.ascontiguousarray(u) for u in
         (lambda g: [np.transpose(fields.taylor_green(b.xsol.reshape(-1, 3), gamma=1.4, mach=0.1)
                                  .reshape(b.nelem, b.ops.n_sol, 5), (1, 2, 0)) for b in g.blocks])(geom)]
    return geom, oph, U


def test_initial_state_closed_forms():
    geom, oph, U = _tgv_case(4, 3)
    d = tgv.diagnostics(geom, oph, U)
    assert abs(d["E"] - 0.125) < 2e-3, d
    assert d["eps2"] == pytest.approx(0.75 * oph.mu, rel=0.03), d
    assert abs(d["eps3"]) < 1e-6 * d["eps2"], d


def test_eps1_is_the_time_derivative_of_the_energy():
    geom, oph, U = _tgv_case(3, 3)
    d0 = tgv.diagnostics(geom, oph, U)
    dt = 5e-5
    E1 = tgv.diagnostics(geom, oph, ores.rk4_step(geom, oph, U, dt))["E"]
    Em = tgv.diagnostics(geom, oph, ores.rk4_step(geom, oph, U, -dt))["E"]
    fd = -(E1 - Em) / (2 * dt)
    assert fd == pytest.approx(d0["eps1"], rel=1e-4), (fd, d0["eps1"])
