"""Pins of the oracle's time integrators (oracle/timestep.py):

* RK54: its linear stability polynomial, derived in exact rational arithmetic
  from the published Carpenter-Kennedy 2N-storage coefficients, is the one the
  paper prints (Eq. "rk_exponential": sum_{i<=4} z^i / i! + z^5 / 200); the
  tableau satisfies the eight conditions of order 4; the two-register
  implementation and the Butcher form give the same step; convergence order
  4 on a nonlinear scalar ODE with a closed-form solution;
* the embedded estimate is third order (local error ~ dt^4) and vanishes for
  polynomial solutions of degree <= 3;
* the PI factor's closed form on scalar inputs.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import timestep as ts


def test_rk54_stability_polynomial_is_the_papers():
    c = ts.rk54_stability_coefficients()
    want = [Fraction(1), Fraction(1), Fraction(1, 2), Fraction(1, 6), Fraction(1, 24), Fraction(1, 200)]
    assert len(c) == 6
    for got, w in zip(c, want):
        # the published coefficients are 13-digit rationals: agreement to 1e-20
        assert abs(float(got - w)) < 1e-20, (got, w)


def test_rk54_order_conditions():
    a, b, c = ts.rk54_butcher()
    assert np.allclose(c, [float(x) for x in ts.RK54_C], atol=1e-14)
    conds = [b.sum() - 1, b @ c - 1 / 2, b @ c ** 2 - 1 / 3, b @ (a @ c) - 1 / 6, b @ c ** 3 - 1 / 4,
             b @ (c * (a @ c)) - 1 / 8, b @ (a @ c ** 2) - 1 / 12, b @ (a @ (a @ c)) - 1 / 24]
    assert np.abs(conds).max() < 1e-14, conds


def _logistic(y):
    return [y[0] * (1 - y[0])]


def _logistic_exact(y0, t):
    return y0 * np.exp(t) / (1 - y0 + y0 * np.exp(t))


def test_rk54_two_register_form_equals_butcher_form_and_converges_at_order_4():
    y0 = np.array([0.2])
    errs = []
    for n in (10, 20, 40):
        dt = 1.0 / n
        y = [y0.copy()]
        for _ in range(n):
            y2 = ts.rk54_step(_logistic, y, dt)
            yb, _ = ts.rk54_embedded_step(_logistic, y, dt)
            assert abs(y2[0][0] - yb[0][0]) < 1e-15
            y = y2
        errs.append(abs(y[0][0] - _logistic_exact(0.2, 1.0)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.8), (errs, rates)


def test_embedded_estimate_is_third_order():
    a, b, c = ts.rk54_butcher()
    bh = ts.embedded_weights()
    assert np.abs([bh.sum() - 1, bh @ c - 0.5, bh @ c ** 2 - 1 / 3, bh @ (a @ c) - 1 / 6]).max() < 1e-14
    assert abs(bh @ c ** 3 - 0.25) > 1e-3          # not fourth order: a genuine estimate
    # the autonomous system t' = 1, z' = 3 t^2 (z = t^3): a cubic, integrated
    # exactly by both solutions, so the estimate vanishes
    rhs = lambda U: [np.ones_like(U[0]), 3 * U[0] ** 2]   # noqa: E731
    Un, Uh = ts.rk54_embedded_step(rhs, [np.array([0.3]), np.array([0.0])], 0.1)
    assert abs(Un[1][0] - Uh[1][0]) < 1e-15 and abs(Un[1][0] - (0.4 ** 3 - 0.3 ** 3)) < 1e-15
    # logistic: local error of the estimate ~ dt^4
    est = []
    for dt in (0.2, 0.1, 0.05):
        Un, Uh = ts.rk54_embedded_step(_logistic, [np.array([0.2])], dt)
        est.append(abs(Un[0][0] - Uh[0][0]))
    r = np.log2(np.array(est[:-1]) / np.array(est[1:]))
    assert np.all(r > 3.7), (est, r)


@pytest.mark.parametrize("err,prev,acc", [(0.5, 1.0, True), (0.8, 0.3, True), (1e-9, 1.0, True), (2.0, 0.8, False)])
def test_pi_factor_closed_form(err, prev, acc):
    k = 4
    want = 0.9 * err ** (-0.7 / k) * (prev ** (0.4 / k) if acc else 1.0)
    want = min(5.0, max(0.2, want))
    assert ts.pi_factor(err, prev, acc) == pytest.approx(want, rel=1e-15)


def test_adaptive_integration_meets_its_tolerance():
    """The controller reaches the end of the span exactly, rejects and shrinks
    a far too large first step, and the global error of the logistic
    solution is of the order of the tolerance."""
    for tol in (1e-6, 1e-9):
        U, dt, nacc, nrej = ts.integrate(_logistic, [np.array([0.2])], 2.0, 1.5, tol, tol)
        err = abs(U[0][0] - _logistic_exact(0.2, 2.0))
        assert nrej >= 1 and nacc >= 3
        assert err < 100 * tol, (tol, err, nacc, nrej)
    # tighter tolerance, more steps
    _, _, n6, _ = ts.integrate(_logistic, [np.array([0.2])], 2.0, 0.1, 1e-6, 1e-6)
    _, _, n9, _ = ts.integrate(_logistic, [np.array([0.2])], 2.0, 0.1, 1e-9, 1e-9)
    assert n9 > n6
