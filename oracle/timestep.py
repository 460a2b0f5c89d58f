"""Explicit time integrators of the paper: classical RK4, the five-stage
fourth-order two-register (2N-storage) RK54 of Carpenter and Kennedy, and a
PI step-size controller.

Oracle (test infrastructure only).

  * RK4: the classical four-stage scheme (paper Sec. 2.1 time marching; its
    stability polynomial is the degree-4 Taylor polynomial, Eq. "rk_exponential").
  * RK54: Carpenter & Kennedy (1994), "Fourth-order 2N-storage Runge-Kutta
    schemes", NASA TM-109112, the five-stage solution the paper cites for its
    RK54.  Two registers: dU <- A_i dU + dt R(U), U <- U + B_i dU.  The
    coefficients below are that report's published rationals.  The paper fixes
    the scheme's linear stability polynomial, sum_{i<=4} z^i/i! + z^5/200
    (Eq. "rk_exponential"); tests/test_oracle_timestep.py derives it from these
    coefficients exactly (rational arithmetic) and checks the eight order
    conditions of a fourth-order method.
  * PI controller (paper Sec. 5.3 runs the Taylor-Green vortex with RK54 and
    a PI controller, citing Butcher's textbook, with absolute and relative
    tolerances and the L-infinity norm of the error estimate): the embedded
    estimate is the difference between the RK54 solution and a third-order
    solution from the same stages; the step factor of an accepted step is
        f = safety * err_n^(-alpha) * err_{n-1}^(beta),
    of a rejected one safety * err_n^(-alpha), clipped to [fmin, fmax], with
    alpha = 0.7/k and beta = 0.4/k (k = the estimator's order + 1), the PI
    gains of the control-theoretic step-size literature (Gustafsson; Hairer &
    Wanner, Sec. IV.2).  The paper does not print its estimator or gains:
    this is the reading stated in the design notes, and the library
    implements the same reading.

Parity: RK54 pinned by the paper's stability polynomial and the fourth-order
conditions; RK4 by its textbook stability polynomial and order; the PI
controller's arithmetic is pinned by its closed-form factor on scalar
problems (tests/test_oracle_timestep.py).
"""
from fractions import Fraction

import numpy as np

# Carpenter-Kennedy (5,4) 2N-storage coefficients (published rationals).
RK54_A = (Fraction(0), Fraction(-567301805773, 1357537059087), Fraction(-2404267990393, 2016746695238),
          Fraction(-3550918686646, 2091501179385), Fraction(-1275806237668, 842570457699))
RK54_B = (Fraction(1432997174477, 9575080441755), Fraction(5161836677717, 13612068292357),
          Fraction(1720146321549, 2090206949498), Fraction(3134564353537, 4481467310338),
          Fraction(2277821191437, 14882151754819))
RK54_C = (Fraction(0), Fraction(1432997174477, 9575080441755), Fraction(2526269341429, 6820363962896),
          Fraction(2006345519317, 3224310063776), Fraction(2802321613138, 2924317926251))


def rk54_step(rhs, U, dt):
    """One RK54 step of dU/dt = rhs(U) (autonomous), two registers.
    U: list of arrays (one per block).  Returns the new state."""
    U = [u.copy() for u in U]
    dU = [np.zeros_like(u) for u in U]
    for a, b in zip(RK54_A, RK54_B):
        R = rhs(U)
        dU = [float(a) * d + dt * r for d, r in zip(dU, R)]
        U = [u + float(b) * d for u, d in zip(U, dU)]
    return U


def rk54_butcher():
    """Butcher tableau (a, b, c) of the 2N-storage RK54, in floating point:
    stage i's input is U0 + sum_j a_ij k_j, the step is U0 + sum_j b_j k_j."""
    s = len(RK54_A)
    a = np.zeros((s, s))
    D = np.zeros(s)           # dU as a combination of the stage slopes k_j
    W = np.zeros(s)           # U - U0 as a combination of the k_j
    for i in range(s):
        a[i] = W
        e = np.zeros(s)
        e[i] = 1.0
        D = float(RK54_A[i]) * D + e
        W = W + float(RK54_B[i]) * D
    return a, W, a.sum(axis=1)


def rk54_stability_coefficients():
    """Exact (rational) coefficients of R(z) for dU/dt = z U, low order first."""
    U = [Fraction(1)]
    dU = [Fraction(0)]
    for a, b in zip(RK54_A, RK54_B):
        zU = [Fraction(0)] + U
        n = max(len(dU), len(zU))
        dU = [a * (dU[i] if i < len(dU) else 0) + (zU[i] if i < len(zU) else 0) for i in range(n)]
        n = max(len(U), len(dU))
        U = [(U[i] if i < len(U) else 0) + b * (dU[i] if i < len(dU) else 0) for i in range(n)]
    return U


def embedded_weights():
    """Weights bh = b - n of the embedded third-order solution: n is the unit
    null vector (last component positive) of the four conditions of order <= 3
    on the five stages (sum n = 0, n.c = 0, n.c^2 = 0, n.(a c) = 0), so bh
    keeps third order and Un - Uh = sum_j n_j k_j is the part of the stage
    slopes those conditions do not see (weights of size <= 1)."""
    a, b, c = rk54_butcher()
    M = np.vstack([np.ones_like(c), c, c ** 2, a @ c])
    n = np.linalg.svd(M)[2][-1]
    if n[-1] < 0:
        n = -n
    return b - n


def rk54_embedded_step(rhs, U, dt):
    """RK54 step and the embedded third-order solution from the same stage
    slopes (Butcher form of the same scheme).  Returns (U_new, U_hat)."""
    a, b, c = rk54_butcher()
    bh = embedded_weights()
    U0 = [u.copy() for u in U]
    ks = []
    for i in range(len(b)):
        Ui = [u0 + sum(a[i, j] * k[m] for j, k in enumerate(ks)) for m, u0 in enumerate(U0)]
        ks.append([dt * r for r in rhs(Ui)])
    Un = [u0 + sum(b[j] * k[m] for j, k in enumerate(ks)) for m, u0 in enumerate(U0)]
    Uh = [u0 + sum(bh[j] * k[m] for j, k in enumerate(ks)) for m, u0 in enumerate(U0)]
    return Un, Uh


def error_norm(Un, Uh, U0, atol, rtol):
    """L-infinity norm (the paper's adaptive runs use it, Sec. 5.3) of
    (Un - Uh) / (atol + rtol max(|U0|, |Un|)) over all values."""
    num = np.concatenate([(n - h).ravel() for n, h in zip(Un, Uh)])
    sc = np.concatenate([(atol + rtol * np.maximum(np.abs(u), np.abs(n))).ravel() for u, n in zip(U0, Un)])
    return float(np.max(np.abs(num) / sc))


def pi_factor(err, err_prev, accepted=True, order=3, safety=0.9, fmin=0.2, fmax=5.0):
    """Step-size factor: accepted steps safety * err^(-0.7/k) * err_prev^(0.4/k),
    rejected ones safety * err^(-0.7/k), k = order + 1, clipped to [fmin, fmax]."""
    k = order + 1
    err = max(err, 1e-16)
    err_prev = max(err_prev, 1e-16)
    f = safety * err ** (-0.7 / k) * (err_prev ** (0.4 / k) if accepted else 1.0)
    return min(fmax, max(fmin, f))


def adaptive_step(rhs, U, dt, atol, rtol, err_prev):
    """One RK54 step attempt with the embedded estimate and the PI controller.
    Returns (U_next, accepted, err, dt_next, err_prev_next); on rejection
    U_next is U."""
    Un, Uh = rk54_embedded_step(rhs, U, dt)
    err = error_norm(Un, Uh, U, atol, rtol)
    acc = err <= 1.0
    dt_next = dt * pi_factor(err, err_prev, acc)
    return (Un if acc else U), acc, err, dt_next, (err if acc else err_prev)


def integrate(rhs, U, t_span, dt, atol, rtol, max_steps=100000):
    """Adaptive RK54 over t_span (the last step shortened to end at t_span).
    Returns (U, dt_next, accepted steps, rejected steps)."""
    t, nacc, nrej, err_prev = 0.0, 0, 0, 1.0
    while t < t_span:
        if nacc + nrej >= max_steps:
            raise RuntimeError("max_steps reached")
        h = min(dt, t_span - t)
        U, acc, err, dt, err_prev = adaptive_step(rhs, U, h, atol, rtol, err_prev)
        if acc:
            t += h
            nacc += 1
        else:
            nrej += 1
    return U, dt, nacc, nrej
