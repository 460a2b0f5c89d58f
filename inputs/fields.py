"""Analytic initial fields at caller-supplied physical points, and seeded noise.

Every field takes X of shape (npts, ND) and returns (npts, V).  Conserved
variables of the Euler / Navier-Stokes systems are (rho, rho u, [rho v, [rho w]], rho E).
"""
import numpy as np


def sine_product(X, k=2 * np.pi):
    """u = prod_i sin(k x_i) (linear advection; config of the 2D test: k = 2 pi)."""
    return np.prod(np.sin(k * X), axis=1)[:, None]


def sine_sum(X, L=1.0):
    """u = sin(sum_i x_i / L) (paper Sec. 5.1 initial condition)."""
    return np.sin(X.sum(axis=1) / L)[:, None]


def constant(X, values):
    return np.tile(np.asarray(values, float)[None, :], (len(X), 1))


def primitive_to_conserved(rho, vel, p, gamma):
    vel = np.atleast_2d(vel)
    mom = rho[:, None] * vel
    E = p / (gamma - 1) + 0.5 * rho * (vel ** 2).sum(axis=1)
    return np.column_stack([rho, mom, E])


def isentropic_vortex(X, gamma=1.4, mach=0.5, S=13.5, R=1.5, t=0.0, center=(0.0, 0.0)):
    """Isentropic vortex of paper Eq. "eulerVortexWitherden", rho_inf = v_inf = 1,
    p_inf = 1 / (gamma Ma^2); in 3D it is extruded along z with w = 0."""
    nd = X.shape[1]
    xh = X[:, 0] - center[0]
    yh = X[:, 1] - center[1] - t
    f = (1 - xh ** 2 - yh ** 2) / (2 * R ** 2)
    ef = np.exp(f)
    rho = (1 - S ** 2 * mach ** 2 * (gamma - 1) * np.exp(2 * f) / (8 * np.pi ** 2)) ** (1 / (gamma - 1))
    p_inf = 1.0 / (gamma * mach ** 2)
    p = p_inf * rho ** gamma
    u = S * yh * ef / (2 * np.pi * R)
    v = 1 - S * xh * ef / (2 * np.pi * R)
    vel = [u, v] + ([np.zeros_like(u)] if nd == 3 else [])
    return primitive_to_conserved(rho, np.column_stack(vel), p, gamma)


def taylor_green(X, gamma=1.4, mach=0.1, L=1.0):
    """Taylor-Green vortex of paper Eq. "tgvInitCondition", rho_inf = v_inf = 1."""
    x, y, z = X[:, 0] / L, X[:, 1] / L, X[:, 2] / L
    p_inf = 1.0 / (gamma * mach ** 2)
    u = np.sin(x) * np.cos(y) * np.cos(z)
    v = -np.cos(x) * np.sin(y) * np.cos(z)
    w = np.zeros_like(u)
    p = p_inf + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2) / 16
    rho = p / p_inf
    return primitive_to_conserved(rho, np.column_stack([u, v, w]), p, gamma)


def uniform_noise(shape, seed, amp=1.0):
    """amp * U(-1, 1) from NumPy's PCG64 with the given seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return amp * rng.uniform(-1.0, 1.0, size=shape)


def normal_noise(shape, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(size=shape)
