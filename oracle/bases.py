"""Monomial modal bases of the solution space and of the Raviart-Thomas flux space.

Oracle (test infrastructure only).  The paper recommends orthonormal modal bases
for conditioning (Sec. 2.1, App. A); the nodal bases do not depend on that
choice, so the oracle uses plain monomials in reference coordinates (the GPU
library builds its operators from a different, Legendre-type basis, so agreement
of the two checks basis independence).

Solution space (App. A):  P_p (triangle, tetrahedron), Q_p (quadrilateral,
hexahedron), P_p(x, y) x P_p(z) (prism).

Raviart-Thomas space (App. A, eqs. for each element type):
  triangle / tetrahedron:  P_p^ND (+) x * Pbar_p          (Pbar = homogeneous degree p)
  quadrilateral:           Q_{p+1,p} x Q_{p,p+1}
  hexahedron:              Q_{p+1,p,p} x Q_{p,p+1,p} x Q_{p,p,p+1}
  prism:                   [P_p(x,y)^2 (+) (x,y) Pbar_p(x,y)] P_p(z)  x  P_p(x,y) P_{p+1}(z)
The divergence of each member is evaluated analytically; for x * m(x) with m
homogeneous of degree k in ND variables, div(x m) = (ND + k) m (Euler's theorem).

Parity: pinned by dim(RT_p) = N_flux (App. A table), by unisolvence, and by the
exact-divergence test against symbolic (sympy) differentiation of independently
built RT fields (tests/test_oracle_operators.py).
"""
import itertools
import numpy as np

from .points import NDIM


def sol_exponents(shape, p):
    nd = NDIM[shape]
    rng = range(p + 1)
    if shape in ("tri", "tet"):
        return [e for e in itertools.product(rng, repeat=nd) if sum(e) <= p]
    if shape in ("quad", "hex"):
        return list(itertools.product(rng, repeat=nd))
    if shape == "pri":
        return [e for e in itertools.product(rng, repeat=3) if e[0] + e[1] <= p]
    raise ValueError(shape)


def _mono(X, e):
    out = np.ones(len(X), dtype=X.dtype)
    for d, k in enumerate(e):
        if k:
            out = out * X[:, d] ** k
    return out


def _dmono(X, e, d):
    if e[d] == 0:
        return np.zeros(len(X), dtype=X.dtype)
    e2 = list(e)
    e2[d] -= 1
    return e[d] * _mono(X, tuple(e2))


def sol_basis(shape, p, X):
    """Values (npts, nmodes) of the monomial solution basis at X."""
    return np.column_stack([_mono(X, e) for e in sol_exponents(shape, p)])


def sol_basis_grad(shape, p, X):
    """Gradients (ND, npts, nmodes) of the monomial solution basis at X."""
    nd = NDIM[shape]
    ex = sol_exponents(shape, p)
    return np.stack([np.column_stack([_dmono(X, e, d) for e in ex]) for d in range(nd)])


def rt_modes(shape, p):
    """List of RT modes.  Each mode is (kind, comp, exps):
    kind 'c' : e_comp * x^exps;
    kind 'x' : (x_0, .., x_{nx-1}, 0..) * x^exps, nx = number of leading components
               multiplied (ND for simplices, 2 for the prism's (x, y) part).
    """
    nd = NDIM[shape]
    modes = []
    if shape in ("tri", "tet"):
        for c in range(nd):
            for e in itertools.product(range(p + 1), repeat=nd):
                if sum(e) <= p:
                    modes.append(("c", c, e))
        for e in itertools.product(range(p + 1), repeat=nd):
            if sum(e) == p:
                modes.append(("x", nd, e))
        return modes
    if shape in ("quad", "hex"):
        for c in range(nd):
            ranges = [range(p + 2) if a == c else range(p + 1) for a in range(nd)]
            for e in itertools.product(*ranges):
                modes.append(("c", c, e))
        return modes
    if shape == "pri":
        for c in range(2):
            for e in itertools.product(range(p + 1), repeat=3):
                if e[0] + e[1] <= p:
                    modes.append(("c", c, e))
        for e in itertools.product(range(p + 1), repeat=3):
            if e[0] + e[1] == p:
                modes.append(("x", 2, e))
        for e in itertools.product(range(p + 1), range(p + 1), range(p + 2)):
            if e[0] + e[1] <= p:
                modes.append(("c", 2, e))
        return modes
    raise ValueError(shape)


def rt_basis(shape, p, X):
    """Values (npts, nmodes, ND) of the RT monomial basis at X."""
    nd = NDIM[shape]
    modes = rt_modes(shape, p)
    out = np.zeros((len(X), len(modes), nd), dtype=X.dtype)
    for m, (kind, c, e) in enumerate(modes):
        v = _mono(X, e)
        if kind == "c":
            out[:, m, c] = v
        else:
            for d in range(c):
                out[:, m, d] = X[:, d] * v
    return out


def rt_divergence(shape, p, X):
    """Divergence (npts, nmodes) of the RT monomial basis at X."""
    nd = NDIM[shape]
    modes = rt_modes(shape, p)
    out = np.zeros((len(X), len(modes)), dtype=X.dtype)
    for m, (kind, c, e) in enumerate(modes):
        if kind == "c":
            out[:, m] = _dmono(X, e, c)
        else:
            k = sum(e[:c])          # degree of the multiplied homogeneous part
            out[:, m] = (c + k) * _mono(X, e)
    return out
