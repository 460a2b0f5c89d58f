"""Von Neumann (Fourier) analysis of the semi-discrete SDRT operator on
uniform periodic meshes, and the CFL_MAX of explicit RK schemes.

Oracle (test infrastructure only).  Paper Sec. 4:
  * a Fourier mode U_c = U^ e^{i kappa . x_c} over the cells c of a uniform
    mesh (Eq. "initial_condition_fourier_mode"); translation invariance of the
    RHS Jacobian (Eq. "jacobian_rhs") reduces dU/dt = J U to dU^/dt =
    G(kappa) U^ with
        G(kappa) = sum_c J_{c, c0} e^{-i kappa . (x_c - x_c0)},
    J_{c, c0} the block coupling the DOFs of the root cell c0 to those of cell
    c (Eq. "patternvar_diagonalized");
  * pure diffusion (Sec. "Von-Neumann analysis with diffusion"): BR1 (beta =
    0) and eta = 0, the stencil reaches two face-neighbour layers, and the CFL
    number is tau = mu dt / h^2 (with h = 1, mu = 1 the eigenvalues of G are
    the scaled ones);
  * CFL_MAX is the largest tau with |P(tau lambda)| <= 1 for every eigenvalue
    (Sec. "Temporal linear stability"), P the RK stability polynomial
    (Eq. "rk_exponential").
The blocks come from the oracle's complex-step JVP (exact for the linear
problems analysed) with one probe per DOF of the root cell, on a periodic box
of ncell^d unit cells; ncell = 5 keeps the two-layer stencil free of periodic
images.  Eigenvalues by numpy.linalg.eigvals.

Parity: pinned by the paper's diffusion CFL_MAX table for quadrilateral SDRT
(RK3 / RK4 / RK54, p = 1..4), by the textbook RK stability limits and by a
closed-form circulant spectrum (tests/test_oracle_fourier.py).
"""
import numpy as np

from . import mesh as omesh
from . import residual as ores
from .timestep import rk54_stability_coefficients


def rk_polynomial(z, scheme):
    """R(z) of RK3, RK4 (truncated exponentials) and RK54 (from its
    published 2N-storage coefficients)."""
    if scheme == "rk3":
        c = [1.0, 1.0, 1 / 2, 1 / 6]
    elif scheme == "rk4":
        c = [1.0, 1.0, 1 / 2, 1 / 6, 1 / 24]
    elif scheme == "rk54":
        c = [float(x) for x in rk54_stability_coefficients()]
    else:
        raise ValueError(scheme)
    return sum(ci * z ** i for i, ci in enumerate(c))


def pattern_blocks(mesh, ncell, degree, phys):
    """Blocks J_{c, c0} (ncell^d, N, N) and cell offsets x_c - x_c0 (nearest
    periodic image, in cells) of a periodic box mesh of ncell^d unit cells
    whose elements are numbered cell by cell (x fastest), one element shape.
    N = elements per cell x solution points x variables (variables fastest
    inside a point)."""
    geom = omesh.build(mesh, degree)
    if len(geom.blocks) != 1:
        raise ValueError("one element shape per cell pattern")
    g = geom.blocks[0]
    nd = geom.nd
    ncells = ncell ** nd
    k = g.nelem // ncells
    ns, V = g.ops.n_sol, phys.nvar
    N = k * ns * V
    c0 = sum((ncell // 2) * ncell ** i for i in range(nd))
    U = [np.zeros((ns, V, g.nelem))]
    blocks = np.zeros((ncells, N, N))
    j = 0
    for el in range(k):
        for s in range(ns):
            for v in range(V):
                dU = [np.zeros((ns, V, g.nelem))]
                dU[0][s, v, c0 * k + el] = 1.0
                JdU = ores.jvp(geom, phys, U, dU)[0]                  # (ns, V, E)
                col = JdU.reshape(ns, V, ncells, k).transpose(2, 3, 0, 1).reshape(ncells, N)
                blocks[:, :, j] = col
                j += 1
    cell = np.array([[(c // ncell ** i) % ncell for i in range(nd)] for c in range(ncells)])
    ref = np.array([(c0 // ncell ** i) % ncell for i in range(nd)])
    off = (cell - ref + ncell // 2) % ncell - ncell // 2
    return blocks, off.astype(float)


def reduced_matrix(blocks, offsets, kappa):
    """G(kappa) for one wavenumber (kappa h per axis)."""
    ph = np.exp(-1j * (offsets @ np.asarray(kappa, float)))
    return np.einsum("c,cij->ij", ph, blocks)


def eigenvalues(blocks, offsets, kappas):
    return np.array([np.linalg.eigvals(reduced_matrix(blocks, offsets, k)) for k in kappas])


def cfl_max(eigs, scheme, tol=1e-10, round_tol=1e-8):
    """Largest tau with |P(tau lambda)| <= 1 + tol for all eigenvalues
    (bisection; positive real parts below round_tol * max |lambda| are the
    eigen-solver's rounding and count as zero)."""
    lam = np.asarray(eigs).ravel()
    amax = np.abs(lam).max()
    re = np.where((lam.real > 0) & (lam.real < round_tol * amax), 0.0, lam.real)
    lam = re + 1j * lam.imag

    def stable(t):
        return bool(np.all(np.abs(rk_polynomial(t * lam, scheme)) <= 1 + tol))

    lo, hi = 0.0, 8.0 / amax
    if stable(hi):
        return hi
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        if stable(mid):
            lo = mid
        else:
            hi = mid
    return lo
