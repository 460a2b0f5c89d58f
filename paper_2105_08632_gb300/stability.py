"""Fourier (von Neumann) stability of the semi-discrete SDRT operator for
linear advection on uniform periodic meshes (paper Sec. 4, Eqs.
"initial_condition_fourier_mode" to "semi_discrete_exponential", and the
temporal linear stability of Sec. 4 with the RK polynomials of Eq.
"rk_exponential"), and of pure diffusion (Sec. "Von-Neumann analysis with
diffusion": BR1, beta = 0, eta = 0, tau = mu dt / h^2).

For a Fourier mode U_c = U e^{i kappa . x_c} over the cells c of a uniform
mesh (each cell split into the same pattern of elements), translation
invariance of the residual's Jacobian J gives dU/dt = G(kappa) U with the
reduced Jacobian

    G(kappa) = sum_c J_{c, c0} e^{-i kappa . (x_c - x_c0)},

J_{c, c0} the block coupling the pattern DOFs of cell c0 to those of cell c.
The blocks come from JVP probes of the library on an n^d periodic box whose
mesh the caller passes (n = 3 for advection, 5 for the two-layer diffusion
stencil, so that every coupled cell is a distinct cell), one probe per
pattern DOF of the root cell.  The eigenvalues of G on a kappa grid are computed in FP64 on
the GPU (wavenumbers along the advection direction, as in the paper's
tables, or the whole zone), and CFL_MAX is the largest tau = |a| dt / h with
|P(tau lambda)| <= 1 for every eigenvalue, P the RK stability polynomial
(h = cell size = 1, |a| = 1 or mu = 1).
"""
import numpy as np


def rk_polynomial(z, scheme="rk4"):
    """Stability polynomial of the explicit RK schemes of the paper."""
    if scheme == "rk3":
        return 1 + z + z ** 2 / 2 + z ** 3 / 6
    if scheme == "rk4":
        return 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24
    if scheme == "rk54":
        return 1 + z + z ** 2 / 2 + z ** 3 / 6 + z ** 4 / 24 + z ** 5 / 200
    raise ValueError(scheme)


def advection_direction(theta0, theta1=None):
    """a = (cos t0, sin t0) in 2D; (cos t0 cos t1, sin t0, cos t0 sin t1) in 3D."""
    if theta1 is None:
        return (np.cos(theta0), np.sin(theta0))
    return (np.cos(theta0) * np.cos(theta1), np.sin(theta0), np.cos(theta0) * np.sin(theta1))


def pattern_blocks(ctx, mesh, ncell, degree, physics):
    """Blocks J_{c, c0} (ncell^d, N, N) and cell offsets x_c - x_c0 (ncell^d, d)
    of a linear system on a periodic box of ncell^d unit cells, N = elements
    per cell x solution points (one variable).  mesh: the box's mesh dict (one
    element shape, elements numbered cell by cell, x fastest); physics: an
    FP64 linear system (advection, or advection-diffusion with mu > 0, whose
    BR1 stencil reaches two neighbour layers: ncell >= 5).  FP64 JVPs on the
    context's device."""
    import torch

    from . import sdrt
    nd = mesh["blocks"][0]["verts"].shape[2]
    if len(mesh["blocks"]) != 1:
        raise ValueError("one element shape per cell pattern")
    M = sdrt.Mesh(ctx, mesh, degree, physics)
    if M.nvar != 1:
        raise ValueError("scalar linear systems only")
    lay = M.layouts[0]
    nsol, ld, nelem = lay["nsol"], lay["ld"], lay["nelem"]
    ncells = ncell ** nd
    if nelem % ncells:
        raise ValueError("element count is not a multiple of the cell count")
    k = nelem // ncells                                  # elements per cell (cells in order, x fastest)
    N = k * nsol
    c0 = sum((ncell // 2) * ncell ** i for i in range(nd))   # the central cell
    dev = torch.device("cuda", ctx.device)
    U = torch.zeros(M.state_len, dtype=torch.float64, device=dev)
    V = torch.zeros_like(U)
    JV = torch.zeros_like(U)
    # column (e_local, rho) of the pattern <-> state index rho * ld + e
    cols = [rho * ld + (c0 * k + el) for el in range(k) for rho in range(nsol)]
    # rows of cell c in the same order
    rows = torch.tensor([[rho * ld + (c * k + el) for el in range(k) for rho in range(nsol)] for c in range(ncells)],
                        device=dev)
    blocks = torch.zeros(ncells, N, N, dtype=torch.float64, device=dev)
    for j, idx in enumerate(cols):
        V.zero_()
        V[idx] = 1.0
        M.jvp(U, V, JV)
        blocks[:, :, j] = JV[rows]
    M.sync()
    cell = np.array([[(c // ncell ** i) % ncell for i in range(nd)] for c in range(ncells)])
    ref = np.array([(c0 // ncell ** i) % ncell for i in range(nd)])
    off = cell - ref
    off = (off + ncell // 2) % ncell - ncell // 2       # nearest periodic image
    return blocks, torch.tensor(off, dtype=torch.float64, device=dev)


def kappa_grid(nd, n):
    """kappa h in [-pi, pi) on an n^d grid (n per direction)."""
    import torch
    k1 = -np.pi + 2 * np.pi * np.arange(n) / n
    g = np.stack(np.meshgrid(*([k1] * nd), indexing="ij"), axis=-1).reshape(-1, nd)
    return torch.tensor(g, dtype=torch.float64)


def kappa_line(a, n, kmax=2 * np.pi):
    """kappa along the direction a, kappa h in [0, kmax] (n samples): the
    wavenumbers of the paper's CFL_MAX tables (advection: along the advection
    direction; diffusion: along a mesh axis; converged by kmax = 2 pi)."""
    import torch
    d = np.asarray(a, float) / np.linalg.norm(a)
    t = np.linspace(0.0, kmax, n)
    return torch.tensor(t[:, None] * d[None, :], dtype=torch.float64)


def reduced_eigenvalues(blocks, offsets, kappas, batch=4096):
    """Eigenvalues of G(kappa) for every kappa (n_kappa, N), complex128, on the
    blocks' device."""
    import torch
    dev = blocks.device
    kap = kappas.to(dev)
    Jc = blocks.to(torch.complex128)
    out = []
    for s in range(0, kap.shape[0], batch):
        ph = torch.exp(-1j * (kap[s:s + batch] @ offsets.T))          # (b, ncells)
        G = torch.einsum("bc,cij->bij", ph, Jc)
        out.append(torch.linalg.eigvals(G))
    return torch.cat(out)


def cfl_max(eigs, scheme="rk4", tol=1e-10, iters=60, round_tol=1e-8):
    """Largest tau with |P(tau lambda)| <= 1 + tol for every eigenvalue.
    Positive real parts below round_tol * max |lambda| are the eigen-solver's
    rounding (the spatial operator is dissipative) and are taken as zero."""
    import torch
    lam = eigs.reshape(-1)
    amax = float(lam.abs().max())
    re = lam.real
    lam = torch.complex(torch.where((re > 0) & (re < round_tol * amax), torch.zeros_like(re), re), lam.imag)
    hi = 8.0 / amax                     # above every RK stability limit used here
    lo = 0.0

    def stable(t):
        return bool((rk_polynomial(t * lam, scheme).abs() <= 1 + tol).all())

    if stable(hi):
        return hi
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if stable(mid):
            lo = mid
        else:
            hi = mid
    return lo


def cfl_table(ctx, mesh, ncell, degrees, physics, kappas, schemes=("rk4",)):
    """CFL_MAX per degree and scheme on the wavenumbers `kappas` (kappa h per
    axis, e.g. kappa_line or kappa_grid), plus the largest real part and the
    largest modulus of the spatial eigenvalues."""
    out = {}
    for p in degrees:
        blocks, off = pattern_blocks(ctx, mesh, ncell, p, physics)
        eig = reduced_eigenvalues(blocks, off, kappas)
        out[p] = {s: cfl_max(eig, s) for s in schemes}
        out[p]["max_real"] = float(eig.real.max())
        out[p]["max_abs"] = float(eig.abs().max())
    return out
