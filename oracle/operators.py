"""Nodal bases and the matrix-form SDRT operators of one element type.

Oracle (test infrastructure only).  Follows paper Sec. 2.1 and App. B:
  solution Vandermonde  V_{rho sigma} = psi_rho(x_sigma),  l = V^{-1} psi;
  flux Vandermonde      Vf_{rho sigma} = psi^f_rho(x_sigma) . n_sigma,  l^f = Vf^{-1} psi^f;
  M0   (N_fe  x N_s)     l_rho(x_fe_sigma)                     (Eq. "interpolation_matrices")
  M12  (N_fiu x N_s)     l_rho(x_fiu_sigma)
  P    (N_fi  x N_fiu)   internal DOF -> unique internal point
  M14  (N_s   x N_fe)    div l^fe_rho(x_sigma)                  (Eq. "flux_matrices")
  M13  (N_s   x N_fi)    div l^fi_rho(x_sigma)
  M16  (ND N_s x N_fe)   n_fe_rho,d div l^fe_rho(x_sigma)       (Eq. "gradient_operators")
  M15  (ND N_s x N_fi)   n_fi_rho,d div l^fi_rho(x_sigma)
Rows of M16 / M15 are ordered (d outer, sigma inner).

Parity: pinned by polynomial reproduction of M0 / M12, exact divergence of RT
fields, FR-SDRT equivalence (Sec. 2.3) and the conservation test
(tests/test_oracle_operators.py, tests/test_oracle_residual.py).
"""
from dataclasses import dataclass

import numpy as np

from . import bases, points


@dataclass
class ElementOps:
    shape: str
    p: int
    nd: int
    xs: np.ndarray        # (N_s, ND) solution points
    xfe: np.ndarray       # (N_fe, ND) external flux points
    nrm_fe: np.ndarray    # (N_fe, ND) unit reference normals
    fe_face: np.ndarray   # (N_fe,) face of each external point
    xfiu: np.ndarray      # (N_fiu, ND) unique internal points
    fi_point: np.ndarray  # (N_fi,) unique point of each internal DOF
    fi_dir: np.ndarray    # (N_fi, ND) direction of each internal DOF
    M0: np.ndarray
    M12: np.ndarray
    P: np.ndarray
    M13: np.ndarray
    M14: np.ndarray
    M15: np.ndarray
    M16: np.ndarray
    Dsol: np.ndarray      # (ND, N_s, N_s) gradient of the solution nodal basis at x_s
    cond_sol: float
    cond_flux: float

    @property
    def n_sol(self):
        return len(self.xs)

    @property
    def n_fe(self):
        return len(self.xfe)

    @property
    def n_fi(self):
        return len(self.fi_point)

    @property
    def n_fiu(self):
        return len(self.xfiu)


def nodal_sol(shape, p, xs, X):
    """Values (npts, N_s) of the solution nodal basis at X: psi(X) V^{-1}."""
    Vs = bases.sol_basis(shape, p, xs)
    return np.linalg.solve(Vs.T, bases.sol_basis(shape, p, X).T).T


def build(shape, p):
    nd = points.NDIM[shape]
    xs = points.sol_points(shape, p)
    xfe, nfe, fe_face = points.ext_points(shape, p)
    xfiu, fi_point, fi_dir = points.internal_points(shape, p)
    xfi = xfiu[fi_point]

    # Solution nodal basis.
    Vs = bases.sol_basis(shape, p, xs)                     # (N_s pts, N_s modes)
    Vs_inv = np.linalg.inv(Vs)
    M0 = bases.sol_basis(shape, p, xfe) @ Vs_inv
    M12 = bases.sol_basis(shape, p, xfiu) @ Vs_inv
    gsol = bases.sol_basis_grad(shape, p, xs)              # (ND, N_s, modes)
    Dsol = np.einsum("dpm,mr->dpr", gsol, Vs_inv)

    # Flux nodal basis: flux points = external then internal DOFs.
    xf = np.vstack([xfe, xfi])
    nf = np.vstack([nfe, fi_dir])
    Phi = bases.rt_basis(shape, p, xf)                     # (N_flux, modes, ND)
    Vf = np.einsum("smd,sd->sm", Phi, nf)                  # row = point, col = mode
    if Vf.shape[0] != Vf.shape[1]:
        raise ValueError(f"{shape} p={p}: {Vf.shape[0]} flux DOFs vs {Vf.shape[1]} RT modes")
    Cf = np.linalg.inv(Vf)                                 # l^f_nu = sum_m Cf[m, nu] psi^f_m
    D = bases.rt_divergence(shape, p, xs) @ Cf             # (N_s, N_flux)
    nfe_ = len(xfe)
    M14 = D[:, :nfe_]
    M13 = D[:, nfe_:]
    M16 = np.vstack([nfe[:, d][None, :] * M14 for d in range(nd)])
    M15 = np.vstack([fi_dir[:, d][None, :] * M13 for d in range(nd)])
    P = np.zeros((len(fi_point), len(xfiu)))
    P[np.arange(len(fi_point)), fi_point] = 1.0
    return ElementOps(shape, p, nd, xs, xfe, nfe, fe_face, xfiu, fi_point, fi_dir,
                      M0, M12, P, M13, M14, M15, M16, Dsol,
                      float(np.linalg.cond(Vs)), float(np.linalg.cond(Vf)))


_CACHE = {}


def get(shape, p):
    key = (shape, p)
    if key not in _CACHE:
        _CACHE[key] = build(shape, p)
    return _CACHE[key]
